// Tabulated property factors f_k(T), f_c(T) (Section 4.2.2 gives k and c at two temperatures
// and interpolates linearly between them; a table generalises this to up to kMaxTablePoints
// increasing temperatures, with the end values held outside the table).
//
// A piecewise-linear factor with points (t_0, v_0) .. (t_{n-1}, v_{n-1}) is evaluated in hinge
// form over u = min(max(T - t_0, 0), t_{n-1} - t_0):
//   f = v_0 + s_0 u + sum_{j=1}^{n-2} (s_j - s_{j-1}) max(u - (t_j - t_0), 0),
// s_j the slope of segment j.  Every term is bounded by the table's own values (no cancellation
// against a large intercept) and the evaluation has no data-dependent branch: one clamp, one
// FMA and three operations per interior point.  Unused hinges carry a zero coefficient.
#pragma once

#include <cuda_runtime.h>

#if defined(__CUDACC__)
#define FEDFEM_UNROLL _Pragma("unroll")
#else
#define FEDFEM_UNROLL
#endif

namespace fedfem {

constexpr int kMaxTablePoints = 8;
constexpr int kHinges = kMaxTablePoints - 2;

template <typename R>
struct HingeLaw {
    R lo, span, v0, s0;
    R u[kHinges];  // t_j - t_0 of the interior points
    R d[kHinges];  // s_j - s_{j-1}
};

// NH: the number of hinges evaluated (the interior points of the table; the unused hinges,
// j >= n - 2, carry zero coefficients, so any NH >= n - 2 gives the same value)
template <int NH = kHinges, typename R>
__host__ __device__ __forceinline__ R hinge_value(const HingeLaw<R> &t, R T)
{
    static_assert(NH >= 0 && NH <= kHinges, "hinge count");
    const R x = T - t.lo;
    const R u = x < (R)0 ? (R)0 : (x > t.span ? t.span : x);
    R f = t.v0 + t.s0 * u;
FEDFEM_UNROLL
    for (int j = 0; j < NH; ++j) {
        const R h = u - t.u[j];
        f += t.d[j] * (h > (R)0 ? h : (R)0);
    }
    return f;
}

// Slope of the factor at T: 0 where the end values are held; at an interior table point the
// slope of the segment below it.
template <typename R>
__host__ __device__ __forceinline__ R hinge_slope(const HingeLaw<R> &t, R T)
{
    const R x = T - t.lo;
    if (!(x > (R)0) || !(x < t.span)) return (R)0;
    R s = t.s0;
FEDFEM_UNROLL
    for (int j = 0; j < kHinges; ++j)
        if (x > t.u[j]) s += t.d[j];
    return s;
}

// Hinge form of the table (T[0..n), v[0..n)), 2 <= n <= kMaxTablePoints, T increasing.
inline HingeLaw<double> make_hinge_law(int n, const double *T, const double *v)
{
    HingeLaw<double> h{};
    h.lo = T[0];
    h.span = T[n - 1] - T[0];
    h.v0 = v[0];
    h.s0 = (v[1] - v[0]) / (T[1] - T[0]);
    double s_prev = h.s0;
    for (int j = 0; j < kHinges; ++j) {
        if (j + 1 < n - 1) {
            const int k = j + 1;  // interior point k, start of segment k
            const double s = (v[k + 1] - v[k]) / (T[k + 1] - T[k]);
            h.u[j] = T[k] - T[0];
            h.d[j] = s - s_prev;
            s_prev = s;
        } else {
            h.u[j] = h.span;
            h.d[j] = 0.0;
        }
    }
    return h;
}

inline HingeLaw<float> hinge_law_f32(const HingeLaw<double> &h)
{
    HingeLaw<float> f;
    f.lo = (float)h.lo;
    f.span = (float)h.span;
    f.v0 = (float)h.v0;
    f.s0 = (float)h.s0;
    for (int j = 0; j < kHinges; ++j) {
        f.u[j] = (float)h.u[j];
        f.d[j] = (float)h.d[j];
    }
    return f;
}

}  // namespace fedfem
