// Nodal update of the explicit step shared by the persistent step kernel and the plain-launch
// variant kernels: physical constants in the working precision, the A coefficient, the update
// of Eq. 16 with its Kahan compensation and Dirichlet handling, and the surface outflow of
// Eq. 4 and Eq. 7 lumped to a node.
#pragma once

#include <cuda_runtime.h>

#include "fedfem_internal.h"

namespace fedfem {

// Physical constants of the step in the working precision (converted once per launch).
template <typename R>
struct Phys {
    R k_lin, c_lin, h, T_inf, eps_sigma, T_amb, T_zero, T_guard, k_a, c_a;
    R qs, qs_prev;  // external-load multiplier of this step and of the previous one
    R dD, dD_prev;  // change of the prescribed temperatures over this step and the previous one
    Phys() = default;
    __device__ explicit Phys(const PhysParams &p)
        : k_lin((R)p.k_lin), c_lin((R)p.c_lin), h((R)p.h), T_inf((R)p.T_inf), eps_sigma((R)p.eps_sigma),
          T_amb((R)p.T_amb), T_zero((R)p.T_zero), T_guard((R)p.T_guard), k_a((R)p.k_a), c_a((R)p.c_a), qs((R)1),
          qs_prev((R)1), dD((R)0), dD_prev((R)0)
    {
    }
};

// A_i = dt / C0_i: FP64 in the FP64 form; in the FP32 form the FP64 value is kept as an
// unevaluated pair of floats (hi + lo, 48 significant bits) and A q is formed with one FMA and
// rounded once.  Dirichlet nodes carry A = -0.0 (dir() reads the sign bit).
template <typename R>
struct ACoef;
template <>
struct ACoef<float> {
    float2 v;
    __device__ __forceinline__ float mul(float q) const { return fmaf(v.x, q, v.y * q); }
    __device__ __forceinline__ bool dir() const { return (__float_as_uint(v.x) >> 31) != 0u; }
};
template <>
struct ACoef<double> {
    double v;
    __device__ __forceinline__ double mul(double q) const { return v * q; }
    __device__ __forceinline__ bool dir() const { return __double_as_longlong(v) < 0; }
};

// Explicit nodal update (Eq. 16): T' = T + A / f_c(T) (Q - F), Kahan-compensated in FP32; a
// Dirichlet node moves by dD, the change of its prescribed value over the step.  f_c is the
// linear law of ph or (TAB) the table tc.
template <typename R, bool KAHAN, bool TAB, int NH = kHinges>
__device__ __forceinline__ R node_update(R T, float comp, ACoef<R> A, R Q, R F, R dD, const Phys<R> &ph,
                                         const HingeLaw<R> &tc, float &comp_out, int32_t *err)
{
    const R fc = TAB ? hinge_value<NH>(tc, T) : ph.c_a + ph.c_lin * T;
    const R inc = A.dir() ? dD : A.mul((Q - F) / fc);
    R Tn;
    if constexpr (KAHAN) {
        const float y = inc - comp;
        const float t = T + y;
        comp_out = (t - T) - y;
        Tn = t;
    } else {
        Tn = T + inc;
        comp_out = 0.0f;
    }
    if (!(fabs(Tn) <= ph.T_guard)) atomicOr(err, ERRBIT_DIVERGED);
    return Tn;
}

// Convection + radiation outflow of a boundary node (Eq. 4 and Eq. 7 lumped to the node);
// the quartic difference is evaluated as (a-b)(a+b)(a^2+b^2).
template <typename R>
__device__ __forceinline__ R surface_outflow(R T, R Ac, R Ar, const Phys<R> &ph)
{
    const R u = T - ph.T_zero, b = ph.T_amb - ph.T_zero;
    const R rad = ph.eps_sigma * ((u - b) * (u + b) * (u * u + b * b));
    return Ac * ph.h * (T - ph.T_inf) + Ar * rad;
}

}  // namespace fedfem
