// The trilinear hexahedron at one point of its natural coordinates (FP64): shape functions,
// physical gradients and det J (Eq. 12, 17, 19).  Shared by the pre-computation of the element
// operators and of the quadrature-point operators.
#pragma once

#include <cuda_runtime.h>

namespace fedfem {

// Natural-coordinate sign of VTK hex node i along axis d (nodes 0-3 bottom counter-clockwise,
// 4-7 top): x: + for 1, 2, 5, 6; y: + for 2, 3, 6, 7; z: + for 4-7.
__device__ __forceinline__ double hex_sign(int i, int d)
{
    const int bit = d == 0 ? ((i + 1) >> 1) & 1 : d == 1 ? (i >> 1) & 1 : (i >> 2) & 1;
    return bit ? 1.0 : -1.0;
}

// N [8], B [8][3] = grad_x N = J^-T grad_xi N and det J at (xi, et, ze) for node coordinates x;
// false (and nothing else valid) when det J <= 0.
__device__ __forceinline__ bool hex_point(const double (&x)[8][3], double xi, double et, double ze, double (&N)[8],
                                          double (&B)[8][3], double &det)
{
    double dN[8][3];
    for (int i = 0; i < 8; ++i) {
        const double sx = hex_sign(i, 0), sy = hex_sign(i, 1), sz = hex_sign(i, 2);
        const double a0 = 1.0 + sx * xi, b0 = 1.0 + sy * et, c0 = 1.0 + sz * ze;
        N[i] = 0.125 * a0 * b0 * c0;
        dN[i][0] = 0.125 * sx * b0 * c0;
        dN[i][1] = 0.125 * sy * a0 * c0;
        dN[i][2] = 0.125 * sz * a0 * b0;
    }
    // Jacobian J[r][s] = d x_r / d xi_s
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < 8; ++i)
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) J[r][s] = fma(x[i][r], dN[i][s], J[r][s]);
    // cofactors: inv(J) = adj(J) / det
    const double C00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double C01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double C02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * C00 + J[0][1] * C01 + J[0][2] * C02;
    if (!(det > 0.0)) return false;
    const double C10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    const double C11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    const double C12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const double C20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    const double C21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    const double C22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    // grad_x N = J^{-T} grad_xi N: (grad_x N)_r = sum_s C[r][s] dN_s / det
    const double id = 1.0 / det;
    for (int i = 0; i < 8; ++i) {
        B[i][0] = (C00 * dN[i][0] + C01 * dN[i][1] + C02 * dN[i][2]) * id;
        B[i][1] = (C10 * dN[i][0] + C11 * dN[i][1] + C12 * dN[i][2]) * id;
        B[i][2] = (C20 * dN[i][0] + C21 * dN[i][1] + C22 * dN[i][2]) * id;
    }
    return true;
}

}  // namespace fedfem
