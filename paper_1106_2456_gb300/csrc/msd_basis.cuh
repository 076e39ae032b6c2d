// msd_basis.cuh -- the Gaussian basis functions of the orbitals and their derivatives at a
// point, shared by the orbital kernels (SIMT and tensor-core).
#pragma once

#include <cuda_runtime.h>

namespace msd {

__device__ __forceinline__ float texp(float x) { return expf(x); }
__device__ __forceinline__ double texp(double x) { return exp(x); }

// chi_mu(r) = (r - A)_c^l exp(-alpha |r - A|^2) (lm = 0 for s, 1 + c for p_c) and its four
// derivative channels, v = (chi, d/dx, d/dy, d/dz, laplacian), from the displacement d = r - A.
template <typename TO>
__device__ __forceinline__ void basis_from_disp(const TO (&d)[3], TO al, int lm, TO (&v)[5]) {
    const TO d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const TO g = texp(-al * d2);
    if (lm == 0) {
        v[0] = g;
        v[1] = TO(-2) * al * d[0] * g;
        v[2] = TO(-2) * al * d[1] * g;
        v[3] = TO(-2) * al * d[2] * g;
        v[4] = (TO(4) * al * al * d2 - TO(6) * al) * g;
    } else {
        const int c = lm - 1;
        const TO dc = d[c];
        v[0] = dc * g;
#pragma unroll
        for (int a = 0; a < 3; ++a) v[1 + a] = ((a == c ? TO(1) : TO(0)) - TO(2) * al * d[a] * dc) * g;
        v[4] = dc * (TO(4) * al * al * d2 - TO(10) * al) * g;
    }
}

// The same at the point rp for b = (A, alpha), the displacement taken in FP64.
template <typename TO>
__device__ __forceinline__ void basis_channels(const double* rp, double4 b, int lm, TO (&v)[5]) {
    const TO d[3] = {TO(rp[0] - b.x), TO(rp[1] - b.y), TO(rp[2] - b.z)};
    basis_from_disp<TO>(d, TO(b.w), lm, v);
}

}  // namespace msd
