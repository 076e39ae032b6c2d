// msd_vmc.cu -- the pieces a VMC energy driver adds around the wavefunction: a Jastrow
// factor exp(J) and the local energy of the electronic Hamiltonian.
//
// The paper runs VMC and DMC on Psi = exp(J) Psi_MD (Section VI) but treats only Psi_MD
// (Section II: the Jastrow factor is left to standard methods).  The Jastrow used here is
// the common two-body Pade form with the cusp coefficients fixed by Kato's conditions:
//   J = sum_{i<j} a_ij r_ij / (1 + b_ee r_ij) + sum_{i,I} (-Z_I) r_iI / (1 + b_en r_iI),
//   a_ij = 1/2 for electrons of unlike spin, 1/4 for like spin.
// The local energy (Hartree atomic units) is
//   E_L = -1/2 sum_i lap_i Psi / Psi + sum_{i<j} 1/r_ij - sum_{i,I} Z_I / r_iI + sum_{I<J} Z_I Z_J / R_IJ,
//   lap_i Psi / Psi = lap_i D / D + lap_i J + |grad_i J|^2 + 2 grad_i J . grad_i D / D,
// with grad_i D / D and lap_i D / D of the multi-determinant part from msd_grad_lap.
// Everything here is FP64 in both precision modes: it is O(n_tot^2) per walker, once per
// sweep for the energy and O(n_tot) per move for the ratio.
#include "msd_internal.h"

namespace msd {
namespace {

constexpr int kLeThreads = 128;      // local energy: one block per walker
constexpr int kJrWarps = 8;          // Jastrow ratio: one warp per walker

// d = |r_a - r_b|, and the difference vector
__device__ __forceinline__ double dist3(double ax, double ay, double az, double bx, double by, double bz, double& dx,
                                        double& dy, double& dz) {
    dx = ax - bx;
    dy = ay - by;
    dz = az - bz;
    return sqrt(dx * dx + dy * dy + dz * dz);
}

// Pade term a r / (1 + b r)
__device__ __forceinline__ double pade(double a, double b, double r) { return a * r / (1.0 + b * r); }

__device__ __forceinline__ double cusp_ee(bool same_spin) { return same_spin ? 0.25 : 0.5; }

// exp(J(R') - J(R)) for a move of electron `elec` to rnew[w]: only the terms that contain
// that electron change.
__global__ void __launch_bounds__(32 * kJrWarps) k_jastrow_ratio(const HamArgs a, int elec, const double* __restrict__ rnew,
                                                                 double* __restrict__ ratio) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * kJrWarps + threadIdx.x / 32;
    if (w >= a.W) return;
    const double* Rw = a.R + (size_t)w * a.n_tot * 3;
    const double ox = Rw[3 * elec], oy = Rw[3 * elec + 1], oz = Rw[3 * elec + 2];
    const double nx = rnew[3 * w], ny = rnew[3 * w + 1], nz = rnew[3 * w + 2];
    const bool up_e = elec < a.n_up;
    double dj = 0.0, dx, dy, dz;
    if (a.b_ee > 0.0)
        for (int j = lane; j < a.n_tot; j += 32) {
            if (j == elec) continue;
            const double xj = Rw[3 * j], yj = Rw[3 * j + 1], zj = Rw[3 * j + 2];
            const double aij = cusp_ee((j < a.n_up) == up_e);
            dj += pade(aij, a.b_ee, dist3(nx, ny, nz, xj, yj, zj, dx, dy, dz)) -
                  pade(aij, a.b_ee, dist3(ox, oy, oz, xj, yj, zj, dx, dy, dz));
        }
    if (a.b_en > 0.0)
        for (int I = lane; I < a.n_nuc; I += 32) {
            const double4 N = a.nuc[I];
            dj += pade(-N.w, a.b_en, dist3(nx, ny, nz, N.x, N.y, N.z, dx, dy, dz)) -
                  pade(-N.w, a.b_en, dist3(ox, oy, oz, N.x, N.y, N.z, dx, dy, dz));
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dj += __shfl_xor_sync(0xffffffffu, dj, o);
    if (lane == 0) ratio[w] *= exp(dj);
}

// Local energy of walker blockIdx.x.  Thread t handles electrons t, t + blockDim, ...: its
// pair terms with every other electron and with every nucleus (each electron pair is visited
// twice, so V_ee is halved), then the block sums kinetic, V_ee and V_en in FP64.
__global__ void __launch_bounds__(kLeThreads) k_local_energy(const HamArgs a, const double* __restrict__ gradD,
                                                             const double* __restrict__ lapD, double* __restrict__ eloc,
                                                             double* __restrict__ parts) {
    extern __shared__ double sR[];  // [n_tot][3]
    __shared__ double red[3][kLeThreads / 32];
    const int w = blockIdx.x;
    const int nt = a.n_tot;
    const double* Rw = a.R + (size_t)w * nt * 3;
    for (int i = threadIdx.x; i < 3 * nt; i += blockDim.x) sR[i] = Rw[i];
    __syncthreads();
    double kin = 0.0, vee = 0.0, ven = 0.0;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const double xi = sR[3 * i], yi = sR[3 * i + 1], zi = sR[3 * i + 2];
        const bool up_i = i < a.n_up;
        double gx = 0.0, gy = 0.0, gz = 0.0, lj = 0.0, dx, dy, dz;
        for (int j = 0; j < nt; ++j) {
            if (j == i) continue;
            const double r = dist3(xi, yi, zi, sR[3 * j], sR[3 * j + 1], sR[3 * j + 2], dx, dy, dz);
            const double rinv = 1.0 / r;
            vee += rinv;
            if (a.b_ee > 0.0) {
                const double aij = cusp_ee((j < a.n_up) == up_i);
                const double t = 1.0 / (1.0 + a.b_ee * r);
                const double d1 = aij * t * t;                 // u'(r)
                const double d2 = -2.0 * aij * a.b_ee * t * t * t;  // u''(r)
                const double s = d1 * rinv;
                gx += s * dx;
                gy += s * dy;
                gz += s * dz;
                lj += d2 + 2.0 * s;
            }
        }
        for (int I = 0; I < a.n_nuc; ++I) {
            const double4 N = a.nuc[I];
            const double r = dist3(xi, yi, zi, N.x, N.y, N.z, dx, dy, dz);
            const double rinv = 1.0 / r;
            ven -= N.w * rinv;
            if (a.b_en > 0.0) {
                const double t = 1.0 / (1.0 + a.b_en * r);
                const double d1 = -N.w * t * t;                // v'(r)
                const double d2 = 2.0 * N.w * a.b_en * t * t * t;  // v''(r)
                const double s = d1 * rinv;
                gx += s * dx;
                gy += s * dy;
                gz += s * dz;
                lj += d2 + 2.0 * s;
            }
        }
        const double* gd = gradD + ((size_t)w * nt + i) * 3;
        const double ld = lapD[(size_t)w * nt + i];
        const double lap_psi = ld + lj + gx * gx + gy * gy + gz * gz + 2.0 * (gx * gd[0] + gy * gd[1] + gz * gd[2]);
        kin -= 0.5 * lap_psi;
    }
    vee *= 0.5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kin += __shfl_xor_sync(0xffffffffu, kin, o);
        vee += __shfl_xor_sync(0xffffffffu, vee, o);
        ven += __shfl_xor_sync(0xffffffffu, ven, o);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = kin;
        red[1][warp] = vee;
        red[2][warp] = ven;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double k = 0.0, ee = 0.0, en = 0.0;
        for (int q = 0; q < kLeThreads / 32; ++q) {
            k += red[0][q];
            ee += red[1][q];
            en += red[2][q];
        }
        eloc[w] = k + ee + en + a.vnn;
        if (parts) {
            parts[4 * (size_t)w + 0] = k;
            parts[4 * (size_t)w + 1] = ee;
            parts[4 * (size_t)w + 2] = en;
            parts[4 * (size_t)w + 3] = a.vnn;
        }
    }
}

}  // namespace

void launch_jastrow_ratio(const Launch& L, const HamArgs& a, int elec, const double* rnew, double* ratio) {
    if (a.W == 0 || (a.b_ee <= 0.0 && a.b_en <= 0.0)) return;
    k_jastrow_ratio<<<(a.W + kJrWarps - 1) / kJrWarps, 32 * kJrWarps, 0, L.stream>>>(a, elec, rnew, ratio);
    L.count();
}

void launch_local_energy(const Launch& L, const HamArgs& a, const double* gradD, const double* lapD, double* eloc,
                         double* parts) {
    if (a.W == 0) return;
    k_local_energy<<<a.W, kLeThreads, sizeof(double) * 3 * a.n_tot, L.stream>>>(a, gradD, lapD, eloc, parts);
    L.count();
}

}  // namespace msd
