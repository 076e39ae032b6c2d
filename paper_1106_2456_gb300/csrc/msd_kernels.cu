// msd_kernels.cu -- CUDA kernels of the multi-determinant table method for sm_103a.
//
// Notation (per spin): n electrons, N orbitals, m = N - n virtuals.
//   A_0[r][c] = phi_c(r_r)            reference Slater matrix   (Section II, M(i,j) = phi_j(r_i))
//   Ainv[c][r] = (A_0^{-1})[c][r]     stored row-major per walker
//   T[c][a] = sum_r Ainv[c][r] phi_{n+a}(r_r)   excitation table (Section III, Algorithm 1 step 3)
// An excitation u of order k (holes h_q, particles p_l) has det A_u / det A_0 = det T_u with
// T_u[q][l] = T[h_q][p_l] (Section III).  Moving electron i to r' gives (Sherman-Morrison,
// Section III) x = Ainv[:, i], rho = phi_occ(r') . x, y = phi_virt(r') - T^T phi_occ(r') and
//   det A_u(R') / det A_0(R) = det [[T_u, x_u], [-y_u^T, rho]]           (bordered form)
// and the same with every phi(r') replaced by d^a phi(r') for the gradient and laplacian
// channels (Section IV-A: the table with the electron's row replaced by derivative rows; the
// bordered determinant is the generalised matrix determinant lemma of Section IV-C).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "msd_basis.cuh"
#include "msd_internal.h"
#include "msd_records.cuh"
#include "msd_smalldet.cuh"

namespace msd {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV values over the block; every thread receives the totals.  red holds 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) red[warp * NV + i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += red[q * NV + i];
        v[i] = s;
    }
}

__device__ __forceinline__ unsigned char* align16(void* p) {
    uintptr_t a = reinterpret_cast<uintptr_t>(p);
    return reinterpret_cast<unsigned char*>((a + 15) & ~uintptr_t(15));
}

// Copy `count` elements global -> shared, 16-byte vectors when both ends allow it.
template <typename TT>
__device__ __forceinline__ void copy_to_smem(TT* dst, const TT* __restrict__ src, long long count) {
    const long long bytes = count * (long long)sizeof(TT);
    if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0 && (bytes & 15) == 0) {
        const long long nv = bytes >> 4;
        const uint4* s = reinterpret_cast<const uint4*>(src);
        uint4* d = reinterpret_cast<uint4*>(dst);
        for (long long i = threadIdx.x; i < nv; i += blockDim.x) d[i] = __ldg(s + i);
    } else {
        for (long long i = threadIdx.x; i < count; i += blockDim.x) dst[i] = src[i];
    }
}

// ------------------------------------------------------------------------------------------
// A1: basis functions and orbitals at a set of points
// ------------------------------------------------------------------------------------------
// chi_mu(r) = (r - A)_c^l exp(-alpha |r - A|^2) with its gradient and laplacian, then
// phi^a_j = sum_mu chi^a_mu B[mu][j] (Algorithm 1 step 2): a [P NC x nb] x [nb x N] product
// whose left factor is generated on the fly.  Block tile: kOrbTP points x kOrbTJ orbitals, all
// NC channels; basis functions in chunks of KC, the chunk of chi (every point and channel) and
// of B staged in shared memory; each thread accumulates 2 points x NC channels x 4 orbitals.
#ifndef MSD_ORB_TP
#define MSD_ORB_TP 32
#endif
constexpr int kOrbTP = MSD_ORB_TP;   // points per tile (16 threads per point group)
constexpr int kOrbPPT = kOrbTP / 16;  // points per thread
constexpr int kOrbTJ = 64;

template <typename TO>
constexpr int orb_kc() {
    return sizeof(TO) == 4 ? 48 : 24;
}

template <typename TO, int NC>
__device__ __forceinline__ void orbitals_tile(int P, int ppw, const double* __restrict__ pos, long long wstride,
                                              int p_off, const double4* __restrict__ bas,
                                              const int8_t* __restrict__ blm, int nb, const TO* __restrict__ B, int N,
                                              TO* __restrict__ out, const int p0, const int j0) {
    constexpr int KC = orb_kc<TO>();
    __shared__ __align__(16) TO chi[KC][kOrbTP * NC];
    __shared__ __align__(16) TO Bs[KC][kOrbTJ];
    const int tid = threadIdx.x, pg = tid >> 4, jg = tid & 15;  // points kOrbPPT pg + q; orbitals 4 jg .. 4 jg + 3
    TO acc[kOrbPPT][NC][4];
#pragma unroll
    for (int q = 0; q < kOrbPPT; ++q)
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[q][a][c] = TO(0);
    for (int k0 = 0; k0 < nb; k0 += KC) {
        const int kc = min(KC, nb - k0);
        for (int idx = tid; idx < kOrbTP * KC; idx += blockDim.x) {
            // consecutive threads take consecutive points: their chi stores fall in distinct banks
            const int kk = idx / kOrbTP, q = idx - kk * kOrbTP, p = p0 + q, mu = k0 + kk;
            TO v[5] = {TO(0), TO(0), TO(0), TO(0), TO(0)};
            if (p < P && kk < kc) {
                const int w = p / ppw, r = p - w * ppw;
                basis_channels<TO>(pos + (long long)w * wstride + (long long)(p_off + r) * 3, bas[mu], blm[mu], v);
            }
#pragma unroll
            for (int a = 0; a < NC; ++a) chi[kk][q * NC + a] = v[a];
        }
        for (int idx = tid; idx < KC * kOrbTJ; idx += blockDim.x) {
            const int kk = idx / kOrbTJ, jj = idx - kk * kOrbTJ, j = j0 + jj;
            Bs[kk][jj] = (kk < kc && j < N) ? __ldg(B + (long long)(k0 + kk) * N + j) : TO(0);
        }
        __syncthreads();
        for (int kk = 0; kk < kc; ++kk) {
            TO b[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][4 * jg + c];
#pragma unroll
            for (int q = 0; q < kOrbPPT; ++q)
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const TO x = chi[kk][(kOrbPPT * pg + q) * NC + a];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][a][c] = fma(x, b[c], acc[q][a][c]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kOrbPPT; ++q) {
        const int p = p0 + kOrbPPT * pg + q;
        if (p >= P) continue;
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = j0 + 4 * jg + c;
                if (j < N) out[((long long)p * NC + a) * N + j] = acc[q][a][c];
            }
    }
}

template <typename TO, int NC>
__global__ void __launch_bounds__(256) k_orbitals(int P, int ppw, const double* __restrict__ pos, long long wstride,
                                                  int p_off, const double4* __restrict__ bas,
                                                  const int8_t* __restrict__ blm, int nb, const TO* __restrict__ B,
                                                  int N, TO* __restrict__ out) {
    orbitals_tile<TO, NC>(P, ppw, pos, wstride, p_off, bas, blm, nb, B, N, out, blockIdx.x * kOrbTP,
                          blockIdx.y * kOrbTJ);
}

// ------------------------------------------------------------------------------------------
// A7: from-scratch inverse of A_0 (Gauss-Jordan with partial pivoting, FP64, one block per walker)
// ------------------------------------------------------------------------------------------
// Block-wide maximum of one value per thread (every thread receives it); red holds 32 doubles.
__device__ __forceinline__ double block_max(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = 0.0;
    for (int q = 0; q < nw; ++q) v = fmax(v, red[q]);
    return v;
}

// cond_out (nullable): ||A_0||_inf ||A_0^{-1}||_inf, the infinity-norm condition number (infinite
// when a pivot vanished) -- the estimate by which the FP32 path decides which walkers it can
// represent.
template <typename TO>
__device__ __forceinline__ void inverse_block(int n, int N, const TO* __restrict__ src, const int* cols,
                                              double* __restrict__ dst, double* __restrict__ logdet_out,
                                              double* __restrict__ sgn_out, int* __restrict__ status,
                                              double* __restrict__ cond_out = nullptr) {
    // A[r][c] = src[r * N + col(c)], col(c) = cols ? cols[c] : c (a shared-memory map)
    extern __shared__ __align__(16) unsigned char smem[];
    const int ld = n + 1;
    double* a = reinterpret_cast<double*>(smem);  // [n][ld]
    double* f = a + (long long)n * ld;            // [n]
    int* piv = reinterpret_cast<int*>(f + n);     // [n]
    __shared__ int s_p, s_bad;
    __shared__ double s_logdet, s_sign, s_amax[32];
    const int tid = threadIdx.x, bd = blockDim.x;
    const int tx = tid & 31, ty = tid >> 5, ny = bd >> 5;
    // Eliminate on B = A_0^T: row operations on B give X with X B = I up to rounding, so
    // A_0 X^T = I has a small residual -- the identity phi_occ(r_i)^T A_0^{-1} = e_i^T that the
    // Sherman-Morrison row update and the table update rely on.
    double amax = 0.0;
    for (int c = ty; c < n; c += ny)
        for (int r = tx; r < n; r += 32) {
            const double v = double(src[(long long)r * N + (cols ? cols[c] : c)]);
            a[c * ld + r] = v;  // a = A_0^T
            amax = fmax(amax, fabs(v));
        }
    __shared__ double s_normA;
    if (cond_out) {
        __syncthreads();
        double rs = 0.0;  // largest row sum of |A_0|: row r is column r of a
        for (int r = tid; r < n; r += bd) {
            double t = 0.0;
            for (int c = 0; c < n; ++c) t += fabs(a[c * ld + r]);
            rs = fmax(rs, t);
        }
        rs = block_max(rs, s_amax);
        if (tid == 0) s_normA = rs;
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (tx == 0) s_amax[ty] = amax;
    if (tid == 0) {
        s_logdet = 0.0;
        s_sign = 1.0;
        s_bad = 0;
    }
    __syncthreads();
    amax = 0.0;
    for (int q = 0; q < ny; ++q) amax = fmax(amax, s_amax[q]);
    // a pivot below n * 8 eps * max|A_0| means A_0 is singular to working precision
    // (e.g. two electrons of one spin at the same point)
    const double tiny = double(n) * 8.0 * 2.220446049250313e-16 * amax;
    for (int k = 0; k < n; ++k) {
        if (ty == 0) {
            double best = -1.0;
            int bi = k;
            for (int r = k + tx; r < n; r += 32) {
                const double v = fabs(a[r * ld + k]);
                if (v > best) { best = v; bi = r; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tx == 0) { s_p = bi; piv[k] = bi; }
        }
        __syncthreads();
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < n; j += bd) {
                const double t = a[k * ld + j];
                a[k * ld + j] = a[p * ld + j];
                a[p * ld + j] = t;
            }
        __syncthreads();
        const double pv = a[k * ld + k];
        const bool bad = !(fabs(pv) > tiny) || !isfinite(pv);
        const double ip = bad ? 0.0 : 1.0 / pv;
        if (tid == 0) {
            if (bad) s_bad = 1;
            else {
                s_logdet += log(fabs(pv));
                if ((pv < 0.0) != (p != k)) s_sign = -s_sign;
            }
        }
        for (int r = tid; r < n; r += bd) f[r] = a[r * ld + k];
        __syncthreads();
        for (int j = tid; j < n; j += bd) a[k * ld + j] = (j == k) ? ip : a[k * ld + j] * ip;
        __syncthreads();
        for (int r = ty; r < n; r += ny) {
            if (r == k) continue;
            const double fr = f[r];
            for (int j = tx; j < n; j += 32) {
                if (j == k) a[r * ld + k] = -fr * ip;
                else a[r * ld + j] = fma(-fr, a[k * ld + j], a[r * ld + j]);
            }
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k)
            for (int r = tid; r < n; r += bd) {
                const double t = a[r * ld + k];
                a[r * ld + k] = a[r * ld + p];
                a[r * ld + p] = t;
            }
        __syncthreads();
    }
    // a now holds (A_0^T)^{-1} = (A_0^{-1})^T; store A_0^{-1}[c][r] = a[r][c]
    for (int c = ty; c < n; c += ny)
        for (int r = tx; r < n; r += 32) dst[c * n + r] = a[r * ld + c];
    if (cond_out) {
        double rs = 0.0;  // largest row sum of |A_0^{-1}|: row c is column c of a
        for (int c = tid; c < n; c += bd) {
            double t = 0.0;
            for (int r = 0; r < n; ++r) t += fabs(a[r * ld + c]);
            rs = fmax(rs, t);
        }
        rs = block_max(rs, s_amax);
        if (tid == 0) *cond_out = s_bad ? INFINITY : s_normA * rs;
    }
    if (tid == 0) {
        *logdet_out = s_bad ? -INFINITY : s_logdet;
        *sgn_out = s_bad ? 0.0 : s_sign;
        if (s_bad && status) atomicOr(status, ST_SINGULAR);
    }
}

template <typename TO>
__global__ void __launch_bounds__(kBlock) k_inverse(int n, int N, const TO* __restrict__ Phi,
                                                    double* __restrict__ Ainv, double* __restrict__ logdet,
                                                    double* __restrict__ sgn, int* __restrict__ status,
                                                    double* __restrict__ cond) {
    const int w = blockIdx.x;
    inverse_block<TO>(n, N, Phi + (long long)w * n * N, nullptr, Ainv + (long long)w * n * n, logdet + w, sgn + w,
                      status, cond ? cond + w : nullptr);
}

// ------------------------------------------------------------------------------------------
// The canonical method (Section III's point of comparison): every determinant A_u keeps its
// own inverse, updated by Sherman-Morrison after each accepted move.  FP64.
// ------------------------------------------------------------------------------------------
// Column map of string j of one spin: col(c) = c, except hole h_q -> n + p_q.
__device__ __forceinline__ bool string_columns(const ExcDev& g, int n, int m, int j, int* cols) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) cols[c] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int k = 0;
        while (k <= g.kmax && j >= g.goff[k + 1]) ++k;
        if (k == 1 && g.dense1) {
            const int q = j - g.goff[1];
            cols[q / m] = n + q % m;
        } else if (k >= 1) {
            const uint8_t* r = g.rec + g.roff[k] + (long long)(j - g.goff[k]) * rec_bytes(k);
            if (r[0] == kEmptyRecord) cols[0] = -1;
            else
                for (int q = 0; q < k; ++q) cols[r[q]] = n + r[k + q];
        }
    }
    __syncthreads();
    return cols[0] >= 0;
}

// Inverse and det A_u / det A_0 of every string (grid: strings x walkers).
__global__ void __launch_bounds__(kBlock) k_canon_build(int n, int N, int m, ExcDev g, const double* __restrict__ Phi,
                                                        const uint8_t* __restrict__ used, const double* __restrict__ ld0,
                                                        const double* __restrict__ sg0, double* __restrict__ D,
                                                        double* __restrict__ t, int* __restrict__ status) {
    __shared__ int cols[MSD_MAX_ORB];
    __shared__ double s_ld, s_sg;
    const int j = blockIdx.x, w = blockIdx.y;
    double* tw = t + (long long)w * g.n_exc + j;
    if (!used[j] || !string_columns(g, n, m, j, cols)) {
        if (threadIdx.x == 0) *tw = 0.0;
        return;
    }
    inverse_block<double>(n, N, Phi + (long long)w * n * N, cols, D + ((long long)w * g.n_exc + j) * n * n, &s_ld, &s_sg,
                          nullptr);
    __syncthreads();
    if (threadIdx.x == 0) *tw = s_sg * sg0[w] * exp(s_ld - ld0[w]);
}

// Ratio, gradient and laplacian of a move of row `row`: every string's row-i replacement
// ratio d^a_u = sum_c d^a phi_col(c)(r') D_u[c][row], combined as sum_u C_u t_u d^a_u.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_canon_ratio(int n, int N, int m, int row, ExcDev g,
                                                        const uint8_t* __restrict__ used, const double* __restrict__ phi,
                                                        const double* __restrict__ D, const double* __restrict__ t,
                                                        const double* __restrict__ C, const double* __restrict__ S,
                                                        double* __restrict__ ru, double* ratio, double* grad,
                                                        double* lap, double* num_out, double* rho_out,
                                                        int* __restrict__ status) {
    __shared__ double red[32 * NC];
    const int w = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* ph = phi + (long long)w * NC * N;
    double acc[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) acc[a] = 0.0;
    for (int j = warp; j < g.n_exc; j += nw) {
        const double cj = C[(long long)w * g.n_exc + j];
        if (!used[j]) continue;
        // this lane's columns c = lane, lane + 32, ...: col(c) from the string's holes
        int k = 0;
        while (k <= g.kmax && j >= g.goff[k + 1]) ++k;
        int hq[MSD_MAX_ORDER], pq[MSD_MAX_ORDER], kk = 0;
        if (k == 1 && g.dense1) {
            const int q = j - g.goff[1];
            hq[0] = q / m;
            pq[0] = q % m;
            kk = 1;
        } else if (k >= 1) {
            const uint8_t* r = g.rec + g.roff[k] + (long long)(j - g.goff[k]) * rec_bytes(k);
            if (r[0] == kEmptyRecord) continue;
            for (int q = 0; q < k; ++q) { hq[q] = r[q]; pq[q] = r[k + q]; }
            kk = k;
        }
        const double* Dj = D + ((long long)w * g.n_exc + j) * n * n;
        double v[NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) v[a] = 0.0;
        for (int c = lane; c < n; c += 32) {
            int col = c;
            for (int q = 0; q < kk; ++q)
                if (hq[q] == c) col = n + pq[q];
            const double dci = Dj[(long long)c * n + row];
#pragma unroll
            for (int a = 0; a < NC; ++a) v[a] = fma(ph[a * N + col], dci, v[a]);
        }
#pragma unroll
        for (int a = 0; a < NC; ++a) v[a] = warp_sum(v[a]);
        if (lane == 0) {
            ru[(long long)w * g.n_exc + j] = v[0];
            const double wt = cj * t[(long long)w * g.n_exc + j];
#pragma unroll
            for (int a = 0; a < NC; ++a) acc[a] = fma(wt, v[a], acc[a]);
        }
    }
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < NC; ++a) red[warp * NC + a] = acc[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        double num[NC];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            double s = 0.0;
            for (int q = 0; q < nw; ++q) s += red[q * NC + a];
            num[a] = s;
        }
        const double r = num[0] / S[w];
        ratio[w] = r;
        if constexpr (NC == 5) {
            for (int d = 0; d < 3; ++d) grad[(long long)w * 3 + d] = num[1 + d] / num[0];
            lap[w] = num[4] / num[0];
        }
        for (int a = 0; a < NCH; ++a) num_out[(long long)w * NCH + a] = a < NC ? num[a] : 0.0;
        rho_out[w] = ru[(long long)w * g.n_exc];  // the reference string's row ratio
        if (!isfinite(r)) atomicOr(status, ST_NONFINITE);
    }
}

// Sherman-Morrison update of every string's inverse of an accepted walker (grid: strings x
// walkers); t_u <- t_u ratio_u / ratio_0.  The row of the old orbitals comes from Phi.
__global__ void __launch_bounds__(kBlock) k_canon_accept(int n, int N, int m, int row, ExcDev g,
                                                         const uint8_t* __restrict__ used,
                                                         const uint8_t* __restrict__ accept,
                                                         const double* __restrict__ phi_new, int nch,
                                                         const double* __restrict__ Phi, double* __restrict__ D,
                                                         double* __restrict__ t, const double* __restrict__ ru) {
    __shared__ int cols[MSD_MAX_ORB];
    extern __shared__ __align__(16) unsigned char smem[];
    double* delta = reinterpret_cast<double*>(smem);  // [n]
    double* uu = delta + n;                           // [n] delta^T D
    double* di = uu + n;                              // [n] column `row` of D
    const int j = blockIdx.x, w = blockIdx.y;
    if (!accept[w] || !used[j] || !string_columns(g, n, m, j, cols)) return;
    double* Dj = D + ((long long)w * g.n_exc + j) * n * n;
    const double* pn = phi_new + (long long)w * nch * N;
    const double* po = Phi + ((long long)w * n + row) * N;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        delta[c] = pn[cols[c]] - po[cols[c]];
        di[c] = Dj[(long long)c * n + row];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double a = 0.0;
        for (int c = 0; c < n; ++c) a = fma(delta[c], Dj[(long long)c * n + r], a);
        uu[r] = a;
    }
    __syncthreads();
    const double rj = ru[(long long)w * g.n_exc + j];  // = 1 + delta^T D e_row
    const double inv = 1.0 / rj;
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) {
        const int c = int(q / n), r = int(q - (long long)c * n);
        Dj[q] = fma(-di[c] * inv, uu[r], Dj[q]);
    }
    if (threadIdx.x == 0) t[(long long)w * g.n_exc + j] *= rj / ru[(long long)w * g.n_exc];
}

// Per accepted walker: the moved row of Phi, the position, the reference determinant and S.
__global__ void k_canon_commit(int W, int n, int N, int row, int elec, int n_tot, int nch,
                               const uint8_t* __restrict__ accept, const double* __restrict__ phi_new,
                               double* __restrict__ Phi, const double* __restrict__ rnew, double* __restrict__ R,
                               const double* __restrict__ rho, const double* __restrict__ num,
                               double* __restrict__ logdet, double* __restrict__ sgn, double* __restrict__ S) {
    const int w = blockIdx.x;
    if (!accept[w]) return;
    for (int jj = threadIdx.x; jj < N; jj += blockDim.x)
        Phi[((long long)w * n + row) * N + jj] = phi_new[(long long)w * nch * N + jj];
    if (threadIdx.x == 0) {
        const double r0 = rho[w];
        logdet[w] += log(fabs(r0));
        if (r0 < 0.0) sgn[w] = -sgn[w];
        S[w] = num[(long long)w * NCH] / r0;
        for (int d = 0; d < 3; ++d) R[((long long)w * n_tot + elec) * 3 + d] = rnew[w * 3 + d];
    }
}

// ------------------------------------------------------------------------------------------
// A7: excitation table T = A_0^{-1} Phi_virt (Algorithm 1 step 3: one matrix product)
// ------------------------------------------------------------------------------------------
// grid (ceil(m / 64), W); each thread owns a 4 x 4 register tile of a 64-column slab.
template <typename TO, typename TT>
__global__ void __launch_bounds__(kBlock) k_table(int n, int N, const double* __restrict__ Ainv,
                                                  const TO* __restrict__ Phi, TT* __restrict__ T) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int m = N - n, a0 = blockIdx.x * 64, w = blockIdx.y;
    const int lda = n + 1;
    TT* As = reinterpret_cast<TT*>(smem);                                  // [n][lda] = Ainv[c][r]
    TT* Bs = reinterpret_cast<TT*>(align16(As + (long long)n * lda));       // [n][64] = Phi[r][n + a0 + a]
    const double* Aw = Ainv + (long long)w * n * n;
    const TO* Pw = Phi + (long long)w * n * N;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int c = idx / n, r = idx - c * n;
        As[c * lda + r] = TT(Aw[idx]);
    }
    for (int idx = threadIdx.x; idx < n * 64; idx += blockDim.x) {
        const int r = idx >> 6, a = idx & 63;
        Bs[idx] = (a0 + a < m) ? TT(Pw[(long long)r * N + n + a0 + a]) : TT(0);
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    TT* Tw = T + (long long)w * n * m;
    for (int c0 = ty * 4; c0 < n; c0 += 64) {
        TT acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = TT(0);
        for (int r = 0; r < n; ++r) {
            TT av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = (c0 + i < n) ? As[(c0 + i) * lda + r] : TT(0);
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[r * 64 + tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = c0 + i;
            if (c >= n) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int a = a0 + tx * 4 + j;
                if (a < m) Tw[(long long)c * m + a] = acc[i][j];
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// excitation records and small determinants (Section III: r x r determinants of T entries)
// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// excitation values t_u = det T_u for every string (used for the CI sums at set-up/refresh)
// ------------------------------------------------------------------------------------------
template <int K, typename TT>
__device__ __forceinline__ void det_group(const ExcDev& g, const TT* Ts, int ld, TT* tw) {
    const int j0 = g.goff[K], j1 = g.goff[K + 1];
    const uint8_t* rec = g.rec + g.roff[K];
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        int h[K], p[K];
        load_rec<K>(rec, j - j0, h, p);
        tw[j] = h[0] == kEmptyRecord ? TT(0) : small_det<K, TT>(Ts, ld, h, p);
    }
}

template <typename TT>
__global__ void __launch_bounds__(kBlock) k_exc_det(int n, int m, ExcDev g, const TT* __restrict__ T,
                                                    TT* __restrict__ t) {
    extern __shared__ __align__(16) unsigned char smem[];
    TT* Ts = reinterpret_cast<TT*>(smem);
    const int w = blockIdx.x;
    copy_to_smem(Ts, T + (long long)w * n * m, (long long)n * m);
    __syncthreads();
    TT* tw = t + (long long)w * g.n_exc;
    for (int j = g.goff[0] + threadIdx.x; j < g.goff[1]; j += blockDim.x) tw[j] = TT(1);
    if (g.dense1) {
        // singles laid out densely: internal index goff[1] + h m + p holds T[h][p]
        for (int q = threadIdx.x; q < n * m; q += blockDim.x) tw[g.goff[1] + q] = Ts[q];
    }
    for (int k = g.dense1 ? 2 : 1; k <= g.kmax; ++k) {
        switch (k) {
            case 1: det_group<1, TT>(g, Ts, m, tw); break;
            case 2: det_group<2, TT>(g, Ts, m, tw); break;
            case 3: det_group<3, TT>(g, Ts, m, tw); break;
            case 4: det_group<4, TT>(g, Ts, m, tw); break;
            case 5: det_group<5, TT>(g, Ts, m, tw); break;
            case 6: det_group<6, TT>(g, Ts, m, tw); break;
            case 7: det_group<7, TT>(g, Ts, m, tw); break;
            case 8: det_group<8, TT>(g, Ts, m, tw); break;
        }
    }
}

// ------------------------------------------------------------------------------------------
// A5 preparation: C_s[u] = sum_{I : s-string of I is u} c_I t_other[other string of I]
// ------------------------------------------------------------------------------------------
template <typename TT>
__global__ void __launch_bounds__(kBlock) k_ci_contract_light(int n_exc, int n_exc_other, const int* __restrict__ off,
                                                              const int* __restrict__ other,
                                                              const double* __restrict__ c,
                                                              const TT* __restrict__ t_other, TT* __restrict__ C,
                                                              int heavy_len) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = blockIdx.y;
    if (u >= n_exc) return;
    const int b = off[u], e = off[u + 1];
    if (e - b > heavy_len) return;  // handled by k_ci_contract_heavy
    const TT* tw = t_other + (long long)w * n_exc_other;
    // accumulated in the table's precision (at most heavy_len terms; the FP32 path stays off
    // the slow FP64 pipe)
    TT acc = TT(0);
    for (int q = b; q < e; ++q) acc = fma(TT(__ldg(c + q)), tw[__ldg(other + q)], acc);
    C[(long long)w * n_exc + u] = acc;
}

template <typename TT>
__global__ void __launch_bounds__(kBlock) k_ci_contract_heavy(int n_exc, int n_exc_other, const int* __restrict__ heavy,
                                                              const int* __restrict__ off,
                                                              const int* __restrict__ other,
                                                              const double* __restrict__ c,
                                                              const TT* __restrict__ t_other, TT* __restrict__ C) {
    __shared__ double red[32];
    const int u = heavy[blockIdx.x];
    const int w = blockIdx.y;
    const TT* tw = t_other + (long long)w * n_exc_other;
    TT part = TT(0);  // per-thread partial in the table's precision, summed across threads in FP64
    for (int q = off[u] + threadIdx.x; q < off[u + 1]; q += blockDim.x)
        part = fma(TT(__ldg(c + q)), tw[__ldg(other + q)], part);
    double v[1] = {double(part)};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) C[(long long)w * n_exc + u] = TT(v[0]);
}

template <typename TT>
__global__ void __launch_bounds__(kBlock) k_ci_dot(int n_exc, const TT* __restrict__ C, const TT* __restrict__ t,
                                                   double* __restrict__ S) {
    __shared__ double red[32];
    const int w = blockIdx.x;
    const TT* Cw = C + (long long)w * n_exc;
    const TT* tw = t + (long long)w * n_exc;
    double v[1] = {0.0};
    for (int u = threadIdx.x; u < n_exc; u += blockDim.x) v[0] = fma(double(Cw[u]), double(tw[u]), v[0]);
    block_sum<1>(v, red);
    if (threadIdx.x == 0) S[w] = v[0];
}

// ------------------------------------------------------------------------------------------
// A2-A5: reference ratio, excitation sweep, virtual-row contraction and CI reduction
// ------------------------------------------------------------------------------------------
// Every channel a shares T_u and x_u, so with d^a_u = det(T_u) s^a + y^a_u . z_u,
// z_u = adj(T_u) x_u:
//   sum_u C_u d^a_u = s^a S_T + sum_p y^a[p] G[p],
//   S_T = sum_u C_u det T_u,   G[p] = sum over (u, slot l with p_l = p) of C_u z_u[l].
// The sweep therefore builds one m-vector G and one scalar S_T per walker; the five channels
// are five length-m dot products afterwards.  Singles are a dense n x m block when most are
// present: G1[p] = sum_h C1[h][p] x[h], S_T += sum_{h,p} C1[h][p] T[h][p].
constexpr int kWarps = kBlock / 32;
#ifndef MSD_SWEEP_DEPTH
#define MSD_SWEEP_DEPTH 2
#endif
constexpr int kSweepDepth = MSD_SWEEP_DEPTH;  // batches of loads in flight per warp

// Orders 1 and 2 take kUnroll12 batches per iteration, orders 3..kUnrollK two: independent
// eliminations whose shared-memory gathers and arithmetic overlap.
#ifndef MSD_UNROLL12
#define MSD_UNROLL12 4
#endif
#ifndef MSD_UNROLL_KMAX
#define MSD_UNROLL_KMAX 2
#endif
constexpr int kUnroll12 = MSD_UNROLL12;
constexpr int kUnrollK = MSD_UNROLL_KMAX;

template <int K>
__device__ __forceinline__ typename RecRaw<K>::type empty_raw() {
    using Raw = typename RecRaw<K>::type;
    if constexpr (K == 1) return Raw(0xffffu);
    else if constexpr (K == 2) return Raw(0xffffffffu);
    else if constexpr (K <= 4) return make_uint2(0xffffffffu, 0xffffffffu);
    else return make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
}

template <int K, typename TT, int NGW>
__device__ __forceinline__ void sweep_group(const ExcDev& g, const TT* Ts, int ld, const TT* xs,
                                            const TT* __restrict__ Cw, TT* Gw, Accum<TT, 1>& sacc, int first) {
    constexpr int U = K <= 2 ? kUnroll12 : K <= kUnrollK ? 2 : 1;  // batches per iteration
    constexpr int QD = U * ((kSweepDepth + U - 1) / U);            // batches of loads in flight
    const int j0 = g.goff[K], j1 = g.goff[K + 1];
    const uint8_t* rec = g.rec + g.roff[K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    TT* Gmine = Gw + (warp % NGW) * ld;
    // Warps take the group's batches of 32 strings round-robin, numbered on from the `first`
    // batches of the groups swept before, so the batches left over at the end of a group fall
    // on different warps.
    const int nb = (j1 - j0) / kBatch;
    int b = (warp - first % nw + nw) % nw;
    // record and C loads of the next QD batches in flight ahead of the arithmetic; a batch past
    // the group's end reads as empty records
    using Raw = typename RecRaw<K>::type;
    Raw rq[QD];
    TT cq[QD];
#pragma unroll
    for (int i = 0; i < QD; ++i) {
        const int bi = b + i * nw;
        rq[i] = empty_raw<K>();
        cq[i] = TT(0);
        if (bi < nb) {
            rq[i] = load_raw<K>(rec, bi * kBatch + lane);
            cq[i] = __ldcs(Cw + j0 + bi * kBatch + lane);
        }
    }
    for (; b < nb; b += U * nw) {
        Raw rc[U];
        TT cu[U];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            rc[i] = rq[i];
            cu[i] = cq[i];
        }
#pragma unroll
        for (int i = 0; i + U < QD; ++i) {
            rq[i] = rq[i + U];
            cq[i] = cq[i + U];
        }
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int bn = b + (QD + i) * nw;
            rq[QD - U + i] = empty_raw<K>();
            cq[QD - U + i] = TT(0);
            if (bn < nb) {
                rq[QD - U + i] = load_raw<K>(rec, bn * kBatch + lane);
                cq[QD - U + i] = __ldcs(Cw + j0 + bn * kBatch + lane);
            }
        }
        int h[U][K], p[U][K];
        bool live[U];
        TT det[U], z[U][K];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            decode_rec<K>(rc[i], h[i], p[i]);
            live[i] = h[i][0] != kEmptyRecord;
            det[i] = TT(0);
#pragma unroll
            for (int l = 0; l < K; ++l) z[i][l] = TT(0);
        }
#pragma unroll
        for (int i = 0; i < U; ++i)
            if (live[i]) {
                adj_solve<K, TT>(Ts, ld, xs, h[i], p[i], det[i], z[i]);
                sacc.add(0, cu[i] * det[i]);
            }
#pragma unroll
        for (int i = 0; i < U; ++i) {
            if constexpr (sizeof(TT) == 4) {
                // FP32 tables come with conflict-free batches: within a slot the 32 lanes'
                // particles are distinct, and every warp owns its copy of G, so a plain
                // read-modify-write per slot, ordered between slots by a warp barrier, needs no
                // atomics
#pragma unroll
                for (int l = 0; l < K; ++l) {
                    if (live[i]) Gmine[p[i][l]] += cu[i] * z[i][l];
                    __syncwarp();
                }
            } else {
                if (live[i])
#pragma unroll
                    for (int l = 0; l < K; ++l) atomicAdd(Gmine + p[i][l], cu[i] * z[i][l]);
            }
        }
    }
}

// Orders 5..8 are rare and need many registers: called out of line so that their register
// pressure (and spills at the 80-register cap of three CTAs per SM) stays out of the code of
// the common orders.
template <int K, typename TT, int NGW>
__device__ __noinline__ void sweep_group_outlined(const ExcDev& g, const TT* Ts, int ld, const TT* xs,
                                                  const TT* __restrict__ Cw, TT* Gw, Accum<TT, 1>& sacc, int first) {
    sweep_group<K, TT, NGW>(g, Ts, ld, xs, Cw, Gw, sacc, first);
}

struct RatioSmem {
    size_t ts, xd, xs, ph, g1, gw, tg, red, total;
};

__host__ __device__ inline RatioSmem ratio_layout(int n, int m, int nch, int tt_bytes, int to_bytes, int ngw) {
    RatioSmem L;
    auto up = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t mm = (size_t)(m > 0 ? m : 1);
    L.ts = 0;
    L.xd = up(L.ts + (size_t)n * m * tt_bytes);
    L.xs = up(L.xd + (size_t)n * 8);
    L.ph = up(L.xs + (size_t)n * tt_bytes);
    L.g1 = up(L.ph + (size_t)nch * n * to_bytes);
    L.gw = up(L.g1 + mm * tt_bytes);
    L.tg = up(L.gw + (size_t)ngw * mm * tt_bytes);
    L.red = up(L.tg + (size_t)n * tt_bytes);
    L.total = up(L.red + (size_t)32 * (NCH + 1) * 8);
    return L;
}

// Copies of G per block: one per warp in FP32, one per warp pair in FP64 so two blocks of 256
// threads fit an SM.
template <typename TT>
__host__ __device__ constexpr int ratio_ngw() {
    return sizeof(TT) == 4 ? kWarps : kWarps / 2;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Asynchronous global -> shared copy of `bytes` (a multiple of 4) by the whole block
// (cp.async, completion awaited with cp_async_wait_all); 16-byte pieces when both ends allow.
__device__ __forceinline__ void cp_async_block(void* dst, const void* src, size_t bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const char* sp = static_cast<const char*>(src);
    if (((reinterpret_cast<uintptr_t>(src) | d) & 15) == 0 && (bytes & 15) == 0) {
        for (size_t o = size_t(threadIdx.x) * 16; o < bytes; o += size_t(blockDim.x) * 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + (uint32_t)o), "l"(sp + o) : "memory");
    } else {
        for (size_t o = size_t(threadIdx.x) * 4; o < bytes; o += size_t(blockDim.x) * 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + (uint32_t)o), "l"(sp + o) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

#ifndef MSD_RATIO_F32_BLOCKS
#define MSD_RATIO_F32_BLOCKS 3
#endif
// One block per walker.  The table is copied to shared memory asynchronously while the block
// loads x and phi(r') and forms rho and s^a; the sweep then builds S_T and G; the epilogue needs
// one table-vector product TG = T G:
//   sum_p y^a[p] G[p] = phi^a_virt . G - phi^a_occ . TG,   y^a = phi^a_virt - T^T phi^a_occ,
// and y^0 itself only when the proposal is kept for msd_accept.  FP32 tables reduce across a
// warp in FP32 and across warps in FP64.
template <typename TO, typename TT, int NC>
__device__ __forceinline__ void ratio_block(const RatioArgs& a, const int w, int* __restrict__ status) {
    constexpr int NGW = ratio_ngw<TT>();
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n, m = a.m, N = a.N;
    const RatioSmem L = ratio_layout(n, m, NC, sizeof(TT), sizeof(TO), NGW);
    TT* Ts = reinterpret_cast<TT*>(smem + L.ts);
    double* xd = reinterpret_cast<double*>(smem + L.xd);
    TT* xs = reinterpret_cast<TT*>(smem + L.xs);
    TO* ph = reinterpret_cast<TO*>(smem + L.ph);
    TT* G1 = reinterpret_cast<TT*>(smem + L.g1);
    TT* Gw = reinterpret_cast<TT*>(smem + L.gw);
    TT* TG = reinterpret_cast<TT*>(smem + L.tg);
    double* red = reinterpret_cast<double*>(smem + L.red);
    __shared__ double s_s[NC];

    const int tid = threadIdx.x, bd = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (m > 0) cp_async_block(Ts, static_cast<const TT*>(a.T) + (long long)w * n * m, (size_t)n * m * sizeof(TT));
    const TO* phw = static_cast<const TO*>(a.phi) + (long long)w * NC * N;
    const double* Aw = a.Ainv + (long long)w * n * n;
    for (int c = tid; c < n; c += bd) {
        const double v = Aw[(long long)c * n + a.row];
        xd[c] = v;
        xs[c] = TT(v);
    }
#pragma unroll
    for (int al = 0; al < NC; ++al)
        for (int c = tid; c < n; c += bd) ph[al * n + c] = phw[al * N + c];
    for (int q = tid; q < (m > 0 ? m : 1); q += bd) G1[q] = TT(0);
    for (int q = tid; q < NGW * (m > 0 ? m : 1); q += bd) Gw[q] = TT(0);
    __syncthreads();
    // A2: rho = phi_occ(r') . x and s^a = d^a phi_occ(r') . x (FP64)
    if (warp < NC) {
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) acc = fma(double(ph[warp * n + c]), xd[c], acc);
        acc = warp_sum(acc);
        if (lane == 0) s_s[warp] = acc;
    }
    cp_async_wait_all();
    __syncthreads();
    // A4: S_T and G over every excitation
    Accum<TT, 1> sacc;
    sacc.zero();
    const TT* Cw = static_cast<const TT*>(a.C) + (long long)w * a.g.n_exc;
    for (int j = a.g.goff[0] + tid; j < a.g.goff[1]; j += bd) sacc.add(0, Cw[j]);
    if (a.g.dense1) {
        // column p of the dense singles block: G1[p] = sum_h C1[h][p] x[h], S_T += C1[h][p] T[h][p];
        // sixteen rows per round so sixteen loads of the C stream are in flight per thread
        const TT* C1 = Cw + a.g.goff[1];
        for (int pv = tid; pv < m; pv += bd) {
            TT g = TT(0), st = TT(0);
            int h = 0;
            for (; h + 16 <= n; h += 16) {
                TT c[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) c[q] = __ldcs(C1 + (h + q) * m + pv);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    g = fma(c[q], xs[h + q], g);
                    st = fma(c[q], Ts[(h + q) * m + pv], st);
                }
            }
            for (; h < n; ++h) {
                const TT c = __ldcs(C1 + h * m + pv);
                g = fma(c, xs[h], g);
                st = fma(c, Ts[h * m + pv], st);
            }
            G1[pv] = g;
            sacc.add(0, st);
        }
    }
    int first = 0;  // batches of the groups swept so far
    for (int k = a.g.dense1 ? 2 : 1; k <= a.g.kmax; ++k) {
        switch (k) {
            case 1: sweep_group<1, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
            case 2: sweep_group<2, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
            case 3: sweep_group<3, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
            case 4: sweep_group<4, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
            case 5: sweep_group_outlined<5, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
            case 6: sweep_group_outlined<6, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
            case 7: sweep_group_outlined<7, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
            case 8: sweep_group_outlined<8, TT, NGW>(a.g, Ts, m, xs, Cw, Gw, sacc, first); break;
        }
        first += (a.g.goff[k + 1] - a.g.goff[k]) / kBatch;
    }
    __syncthreads();
    // G = G1 + the per-warp copies, kept in G1
    for (int pv = tid; pv < m; pv += bd) {
        TT gp = G1[pv];
#pragma unroll
        for (int q = 0; q < NGW; ++q) gp += Gw[q * m + pv];
        G1[pv] = gp;
    }
    __syncthreads();
    // TG[c] = sum_p T[c][p] G[p], one warp per row
    for (int c = warp; c < n; c += bd >> 5) {
        TT acc = TT(0);
        for (int pv = lane; pv < m; pv += 32) acc = fma(Ts[c * m + pv], G1[pv], acc);
        acc = warp_sum_t(acc);
        if (lane == 0) TG[c] = acc;
    }
    // A3 (kept for msd_accept): y^0[p] = phi_virt(r')[p] - sum_c T[c][p] phi_occ(r')[c]
    if (a.y0) {
        TT* yw = static_cast<TT*>(a.y0) + (long long)w * m;
        for (int pv = tid; pv < m; pv += bd) {
            TT y = TT(phw[n + pv]);
            for (int c = 0; c < n; ++c) y = fma(-Ts[c * m + pv], TT(ph[c]), y);
            yw[pv] = y;
        }
    }
    __syncthreads();
    // A5: sum_p y^a[p] G[p] per channel, and S_T
    TT v[NC + 1];
#pragma unroll
    for (int al = 0; al < NC; ++al) v[al] = TT(0);
    v[NC] = TT(sacc.get(0));
    for (int pv = tid; pv < m; pv += bd) {
        const TT gp = G1[pv];
#pragma unroll
        for (int al = 0; al < NC; ++al) v[al] = fma(TT(phw[al * N + n + pv]), gp, v[al]);
    }
    for (int c = tid; c < n; c += bd) {
        const TT tg = TG[c];
#pragma unroll
        for (int al = 0; al < NC; ++al) v[al] = fma(-TT(ph[al * n + c]), tg, v[al]);
    }
#pragma unroll
    for (int i = 0; i <= NC; ++i) v[i] = warp_sum_t(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i <= NC; ++i) red[warp * (NC + 1) + i] = double(v[i]);
    __syncthreads();
    if (tid == 0) {
        double tot[NC + 1];
#pragma unroll
        for (int i = 0; i <= NC; ++i) {
            double t = 0.0;
            for (int q = 0; q < (bd >> 5); ++q) t += red[q * (NC + 1) + i];
            tot[i] = t;
        }
        const double ST = tot[NC];
        double num[NC];
#pragma unroll
        for (int al = 0; al < NC; ++al) num[al] = fma(s_s[al], ST, tot[al]);
        const double ratio = num[0] / a.S[w];
        a.ratio[(long long)w * a.rs] = ratio;
        if constexpr (NC == 5) {
            const double inv = 1.0 / num[0];
            for (int d = 0; d < 3; ++d) a.grad[(long long)w * a.gs + d] = num[1 + d] * inv;
            a.lap[(long long)w * a.ls] = num[4] * inv;
        }
        if (a.rho) a.rho[w] = s_s[0];
        if (a.num)
            for (int al = 0; al < NCH; ++al) a.num[(long long)w * NCH + al] = al < NC ? num[al] : 0.0;
        if (!isfinite(ratio)) atomicOr(status, ST_NONFINITE);
    }
}

template <typename TO, typename TT, int NC>
__global__ void __launch_bounds__(kBlock, sizeof(TT) == 4 ? MSD_RATIO_F32_BLOCKS : 2)
    k_ratio(const __grid_constant__ RatioArgs a, int* __restrict__ status) {
    ratio_block<TO, TT, NC>(a, blockIdx.x, status);
}

// ------------------------------------------------------------------------------------------
// A6: accept -- Sherman-Morrison update of A_0^{-1} (FP64), rank-1 update of T (Section III)
// ------------------------------------------------------------------------------------------
// Ainv' = Ainv - x v^T / rho with v = phi_occ(r')^T Ainv - e_i^T, T' = T + x y^T / rho.
template <typename TO, typename TT>
__device__ __forceinline__ void accept_block(const AcceptArgs& a, const int w, int* __restrict__ status) {
    if (!a.accept[w]) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = a.n, m = a.m, tid = threadIdx.x, bd = blockDim.x;
    // np partial sums per entry of v so that all threads share the n-term FP64 dot products
    const int np = bd >= 2 * n ? bd / n : 1;
    double* xr = reinterpret_cast<double*>(smem);  // [n] x[c] / rho
    double* pd = xr + n;                           // [n] phi_occ(r')
    double* v = pd + n;                            // [n]
    double* vp = v + n;                            // [np][n] partial sums
    double* Aw = a.Ainv + (long long)w * n * n;
    const TO* phw = static_cast<const TO*>(a.phi) + (long long)w * a.nch * a.N;
    const double rho = a.rho[w];
    const double irho = 1.0 / rho;
    for (int c = tid; c < n; c += bd) {
        xr[c] = Aw[(long long)c * n + a.row] * irho;
        pd[c] = double(phw[c]);
    }
    __syncthreads();
    if (np > 1) {
        const int r = tid % n, part = tid / n;
        if (part < np) {
            double acc = 0.0;
            for (int c = part; c < n; c += np) acc = fma(pd[c], Aw[(long long)c * n + r], acc);
            vp[part * n + r] = acc;
        }
        __syncthreads();
        for (int r2 = tid; r2 < n; r2 += bd) {
            double acc = 0.0;
            for (int q = 0; q < np; ++q) acc += vp[q * n + r2];
            v[r2] = acc - (r2 == a.row ? 1.0 : 0.0);
        }
    } else {
        for (int r = tid; r < n; r += bd) {
            double acc = 0.0;
            for (int c = 0; c < n; ++c) acc = fma(pd[c], Aw[(long long)c * n + r], acc);
            v[r] = acc - (r == a.row ? 1.0 : 0.0);
        }
    }
    __syncthreads();
    const int lane = tid & 31, nw = bd >> 5;
    for (int c = tid >> 5; c < n; c += nw) {
        double* row = Aw + (long long)c * n;
        const double xc = xr[c];
        for (int r = lane; r < n; r += 32) row[r] = fma(-xc, v[r], row[r]);
    }
    TT* Tw = static_cast<TT*>(a.T) + (long long)w * n * m;
    const TT* yw = static_cast<const TT*>(a.y0) + (long long)w * m;
    const bool vec = sizeof(TT) == 4 && (m & 3) == 0 && ((reinterpret_cast<uintptr_t>(Tw) | reinterpret_cast<uintptr_t>(yw)) & 15) == 0;
    if (vec) {
        // FP32 rows as float4: m / 4 vectors per row, one row per warp at a time
        const int m4 = m >> 2;
        const float4* y4 = reinterpret_cast<const float4*>(yw);
        for (int c = tid >> 5; c < n; c += nw) {
            float4* row = reinterpret_cast<float4*>(Tw + (long long)c * m);
            const float xc = float(xr[c]);
            for (int q = lane; q < m4; q += 32) {
                float4 t = row[q];
                const float4 y = y4[q];
                t.x = fmaf(xc, y.x, t.x);
                t.y = fmaf(xc, y.y, t.y);
                t.z = fmaf(xc, y.z, t.z);
                t.w = fmaf(xc, y.w, t.w);
                row[q] = t;
            }
        }
    } else {
        for (int c = tid >> 5; c < n; c += nw) {
            TT* row = Tw + (long long)c * m;
            const TT xc = TT(xr[c]);
            for (int av = lane; av < m; av += 32) row[av] = fma(xc, yw[av], row[av]);
        }
    }
    if (tid == 0) {
        if ((!(rho != 0.0) || !isfinite(rho)) && !(a.skip && a.skip[w] >= 0)) atomicOr(status, ST_SINGULAR);
        a.logdet[w] += log(fabs(rho));
        if (rho < 0.0) a.sgn[w] = -a.sgn[w];
        a.S[w] = a.num[(long long)w * NCH] * irho;
        for (int d = 0; d < 3; ++d) a.R[((long long)w * a.n_tot + a.elec) * 3 + d] = a.rnew[w * 3 + d];
    }
}

template <typename TO, typename TT>
__global__ void __launch_bounds__(kBlock) k_accept(const __grid_constant__ AcceptArgs a, int* __restrict__ status) {
    accept_block<TO, TT>(a, blockIdx.x, status);
}

__global__ void k_propose(int W, int n_tot, int elec, const double* __restrict__ R, const double* __restrict__ eta,
                          double tau, double* __restrict__ rnew) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * 3) return;
    const int w = i / 3, d = i - w * 3;
    rnew[i] = fma(tau, eta[i], R[((long long)w * n_tot + elec) * 3 + d]);
}

__global__ void k_gather_rows(int n, const int* __restrict__ map, int row, const double* __restrict__ src,
                              double* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * row) return;
    const int s = int(i / row), k = int(i - (long long)s * row);
    dst[i] = src[(long long)map[s] * row + k];
}

__global__ void k_gather_bytes(int n, const int* __restrict__ map, const uint8_t* __restrict__ src,
                               uint8_t* __restrict__ dst) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) dst[s] = src[map[s]];
}

__global__ void k_scatter_rows(int n, const int* __restrict__ map, int row, const double* __restrict__ src,
                               double* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * row) return;
    const int s = int(i / row), k = int(i - (long long)s * row);
    dst[(long long)map[s] * row + k] = src[i];
}

__global__ void k_check_finite_batched(int W, const double* __restrict__ ratio, const int* __restrict__ wsys,
                                       const BatchSys* __restrict__ sys) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < W && !isfinite(ratio[w])) atomicOr(sys[wsys[w]].status, ST_NONFINITE);
}

__global__ void k_check_finite(int W, const double* __restrict__ ratio, int* __restrict__ status) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < W && !isfinite(ratio[w])) atomicOr(status, ST_NONFINITE);
}

__global__ void k_metropolis(int W, const double* __restrict__ u, const double* __restrict__ ratio,
                             uint8_t* __restrict__ accept) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const double r = ratio[w];
    accept[w] = (u[w] < r * r) ? 1 : 0;
}

__global__ void k_state(int W, const double* __restrict__ ld0, const double* __restrict__ sg0,
                        const double* __restrict__ ld1, const double* __restrict__ sg1, const double* __restrict__ S,
                        double* __restrict__ logabs, double* __restrict__ sign) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const double s = S[w];
    if (logabs) logabs[w] = ld0[w] + ld1[w] + log(fabs(s));
    if (sign) sign[w] = sg0[w] * sg1[w] * (s < 0.0 ? -1.0 : (s > 0.0 ? 1.0 : 0.0));
}

// ------------------------------------------------------------------------------------------
// Batched systems: one launch per stage for every system (per-system descriptors)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int batch_spin(const BatchSys& B, int t, int& e) {
    e = t % B.n_tot;
    return e < B.n_up ? 0 : 1;
}

template <typename TO, int NC>
__global__ void __launch_bounds__(256) k_orbitals_batched(const BatchSys* __restrict__ sys, const int4* __restrict__ tiles,
                                                          int t, const double* __restrict__ rnew) {
    const int4 tl = tiles[blockIdx.x];
    const BatchSys& B = sys[tl.x];
    int e;
    const OrbArgs& o = B.orb[batch_spin(B, t, e)];
    if (tl.z >= o.N) return;  // tile beyond this spin's orbitals (uniform over the block)
    orbitals_tile<TO, NC>(B.W, 1, rnew + 3LL * B.w_off, 3, 0, o.bas, o.blm, o.nb, static_cast<const TO*>(o.B), o.N,
                          static_cast<TO*>(o.out), tl.y, tl.z);
}

template <typename TO, typename TT, int NC>
__global__ void __launch_bounds__(kBlock, sizeof(TT) == 4 ? MSD_RATIO_F32_BLOCKS : 2)
    k_ratio_batched(const BatchSys* __restrict__ sys, const int2* __restrict__ blk, int t, double* ratio,
                    double* grad, double* lap) {
    __shared__ RatioArgs sa;
    __shared__ int* s_status;
    const int2 bw = blk[blockIdx.x];  // blk already offset to this launch's group
    if (threadIdx.x == 0) {
        const BatchSys& B = sys[bw.x];
        int e;
        const int sp = batch_spin(B, t, e);
        sa = B.ratio[sp];
        sa.row = e - (sp ? B.n_up : 0);
        sa.nch = NC;
        sa.ratio = ratio + B.w_off;
        sa.rs = 1;
        sa.grad = grad ? grad + 3LL * B.w_off : nullptr;
        sa.gs = 3;
        sa.lap = lap ? lap + B.w_off : nullptr;
        sa.ls = 1;
        s_status = B.ratio_status ? B.ratio_status : B.status;
    }
    __syncthreads();
    ratio_block<TO, TT, NC>(sa, bw.y, s_status);
}

template <typename TO, typename TT>
__global__ void __launch_bounds__(kBlock) k_accept_batched(const BatchSys* __restrict__ sys, const int2* __restrict__ blk,
                                                           int t, int nch, const uint8_t* __restrict__ accept,
                                                           const double* __restrict__ rnew) {
    __shared__ AcceptArgs sa;
    __shared__ int* s_status;
    const int2 bw = blk[blockIdx.x];
    if (threadIdx.x == 0) {
        const BatchSys& B = sys[bw.x];
        int e;
        const int sp = batch_spin(B, t, e);
        sa = B.accept[sp];
        sa.row = e - (sp ? B.n_up : 0);
        sa.elec = e;
        sa.nch = nch;
        sa.accept = accept + B.w_off;
        sa.rnew = rnew + 3LL * B.w_off;
        s_status = B.status;
    }
    __syncthreads();
    accept_block<TO, TT>(sa, bw.y, s_status);
}

// ------------------------------------------------------------------------------------------
// One Metropolis step of every walker of every system in one persistent launch per group of
// systems: a block takes (system, walker) items from a device counter until none is left and, for
// each, proposes r' = r + tau eta, evaluates the moving spin's orbitals at r' (SIMT, all five
// channels), runs the ratio sweep (ratio_block), takes the Metropolis decision u < ratio^2 and
// applies the update (accept_block).  The last block to run out resets the counter for the next
// launch (no block waits on another).
// ------------------------------------------------------------------------------------------
template <typename TO>
__device__ __forceinline__ void orbitals_walker(const double* rp, const double4* __restrict__ bas,
                                                const int8_t* __restrict__ blm, int nb, const TO* __restrict__ Bm,
                                                int N, TO* __restrict__ out, TO* chi) {
    for (int mu = threadIdx.x; mu < nb; mu += blockDim.x) {
        TO v[5];
        basis_channels<TO>(rp, bas[mu], blm[mu], v);
#pragma unroll
        for (int a = 0; a < 5; ++a) chi[a * nb + mu] = v[a];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        TO acc[5] = {TO(0), TO(0), TO(0), TO(0), TO(0)};
        for (int mu = 0; mu < nb; ++mu) {
            const TO b = __ldg(Bm + (long long)mu * N + j);
#pragma unroll
            for (int a = 0; a < 5; ++a) acc[a] = fma(chi[a * nb + mu], b, acc[a]);
        }
#pragma unroll
        for (int a = 0; a < 5; ++a) out[a * N + j] = acc[a];
    }
}

template <typename TO, typename TT>
__global__ void __launch_bounds__(kBlock, sizeof(TT) == 4 ? MSD_RATIO_F32_BLOCKS : 2)
    k_step_batched(const BatchSys* __restrict__ sys, const int2* __restrict__ items, int n_items, int t,
                   const double* __restrict__ eta, double tau, const double* __restrict__ u, double* ratio,
                   double* grad, double* lap, uint8_t* accept, double* rnew, int* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ RatioArgs sa;
    __shared__ AcceptArgs sb;
    __shared__ int* s_rstatus;
    __shared__ int* s_status;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 sw = items[it];
        const BatchSys& B = sys[sw.x];
        const int w = sw.y, gw = B.w_off + w;
        int e;
        const int sp = batch_spin(B, t, e);
        if (tid < 3) rnew[3LL * gw + tid] = fma(tau, eta[3LL * gw + tid], B.R[((long long)w * B.n_tot + e) * 3 + tid]);
        if (tid == 0) {
            sa = B.ratio[sp];
            sa.row = e - (sp ? B.n_up : 0);
            sa.nch = NCH;
            sa.ratio = ratio + B.w_off;
            sa.rs = 1;
            sa.grad = grad + 3LL * B.w_off;
            sa.gs = 3;
            sa.lap = lap + B.w_off;
            sa.ls = 1;
            sb = B.accept[sp];
            sb.row = sa.row;
            sb.elec = e;
            sb.nch = NCH;
            sb.accept = accept + B.w_off;
            sb.rnew = rnew + 3LL * B.w_off;
            s_rstatus = B.ratio_status ? B.ratio_status : B.status;
            s_status = B.status;
        }
        __syncthreads();
        const OrbArgs& o = B.orb[sp];
        orbitals_walker<TO>(rnew + 3LL * gw, o.bas, o.blm, o.nb, static_cast<const TO*>(o.B), o.N,
                            static_cast<TO*>(o.out) + (long long)w * NCH * o.N, reinterpret_cast<TO*>(smem));
        __syncthreads();
        ratio_block<TO, TT, NCH>(sa, w, s_rstatus);
        __syncthreads();
        if (tid == 0) {
            const double r = ratio[gw];
            accept[gw] = (u[gw] < r * r) ? 1 : 0;
        }
        __syncthreads();
        accept_block<TO, TT>(sb, w, s_status);
        __syncthreads();
    }
    if (tid == 0 && atomicAdd(counter + 1, 1) == (int)gridDim.x - 1) {
        counter[0] = 0;  // every block has left the loop: no item is taken any more in this launch
        counter[1] = 0;
    }
}

__global__ void k_propose_batched(const BatchSys* __restrict__ sys, const int* __restrict__ wsys, int Wt, int t,
                                  const double* __restrict__ eta, double tau, double* __restrict__ rnew) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wt * 3) return;
    const int gw = i / 3, d = i - gw * 3;
    const BatchSys& B = sys[wsys[gw]];
    const int w = gw - B.w_off, e = t % B.n_tot;
    rnew[i] = fma(tau, eta[i], B.R[((long long)w * B.n_tot + e) * 3 + d]);
}

template <typename Kern>
void set_smem(Kern kern, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------------
template <typename TO>
static void orbitals_impl(const Launch& L, int nch, int P, int ppw, const double* pos, long long wstride, int p_off,
                          const double4* bas, const int8_t* blm, int nb, const TO* B, int N, TO* out) {
    if (P <= 0 || N <= 0) return;
    const dim3 grid((P + kOrbTP - 1) / kOrbTP, (N + kOrbTJ - 1) / kOrbTJ);
    L.count();
    if (nch == 5)
        k_orbitals<TO, 5><<<grid, 256, 0, L.stream>>>(P, ppw, pos, wstride, p_off, bas, blm, nb, B, N, out);
    else
        k_orbitals<TO, 1><<<grid, 256, 0, L.stream>>>(P, ppw, pos, wstride, p_off, bas, blm, nb, B, N, out);
}

void launch_orbitals(const Launch& L, bool mixed, int nch, int P, int ppw, const double* pos, long long wstride,
                     int p_off, const double4* bas, const int8_t* blm, int nb, const void* B, int N, void* out) {
    if (mixed)
        orbitals_impl<float>(L, nch, P, ppw, pos, wstride, p_off, bas, blm, nb, static_cast<const float*>(B), N,
                             static_cast<float*>(out));
    else
        orbitals_impl<double>(L, nch, P, ppw, pos, wstride, p_off, bas, blm, nb, static_cast<const double*>(B), N,
                              static_cast<double*>(out));
}

void launch_inverse(const Launch& L, bool mixed, int W, int n, int N, const void* Phi, double* Ainv, double* logdet,
                    double* sgn, double* cond) {
    const size_t sm = (size_t)n * (n + 1) * 8 + (size_t)n * 8 + (size_t)n * 4 + 16;
    if (mixed) {
        set_smem(k_inverse<float>, sm);
        L.count();
        k_inverse<float><<<W, kBlock, sm, L.stream>>>(n, N, static_cast<const float*>(Phi), Ainv, logdet, sgn,
                                                      L.status, cond);
    } else {
        set_smem(k_inverse<double>, sm);
        L.count();
        k_inverse<double><<<W, kBlock, sm, L.stream>>>(n, N, static_cast<const double*>(Phi), Ainv, logdet, sgn,
                                                       L.status, cond);
    }
}

void launch_table(const Launch& L, bool mixed, int W, int n, int N, const double* Ainv, const void* Phi, void* T) {
    const int m = N - n;
    if (m <= 0) return;
    dim3 grid((m + 63) / 64, W);
    if (mixed) {
        const size_t sm = (((size_t)n * (n + 1) * 4 + 15) & ~size_t(15)) + (size_t)n * 64 * 4;
        set_smem(k_table<float, float>, sm);
        L.count();
        k_table<float, float><<<grid, kBlock, sm, L.stream>>>(n, N, Ainv, static_cast<const float*>(Phi),
                                                              static_cast<float*>(T));
    } else {
        const size_t sm = (((size_t)n * (n + 1) * 8 + 15) & ~size_t(15)) + (size_t)n * 64 * 8;
        set_smem(k_table<double, double>, sm);
        L.count();
        k_table<double, double><<<grid, kBlock, sm, L.stream>>>(n, N, Ainv, static_cast<const double*>(Phi),
                                                                static_cast<double*>(T));
    }
}

void launch_exc_det(const Launch& L, bool mixed, int W, int n, int m, const ExcDev& g, const void* T, void* t) {
    if (mixed) {
        const size_t sm = (size_t)n * m * 4 + 16;
        set_smem(k_exc_det<float>, sm);
        L.count();
        k_exc_det<float><<<W, kBlock, sm, L.stream>>>(n, m, g, static_cast<const float*>(T), static_cast<float*>(t));
    } else {
        const size_t sm = (size_t)n * m * 8 + 16;
        set_smem(k_exc_det<double>, sm);
        L.count();
        k_exc_det<double><<<W, kBlock, sm, L.stream>>>(n, m, g, static_cast<const double*>(T),
                                                       static_cast<double*>(t));
    }
}

static constexpr int kHeavyLen = 128;

void launch_ci_contract(const Launch& L, bool mixed, int W, int n_exc, int n_exc_other, const int* off,
                        const int* other, const double* c, const void* t_other, void* C) {
    dim3 grid((n_exc + kBlock - 1) / kBlock, W);
    L.count();
    if (mixed)
        k_ci_contract_light<float><<<grid, kBlock, 0, L.stream>>>(n_exc, n_exc_other, off, other, c,
                                                                  static_cast<const float*>(t_other),
                                                                  static_cast<float*>(C), kHeavyLen);
    else
        k_ci_contract_light<double><<<grid, kBlock, 0, L.stream>>>(n_exc, n_exc_other, off, other, c,
                                                                   static_cast<const double*>(t_other),
                                                                   static_cast<double*>(C), kHeavyLen);
}

void launch_ci_contract_heavy(const Launch& L, bool mixed, int W, int n_exc, int n_exc_other, int n_heavy,
                              const int* heavy, const int* off, const int* other, const double* c,
                              const void* t_other, void* C) {
    if (n_heavy <= 0) return;
    dim3 grid(n_heavy, W);
    L.count();
    if (mixed)
        k_ci_contract_heavy<float><<<grid, kBlock, 0, L.stream>>>(n_exc, n_exc_other, heavy, off, other, c,
                                                                  static_cast<const float*>(t_other),
                                                                  static_cast<float*>(C));
    else
        k_ci_contract_heavy<double><<<grid, kBlock, 0, L.stream>>>(n_exc, n_exc_other, heavy, off, other, c,
                                                                   static_cast<const double*>(t_other),
                                                                   static_cast<double*>(C));
}

int heavy_threshold() { return kHeavyLen; }

void launch_ci_dot(const Launch& L, bool mixed, int W, int n_exc, const void* C, const void* t, double* S) {
    L.count();
    if (mixed)
        k_ci_dot<float><<<W, kBlock, 0, L.stream>>>(n_exc, static_cast<const float*>(C), static_cast<const float*>(t),
                                                    S);
    else
        k_ci_dot<double><<<W, kBlock, 0, L.stream>>>(n_exc, static_cast<const double*>(C),
                                                     static_cast<const double*>(t), S);
}

size_t ratio_smem_bytes(bool mixed, int n, int m, int nch) {
    return mixed ? ratio_layout(n, m, nch, 4, 4, ratio_ngw<float>()).total
                 : ratio_layout(n, m, nch, 8, 8, ratio_ngw<double>()).total;
}

template <typename TO, typename TT>
static void ratio_impl(const Launch& L, const RatioArgs& a) {
    const size_t sm = ratio_layout(a.n, a.m, a.nch, sizeof(TT), sizeof(TO), ratio_ngw<TT>()).total;
    if (L.t0) cudaEventRecord(L.t0, L.stream);
    if (a.nch == 5) {
        set_smem(k_ratio<TO, TT, 5>, sm);
        L.count();
        k_ratio<TO, TT, 5><<<a.W, kBlock, sm, L.stream>>>(a, L.status);
    } else {
        set_smem(k_ratio<TO, TT, 1>, sm);
        L.count();
        k_ratio<TO, TT, 1><<<a.W, kBlock, sm, L.stream>>>(a, L.status);
    }
    if (L.t1) cudaEventRecord(L.t1, L.stream);
}

void launch_ratio(const Launch& L, bool mixed, const RatioArgs& a) {
    if (mixed) ratio_impl<float, float>(L, a);
    else ratio_impl<double, double>(L, a);
}

void launch_accept(const Launch& L, bool mixed, const AcceptArgs& a) {
    const size_t sm = accept_smem_bytes(a.n);
    L.count();
    if (mixed) k_accept<float, float><<<a.W, kBlock, sm, L.stream>>>(a, L.status);
    else k_accept<double, double><<<a.W, kBlock, sm, L.stream>>>(a, L.status);
}

void launch_propose(const Launch& L, int W, int n_tot, int elec, const double* R, const double* eta, double tau,
                    double* rnew) {
    L.count();
    k_propose<<<(W * 3 + 255) / 256, 256, 0, L.stream>>>(W, n_tot, elec, R, eta, tau, rnew);
}

void launch_gather_rows(const Launch& L, int n_slots, const int* map, int row, const double* src, double* dst) {
    const long long tot = (long long)n_slots * row;
    if (tot <= 0) return;
    L.count();
    k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(n_slots, map, row, src, dst);
}

void launch_gather_bytes(const Launch& L, int n_slots, const int* map, const uint8_t* src, uint8_t* dst) {
    if (n_slots <= 0) return;
    L.count();
    k_gather_bytes<<<(n_slots + 255) / 256, 256, 0, L.stream>>>(n_slots, map, src, dst);
}

void launch_scatter_rows(const Launch& L, int n_real, const int* map, int row, const double* src, double* dst) {
    const long long tot = (long long)n_real * row;
    if (tot <= 0) return;
    L.count();
    k_scatter_rows<<<(unsigned)((tot + 255) / 256), 256, 0, L.stream>>>(n_real, map, row, src, dst);
}

void launch_check_finite_batched(const Launch& L, const BatchPlan& P, int W, const double* ratio) {
    L.count();
    k_check_finite_batched<<<(W + 255) / 256, 256, 0, L.stream>>>(W, ratio, P.wsys, P.sys);
}

void launch_check_finite(const Launch& L, int W, const double* ratio) {
    L.count();
    k_check_finite<<<(W + 255) / 256, 256, 0, L.stream>>>(W, ratio, L.status);
}

void launch_metropolis(const Launch& L, int W, const double* u, const double* ratio, uint8_t* accept) {
    L.count();
    k_metropolis<<<(W + 255) / 256, 256, 0, L.stream>>>(W, u, ratio, accept);
}

void launch_state(const Launch& L, int W, const double* ld0, const double* sg0, const double* ld1, const double* sg1,
                  const double* S, double* logabs, double* sign) {
    L.count();
    k_state<<<(W + 255) / 256, 256, 0, L.stream>>>(W, ld0, sg0, ld1, sg1, S, logabs, sign);
}

// ------------------------------------------------------------------------------------------
// Fixed device scratch for msd_ratio_noalloc
// ------------------------------------------------------------------------------------------
// Some callers may not allocate device memory at the moment they need a ratio: cudaMalloc and
// cudaFree can synchronise the whole device (stalling every other stream of the process), and a
// process whose device memory is already reserved by another framework's caching allocator
// may have nothing left to give.  For them msd_ratio_noalloc keeps the orbitals at the trial
// positions in this file-scope array instead of a buffer of the context.  One array exists per
// device and every call on that device uses all of it, so two calls that overlap in time on one
// device (two streams, two host threads, two contexts) race on it; callers serialise them.
// Nothing in it needs to start at zero: the orbital kernel writes every entry the sweep reads.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static constexpr int kNoAllocMaxDevices = 64;

cudaError_t noalloc_scratch(void** ptr) {
    // Address looked up once per device, with that device current, on its first use (a runtime
    // query, not an allocation); a caller's first call on a device must therefore come before
    // any stream capture it starts.
    static std::mutex mu;
    static void* addr[kNoAllocMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

template <typename TO>
static void orbitals_batched_impl(const Launch& L, const BatchPlan& P, int t, int nch, const double* rnew) {
    if (P.n_tiles <= 0) return;
    L.count();
    if (nch == 5)
        k_orbitals_batched<TO, 5><<<P.n_tiles, 256, 0, L.stream>>>(P.sys, P.tiles, t, rnew);
    else
        k_orbitals_batched<TO, 1><<<P.n_tiles, 256, 0, L.stream>>>(P.sys, P.tiles, t, rnew);
}

void launch_orbitals_batched(const Launch& L, bool mixed, const BatchPlan& P, int t, int nch, const double* rnew) {
    if (mixed) orbitals_batched_impl<float>(L, P, t, nch, rnew);
    else orbitals_batched_impl<double>(L, P, t, nch, rnew);
}

template <typename TO, typename TT>
static void ratio_batched_impl(const Launch& L, const BatchPlan& P, int t, int nch, double* ratio, double* grad,
                               double* lap) {
    if (L.t0) cudaEventRecord(L.t0, L.stream);
    set_smem(k_ratio_batched<TO, TT, 5>, P.ratio_smem);
    set_smem(k_ratio_batched<TO, TT, 1>, P.ratio_smem);
    for (int g = 0; g < P.n_groups; ++g) {
        const int nb = P.gfirst[g + 1] - P.gfirst[g];
        if (nb <= 0) continue;
        L.count();
        if (nch == 5)
            k_ratio_batched<TO, TT, 5><<<nb, kBlock, P.gsmem[g], L.stream>>>(P.sys, P.blk + P.gfirst[g], t, ratio,
                                                                             grad, lap);
        else
            k_ratio_batched<TO, TT, 1><<<nb, kBlock, P.gsmem[g], L.stream>>>(P.sys, P.blk + P.gfirst[g], t, ratio,
                                                                             grad, lap);
    }
    if (L.t1) cudaEventRecord(L.t1, L.stream);
}

void launch_ratio_batched(const Launch& L, bool mixed, const BatchPlan& P, int t, int nch, double* ratio, double* grad,
                          double* lap) {
    if (mixed) ratio_batched_impl<float, float>(L, P, t, nch, ratio, grad, lap);
    else ratio_batched_impl<double, double>(L, P, t, nch, ratio, grad, lap);
}

void launch_accept_batched(const Launch& L, bool mixed, const BatchPlan& P, int t, int nch, const uint8_t* accept,
                           const double* rnew) {
    L.count();
    if (mixed)
        k_accept_batched<float, float><<<P.n_blk, kBlock, P.accept_smem, L.stream>>>(P.sys, P.blk, t, nch, accept, rnew);
    else
        k_accept_batched<double, double><<<P.n_blk, kBlock, P.accept_smem, L.stream>>>(P.sys, P.blk, t, nch, accept,
                                                                                       rnew);
}

void launch_propose_batched(const Launch& L, const BatchPlan& P, int W_total, int t, const double* eta, double tau,
                            double* rnew) {
    L.count();
    k_propose_batched<<<(W_total * 3 + 255) / 256, 256, 0, L.stream>>>(P.sys, P.wsys, W_total, t, eta, tau, rnew);
}

template <typename TO, typename TT>
static void step_batched_impl(const Launch& L, const BatchPlan& P, int group, int grid, int t, const double* eta,
                              double tau, const double* u, double* ratio, double* grad, double* lap, uint8_t* accept,
                              double* rnew) {
    const int first = P.gfirst[group], n = P.gfirst[group + 1] - first;
    if (n <= 0) return;
    const size_t sm = P.step_smem[group];
    set_smem(k_step_batched<TO, TT>, sm);
    L.count();
    k_step_batched<TO, TT><<<grid, kBlock, sm, L.stream>>>(P.sys, P.items + first, n, t, eta, tau, u, ratio, grad, lap,
                                                          accept, rnew, P.counters + 2 * group);
}

void launch_step_batched(const Launch& L, bool mixed, const BatchPlan& P, int group, int grid, int t,
                         const double* eta, double tau, const double* u, double* ratio, double* grad, double* lap,
                         uint8_t* accept, double* rnew) {
    if (mixed) step_batched_impl<float, float>(L, P, group, grid, t, eta, tau, u, ratio, grad, lap, accept, rnew);
    else step_batched_impl<double, double>(L, P, group, grid, t, eta, tau, u, ratio, grad, lap, accept, rnew);
}

int step_blocks_per_sm(bool mixed, size_t smem) {
    int b = 0;
    if (mixed) {
        set_smem(k_step_batched<float, float>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_batched<float, float>, kBlock, smem);
    } else {
        set_smem(k_step_batched<double, double>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step_batched<double, double>, kBlock, smem);
    }
    return b;
}

size_t accept_smem_bytes(int n) {
    const int np = kBlock >= 2 * n ? kBlock / n : 1;
    return (size_t)n * (3 + np) * 8;
}

int orbital_tile_points() { return kOrbTP; }
int orbital_tile_orbitals() { return kOrbTJ; }

void launch_canon_build(const Launch& L, int W, int n, int N, int m, const ExcDev& g, const double* Phi,
                        const uint8_t* used, const double* ld0, const double* sg0, double* D, double* t) {
    const size_t sm = (size_t)n * (n + 1) * 8 + (size_t)n * 12 + 16;
    set_smem(k_canon_build, sm);
    L.count();
    k_canon_build<<<dim3(g.n_exc, W), kBlock, sm, L.stream>>>(n, N, m, g, Phi, used, ld0, sg0, D, t, L.status);
}

void launch_canon_ratio(const Launch& L, int W, int n, int N, int m, int row, int nch, const ExcDev& g,
                        const uint8_t* used, const double* phi, const double* D, const double* t, const double* C,
                        const double* S, double* ru, double* ratio, double* grad, double* lap, double* num,
                        double* rho) {
    if (L.t0) cudaEventRecord(L.t0, L.stream);
    L.count();
    if (nch == 5)
        k_canon_ratio<5><<<W, kBlock, 0, L.stream>>>(n, N, m, row, g, used, phi, D, t, C, S, ru, ratio, grad, lap, num,
                                                     rho, L.status);
    else
        k_canon_ratio<1><<<W, kBlock, 0, L.stream>>>(n, N, m, row, g, used, phi, D, t, C, S, ru, ratio, grad, lap, num,
                                                     rho, L.status);
    if (L.t1) cudaEventRecord(L.t1, L.stream);
}

void launch_canon_accept(const Launch& L, int W, int n, int N, int m, int row, int elec, int n_tot, const ExcDev& g,
                         const uint8_t* used, const uint8_t* accept, const double* phi_new, int nch, double* Phi,
                         double* D, double* t, const double* ru, const double* rnew, double* R, const double* rho,
                         const double* num, double* logdet, double* sgn, double* S) {
    L.count();
    k_canon_accept<<<dim3(g.n_exc, W), kBlock, (size_t)3 * n * 8, L.stream>>>(n, N, m, row, g, used, accept, phi_new,
                                                                              nch, Phi, D, t, ru);
    L.count();
    k_canon_commit<<<W, 128, 0, L.stream>>>(W, n, N, row, elec, n_tot, nch, accept, phi_new, Phi, rnew, R, rho, num,
                                            logdet, sgn, S);
}

}  // namespace msd
