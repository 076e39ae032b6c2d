// msd_backward.cu -- adjoint of log|Psi| with respect to the CI coefficients c_I and the
// orbital coefficients B of each spin, accumulated over walkers with weights gbar[w]
// (the gradient a parameter optimisation needs; the paper is silent on it).
//
// Per walker, with S = Psi / (det A_up,0 det A_dn,0) = sum_I c_I t_up[u_I] t_dn[d_I]:
//   d log|Psi| / d c_I   = t_up[u_I] t_dn[d_I] / S
//   d log|Psi| / d T[h][p] = Tbar[h][p] = (1/S) sum_u C_u cof(T_u)[q][l]   (h = h_q, p = p_l)
//   d log|Psi| / d Phi  = Ainv^T [ I - Tbar T^T | Tbar ]    (log|det A_0| and T = A_0^{-1} Phi_virt)
//   d log|Psi| / d B[mu][j] = sum_r chi_mu(r_r) Phibar[r][j]
// where cof(T_u) is the cofactor matrix of the k x k excitation block (Section III: t_u =
// det T_u) and C_u the spin's CI weight of string u.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "msd_internal.h"
#include "msd_records.cuh"
#include "msd_smalldet.cuh"

namespace msd {
namespace {

constexpr int kBB = 256;

// ------------------------------------------------------------------------------------------
// d log|Psi| / d c_I, summed over walkers: one thread per term, a slice of walkers per block row
// ------------------------------------------------------------------------------------------
template <typename TT>
__global__ void __launch_bounds__(kBB) k_dci(int W, int wchunk, long long n_det, const int* __restrict__ iu,
                                            const int* __restrict__ id, const double* __restrict__ gbar,
                                            const double* __restrict__ S, const TT* __restrict__ t0, int ld0,
                                            const TT* __restrict__ t1, int ld1, double* __restrict__ dci) {
    const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n_det) return;
    const int a = iu[I], b = id[I];
    const int w0 = blockIdx.y * wchunk, w1 = min(W, w0 + wchunk);
    double acc = 0.0;
    for (int w = w0; w < w1; ++w)
        acc = fma(gbar[w] / S[w], double(t0[(long long)w * ld0 + a]) * double(t1[(long long)w * ld1 + b]), acc);
    atomicAdd(dci + I, acc);
}

// ------------------------------------------------------------------------------------------
// Tbar: scatter of cofactors of every excitation block, one block per walker
// ------------------------------------------------------------------------------------------
// cof(T_u)[q][l] = (-1)^(q+l) det(T_u without row q and column l), each minor by the same
// pivoted small-determinant code the sweep uses.
template <int K, typename TT>
__device__ __forceinline__ void scatter_cofactors(const TT* Ts, int m, const int (&h)[K], const int (&p)[K], TT cu,
                                                  TT* Tb) {
    if constexpr (K == 1) {
        atomicAdd(Tb + h[0] * m + p[0], cu);
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            int hh[K - 1];
#pragma unroll
            for (int i = 0; i < K - 1; ++i) hh[i] = h[i < q ? i : i + 1];
#pragma unroll
            for (int l = 0; l < K; ++l) {
                int pp[K - 1];
#pragma unroll
                for (int i = 0; i < K - 1; ++i) pp[i] = p[i < l ? i : i + 1];
                const TT minor = small_det<K - 1, TT>(Ts, m, hh, pp);
                atomicAdd(Tb + h[q] * m + p[l], ((q + l) & 1) ? -cu * minor : cu * minor);
            }
        }
    }
}

// The same scatter from the adjugate as a whole: row q of cof(T_u) is column q of adj(T_u),
// i.e. adj(T_u) e_q, which the pivoted elimination of the ratio sweep (adj_solve) gives for one
// LU per column.  For K >= 5 that is far less work than K^2 separate (K-1) x (K-1) minors.
template <int K, typename TT>
__device__ __forceinline__ void scatter_adjugate(const TT* Ts, int m, const int (&h)[K], const int (&p)[K], TT cu,
                                                 TT* Tb) {
    TT Tu[K * K];
    int id[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        id[q] = q;
#pragma unroll
        for (int l = 0; l < K; ++l) Tu[q * K + l] = Ts[h[q] * m + p[l]];
    }
#pragma unroll 1
    for (int q = 0; q < K; ++q) {
        TT e[K], z[K], det;
#pragma unroll
        for (int j = 0; j < K; ++j) e[j] = j == q ? TT(1) : TT(0);
        adj_solve<K, TT>(Tu, K, e, id, id, det, z);
        TT* row = Tb + h[q] * m;
#pragma unroll
        for (int l = 0; l < K; ++l) atomicAdd(row + p[l], cu * z[l]);
    }
}

template <int K, typename TT>
__device__ __forceinline__ void tbar_group(const ExcDev& g, const TT* Ts, int m, const TT* __restrict__ Cw,
                                           TT* Tb) {
    const int j0 = g.goff[K], j1 = g.goff[K + 1];
    const uint8_t* rec = g.rec + g.roff[K];
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        int h[K], p[K];
        load_rec<K>(rec, j - j0, h, p);
        const TT cu = Cw[j];
        if (h[0] == kEmptyRecord || cu == TT(0)) continue;
        if constexpr (K >= 5)
            scatter_adjugate<K, TT>(Ts, m, h, p, cu, Tb);
        else
            scatter_cofactors<K, TT>(Ts, m, h, p, cu, Tb);
    }
}

// Orders 5-8 are rare: out of line, so that their registers do not limit orders 1-4.
template <int K, typename TT>
__device__ __noinline__ void tbar_group_outlined(const ExcDev& g, const TT* Ts, int m, const TT* __restrict__ Cw,
                                                 TT* Tb) {
    tbar_group<K, TT>(g, Ts, m, Cw, Tb);
}

// Threads per block: FP64 tables and their adjoint fill an SM's shared memory (one block of 512);
// FP32 ones take half, so two blocks of 256 share an SM.
template <typename TT>
__host__ __device__ constexpr int tbar_threads() {
    return sizeof(TT) == 4 ? 256 : 512;
}

// Writes Tbar / S into columns n..N-1 of M[w] (n x N, row stride N).  The cofactors are summed in
// the table's precision (FP32 tables: FP32 shared-memory atomics, off the slow FP64 pipe).
template <typename TT>
__global__ void __launch_bounds__(tbar_threads<TT>(), sizeof(TT) == 4 ? 2 : 1)
    k_tbar(int n, int m, int N, ExcDev g, const TT* __restrict__ T, const TT* __restrict__ C,
           const double* __restrict__ S, double* __restrict__ M) {
    extern __shared__ __align__(16) unsigned char smem[];
    TT* Tb = reinterpret_cast<TT*>(smem);                                                   // [n][m]
    TT* Ts = reinterpret_cast<TT*>(smem + (((size_t)n * m * sizeof(TT) + 15) & ~size_t(15)));  // [n][m]
    const int w = blockIdx.x;
    const TT* Tw = T + (long long)w * n * m;
    const TT* Cw = C + (long long)w * g.n_exc;
    for (int q = threadIdx.x; q < n * m; q += blockDim.x) {
        Ts[q] = Tw[q];
        Tb[q] = g.dense1 ? Cw[g.goff[1] + q] : TT(0);  // dense singles: d det T_u / d T[h][p] = 1
    }
    __syncthreads();
    for (int k = g.dense1 ? 2 : 1; k <= g.kmax; ++k) {
        switch (k) {
            case 1: tbar_group<1, TT>(g, Ts, m, Cw, Tb); break;
            case 2: tbar_group<2, TT>(g, Ts, m, Cw, Tb); break;
            case 3: tbar_group<3, TT>(g, Ts, m, Cw, Tb); break;
            case 4: tbar_group<4, TT>(g, Ts, m, Cw, Tb); break;
            case 5: tbar_group_outlined<5, TT>(g, Ts, m, Cw, Tb); break;
            case 6: tbar_group_outlined<6, TT>(g, Ts, m, Cw, Tb); break;
            case 7: tbar_group_outlined<7, TT>(g, Ts, m, Cw, Tb); break;
            case 8: tbar_group_outlined<8, TT>(g, Ts, m, Cw, Tb); break;
        }
    }
    __syncthreads();
    const double inv = 1.0 / S[w];
    double* Mw = M + (long long)w * n * N;
    for (int q = threadIdx.x; q < n * m; q += blockDim.x) {
        const int c = q / m, a = q - c * m;
        Mw[(long long)c * N + n + a] = double(Tb[q]) * inv;
    }
}

// M[w][:, 0:n] = I - Tbar T^T  (Tbar read from M[w][:, n:N]); one block per walker.
template <typename TT>
__global__ void __launch_bounds__(kBB) k_tbar_tt(int n, int m, int N, const TT* __restrict__ T, double* __restrict__ M) {
    const int w = blockIdx.x;
    const TT* Tw = T + (long long)w * n * m;
    double* Mw = M + (long long)w * n * N;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int c1 = idx / n, c = idx - c1 * n;
        const double* tb = Mw + (long long)c1 * N + n;
        const TT* tr = Tw + (long long)c * m;
        double acc = 0.0;
        for (int a = 0; a < m; ++a) acc = fma(tb[a], double(tr[a]), acc);
        Mw[(long long)c1 * N + c] = (c1 == c ? 1.0 : 0.0) - acc;
    }
}

// M[w] <- gbar[w] Ainv[w]^T M[w] in place, one block per (walker, 32-column tile).
__global__ void __launch_bounds__(kBB) k_phibar(int n, int N, const double* __restrict__ Ainv,
                                               const double* __restrict__ gbar, double* __restrict__ M) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* A = reinterpret_cast<double*>(smem);  // [n][n], A[c][r]
    double* Mt = A + (size_t)n * n;               // [n][32]
    const int w = blockIdx.x, j0 = blockIdx.y * 32;
    const int nj = min(32, N - j0);
    const double* Aw = Ainv + (long long)w * n * n;
    double* Mw = M + (long long)w * n * N;
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) A[q] = Aw[q];
    for (int q = threadIdx.x; q < n * 32; q += blockDim.x) {
        const int c = q >> 5, j = q & 31;
        Mt[q] = j < nj ? Mw[(long long)c * N + j0 + j] : 0.0;
    }
    __syncthreads();
    const double gw = gbar[w];
    for (int q = threadIdx.x; q < n * 32; q += blockDim.x) {
        const int r = q >> 5, j = q & 31;
        if (j >= nj) continue;
        double acc = 0.0;
        for (int c = 0; c < n; ++c) acc = fma(A[c * n + r], Mt[c * 32 + j], acc);
        Mw[(long long)r * N + j0 + j] = gw * acc;
    }
}

// chi[p][mu] = chi_mu(r_p) (values only, FP64) at the electrons of one spin.
__global__ void __launch_bounds__(kBB) k_chi(int P, int ppw, const double* __restrict__ pos, long long wstride,
                                            int p_off, const double4* __restrict__ bas,
                                            const int8_t* __restrict__ blm, int nb, double* __restrict__ chi) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * nb) return;
    const int p = int(idx / nb), mu = int(idx - (long long)p * nb);
    const int w = p / ppw, r = p - w * ppw;
    const double* rp = pos + (long long)w * wstride + (long long)(p_off + r) * 3;
    const double4 b = bas[mu];
    const double d[3] = {rp[0] - b.x, rp[1] - b.y, rp[2] - b.z};
    const double g = exp(-b.w * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
    const int lm = blm[mu];
    chi[idx] = lm == 0 ? g : d[lm - 1] * g;
}

// dB[mu][j] += sum_p chi[p][mu] Phibar[p][j] over a slice of points; 32 x 32 output tile per
// block, 32-point steps through shared memory, one FP64 atomic per output at the end.
__global__ void __launch_bounds__(kBB) k_dB(int P, int nb, int N, int pchunk, const double* __restrict__ chi,
                                           const double* __restrict__ Phib, double* __restrict__ dB) {
    __shared__ double Xs[32][33];
    __shared__ double Ys[32][33];
    const int mu0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int pa = blockIdx.z * pchunk, pb = min(P, pa + pchunk);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int p0 = pa; p0 < pb; p0 += 32) {
        for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
            const int pp = q >> 5, cc = q & 31;
            const int p = p0 + pp;
            Xs[pp][cc] = (p < pb && mu0 + cc < nb) ? chi[(long long)p * nb + mu0 + cc] : 0.0;
            Ys[pp][cc] = (p < pb && j0 + cc < N) ? Phib[(long long)p * N + j0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < 32; ++pp) {
            const double y = Ys[pp][tx];
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i] = fma(Xs[pp][ty + 8 * i], y, acc[i]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int mu = mu0 + ty + 8 * i, j = j0 + tx;
        if (mu < nb && j < N) atomicAdd(dB + (long long)mu * N + j, acc[i]);
    }
}

// All-electron gradient and laplacian at the current positions (one spin), from Tbar:
//   d^a Psi / Psi for electron i = s^a(i) + sum_p y^a_i[p] G'[i][p],
//   s^a(i) = d^a phi_occ(r_i) . A_0^{-1}[:, i],  y^a_i = d^a phi_virt(r_i) - T^T d^a phi_occ(r_i),
//   G'[i][p] = sum_h A_0^{-1}[h][i] Tbar[h][p]  (the G of a move of electron i, divided by S).
// With U = T G'^T (n x n) this is
//   num^a[i] = sum_c d^a phi_occ(r_i)[c] (A_0^{-1} - U)[c][i] + sum_p d^a phi_virt(r_i)[p] G'[i][p].
// One block per walker, two tiled products in shared memory: G' = A_0^{-T} Tbar in 64 x 64 output
// tiles (written to global scratch), then U in 64 x 64 tiles, each turned into V = A_0^{-1} - U
// and contracted with the occupied orbital derivatives at once.  Every thread owns a 4 x 4
// register tile; products run in TC (FP32 on the mixed path, whose table is FP32, FP64 otherwise).
constexpr int kGT = 64;       // output tile edge
constexpr int kGK = 32;       // depth of one staged slab
constexpr int kGLd = kGT + 4; // row stride of the staged tiles (16-byte aligned rows)

template <typename TC>
__host__ __device__ constexpr size_t gradlap_smem_bytes() {
    return sizeof(TC) * (2 * (size_t)kGK * kGLd + (size_t)kGT * kGLd) + sizeof(double) * 4 * 256;
}

template <typename TO, typename TT, typename TC>
__global__ void __launch_bounds__(kBB) k_all_gradlap(int n, int m, int N, int n_tot, int e_off,
                                                    const double* __restrict__ Ainv, const TT* __restrict__ T,
                                                    const double* __restrict__ M, const TO* __restrict__ phid,
                                                    TC* __restrict__ Gp, double* __restrict__ grad,
                                                    double* __restrict__ lap) {
    extern __shared__ __align__(16) unsigned char smem[];
    TC* Xs = reinterpret_cast<TC*>(smem);          // [kGK][kGLd] left slab, [k][row]
    TC* Ys = Xs + kGK * kGLd;                       // [kGK][kGLd] right slab, [k][col]
    TC* Vs = Ys + kGK * kGLd;                       // [kGT][kGLd] V tile, [c][i]
    double* nums = reinterpret_cast<double*>(Vs + kGT * kGLd);  // [4][256] per-electron sums (n <= 256)
    const int w = blockIdx.x, tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;         // output rows 4 ty .. 4 ty + 3, cols 4 tx .. 4 tx + 3
    const double* Aw = Ainv + (long long)w * n * n;  // A_0^{-1}[c][r] at Aw[c n + r]
    const TT* Tw = T + (long long)w * n * m;
    const double* Mw = M + (long long)w * n * N;    // Tbar[h][p] at Mw[h N + n + p]
    TC* Gw = Gp + (long long)w * n * m;
    const TO* phw = phid + (long long)w * n * 5 * N;  // d^a phi(r_i)[j] at phw[(i 5 + a) N + j]
    for (int q = tid; q < 4 * 256; q += kBB) nums[q] = 0.0;

    // G'[i][p] = sum_h A[h][i] Tbar[h][p]: left slab Xs[k][i] = A[h0 + k][i0 + i], right Ys[k][p] = Tbar
    for (int i0 = 0; i0 < n; i0 += kGT)
        for (int p0 = 0; p0 < m; p0 += kGT) {
            TC acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = TC(0);
            for (int h0 = 0; h0 < n; h0 += kGK) {
                __syncthreads();
                for (int q = tid; q < kGK * kGT; q += kBB) {
                    const int k = q / kGT, j = q - k * kGT, h = h0 + k;
                    Xs[k * kGLd + j] = (h < n && i0 + j < n) ? TC(Aw[(long long)h * n + i0 + j]) : TC(0);
                    Ys[k * kGLd + j] = (h < n && p0 + j < m) ? TC(Mw[(long long)h * N + n + p0 + j]) : TC(0);
                }
                __syncthreads();
#pragma unroll 4
                for (int k = 0; k < kGK; ++k) {
                    TC xa[4], yb[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) xa[a] = Xs[k * kGLd + 4 * ty + a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) yb[b] = Ys[k * kGLd + 4 * tx + b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int i = i0 + 4 * ty + a;
                if (i >= n) continue;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int p = p0 + 4 * tx + b;
                    if (p < m) Gw[(long long)i * m + p] = acc[a][b];
                }
            }
        }
    __syncthreads();  // G' of this walker complete (block-wide visibility of its global writes)

    // U[c][i] = sum_p T[c][p] G'[i][p] per 64 x 64 tile; V = A - U; num^a[i] += sum_c dphi^a[i][c] V[c][i]
    for (int i0 = 0; i0 < n; i0 += kGT)
        for (int c0 = 0; c0 < n; c0 += kGT) {
            TC acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = TC(0);
            for (int q0 = 0; q0 < m; q0 += kGK) {
                __syncthreads();
                for (int q = tid; q < kGK * kGT; q += kBB) {
                    // consecutive threads read consecutive p of one row (coalesced), stored [p][row]
                    const int j = q / kGK, k = q - j * kGK, pp = q0 + k;
                    Xs[k * kGLd + j] = (pp < m && c0 + j < n) ? TC(Tw[(long long)(c0 + j) * m + pp]) : TC(0);
                    Ys[k * kGLd + j] = (pp < m && i0 + j < n) ? Gw[(long long)(i0 + j) * m + pp] : TC(0);
                }
                __syncthreads();
#pragma unroll 4
                for (int k = 0; k < kGK; ++k) {
                    TC xa[4], yb[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) xa[a] = Xs[k * kGLd + 4 * ty + a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) yb[b] = Ys[k * kGLd + 4 * tx + b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
                }
            }
            // V tile [c][i] = A[c][i] - U[c][i]
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int c = c0 + 4 * ty + a;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int i = i0 + 4 * tx + b;
                    Vs[(4 * ty + a) * kGLd + 4 * tx + b] =
                        (c < n && i < n) ? TC(Aw[(long long)c * n + i]) - acc[a][b] : TC(0);
                }
            }
            __syncthreads();
            // thread (electron i0 + ii, channel 1 + ch): sum over this tile's occupied orbitals c
            {
                const int ii = tid & 63, ch = tid >> 6, i = i0 + ii;
                if (i < n) {
                    const TO* pa = phw + ((long long)i * 5 + 1 + ch) * N + c0;
                    TC v = TC(0);
                    const int cn = min(kGT, n - c0);
                    for (int cc = 0; cc < cn; ++cc) v = fma(TC(pa[cc]), Vs[cc * kGLd + ii], v);
                    nums[ch * 256 + i] += double(v);
                }
            }
        }
    __syncthreads();
    // the virtual part: num^a[i] += sum_p d^a phi_virt(r_i)[p] G'[i][p], one warp per (electron, channel)
    const int lane = tid & 31, warp = tid >> 5;
    for (int q = warp; q < 4 * n; q += kBB / 32) {
        const int i = q >> 2, ch = q & 3;
        const TO* pa = phw + ((long long)i * 5 + 1 + ch) * N + n;
        const TC* gi = Gw + (long long)i * m;
        TC v = TC(0);
        for (int p = lane; p < m; p += 32) v = fma(TC(pa[p]), gi[p], v);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) nums[ch * 256 + i] += double(v);
    }
    __syncthreads();
    for (int i = tid; i < n; i += kBB) {
        const long long e = (long long)w * n_tot + e_off + i;
        for (int d = 0; d < 3; ++d) grad[e * 3 + d] = nums[d * 256 + i];
        lap[e] = nums[3 * 256 + i];
    }
}

}  // namespace

void launch_dci(const Launch& L, bool mixed, int W, long long n_det, const int* iu, const int* id, const double* gbar,
                const double* S, const void* t0, int ld0, const void* t1, int ld1, double* dci) {
    const int wchunk = 64;
    dim3 grid((unsigned)((n_det + kBB - 1) / kBB), (unsigned)((W + wchunk - 1) / wchunk));
    L.count();
    if (mixed)
        k_dci<float><<<grid, kBB, 0, L.stream>>>(W, wchunk, n_det, iu, id, gbar, S, static_cast<const float*>(t0), ld0,
                                                  static_cast<const float*>(t1), ld1, dci);
    else
        k_dci<double><<<grid, kBB, 0, L.stream>>>(W, wchunk, n_det, iu, id, gbar, S, static_cast<const double*>(t0),
                                                   ld0, static_cast<const double*>(t1), ld1, dci);
}

size_t tbar_smem_bytes(bool mixed, int n, int m) {
    const size_t b = mixed ? 4 : 8;
    return (((size_t)n * m * b + 15) & ~size_t(15)) + (size_t)n * m * b;
}

void launch_phibar(const Launch& L, bool mixed, int W, int n, int m, int N, const ExcDev& g, const void* T,
                   const void* C, const double* S, const double* Ainv, const double* gbar, double* M) {
    const size_t sm = tbar_smem_bytes(mixed, n, m);
    if (m > 0) {
        if (mixed) {
            cudaFuncSetAttribute(k_tbar<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            L.count();
            k_tbar<float><<<W, tbar_threads<float>(), sm, L.stream>>>(n, m, N, g, static_cast<const float*>(T),
                                                    static_cast<const float*>(C), S, M);
            L.count();
            k_tbar_tt<float><<<W, kBB, 0, L.stream>>>(n, m, N, static_cast<const float*>(T), M);
        } else {
            cudaFuncSetAttribute(k_tbar<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            L.count();
            k_tbar<double><<<W, tbar_threads<double>(), sm, L.stream>>>(n, m, N, g, static_cast<const double*>(T),
                                                     static_cast<const double*>(C), S, M);
            L.count();
            k_tbar_tt<double><<<W, kBB, 0, L.stream>>>(n, m, N, static_cast<const double*>(T), M);
        }
    } else {
        // no virtual orbitals: Phibar = gbar Ainv^T, M = I
        L.count();
        k_tbar_tt<double><<<W, kBB, 0, L.stream>>>(n, 0, N, nullptr, M);
    }
    const size_t sp = ((size_t)n * n + (size_t)n * 32) * 8;
    cudaFuncSetAttribute(k_phibar, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
    L.count();
    k_phibar<<<dim3(W, (N + 31) / 32), kBB, sp, L.stream>>>(n, N, Ainv, gbar, M);
}

void launch_chi(const Launch& L, int P, int ppw, const double* pos, long long wstride, int p_off, const double4* bas,
                const int8_t* blm, int nb, double* chi) {
    const long long total = (long long)P * nb;
    L.count();
    k_chi<<<(unsigned)((total + kBB - 1) / kBB), kBB, 0, L.stream>>>(P, ppw, pos, wstride, p_off, bas, blm, nb, chi);
}

void launch_dB(const Launch& L, int P, int nb, int N, const double* chi, const double* Phib, double* dB) {
    const int pchunk = 4096;
    dim3 grid((nb + 31) / 32, (N + 31) / 32, (P + pchunk - 1) / pchunk);
    L.count();
    k_dB<<<grid, kBB, 0, L.stream>>>(P, nb, N, pchunk, chi, Phib, dB);
}

void launch_tbar(const Launch& L, bool mixed, int W, int n, int m, int N, const ExcDev& g, const void* T, const void* C,
                 const double* S, double* M) {
    const size_t sm = tbar_smem_bytes(mixed, n, m);
    if (m <= 0) return;
    if (mixed) {
        cudaFuncSetAttribute(k_tbar<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        L.count();
        k_tbar<float><<<W, tbar_threads<float>(), sm, L.stream>>>(n, m, N, g, static_cast<const float*>(T), static_cast<const float*>(C),
                                                S, M);
    } else {
        cudaFuncSetAttribute(k_tbar<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        L.count();
        k_tbar<double><<<W, tbar_threads<double>(), sm, L.stream>>>(n, m, N, g, static_cast<const double*>(T),
                                                 static_cast<const double*>(C), S, M);
    }
}

void launch_all_gradlap(const Launch& L, bool mixed, int W, int n, int m, int N, int n_tot, int e_off,
                        const double* Ainv, const void* T, const double* M, const void* phid, void* Gp, double* grad,
                        double* lap) {
    L.count();
    if (mixed) {
        const size_t sm = gradlap_smem_bytes<float>();
        cudaFuncSetAttribute(k_all_gradlap<float, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_all_gradlap<float, float, float><<<W, kBB, sm, L.stream>>>(n, m, N, n_tot, e_off, Ainv,
                                                                   static_cast<const float*>(T), M,
                                                                   static_cast<const float*>(phid),
                                                                   static_cast<float*>(Gp), grad, lap);
    } else {
        const size_t sm = gradlap_smem_bytes<double>();
        cudaFuncSetAttribute(k_all_gradlap<double, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
        k_all_gradlap<double, double, double><<<W, kBB, sm, L.stream>>>(n, m, N, n_tot, e_off, Ainv,
                                                                      static_cast<const double*>(T), M,
                                                                      static_cast<const double*>(phid),
                                                                      static_cast<double*>(Gp), grad, lap);
    }
}

}  // namespace msd
