// msd_smalldet.cuh -- small determinants of excitation-table entries (Section III), as
// __host__ __device__ code so the arithmetic the excitation sweep runs can be unit-tested on
// the host.
//
// For an excitation u of order k with holes h_q and particles p_l, T_u[q][l] = T[h_q][p_l].
//   small_det : det T_u                               (= det A_u / det A_0, Section III)
//   adj_solve : det T_u and z = adj(T_u) x_u          (the two ingredients of every bordered
//               determinant det [[T_u, x_u], [-y^T, s]] = det(T_u) s + y . z, Section IV-A/C)
// Both eliminate the first k-2 columns by LU with partial pivoting held in registers and
// finish the remaining 2 x 2 Schur complement in closed form, each 2 x 2 determinant
// a d - b c evaluated with one FMA-based error correction (Kahan's method), so it is accurate
// to a few units in the last place whatever the cancellation.  Plain closed-form cofactor
// expansions are not used for k >= 3: when A_0 is nearly singular, T = A_0^{-1} Phi_virt
// carries a large rank-1 component and products of its entries cancel catastrophically,
// while the pivoted elimination removes that component in its first step.  The only division
// is one reciprocal per eliminated column (none for k <= 2).
#pragma once

#include <cmath>

#include "msd.h"

#if defined(__CUDACC__)
#define MSD_HD __host__ __device__ __forceinline__
#define MSD_HD_NOINLINE __host__ __device__ __noinline__
#else
#define MSD_HD inline
#define MSD_HD_NOINLINE
#endif

namespace msd {

#if !defined(__CUDACC__)
using std::fma;
#endif

template <typename T>
MSD_HD T tabs(T x) {
    return x < T(0) ? -x : x;
}

// 1 / x.  FP64: IEEE division.  FP32 on the device: the hardware approximation (PTX
// rcp.approx.f32, at most 1 ulp from the exact reciprocal), one instruction instead of a
// correctly rounded sequence; an LU multiplier then carries one extra rounding of that size.
MSD_HD double recip(double x) { return 1.0 / x; }
MSD_HD float recip(float x) {
#if defined(__CUDA_ARCH__)
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;
#endif
}

// a b - c d with the rounding error of c d added back (Kahan's 2 x 2 determinant): the result
// is within about 2 ulp of the exact value even when the two products nearly cancel.
template <typename T>
MSD_HD T dop(T a, T b, T c, T d) {
    const T w = c * d;
    const T e = fma(-c, d, w);
    const T f = fma(a, b, -w);
    return f + e;
}

// S steps of LU with partial pivoting on the K x K block M, the right-hand side b permuted and
// eliminated alongside.  On return rows/columns < S hold U with 1/u_kk on the diagonal, the
// trailing (K-S) x (K-S) block holds the Schur complement, and the return value is
// sign(P) * prod u_kk, starting from dp.  The first K0 steps take their pivot row as it stands
// (the caller has already put the pivot there).  `singular` is set if a pivot is exactly zero (the column below the
// diagonal is then zero and T_u is singular).
template <int K, int S, typename TT, int K0 = 0>
MSD_HD TT lu_steps(TT (&M)[K][K], TT (&b)[K], bool& singular, TT dp = TT(1)) {
    singular = false;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        if (k < K0) {  // pivot already in place (rows ordered before loading)
            const TT pv = M[k][k];
            dp *= pv;
            singular |= (pv == TT(0));
            const TT ip = recip(pv);
#pragma unroll
            for (int r = k + 1; r < K; ++r) {
                const TT fct = M[r][k] * ip;
#pragma unroll
                for (int j = k + 1; j < K; ++j) M[r][j] = fma(-fct, M[k][j], M[r][j]);
                b[r] = fma(-fct, b[k], b[r]);
            }
            M[k][k] = ip;
            continue;
        }
        int piv = k;
        TT best = tabs(M[k][k]);
#pragma unroll
        for (int r = k + 1; r < K; ++r) {
            const TT v = tabs(M[r][k]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
#pragma unroll
        for (int r = k + 1; r < K; ++r) {
            const bool sw = (piv == r);
#pragma unroll
            for (int j = k; j < K; ++j) {
                const TT x = M[k][j], y = M[r][j];
                M[k][j] = sw ? y : x;
                M[r][j] = sw ? x : y;
            }
            const TT x = b[k], y = b[r];
            b[k] = sw ? y : x;
            b[r] = sw ? x : y;
        }
        const TT pv = M[k][k];
        dp = (piv != k) ? -dp * pv : dp * pv;
        singular |= (pv == TT(0));
        const TT ip = recip(pv);
#pragma unroll
        for (int r = k + 1; r < K; ++r) {
            const TT fct = M[r][k] * ip;
#pragma unroll
            for (int j = k + 1; j < K; ++j) M[r][j] = fma(-fct, M[k][j], M[r][j]);
            b[r] = fma(-fct, b[k], b[r]);
        }
        M[k][k] = ip;
    }
    return dp;
}

// det T_u.
template <int K, typename TT>
MSD_HD TT small_det(const TT* Ts, int ld, const int (&h)[K], const int (&p)[K]) {
    if constexpr (K == 1) {
        return Ts[h[0] * ld + p[0]];
    } else if constexpr (K == 2) {
        return dop(Ts[h[0] * ld + p[0]], Ts[h[1] * ld + p[1]], Ts[h[0] * ld + p[1]], Ts[h[1] * ld + p[0]]);
    } else {
        TT M[K][K], b[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            b[q] = TT(0);
#pragma unroll
            for (int l = 0; l < K; ++l) M[q][l] = Ts[h[q] * ld + p[l]];
        }
        bool singular;
        const TT dp = lu_steps<K, K - 2, TT>(M, b, singular);
        constexpr int a = K - 2, c = K - 1;
        return singular ? TT(0) : dp * dop(M[a][a], M[c][c], M[a][c], M[c][a]);
    }
}

// Exactly singular T_u: z_l = det(T_u with column l replaced by x_u) (Cramer's rule for the
// adjugate), each by its own pivoted LU.  Never taken for generic inputs.
template <typename TT>
MSD_HD_NOINLINE void adj_cramer(int K, const TT* Ts, int ld, const TT* xs, const int* h, const int* p, TT* z) {
    TT M[MSD_MAX_ORDER][MSD_MAX_ORDER];
    for (int l = 0; l < K; ++l) {
        for (int q = 0; q < K; ++q)
            for (int j = 0; j < K; ++j) M[q][j] = (j == l) ? xs[h[q]] : Ts[h[q] * ld + p[j]];
        TT det = TT(1);
        for (int k = 0; k < K && det != TT(0); ++k) {
            int piv = k;
            for (int r = k + 1; r < K; ++r)
                if (tabs(M[r][k]) > tabs(M[piv][k])) piv = r;
            if (M[piv][k] == TT(0)) {
                det = TT(0);
                break;
            }
            if (piv != k) {
                for (int j = 0; j < K; ++j) {
                    const TT t = M[k][j];
                    M[k][j] = M[piv][j];
                    M[piv][j] = t;
                }
                det = -det;
            }
            det *= M[k][k];
            for (int r = k + 1; r < K; ++r) {
                const TT fct = M[r][k] / M[k][k];
                for (int j = k + 1; j < K; ++j) M[r][j] -= fct * M[k][j];
            }
        }
        z[l] = det;
    }
}

// det T_u and z = adj(T_u) x_u = det(T_u) T_u^{-1} x_u, z indexed by particle slot l.
// With U_11 (pivots u_jj), U_12, Schur block S and b' = (b'_1, b'_2) after the first K-2
// elimination steps: z_2 = sign(P) prod u_jj adj(S) b'_2 and z_1 = U_11^{-1}(det b'_1 - U_12 z_2),
// which needs no division beyond the stored 1/u_jj and stays valid when det S = 0.
template <int K, typename TT>
MSD_HD void adj_solve(const TT* Ts, int ld, const TT* xs, const int (&h)[K], const int (&p)[K], TT& det,
                      TT (&z)[K]) {
    if constexpr (K == 1) {
        det = Ts[h[0] * ld + p[0]];
        z[0] = xs[h[0]];
    } else if constexpr (K == 2) {
        TT M[K][K], b[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
#pragma unroll
            for (int l = 0; l < K; ++l) M[q][l] = Ts[h[q] * ld + p[l]];
            b[q] = xs[h[q]];
        }
        det = dop(M[0][0], M[1][1], M[0][1], M[1][0]);
        z[0] = dop(M[1][1], b[0], M[0][1], b[1]);
        z[1] = dop(M[0][0], b[1], M[1][0], b[0]);
    } else {
        // The first elimination step's row exchange is made on the hole indices before the rest
        // of T_u is gathered: the first column alone decides the pivot, and exchanging two
        // holes then costs a few integer selects instead of exchanging K values in every row.
        TT M[K][K], b[K];
        int hp[K];
        TT c0[K];
#pragma unroll
        for (int q = 0; q < K; ++q) c0[q] = Ts[h[q] * ld + p[0]];
        int piv = 0;
        TT best = tabs(c0[0]);
#pragma unroll
        for (int r = 1; r < K; ++r) {
            const TT v = tabs(c0[r]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        int h0 = h[0];
        TT v0 = c0[0];
#pragma unroll
        for (int r = 1; r < K; ++r) {
            const bool sw = piv == r;
            h0 = sw ? h[r] : h0;
            v0 = sw ? c0[r] : v0;
            hp[r] = sw ? h[0] : h[r];
            M[r][0] = sw ? c0[0] : c0[r];
        }
        hp[0] = h0;
        M[0][0] = v0;
#pragma unroll
        for (int q = 0; q < K; ++q) {
#pragma unroll
            for (int l = 1; l < K; ++l) M[q][l] = Ts[hp[q] * ld + p[l]];
            b[q] = xs[hp[q]];
        }
        bool singular;
        const TT dp = lu_steps<K, K - 2, TT, 1>(M, b, singular, piv != 0 ? TT(-1) : TT(1));
        if (singular) {
            int hh[MSD_MAX_ORDER], pp[MSD_MAX_ORDER];
            TT zz[MSD_MAX_ORDER];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                hh[q] = h[q];
                pp[q] = p[q];
            }
            adj_cramer<TT>(K, Ts, ld, xs, hh, pp, zz);
            det = TT(0);
#pragma unroll
            for (int q = 0; q < K; ++q) z[q] = zz[q];
            return;
        }
        constexpr int a = K - 2, c = K - 1;
        det = dp * dop(M[a][a], M[c][c], M[a][c], M[c][a]);
        z[a] = dp * dop(M[c][c], b[a], M[a][c], b[c]);
        z[c] = dp * dop(M[a][a], b[c], M[c][a], b[a]);
#pragma unroll
        for (int q = K - 3; q >= 0; --q) {
            TT acc = det * b[q];
#pragma unroll
            for (int j = q + 1; j < K; ++j) acc = fma(-M[q][j], z[j], acc);
            z[q] = acc * M[q][q];
        }
    }
}

// Per-thread accumulators of CI sums in the table's precision.  A thread adds at most a few
// hundred terms of one walker's sum (the strings are spread over 256 threads), so plain FP32
// accumulation adds a relative error of order 1e-5 of the sum of magnitudes, well inside the
// FP32 path's accuracy; partial sums are combined across warps in FP64.
template <typename TT, int NV>
struct Accum {
    TT s[NV];
    MSD_HD void zero() {
        for (int a = 0; a < NV; ++a) s[a] = TT(0);
    }
    MSD_HD void add(int a, TT x) { s[a] += x; }
    MSD_HD double get(int a) const { return double(s[a]); }
};

}  // namespace msd
