// msd_smalldet.cuh -- small determinants of excitation-table entries (Section III) and the
// bordered determinants of a single-electron move (Section IV-A/IV-C), as __host__ __device__
// code so the same arithmetic can be unit-tested on the host.
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

// det T_u by LU with partial pivoting held in registers (k >= 2).  Closed-form cofactor
// expansions are not used: when A_0 is nearly singular, T = A_0^{-1} Phi_virt carries a large
// rank-1 component and products of its entries cancel catastrophically, while the pivoted
// elimination removes that component in its first step.
template <int K, typename TT>
MSD_HD TT small_det(const TT* Ts, int ld, const int (&h)[K], const int (&p)[K]) {
    if constexpr (K == 1) {
        return Ts[h[0] * ld + p[0]];
    } else {
        TT M[K][K];
#pragma unroll
        for (int q = 0; q < K; ++q)
#pragma unroll
            for (int l = 0; l < K; ++l) M[q][l] = Ts[h[q] * ld + p[l]];
        TT det = TT(1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int piv = k;
            TT best = tabs(M[k][k]);
#pragma unroll
            for (int r = k + 1; r < K; ++r) {
                const TT v = tabs(M[r][k]);
                if (v > best) { best = v; piv = r; }
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
            }
            const TT pv = M[k][k];
            det = (piv != k) ? -det * pv : det * pv;
            if (pv == TT(0)) return TT(0);
            const TT ip = TT(1) / pv;
#pragma unroll
            for (int r = k + 1; r < K; ++r) {
                const TT fct = M[r][k] * ip;
#pragma unroll
                for (int j = k + 1; j < K; ++j) M[r][j] = fma(-fct, M[k][j], M[r][j]);
            }
        }
        return det;
    }
}

// Slow path for an exactly singular T_u (k >= 4): the (k+1) x (k+1) bordered determinant of
// each channel by its own LU.  Never taken for generic inputs.
template <typename TT>
MSD_HD_NOINLINE TT bordered_direct(int K, const TT* Ts, int ld, const TT* xs, const TT* ysa, const int* h,
                                           const int* p, TT s) {
    TT M[MSD_MAX_ORDER + 1][MSD_MAX_ORDER + 1];
    const int n1 = K + 1;
    for (int q = 0; q < K; ++q) {
        for (int l = 0; l < K; ++l) M[q][l] = Ts[h[q] * ld + p[l]];
        M[q][K] = xs[h[q]];
    }
    for (int l = 0; l < K; ++l) M[K][l] = -ysa[p[l]];
    M[K][K] = s;
    TT det = TT(1);
    for (int k = 0; k < n1; ++k) {
        int piv = k;
        TT best = tabs(M[k][k]);
        for (int r = k + 1; r < n1; ++r)
            if (tabs(M[r][k]) > best) { best = tabs(M[r][k]); piv = r; }
        if (best == TT(0)) return TT(0);
        if (piv != k) {
            for (int j = 0; j < n1; ++j) { TT t = M[k][j]; M[k][j] = M[piv][j]; M[piv][j] = t; }
            det = -det;
        }
        det *= M[k][k];
        for (int r = k + 1; r < n1; ++r) {
            const TT fct = M[r][k] / M[k][k];
            for (int j = k + 1; j < n1; ++j) M[r][j] -= fct * M[k][j];
        }
    }
    return det;
}

// Bordered determinants d^a = det [[T_u, x_u], [-y^a_u^T, s^a]] = det(T_u) s^a + y^a_u . adj(T_u) x_u
// for NC channels sharing one factorisation of T_u (adj(T_u) x_u = det(T_u) T_u^{-1} x_u from
// the pivoted LU).  ys is [NC][ldy].
template <int K, int NC, typename TT>
MSD_HD void bordered(const TT* Ts, int ld, const TT* xs, const TT* ys, int ldy,
                                         const TT (&s)[NC], const int (&h)[K], const int (&p)[K], TT (&d)[NC]) {
    TT z[K];  // adj(T_u) x_u, indexed by particle slot
    TT det;
    if constexpr (K == 1) {
        det = Ts[h[0] * ld + p[0]];
        z[0] = xs[h[0]];
    } else {
        TT M[K][K], b[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
#pragma unroll
            for (int l = 0; l < K; ++l) M[q][l] = Ts[h[q] * ld + p[l]];
            b[q] = xs[h[q]];
        }
        det = TT(1);
        bool singular = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int piv = k;
            TT best = tabs(M[k][k]);
#pragma unroll
            for (int r = k + 1; r < K; ++r) {
                const TT v = tabs(M[r][k]);
                if (v > best) { best = v; piv = r; }
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
            det = (piv != k) ? -det * pv : det * pv;
            singular |= (pv == TT(0));
            const TT ip = TT(1) / pv;
#pragma unroll
            for (int r = k + 1; r < K; ++r) {
                const TT fct = M[r][k] * ip;
#pragma unroll
                for (int j = k + 1; j < K; ++j) M[r][j] = fma(-fct, M[k][j], M[r][j]);
                b[r] = fma(-fct, b[k], b[r]);
            }
            M[k][k] = ip;
        }
        if (singular) {
            int hh[MSD_MAX_ORDER], pp[MSD_MAX_ORDER];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                hh[q] = h[q];
                pp[q] = p[q];
            }
            for (int a = 0; a < NC; ++a) d[a] = bordered_direct<TT>(K, Ts, ld, xs, ys + a * ldy, hh, pp, s[a]);
            return;
        }
        // back substitution U z' = b, then z = det * z'
#pragma unroll
        for (int q = K - 1; q >= 0; --q) {
            TT acc = b[q];
#pragma unroll
            for (int j = q + 1; j < K; ++j) acc = fma(-M[q][j], z[j], acc);
            z[q] = acc * M[q][q];
        }
#pragma unroll
        for (int q = 0; q < K; ++q) z[q] *= det;
    }
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        TT acc = det * s[a];
#pragma unroll
        for (int l = 0; l < K; ++l) acc = fma(ys[a * ldy + p[l]], z[l], acc);
        d[a] = acc;
    }
}

// Per-thread accumulators of the CI sums: plain FP64, or FP32 with Kahan compensation.
template <typename TT, int NC>
struct Accum;
template <int NC>
struct Accum<double, NC> {
    double s[NC];
    MSD_HD void zero() {
#pragma unroll
        for (int a = 0; a < NC; ++a) s[a] = 0.0;
    }
    MSD_HD void add(int a, double x) { s[a] += x; }
    MSD_HD void get(double (&v)[NC]) const {
#pragma unroll
        for (int a = 0; a < NC; ++a) v[a] = s[a];
    }
};
template <int NC>
struct Accum<float, NC> {
    float s[NC], c[NC];
    MSD_HD void zero() {
#pragma unroll
        for (int a = 0; a < NC; ++a) s[a] = c[a] = 0.0f;
    }
    MSD_HD void add(int a, float x) {
        const float y = x - c[a];
        const float t = s[a] + y;
        c[a] = (t - s[a]) - y;
        s[a] = t;
    }
    MSD_HD void get(double (&v)[NC]) const {
#pragma unroll
        for (int a = 0; a < NC; ++a) v[a] = double(s[a]) - double(c[a]);
    }
};

}  // namespace msd
