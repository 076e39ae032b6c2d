// Host build of the library's small-determinant arithmetic (msd_smalldet.cuh) for unit tests:
// the exact code the excitation-sweep kernel runs, compiled by the host compiler.
#include "msd_smalldet.cuh"

namespace {
template <typename TT, int K>
TT det_k(const TT* T, int ld, const int* h, const int* p) {
    int hh[K], pp[K];
    for (int q = 0; q < K; ++q) { hh[q] = h[q]; pp[q] = p[q]; }
    return msd::small_det<K, TT>(T, ld, hh, pp);
}
template <typename TT, int K>
TT adj_k(const TT* T, int ld, const TT* x, const int* h, const int* p, TT* z) {
    int hh[K], pp[K];
    for (int q = 0; q < K; ++q) { hh[q] = h[q]; pp[q] = p[q]; }
    TT det, zz[K];
    msd::adj_solve<K, TT>(T, ld, x, hh, pp, det, zz);
    for (int q = 0; q < K; ++q) z[q] = zz[q];
    return det;
}
template <typename TT>
TT det_any(int K, const TT* T, int ld, const int* h, const int* p) {
    switch (K) {
        case 1: return det_k<TT, 1>(T, ld, h, p);
        case 2: return det_k<TT, 2>(T, ld, h, p);
        case 3: return det_k<TT, 3>(T, ld, h, p);
        case 4: return det_k<TT, 4>(T, ld, h, p);
        case 5: return det_k<TT, 5>(T, ld, h, p);
        case 6: return det_k<TT, 6>(T, ld, h, p);
        case 7: return det_k<TT, 7>(T, ld, h, p);
        default: return det_k<TT, 8>(T, ld, h, p);
    }
}
template <typename TT>
TT adj_any(int K, const TT* T, int ld, const TT* x, const int* h, const int* p, TT* z) {
    switch (K) {
        case 1: return adj_k<TT, 1>(T, ld, x, h, p, z);
        case 2: return adj_k<TT, 2>(T, ld, x, h, p, z);
        case 3: return adj_k<TT, 3>(T, ld, x, h, p, z);
        case 4: return adj_k<TT, 4>(T, ld, x, h, p, z);
        case 5: return adj_k<TT, 5>(T, ld, x, h, p, z);
        case 6: return adj_k<TT, 6>(T, ld, x, h, p, z);
        case 7: return adj_k<TT, 7>(T, ld, x, h, p, z);
        default: return adj_k<TT, 8>(T, ld, x, h, p, z);
    }
}
}  // namespace

extern "C" {
double sd_det_f64(int K, const double* T, int ld, const int* h, const int* p) { return det_any<double>(K, T, ld, h, p); }
float sd_det_f32(int K, const float* T, int ld, const int* h, const int* p) { return det_any<float>(K, T, ld, h, p); }
double sd_adj_f64(int K, const double* T, int ld, const double* x, const int* h, const int* p, double* z) {
    return adj_any<double>(K, T, ld, x, h, p, z);
}
float sd_adj_f32(int K, const float* T, int ld, const float* x, const int* h, const int* p, float* z) {
    return adj_any<float>(K, T, ld, x, h, p, z);
}
}
