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
void bord_k(const TT* T, int ld, const TT* x, const TT* y, int ldy, const TT* s, const int* h, const int* p, TT* d) {
    int hh[K], pp[K];
    for (int q = 0; q < K; ++q) { hh[q] = h[q]; pp[q] = p[q]; }
    TT ss[5] = {s[0], s[1], s[2], s[3], s[4]};
    TT dd[5];
    msd::bordered<K, 5, TT>(T, ld, x, y, ldy, ss, hh, pp, dd);
    for (int a = 0; a < 5; ++a) d[a] = dd[a];
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
void bord_any(int K, const TT* T, int ld, const TT* x, const TT* y, int ldy, const TT* s, const int* h, const int* p,
              TT* d) {
    switch (K) {
        case 1: bord_k<TT, 1>(T, ld, x, y, ldy, s, h, p, d); break;
        case 2: bord_k<TT, 2>(T, ld, x, y, ldy, s, h, p, d); break;
        case 3: bord_k<TT, 3>(T, ld, x, y, ldy, s, h, p, d); break;
        case 4: bord_k<TT, 4>(T, ld, x, y, ldy, s, h, p, d); break;
        case 5: bord_k<TT, 5>(T, ld, x, y, ldy, s, h, p, d); break;
        case 6: bord_k<TT, 6>(T, ld, x, y, ldy, s, h, p, d); break;
        case 7: bord_k<TT, 7>(T, ld, x, y, ldy, s, h, p, d); break;
        default: bord_k<TT, 8>(T, ld, x, y, ldy, s, h, p, d); break;
    }
}
}  // namespace

extern "C" {
double sd_det_f64(int K, const double* T, int ld, const int* h, const int* p) { return det_any<double>(K, T, ld, h, p); }
float sd_det_f32(int K, const float* T, int ld, const int* h, const int* p) { return det_any<float>(K, T, ld, h, p); }
void sd_bordered_f64(int K, const double* T, int ld, const double* x, const double* y, int ldy, const double* s,
                     const int* h, const int* p, double* d) { bord_any<double>(K, T, ld, x, y, ldy, s, h, p, d); }
void sd_bordered_f32(int K, const float* T, int ld, const float* x, const float* y, int ldy, const float* s,
                     const int* h, const int* p, float* d) { bord_any<float>(K, T, ld, x, y, ldy, s, h, p, d); }
}
