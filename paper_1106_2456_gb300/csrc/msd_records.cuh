// msd_records.cuh -- device decoding of the excitation records built by the host plan
// (msd_api.cu): k hole bytes then k particle bytes, padded to 2, 4, 8 or 16 bytes.
#pragma once

#include <cstdint>
#include <type_traits>

namespace msd {

// Raw record of order K as one vector load, and its decoding into hole/particle indices.
template <int K>
struct RecRaw {
    using type = typename std::conditional<K == 1, unsigned short,
                 typename std::conditional<K == 2, unsigned,
                 typename std::conditional<(K <= 4), uint2, uint4>::type>::type>::type;
};

template <int K>
__device__ __forceinline__ typename RecRaw<K>::type load_raw(const uint8_t* __restrict__ base, int i) {
    return __ldg(reinterpret_cast<const typename RecRaw<K>::type*>(base) + i);
}

template <int K>
__device__ __forceinline__ void decode_rec(const typename RecRaw<K>::type& v, int (&h)[K], int (&p)[K]) {
    if constexpr (K == 1) {
        h[0] = v & 0xff;
        p[0] = (v >> 8) & 0xff;
    } else if constexpr (K == 2) {
        h[0] = v & 0xff;
        h[1] = (v >> 8) & 0xff;
        p[0] = (v >> 16) & 0xff;
        p[1] = (v >> 24) & 0xff;
    } else if constexpr (K <= 4) {
        const unsigned wd[2] = {v.x, v.y};
#pragma unroll
        for (int q = 0; q < K; ++q) {
            h[q] = (wd[q >> 2] >> ((q & 3) * 8)) & 0xff;
            p[q] = (wd[(K + q) >> 2] >> (((K + q) & 3) * 8)) & 0xff;
        }
    } else {
        const unsigned wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < K; ++q) {
            h[q] = (wd[q >> 2] >> ((q & 3) * 8)) & 0xff;
            p[q] = (wd[(K + q) >> 2] >> (((K + q) & 3) * 8)) & 0xff;
        }
    }
}

template <int K>
__device__ __forceinline__ void load_rec(const uint8_t* __restrict__ base, int i, int (&h)[K], int (&p)[K]) {
    if constexpr (K == 1) {
        const unsigned v = __ldg(reinterpret_cast<const unsigned short*>(base) + i);
        h[0] = v & 0xff;
        p[0] = (v >> 8) & 0xff;
    } else if constexpr (K == 2) {
        const unsigned v = __ldg(reinterpret_cast<const unsigned*>(base) + i);
        h[0] = v & 0xff;
        h[1] = (v >> 8) & 0xff;
        p[0] = (v >> 16) & 0xff;
        p[1] = (v >> 24) & 0xff;
    } else if constexpr (K <= 4) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + i);
        const unsigned wd[2] = {v.x, v.y};
#pragma unroll
        for (int q = 0; q < K; ++q) {
            h[q] = (wd[q >> 2] >> ((q & 3) * 8)) & 0xff;
            p[q] = (wd[(K + q) >> 2] >> (((K + q) & 3) * 8)) & 0xff;
        }
    } else {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(base) + i);
        const unsigned wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < K; ++q) {
            h[q] = (wd[q >> 2] >> ((q & 3) * 8)) & 0xff;
            p[q] = (wd[(K + q) >> 2] >> (((K + q) & 3) * 8)) & 0xff;
        }
    }
}

}  // namespace msd
