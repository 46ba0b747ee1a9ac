// spectrum_store.cuh - writing packed spectra into the engine's layouts
// (FDL ring rows and tiled filter spectra), in storage precision.
//
// Shared by the 2 n_x kernels (kernels.cu) and the 3 n_x spectrum-reuse
// kernels (reuse.cu).  `B` below is the number of packed bins of a row (n_f / 2).
#pragma once
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "kernels.h"

namespace gbconv {

// Largest value of v over the CTA (every thread gets it); red: 32 floats.
__device__ inline float block_max(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? red[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    const float r = red[0];
    return r;
}

// Element index of bin k of ring slot `slot` of channel c (layout X[kt][slot][c][BT]).
struct RingIndex {
    int BT, n_ch, c, K, slot;
    __device__ size_t operator()(int k) const {
        const int kt = k / BT, kl = k - kt * BT;
        return (((size_t)kt * K + slot) * n_ch + c) * BT + kl;
    }
};

// Element index of bin k of sub-filter r of output l: tile (kt, lt) starts at
// (kt * n_lt + lt) * tile_elems, then [r][LTt][BT].
struct FilterIndex {
    int BT, n_lt, lt, r, LTt, ll;
    size_t tile_elems;
    __device__ size_t operator()(int k) const {
        const int kt = k / BT, kl = k - kt * BT;
        return ((size_t)kt * n_lt + lt) * tile_elems + ((size_t)r * LTt + ll) * BT + kl;
    }
};

// Largest |re| or |im| of the packed spectrum Xs[0..B) (shared memory).
__device__ inline float spectrum_max(const float2* Xs, int B, float* red) {
    float mx = 0.0f;
    for (int k = threadIdx.x; k < B; k += blockDim.x) mx = fmaxf(mx, fmaxf(fabsf(Xs[k].x), fabsf(Xs[k].y)));
    return block_max(mx, red);
}

// Writes the packed spectrum Xs[0..B) divided by `scale` (a power of two, so
// exactly) in storage precision; `dst_index(k)` gives the element of bin k.
template <int PREC, typename IndexFn>
__device__ void store_scaled(const float2* Xs, int B, int BT, void* dst, IndexFn dst_index, float scale) {
    const float inv = 1.0f / scale;
    for (int k = threadIdx.x; k < B; k += blockDim.x)
        Store<PREC>::store1(dst, dst_index(k), k % BT, BT, cscale(Xs[k], inv));
}

// Writes Xs with its own power-of-two scale (FP32: scale 1).  Returns the scale.
template <int PREC, typename IndexFn>
__device__ float store_spectrum(const float2* Xs, int B, int BT, void* dst, IndexFn dst_index, float* red) {
    const float scale = PREC == PREC_FP32 ? 1.0f : block_scale<PREC>(spectrum_max(Xs, B, red));
    store_scaled<PREC>(Xs, B, BT, dst, dst_index, scale);
    return scale;
}

}  // namespace gbconv
