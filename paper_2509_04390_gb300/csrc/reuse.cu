// reuse.cu - kernels of the n_f = 3 n_x form of the synthesis + feedback
// canceller (the remark closing Sec. 5).
//
// With n_f = 3 n_x, the synthesis accumulated spectrum Y_n is the spectrum of
// a 3 n_x window whose last 2 n_x samples are [l_{n-1}, l_n] (only the first
// n_x samples wrap around: the sub-filters have n_x taps).  The canceller's
// n_x-tap sub-filters reach at most n_x - 1 samples back from its kept last
// n_x output samples, so Y_n can enter the canceller's FDL as it is: the output
// kernel of the synthesis pushes Y_n into the canceller's ring and the
// canceller's C_out input R2C transforms disappear.  The price: 3 n_x-point
// transforms, and 3 n_x / 2 bins instead of n_x in every spectrum of both
// convolutions (1.5x the bytes of both FDL MACs).
//
// Transforms.  The real FFT of n_f = 3 n_x samples w is the complex FFT of the
// N = 3 n_x / 2 points z[n] = w[2n] + i w[2n+1] followed by the same
// post-processing as the 2 n_x kernels (r2c_post / c2r_pre with N in place of
// n_x).  The complex FFT is a mixed-radix Stockham transform: one radix-3
// stage, then radix 2 (when log2(N / 3) is odd) and radix 4.  Twiddles
// tw[j] = W_{3 n_x}^j = exp(-2 pi i j / (3 n_x)), j in [0, 3 n_x), are
// computed in FP64 on the host and rounded once.
//
// Spectra are packed as in kernels.h (N complex values per row, the real
// Nyquist bin in the imaginary slot of bin 0).  The FDL MAC is the 2 n_x one,
// planned over N bins.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "kernels.h"
#include "spectrum_store.cuh"

namespace gbconv {
namespace {

constexpr float SQRT3_2 = 0.866025403784438646763723170752936183f;  // sqrt(3) / 2

// Complex FFT of N = 3 * 2^log2M points in shared memory, Stockham autosort:
// a stage with radix R and span Ns reads element j + r*N/R, multiplies it by
// W_{Ns R}^{r (j mod Ns)} (= tw[r (j mod Ns) twN / (Ns R)]), does an R-point
// DFT and writes output r to (j / Ns) * Ns * R + (j mod Ns) + r * Ns.  INV
// selects the conjugate roots (unscaled inverse).  Every stage ends with
// __syncthreads(); the caller synchronises before the first one.  Returns the
// buffer that holds the result (a or b).
template <bool INV>
__device__ float2* fft_mixed_smem(float2* a, float2* b, int N, int log2M, const float2* tw, int twN, int tid,
                                  int nth) {
    // radix 3 at span 1 (no twiddles).  W_3 = -1/2 - i sqrt(3)/2:
    // y0 = v0 + s, y1 = t - i r, y2 = t + i r with s = v1 + v2, t = v0 - s/2,
    // r = sqrt(3)/2 (v1 - v2); the inverse swaps y1 and y2.
    {
        const int T = N / 3;
        for (int j = tid; j < T; j += nth) {
            const float2 v0 = a[j], v1 = a[j + T], v2 = a[j + 2 * T];
            const float2 s = cadd(v1, v2);
            const float2 r = cscale(csub(v1, v2), SQRT3_2);
            const float2 t = make_float2(v0.x - 0.5f * s.x, v0.y - 0.5f * s.y);
            const float2 mir = make_float2(r.y, -r.x);  // -i r
            b[3 * j] = cadd(v0, s);
            b[3 * j + 1] = INV ? csub(t, mir) : cadd(t, mir);
            b[3 * j + 2] = INV ? cadd(t, mir) : csub(t, mir);
        }
        __syncthreads();
        float2* x = a;
        a = b;
        b = x;
    }
    int Ns = 3;
    if (log2M & 1) {
        const int H = N >> 1;
        const int step = twN / (2 * Ns);
        for (int j = tid; j < H; j += nth) {
            const int k = j % Ns;
            const float2 v0 = a[j];
            const float2 v1 = cmul(a[j + H], tw_at<INV>(tw, k * step));
            const int o = (j - k) * 2 + k;
            b[o] = cadd(v0, v1);
            b[o + Ns] = csub(v0, v1);
        }
        __syncthreads();
        float2* x = a;
        a = b;
        b = x;
        Ns *= 2;
    }
    while (Ns < N) {
        const int Q = N >> 2;
        const int step = twN / (4 * Ns);
        for (int j = tid; j < Q; j += nth) {
            const int k = j % Ns;
            const int base = k * step;
            const float2 v0 = a[j];
            const float2 v1 = cmul(a[j + Q], tw_at<INV>(tw, base));
            const float2 v2 = cmul(a[j + 2 * Q], tw_at<INV>(tw, 2 * base));
            const float2 v3 = cmul(a[j + 3 * Q], tw_at<INV>(tw, 3 * base));
            const float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
            const float2 s13 = cadd(v1, v3), d13 = csub(v1, v3);
            // forward: -i * d13 ; inverse: +i * d13
            const float2 rot = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
            const int o = (j - k) * 4 + k;
            b[o] = cadd(s02, s13);
            b[o + Ns] = cadd(d02, rot);
            b[o + 2 * Ns] = csub(s02, s13);
            b[o + 3 * Ns] = csub(d02, rot);
        }
        __syncthreads();
        float2* x = a;
        a = b;
        b = x;
        Ns *= 4;
    }
    return a;
}

__device__ __forceinline__ void load_twiddles3(float2* dst, const float2* __restrict__ tw, int twN) {
    for (int j = threadIdx.x; j < twN; j += blockDim.x) dst[j] = __ldg(tw + j);
}

// ------------------------------------------------------- pack + R2C (3 n_x)
// One CTA per channel.  w = [two previous blocks, in - sub] (3 n_x samples);
// N-point complex FFT of z[n] = w[2n] + i w[2n+1]; real-FFT post-processing;
// push into the ring slot.  win holds [n_ch][2 n_x].
template <int PREC>
__device__ __forceinline__ void pack3_body(const PackArgs& a, const int c) {
    extern __shared__ float2 fsm[];
    __shared__ float red[32];
    const int B = a.B, N = 3 * (B >> 1), tid = threadIdx.x, nth = blockDim.x;
    float2* bufA = fsm;
    float2* bufB = fsm + N;
    float2* tws = fsm + 2 * N;
    griddep_launch_dependents();
    load_twiddles3(tws, a.tw, 2 * N);
    griddep_wait();  // input, feedback prediction and ring slot belong to earlier work
    const float* in = a.in + (size_t)c * a.in_stride;
    const float* sub = a.sub ? a.sub + (size_t)c * B : nullptr;
    float* win = a.win + (size_t)c * 2 * B;
    for (int n = tid; n < N; n += nth) {
        float2 z;
        if (n < B) {
            z = make_float2(win[2 * n], win[2 * n + 1]);
        } else {
            const int t = 2 * n - 2 * B;
            float v0 = in[t], v1 = in[t + 1];
            if (sub) {
                v0 -= sub[t];
                v1 -= sub[t + 1];
            }
            z = make_float2(v0, v1);
        }
        bufA[n] = z;
    }
    __syncthreads();
    // slide the history by one block: win = [w[B..2B), in - sub].  bufA is
    // first overwritten by the FFT's second stage, after its first barrier.
    float* e_out = a.e_out ? a.e_out + (size_t)c * (a.e_stride ? a.e_stride : B) : nullptr;
    for (int t = tid; t < B; t += nth) {
        const int u = B + t;
        const float2 zz = bufA[u >> 1];
        win[t] = (u & 1) ? zz.y : zz.x;
        const float v = sub ? in[t] - sub[t] : in[t];
        win[B + t] = v;
        if (e_out) e_out[t] = v;
    }
    float2* Z = fft_mixed_smem<false>(bufA, bufB, N, a.log2B - 1, tws, 2 * N, tid, nth);
    float2* Xs = (Z == bufA) ? bufB : bufA;
    for (int k = tid; k < N; k += nth) Xs[k] = r2c_post(Z, k, N, tws);
    __syncthreads();
    const float scale = store_spectrum<PREC>(Xs, N, a.BT, a.X, RingIndex{a.BT, a.n_ch, c, a.K, a.slot}, red);
    if (PREC != PREC_FP32 && tid == 0) a.sX[(size_t)a.slot * a.n_ch + c] = scale;
}

template <int PREC>
__global__ void k_pack3(const PackArgs a) {
    pack3_body<PREC>(a, blockIdx.x);
}

// ---------------------------------------------- filter partitions R2C (3 n_x)
// One CTA per (l, q, p): sub-filter h_lq[pB, pB+B) zero-padded to 3B, R2C,
// stored at reduction index p * n_src + q; the two reduced-precision passes
// as in the 2 n_x filter kernel (pass 0 records maxima, pass 1 stores scaled).
template <int PREC>
__global__ void k_filter3(const FilterArgs a) {
    extern __shared__ float2 fsm[];
    __shared__ float red[32];
    const int B = a.B, half = B >> 1, N = 3 * half, tid = threadIdx.x, nth = blockDim.x;
    const int K = a.K, R = a.n_src * K;
    const int l = blockIdx.x / R;
    const int qp = blockIdx.x - l * R;
    const int q = qp / K, p = qp - q * K;
    const int r = p * a.n_src + q;
    const float* h = a.h + ((size_t)l * a.n_src + q) * (size_t)a.taps;
    const long long t0 = (long long)p * B;
    float2* bufA = fsm;
    float2* bufB = fsm + N;
    float2* tws = fsm + 2 * N;
    load_twiddles3(tws, a.tw, 2 * N);
    for (int n = tid; n < N; n += nth) {
        float2 z = make_float2(0.0f, 0.0f);
        if (n < half) {
            const long long t = t0 + 2 * n;
            z.x = t < a.taps ? h[t] : 0.0f;
            z.y = t + 1 < a.taps ? h[t + 1] : 0.0f;
        }
        bufA[n] = z;
    }
    __syncthreads();
    float2* Z = fft_mixed_smem<false>(bufA, bufB, N, a.log2B - 1, tws, 2 * N, tid, nth);
    float2* Xs = (Z == bufA) ? bufB : bufA;
    for (int k = tid; k < N; k += nth) Xs[k] = r2c_post(Z, k, N, tws);
    __syncthreads();
    const int l0 = (l / a.LT) * a.LT;
    const int LTt = min(a.LT, a.n_dst - l0), ll = l - l0;
    if (PREC != PREC_FP32 && a.pass == 0) {
        const float mx = spectrum_max(Xs, N, red);
        if (tid == 0) a.maxabs[(size_t)l * R + r] = mx;
        return;
    }
    const float scale = PREC == PREC_FP32 ? 1.0f : __ldg(a.sH + (size_t)(l / a.LT) * R + r);
    const int n_lt = (a.n_dst + a.LT - 1) / a.LT;
    store_scaled<PREC>(Xs, N, a.BT, a.H, FilterIndex{a.BT, n_lt, l / a.LT, r, LTt, ll, a.tile_elems}, scale);
}

// --------------------------------------------------- output (3 n_x) + reuse
// One CTA per output channel l: fixed-order sum of the tail's split partials,
// partition 0 of this block (the head), then
//   * if push.X is set: the accumulated spectrum Y goes, as it is, into ring
//     slot push.slot of channel l of the next convolution (the canceller:
//     the reuse of the synthesis output spectrum);
//   * C2R of Y (N-point inverse FFT, scaled by 1/N) and overlap-save: the last
//     n_x of the 3 n_x samples are the output block.
template <int PREC>
__device__ __forceinline__ void out3_body(const OutArgs& a, const PackArgs& push, const int l) {
    using St = Store<PREC>;
    extern __shared__ float2 fsm[];
    __shared__ float red[32];
    const int B = a.B, N = 3 * (B >> 1), tid = threadIdx.x, nth = blockDim.x;
    float2* P = fsm;
    float2* W = fsm + N;
    float2* tws = fsm + 2 * N;
    griddep_launch_dependents();
    load_twiddles3(tws, a.tw, 2 * N);
    const size_t stride = (size_t)a.n_dst * N;
    const int S = a.S;
    const int l0 = (l / a.LT) * a.LT;
    const int LTt = min(a.LT, a.n_dst - l0), ll = l - l0;
    const int n_lt = (a.n_dst + a.LT - 1) / a.LT;
    // the tail partials come from another stream, complete before this launch
    // (early_partials), so they are summed before waiting for the previous kernel
    if (!a.early_partials) griddep_wait();
    for (int k = tid; k < N; k += nth) {
        const float2* src = a.partial + (size_t)l * N + k;
        float2 tot = make_float2(0.0f, 0.0f);
        int s = 0;
        for (; s + 8 <= S; s += 8) {
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = src[(size_t)(s + i) * stride];
            const float2 g = cadd(cadd(cadd(v[0], v[1]), cadd(v[2], v[3])), cadd(cadd(v[4], v[5]), cadd(v[6], v[7])));
            tot = cadd(tot, g);
        }
        for (; s < S; ++s) tot = cadd(tot, src[(size_t)s * stride]);
        P[k] = tot;
    }
    griddep_wait();
    if (a.head) {
        for (int k = tid; k < N; k += nth) {
            const int kt = k / a.BT, kl = k - kt * a.BT;
            const size_t hbase = ((size_t)kt * n_lt + l / a.LT) * a.tile_elems + (size_t)ll * a.BT + kl;
            const size_t xbase = (((size_t)kt * a.K + a.slot0) * a.n_src) * a.BT + kl;
            float2 hd = make_float2(0.0f, 0.0f);
            for (int q = 0; q < a.n_src; ++q) {
                const float2 h = St::load1(a.H, hbase + (size_t)q * LTt * a.BT, kl, a.BT);
                const float2 x = St::load1(a.X, xbase + (size_t)q * a.BT, kl, a.BT);
                float2 t = make_float2(0.0f, 0.0f);
                if (k == 0)
                    rmac2(t, h, x);
                else
                    cmac(t, h, x);
                const float sc = PREC == PREC_FP32 ? 1.0f
                                                   : __ldg(a.sH + (size_t)(l / a.LT) * a.R + q) *
                                                         __ldg(a.sX + (size_t)a.slot0 * a.n_src + q);
                hd.x = fmaf(sc, t.x, hd.x);
                hd.y = fmaf(sc, t.y, hd.y);
            }
            P[k] = cadd(P[k], hd);
        }
    }
    __syncthreads();
    if (push.X) {
        const float scale =
            store_spectrum<PREC>(P, N, push.BT, push.X, RingIndex{push.BT, push.n_ch, l, push.K, push.slot}, red);
        if (PREC != PREC_FP32 && tid == 0) push.sX[(size_t)push.slot * push.n_ch + l] = scale;
    }
    for (int k = tid; k < N; k += nth) W[k] = c2r_pre(P, k, N, tws);
    __syncthreads();
    const float2* z = fft_mixed_smem<true>(W, P, N, a.log2B - 1, tws, 2 * N, tid, nth);
    const float invN = 1.0f / (float)N;
    float* out = a.out + (size_t)l * a.out_stride;
    for (int t = tid; t < B; t += nth) {
        const int u = 2 * B + t, n = u >> 1;
        out[t] = ((u & 1) ? z[n].y : z[n].x) * invN;
    }
}

template <int PREC>
__global__ void k_out3(const OutArgs a, const PackArgs push) {
    out3_body<PREC>(a, push, blockIdx.x);
}

// Launch with programmatic stream serialization (see launch_pdl in kernels.cu).
template <typename Kern, typename... Args>
cudaError_t launch_pdl3(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

size_t fft3_smem_bytes(int B) { return (size_t)4 * (3 * (size_t)B / 2) * sizeof(float2); }

cudaError_t prepare_reuse_kernels() {
    const int mx = (int)fft3_smem_bytes(4096);
    cudaError_t e;
#define GB_ATTR3(kern)                                                                        \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
    if (e != cudaSuccess) return e;
    GB_ATTR3(k_pack3<PREC_FP32>)
    GB_ATTR3(k_pack3<PREC_FP16>)
    GB_ATTR3(k_pack3<PREC_BF16>)
    GB_ATTR3(k_filter3<PREC_FP32>)
    GB_ATTR3(k_filter3<PREC_FP16>)
    GB_ATTR3(k_filter3<PREC_BF16>)
    GB_ATTR3(k_out3<PREC_FP32>)
    GB_ATTR3(k_out3<PREC_FP16>)
    GB_ATTR3(k_out3<PREC_BF16>)
#undef GB_ATTR3
    return cudaSuccess;
}

cudaError_t launch_pack3(int prec, const PackArgs& a, cudaStream_t s) {
    if (a.B < 32 || a.B > 4096 || (a.B & (a.B - 1))) return cudaErrorInvalidValue;
    const dim3 grid(a.n_ch), block(out_threads(a.B));
    const size_t sm = fft3_smem_bytes(a.B);
    switch (prec) {
        case PREC_FP32: return launch_pdl3(k_pack3<PREC_FP32>, grid, block, sm, s, a);
        case PREC_FP16: return launch_pdl3(k_pack3<PREC_FP16>, grid, block, sm, s, a);
        case PREC_BF16: return launch_pdl3(k_pack3<PREC_BF16>, grid, block, sm, s, a);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_filter3(int prec, const FilterArgs& a, cudaStream_t s) {
    if (a.B < 32 || a.B > 4096 || (a.B & (a.B - 1))) return cudaErrorInvalidValue;
    const long long n = (long long)a.n_dst * a.n_src * a.K;
    if (n <= 0 || n > 0x7fffffffLL) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)n), block(fft_threads(2 * a.B));
    const size_t sm = fft3_smem_bytes(a.B);
    switch (prec) {
        case PREC_FP32: k_filter3<PREC_FP32><<<grid, block, sm, s>>>(a); break;
        case PREC_FP16: k_filter3<PREC_FP16><<<grid, block, sm, s>>>(a); break;
        case PREC_BF16: k_filter3<PREC_BF16><<<grid, block, sm, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_out3(int prec, const OutArgs& a, const PackArgs& push, cudaStream_t s) {
    if (a.B < 32 || a.B > 4096 || (a.B & (a.B - 1))) return cudaErrorInvalidValue;
    if (push.X && (push.n_ch != a.n_dst || push.B != a.B)) return cudaErrorInvalidValue;
    const dim3 grid(a.n_dst), block(out_threads(a.B));
    const size_t sm = fft3_smem_bytes(a.B);
    switch (prec) {
        case PREC_FP32: return launch_pdl3(k_out3<PREC_FP32>, grid, block, sm, s, a, push);
        case PREC_FP16: return launch_pdl3(k_out3<PREC_FP16>, grid, block, sm, s, a, push);
        case PREC_BF16: return launch_pdl3(k_out3<PREC_BF16>, grid, block, sm, s, a, push);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbconv
