// nlms.cu - kernels of the adaptive feedback canceller (partitioned-block
// frequency-domain NLMS on the canceller's sub-filter spectra; see nlms.h).
//
//   nlms_prep    one CTA per microphone: R2C of [0_B | e_p] (shared-memory
//                FFT), the per-bin power recursion over the loudspeakers'
//                newest spectra, and G_p = mu E_p / (K pow + delta)
//   nlms_update  F_hat[p][l][j][k] += G_p[k] conj(U_l,j[k]) over every filter
//                tile; streams F_hat once (read + write), the delay line and
//                G come from L2
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "nlms.h"

namespace gbconv {

namespace {

__global__ void k_nlms_prep(const NlmsPrepArgs a) {
    extern __shared__ float2 fsm[];
    const int B = a.B, half = B >> 1, tid = threadIdx.x, nth = blockDim.x;
    float2* bufA = fsm;
    float2* bufB = fsm + B;
    float2* tws = fsm + 2 * B;
    const int p = blockIdx.x;
    load_twiddles(tws, a.tw, B);
    // z[n] = w[2n] + i w[2n+1] with w = [0_B | e_p]
    const float* e = a.e + (size_t)p * B;
    for (int n = tid; n < B; n += nth)
        bufA[n] = n < half ? make_float2(0.0f, 0.0f) : make_float2(e[2 * n - B], e[2 * n - B + 1]);
    __syncthreads();
    const float2* Z = fft_smem<false>(bufA, bufB, B, a.log2B, tws, a.log2B + 1, tid, nth);
    const float kf = (float)a.K;
    for (int k = tid; k < B; k += nth) {
        const float2 E = r2c_post(Z, k, B, tws);
        const int kt = k / a.BT, kl = k - kt * a.BT;
        const float2* u = a.U + ((size_t)kt * a.K + a.slot0) * a.L * a.BT + kl;
        float px = 0.0f, py = 0.0f;
        // eight loudspeaker rows per batch of independent loads, summed in order
        int l = 0;
        for (; l + 8 <= a.L; l += 8) {
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __ldg(u + (size_t)(l + i) * a.BT);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (k == 0) {
                    px = fmaf(v[i].x, v[i].x, px);
                    py = fmaf(v[i].y, v[i].y, py);
                } else {
                    px = fmaf(v[i].x, v[i].x, fmaf(v[i].y, v[i].y, px));
                }
            }
        }
        for (; l < a.L; ++l) {
            const float2 v = __ldg(u + (size_t)l * a.BT);
            if (k == 0) {
                px = fmaf(v.x, v.x, px);
                py = fmaf(v.y, v.y, py);
            } else {
                px = fmaf(v.x, v.x, fmaf(v.y, v.y, px));
            }
        }
        const float2 old = a.pow_in[k];
        float2 pw;
        pw.x = a.lam * old.x + (1.0f - a.lam) * px;
        pw.y = k == 0 ? a.lam * old.y + (1.0f - a.lam) * py : 0.0f;
        if (p == 0) a.pow_out[k] = pw;
        float2 g;
        if (k == 0) {
            g.x = a.mu * E.x / (kf * pw.x + a.delta);
            g.y = a.mu * E.y / (kf * pw.y + a.delta);
        } else {
            const float st = a.mu / (kf * pw.x + a.delta);
            g = cscale(E, st);
        }
        a.G[(size_t)p * B + k] = g;
    }
}

__global__ void __launch_bounds__(256) k_nlms_update(const NlmsUpdateArgs a) {
    const int tile = blockIdx.y;
    const int kt = tile / a.n_lt, lt = tile - kt * a.n_lt;
    const int LTt = min(a.LT, a.P - lt * a.LT);
    const int R = a.L * a.K;
    const int r0 = blockIdx.x * a.rows_per_cta;
    const int r1 = min(R, r0 + a.rows_per_cta);
    if (r0 >= r1) return;
    const int row = LTt * a.BT;
    float2* __restrict__ Ft = a.F + (size_t)tile * a.tile_elems;
    const float2* __restrict__ U = a.U;
    const float2* __restrict__ G = a.G;
    for (int e = threadIdx.x; e < row; e += blockDim.x) {
        const int ll = e / a.BT, kl = e - ll * a.BT;
        const int p = lt * a.LT + ll, k = kt * a.BT + kl;
        const float2 g = G[(size_t)p * a.B + k];
        int l = r0 % a.L;
        int slot = a.slot0 + r0 / a.L;
        if (slot >= a.K) slot -= a.K;
#pragma unroll 4
        for (int r = r0; r < r1; ++r) {
            const float2 u = U[((size_t)(kt * a.K + slot) * a.L + l) * a.BT + kl];
            float2* f = Ft + (size_t)r * row + e;
            float2 v = *f;
            if (k == 0) {  // packed DC and Nyquist: two real products
                v.x = fmaf(g.x, u.x, v.x);
                v.y = fmaf(g.y, u.y, v.y);
            } else {  // v += g * conj(u)
                v.x = fmaf(g.x, u.x, fmaf(g.y, u.y, v.x));
                v.y = fmaf(g.y, u.x, fmaf(-g.x, u.y, v.y));
            }
            *f = v;
            if (++l == a.L) {
                l = 0;
                if (++slot == a.K) slot = 0;
            }
        }
    }
}

}  // namespace

cudaError_t launch_nlms_prep(const NlmsPrepArgs& a, int P, cudaStream_t s) {
    static_assert(sizeof(float2) == 8, "packed spectra are float pairs");
    const size_t sm = fft_smem_bytes(a.B);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_nlms_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    // one thread per bin (up to 256): the power sums are latency-bound loads
    const int threads = a.B < 256 ? (a.B < 64 ? 64 : a.B) : 256;
    k_nlms_prep<<<P, threads, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nlms_update(const NlmsUpdateArgs& a, cudaStream_t s) {
    const int R = a.L * a.K;
    if (a.rows_per_cta < 1 || R < 1) return cudaErrorInvalidValue;
    const int row = a.LT * a.BT;
    int threads = ((row + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    const dim3 grid((unsigned)((R + a.rows_per_cta - 1) / a.rows_per_cta), (unsigned)(a.n_kt * a.n_lt));
    k_nlms_update<<<grid, threads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbconv
