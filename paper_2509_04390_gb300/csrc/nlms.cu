// nlms.cu - kernels of the adaptive feedback canceller (partitioned-block
// frequency-domain NLMS on the canceller's sub-filter spectra; see nlms.h).
//
//   nlms_prep    one CTA per microphone: R2C of [0_B | e_p] (shared-memory
//                FFT in float-float arithmetic), the per-bin power recursion
//                over the loudspeakers' newest spectra, G_p = mu E_p /
//                (K pow + delta), and the step on partition 0
//   nlms_update  F_hat[p][l][j][k] += G_p[k] conj(U_l,j[k]) over the tail
//                partitions of every filter tile; streams them once (read +
//                write), the delay line and G come from L2
//   nlms_update_mac  the same step fused with the canceller's tail MAC of a
//                later block: each spectrum is read, stepped, written back and
//                multiplied by its delay-line entry in one pass (split partials)
//   nlms_corr    chunks of the lag-one and lag-two correlations of the delay
//                line (the deferred update's correction terms), summed by the
//                last CTA of each bin range
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "nlms.h"

namespace gbconv {

namespace {

// ------------------------------------------- float-float (compensated) FFT
// The error spectrum E = R2C([0_B | e]) sets the step of every update, and an
// FP32 FFT's rounding (~1.5e-7 relative) in E accumulates in F_hat over the
// blocks.  E is therefore computed with float-float arithmetic: each value is
// an unevaluated sum hi + lo of two floats, sums use Knuth's TwoSum and
// products the exact FMA residual, so the transform carries about 44
// significant bits before E is rounded to FP32 once.  Only FP32 operations.
struct ff {
    float hi, lo;
};
struct cff {
    ff re, im;
};

__device__ __forceinline__ ff ff_norm(float s, float e) {  // |s| >= |e| after a sum: fast renormalisation
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));  // TwoSum residual
    return ff_norm(s, __fadd_rn(err, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact residual of the product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_norm(p, e);
}
__device__ __forceinline__ cff cff_add(cff a, cff b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ __forceinline__ cff cff_sub(cff a, cff b) { return {ff_add(a.re, ff_neg(b.re)), ff_add(a.im, ff_neg(b.im))}; }
__device__ __forceinline__ cff cff_mul(cff a, cff w) {
    return {ff_add(ff_mul(a.re, w.re), ff_neg(ff_mul(a.im, w.im))), ff_add(ff_mul(a.re, w.im), ff_mul(a.im, w.re))};
}
// W_2B^j as float-float from the FP32 table and its residual table
__device__ __forceinline__ cff tw_ff(const float2* tw, const float2* tw_lo, int j) {
    const float2 h = __ldg(tw + j), l = __ldg(tw_lo + j);
    return {{h.x, l.x}, {h.y, l.y}};
}

// E[k], k < B (packed: bin 0 = (DC, Nyquist)), of the 2B-point R2C of
// w = [0_B | e]: a B-point radix-2 Stockham FFT of z[n] = w[2n] + i w[2n+1],
// then the real-FFT post-processing, all in float-float.  `a`, `b`: two
// shared buffers of B values; returns E for the calling thread's bins via
// `out` (indexed like the kernel's bin loop).
__device__ void error_spectrum_ff(const float* e, cff* a, cff* b, int B, const float2* tw, const float2* tw_lo,
                                  float2* out) {
    const int tid = threadIdx.x, nth = blockDim.x, half = B >> 1;
    const cff zero = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int n = tid; n < B; n += nth)
        a[n] = n < half ? zero : cff{{e[2 * n - B], 0.0f}, {e[2 * n - B + 1], 0.0f}};
    __syncthreads();
    for (int Ns = 1; Ns < B; Ns <<= 1) {
        for (int j = tid; j < half; j += nth) {
            const int k = j & (Ns - 1);
            const cff v0 = a[j];
            cff v1 = a[j + half];
            if (k) v1 = cff_mul(v1, tw_ff(tw, tw_lo, k * (B / Ns)));  // W_2Ns^k = W_2B^(k B / Ns)
            const int o = ((j - k) << 1) + k;
            b[o] = cff_add(v0, v1);
            b[o + Ns] = cff_sub(v0, v1);
        }
        __syncthreads();
        cff* t = a;
        a = b;
        b = t;
    }
    // a holds Z = FFT_B(z); E[k] = (Z[k] + conj Z[B-k]) / 2 + W_2B^k (Z[k] - conj Z[B-k]) / 2i
    for (int k = tid; k < B; k += nth) {
        const cff Z = a[k];
        if (k == 0) {
            out[k] = make_float2(ff_add(Z.re, Z.im).hi, ff_add(Z.re, ff_neg(Z.im)).hi);
            continue;
        }
        const cff Zm = a[B - k];
        const ff half_f = {0.5f, 0.0f};
        const cff Ev = {ff_mul(ff_add(Z.re, Zm.re), half_f), ff_mul(ff_add(Z.im, ff_neg(Zm.im)), half_f)};
        const cff D = {ff_mul(ff_add(Z.re, ff_neg(Zm.re)), half_f), ff_mul(ff_add(Z.im, Zm.im), half_f)};
        const cff O = {D.im, ff_neg(D.re)};  // D / i
        const cff r = cff_add(Ev, cff_mul(O, tw_ff(tw, tw_lo, k)));
        out[k] = make_float2(r.re.hi + r.re.lo, r.im.hi + r.im.lo);
    }
}

__global__ void k_nlms_prep(const NlmsPrepArgs a) {
    extern __shared__ __align__(16) unsigned char prep_smem[];
    const int B = a.B, tid = threadIdx.x, nth = blockDim.x;
    cff* bufA = reinterpret_cast<cff*>(prep_smem);
    cff* bufB = bufA + B;
    float2* Es = reinterpret_cast<float2*>(bufB + B);  // [B] the error spectrum, rounded once
    const int p = blockIdx.x;
    error_spectrum_ff(a.e + (size_t)p * B, bufA, bufB, B, a.tw, a.tw_lo, Es);
    __syncthreads();
    const float kf = (float)a.K;
    for (int k = tid; k < B; k += nth) {
        const float2 E = Es[k];
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
        const float2 old = a.pow_in[k];  // (the ring loads below repeat from L1/L2)
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
        // partition 0: F[p][l][0][k] += g conj(U_l,0[k])
        const int lt = p / a.LT, ll = p - lt * a.LT;
        const int LTt = min(a.LT, (int)gridDim.x - lt * a.LT);
        float2* f = a.F + (size_t)(kt * a.n_lt + lt) * a.tile_elems + (size_t)ll * a.BT + kl;
        const size_t fr = (size_t)LTt * a.BT;  // row pitch
        for (int l0 = 0; l0 < a.L; l0 += 8) {
            const int nl = min(8, a.L - l0);
            float2 v[8], w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < nl) {
                    v[i] = __ldg(u + (size_t)(l0 + i) * a.BT);
                    w[i] = f[(size_t)(l0 + i) * fr];
                }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < nl) {
                    if (k == 0) {
                        w[i].x = fmaf(g.x, v[i].x, w[i].x);
                        w[i].y = fmaf(g.y, v[i].y, w[i].y);
                    } else {
                        w[i].x = fmaf(g.x, v[i].x, fmaf(g.y, v[i].y, w[i].x));
                        w[i].y = fmaf(g.y, v[i].x, fmaf(-g.x, v[i].y, w[i].y));
                    }
                    f[(size_t)(l0 + i) * fr] = w[i];
                }
        }
    }
}

__global__ void __launch_bounds__(256) k_nlms_update(const NlmsUpdateArgs a) {
    const int tile = blockIdx.y;
    const int kt = tile / a.n_lt, lt = tile - kt * a.n_lt;
    const int LTt = min(a.LT, a.P - lt * a.LT);
    const int R = a.L * a.K;
    const int r0 = a.r_begin + blockIdx.x * a.rows_per_cta;
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
        int l = r0 % a.L, j = r0 / a.L;
        int slot = a.slot0 + j;
        if (slot >= a.K) slot -= a.K;
#pragma unroll 4
        for (int r = r0; r < r1; ++r) {
            float2 u;
            if (j == a.K - 1 && a.U_old[0])
                u = a.U_old[0][((size_t)kt * a.L + l) * a.BT + kl];
            else if (j == a.K - 2 && a.U_old[1])
                u = a.U_old[1][((size_t)kt * a.L + l) * a.BT + kl];
            else
                u = U[((size_t)(kt * a.K + slot) * a.L + l) * a.BT + kl];
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
                ++j;
                if (++slot == a.K) slot = 0;
            }
        }
    }
}

// CTA (split, filter tile); thread (element of the tile row, row lane).  Each
// lane walks every NRL-th row of the split: read F, take the step, write F
// back, accumulate F x (MAC entry); the lanes' sums are combined in shared
// memory in a fixed order into the split's partial.
__global__ void __launch_bounds__(512) k_nlms_update_mac(const NlmsUpdateMacArgs a) {
    extern __shared__ float2 lanes[];  // [NRL][row]
    const NlmsUpdateArgs& u = a.u;
    const int tile = blockIdx.y, split = blockIdx.x;
    const int kt = tile / u.n_lt, lt = tile - kt * u.n_lt;
    const int LTt = min(u.LT, u.P - lt * u.LT);
    const int R = u.L * u.K, Rt = R - u.r_begin;
    const int r0 = u.r_begin + (int)((long long)split * Rt / a.S);
    const int r1 = u.r_begin + (int)((long long)(split + 1) * Rt / a.S);
    const int row = LTt * u.BT;
    const int ET = blockDim.x, NRL = blockDim.y, ly = threadIdx.y;
    float2* __restrict__ Ft = u.F + (size_t)tile * u.tile_elems;
    for (int e = threadIdx.x; e < row; e += ET) {
        const int ll = e / u.BT, kl = e - ll * u.BT;
        const int p = lt * u.LT + ll, k = kt * u.BT + kl;
        const bool step = u.G != nullptr;
        const float2 g = step ? u.G[(size_t)p * u.B + k] : make_float2(0.0f, 0.0f);
        float2 acc = make_float2(0.0f, 0.0f);
        // eight rows per trip: all their loads are issued before any store
        for (int rb = r0 + ly; rb < r1; rb += 8 * NRL) {
            float2 fv[8], wv[8], xv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = rb + i * NRL;
                if (r < r1) {
                    const int j = r / u.L, l = r - j * u.L;
                    fv[i] = Ft[(size_t)r * row + e];
                    int sm = a.mac_slot0 + j;
                    if (sm >= u.K) sm -= u.K;
                    xv[i] = u.U[((size_t)(kt * u.K + sm) * u.L + l) * u.BT + kl];
                    if (step) {
                        if (j == u.K - 1 && u.U_old[0]) {
                            wv[i] = u.U_old[0][((size_t)kt * u.L + l) * u.BT + kl];
                        } else if (j == u.K - 2 && u.U_old[1]) {
                            wv[i] = u.U_old[1][((size_t)kt * u.L + l) * u.BT + kl];
                        } else {
                            int sl = u.slot0 + j;
                            if (sl >= u.K) sl -= u.K;
                            wv[i] = u.U[((size_t)(kt * u.K + sl) * u.L + l) * u.BT + kl];
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = rb + i * NRL;
                if (r < r1) {
                    float2 v = fv[i];
                    if (step) {
                        const float2 w = wv[i];
                        if (k == 0) {
                            v.x = fmaf(g.x, w.x, v.x);
                            v.y = fmaf(g.y, w.y, v.y);
                        } else {  // v += g * conj(w)
                            v.x = fmaf(g.x, w.x, fmaf(g.y, w.y, v.x));
                            v.y = fmaf(g.y, w.x, fmaf(-g.x, w.y, v.y));
                        }
                        Ft[(size_t)r * row + e] = v;
                    }
                    const float2 x = xv[i];
                    if (k == 0) {
                        acc.x = fmaf(v.x, x.x, acc.x);
                        acc.y = fmaf(v.y, x.y, acc.y);
                    } else {
                        acc.x = fmaf(v.x, x.x, fmaf(-v.y, x.y, acc.x));
                        acc.y = fmaf(v.x, x.y, fmaf(v.y, x.x, acc.y));
                    }
                }
            }
        }
        lanes[(size_t)ly * row + e] = acc;
    }
    __syncthreads();
    if (ly != 0) return;
    for (int e = threadIdx.x; e < row; e += ET) {
        const int ll = e / u.BT, kl = e - ll * u.BT;
        const int p = lt * u.LT + ll, k = kt * u.BT + kl;
        float2 t = lanes[e];
        for (int y = 1; y < NRL; ++y) t = cadd(t, lanes[(size_t)y * row + e]);
        a.partial[((size_t)split * u.P + p) * u.B + k] = t;
    }
}

// CTA (bin chunk, j chunk); thread (l, bin).  A window of three consecutive
// delay-line entries slides over the chunk, so each thread loads every entry
// once; the sums over loudspeakers run in shared memory in a fixed order.
__device__ __forceinline__ void conj_mac(float2& acc, float2 o, float2 n, bool packed0) {
    if (packed0) {  // DC and Nyquist: real products
        acc.x = fmaf(o.x, n.x, acc.x);
        acc.y = fmaf(o.y, n.y, acc.y);
    } else {  // acc += conj(o) n
        acc.x = fmaf(o.x, n.x, fmaf(o.y, n.y, acc.x));
        acc.y = fmaf(o.x, n.y, fmaf(-o.y, n.x, acc.y));
    }
}

__global__ void __launch_bounds__(256) k_nlms_corr(const NlmsCorrArgs a, const int BA) {
    extern __shared__ float2 red[];  // [2][L][BA]
    const int c = blockIdx.y, J = a.K - 1;
    const int j0 = 1 + (int)((long long)c * J / a.C), j1 = 1 + (int)((long long)(c + 1) * J / a.C);
    const size_t ss = (size_t)a.L * a.BT;  // slot pitch
    const int LB = a.L * BA;
    for (int e = threadIdx.x; e < LB; e += blockDim.x) {
        const int l = e / BA, kb = e - l * BA;
        const int k = blockIdx.x * BA + kb;
        const int kt = k / a.BT, kl = k - kt * a.BT;
        const float2* base = a.U + (size_t)kt * a.K * ss + (size_t)l * a.BT + kl;
        const float2 oldest = j1 == a.K ? __ldg(a.oldest + ((size_t)kt * a.L + l) * a.BT + kl) : make_float2(0.0f, 0.0f);
        int s = (a.slot_m + j0 - 1) % a.K;  // entry j0 - 1 (block m+1-j0)
        float2 nv = __ldg(base + s * ss);
        if (++s == a.K) s = 0;
        float2 o1 = __ldg(base + s * ss);  // entry j0
        float2 acc1 = make_float2(0.0f, 0.0f), acc2 = make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
            if (++s == a.K) s = 0;
            const float2 o2 = j + 1 == a.K ? oldest : __ldg(base + s * ss);  // entry j + 1
            conj_mac(acc1, o1, nv, k == 0);
            conj_mac(acc2, o2, nv, k == 0);
            nv = o1;
            o1 = o2;
        }
        red[e] = acc1;
        red[LB + e] = acc2;
    }
    __syncthreads();
    for (int kb = threadIdx.x; kb < BA; kb += blockDim.x) {
        float2 t1 = make_float2(0.0f, 0.0f), t2 = make_float2(0.0f, 0.0f);
        for (int l = 0; l < a.L; ++l) {
            t1 = cadd(t1, red[l * BA + kb]);
            t2 = cadd(t2, red[LB + l * BA + kb]);
        }
        a.A1[(size_t)c * a.B + blockIdx.x * BA + kb] = t1;
        a.A2[(size_t)c * a.B + blockIdx.x * BA + kb] = t2;
    }
    // the last of the range's C CTAs adds the chunks in order
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.ticket + blockIdx.x, 1u) == (unsigned)(a.C - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int kb = threadIdx.x; kb < BA; kb += blockDim.x) {
        const size_t k = (size_t)blockIdx.x * BA + kb;
        float2 t1 = make_float2(0.0f, 0.0f), t2 = make_float2(0.0f, 0.0f);
        for (int cc = 0; cc < a.C; ++cc) {
            t1 = cadd(t1, __ldcg(a.A1 + (size_t)cc * a.B + k));
            t2 = cadd(t2, __ldcg(a.A2 + (size_t)cc * a.B + k));
        }
        a.A1f[k] = t1;
        a.A2f[k] = t2;
    }
    if (threadIdx.x == 0) a.ticket[blockIdx.x] = 0u;
}

}  // namespace

int nlms_corr_chunks(int K) { return K < 2 ? 0 : (K - 1 < 8 ? K - 1 : 8); }

cudaError_t launch_nlms_corr(const NlmsCorrArgs& a, cudaStream_t s) {
    if (a.K < 2 || a.C < 1 || a.C > a.K - 1 || a.L < 1 || a.L > 1024 || a.B < 16 || (a.B & (a.B - 1)))
        return cudaErrorInvalidValue;
    // small CTAs (<= 256 threads) that fit beside a MAC CTA on its SM
    int BA = 1;
    while (BA * 2 * a.L <= 256 && BA * 2 <= a.B) BA *= 2;
    int threads = ((a.L * BA + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    const dim3 grid((unsigned)(a.B / BA), (unsigned)a.C);
    k_nlms_corr<<<grid, threads, 2 * (size_t)a.L * BA * sizeof(float2), s>>>(a, BA);
    return cudaGetLastError();
}

cudaError_t launch_nlms_update_mac(const NlmsUpdateMacArgs& a, cudaStream_t s) {
    const NlmsUpdateArgs& u = a.u;
    if (a.S < 1 || u.r_begin < 0 || u.L * u.K - u.r_begin < 1) return cudaErrorInvalidValue;
    const int row = u.LT * u.BT;
    const int ET = row < 256 ? ((row + 31) / 32) * 32 : 256;
    int NRL = 512 / ET;
    if (NRL > 4) NRL = 4;
    while (NRL > 1 && (size_t)NRL * row * sizeof(float2) > 48 * 1024) --NRL;
    const size_t smem = (size_t)NRL * row * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_nlms_update_mac, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_nlms_update_mac<<<dim3((unsigned)a.S, (unsigned)(u.n_kt * u.n_lt)), dim3(ET, NRL), smem, s>>>(a);
    return cudaGetLastError();
}

// two float-float buffers of B complex values and the rounded spectrum
static size_t nlms_prep_smem(int B) { return (size_t)B * (2 * sizeof(float) * 4 + sizeof(float2)); }

cudaError_t launch_nlms_prep(const NlmsPrepArgs& a, int P, cudaStream_t s) {
    static_assert(sizeof(float2) == 8, "packed spectra are float pairs");
    if (!a.tw_lo) return cudaErrorInvalidValue;
    const size_t sm = nlms_prep_smem(a.B);
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
    const int R = a.L * a.K - a.r_begin;  // rows that take the step
    if (a.rows_per_cta < 1 || a.r_begin < 0 || R < 1) return cudaErrorInvalidValue;
    const int row = a.LT * a.BT;
    int threads = ((row + 31) / 32) * 32;
    if (threads > 256) threads = 256;
    const dim3 grid((unsigned)((R + a.rows_per_cta - 1) / a.rows_per_cta), (unsigned)(a.n_kt * a.n_lt));
    k_nlms_update<<<grid, threads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbconv
