// group.cu - kernels of shared-filter session groups (see group.h): filter
// tiles, pack + R2C into the duplicated-slot ring, the tcgen05 tensor-core
// FDL MAC, and the split reduction + C2R.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "device_util.cuh"
#include "group.h"

namespace gbconv {

namespace {

constexpr uint64_t GRP_WAIT_NS = 1000000000ull;  // 1 s: far beyond any legitimate wait
constexpr int TILE_BYTES = 8192;                 // one K-step of filter tiles: Hr 4 KiB + Hi 4 KiB

// ------------------------------------------------------------ tcgen05 helpers

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// byte offset (between core matrices along K), stride byte offset (between
// 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// D[tmem] (+)= A * B, kind::f16, issued by one thread.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

// The mbarrier receives one arrival when every tcgen05 operation this thread
// issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Eight consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

template <int PREC>
__device__ __forceinline__ uint16_t to16(float v) {
    if (PREC == PREC_FP16) {
        v = fminf(fmaxf(v, -65504.0f), 65504.0f);  // saturate instead of overflowing to inf
        const __half h = __float2half_rn(v);
        return *reinterpret_cast<const uint16_t*>(&h);
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&h);
}

__device__ void report(int* err, volatile int* abort_flag, int code) {
    *abort_flag = 1;
    if (err) atomicExch(err, code);
}

// --------------------------------------------------------------- filter tiles
// One CTA per (output l, input q, partition p < K).  Pass 0 records the
// largest component per (bin, output); pass 1 stores the spectrum divided by
// the row's power-of-two scale into the tile layout of group.h.
template <int PREC>
__global__ void k_group_filter(const GroupFilterArgs a) {
    extern __shared__ float2 fsm[];
    const int B = a.B, half = B >> 1, tid = threadIdx.x, nth = blockDim.x;
    float2* bufA = fsm;
    float2* bufB = fsm + B;
    float2* tws = fsm + 2 * B;
    const long long id = blockIdx.x;
    const int p = (int)(id % a.K);
    const long long rest = id / a.K;
    const int q = (int)(rest % a.n_src);
    const int l = (int)(rest / a.n_src);
    load_twiddles(tws, a.tw, B);
    const float* h = a.h + ((size_t)l * a.n_src + q) * (size_t)a.taps;
    const long long t0 = (long long)p * B;
    for (int n = tid; n < B; n += nth) {
        float2 z = make_float2(0.0f, 0.0f);
        if (n < half) {
            const long long t = t0 + 2 * n;
            if (t < a.taps) z.x = h[t];
            if (t + 1 < a.taps) z.y = h[t + 1];
        }
        bufA[n] = z;
    }
    __syncthreads();
    const float2* Z = fft_smem<false>(bufA, bufB, B, a.log2B, tws, a.log2B + 1, tid, nth);
    for (int k = tid; k < B; k += nth) {
        const float2 X = r2c_post(Z, k, B, tws);
        unsigned* mb = a.maxbits + (size_t)k * a.n_dst + l;
        if (a.pass == 0) {
            atomicMax(mb, __float_as_uint(fmaxf(fabsf(X.x), fabsf(X.y))));  // non-negative floats order as integers
            continue;
        }
        const float scale = block_scale<PREC>(__uint_as_float(*mb));
        const int g = k / a.G, b = k - g * a.G;
        const int row = b * a.n_dst + l;
        if (q == 0 && p == 0) a.sH[(size_t)g * 128 + row] = scale;
        const int c = p / a.KP;
        const int kk = (p - c * a.KP) * a.n_src + q;
        const size_t off = ((size_t)g * a.NKS + c) * TILE_BYTES + (size_t)(kk >> 3) * 2048 + (size_t)(row >> 3) * 128 +
                           (size_t)(row & 7) * 16 + (size_t)(kk & 7) * 2;
        unsigned char* H = static_cast<unsigned char*>(a.H);
        const float inv = 1.0f / scale;
        *reinterpret_cast<uint16_t*>(H + off) = to16<PREC>(X.x * inv);
        *reinterpret_cast<uint16_t*>(H + off + 4096) = to16<PREC>(X.y * inv);
    }
}

// ------------------------------------------------------------- pack + R2C
// One CTA per (input q, session s): w = [previous block, this block], R2C,
// then every bin's (re, im) goes to the D ring rows that hold this slot.
template <int PREC>
__global__ void k_group_pack(const GroupPackArgs a) {
    extern __shared__ float2 fsm[];
    const int B = a.B, half = B >> 1, tid = threadIdx.x, nth = blockDim.x;
    float2* bufA = fsm;
    float2* bufB = fsm + B;
    float2* tws = fsm + 2 * B;
    const int q = blockIdx.x, s = blockIdx.y;
    load_twiddles(tws, a.tw, B);
    const float* in = a.in + ((size_t)s * a.n_src + q) * a.in_stride;
    float* win = a.win + ((size_t)s * a.n_src + q) * B;
    for (int n = tid; n < B; n += nth) {
        bufA[n] = n < half ? make_float2(win[2 * n], win[2 * n + 1]) : make_float2(in[2 * n - B], in[2 * n - B + 1]);
    }
    __syncthreads();
    for (int t = tid; t < B; t += nth) win[t] = in[t];
    const float2* Z = fft_smem<false>(bufA, bufB, B, a.log2B, tws, a.log2B + 1, tid, nth);
    unsigned char* X = static_cast<unsigned char*>(a.X);
    const int rows_per_class = a.KR / a.D;
    for (int k = tid; k < B; k += nth) {
        const float2 v = r2c_post(Z, k, B, tws);
        const int g = k / a.G, b = k - g * a.G;
        const uint16_t re = to16<PREC>(v.x), im = to16<PREC>(v.y);
        for (int u = 0; u < a.D; ++u) {
            int t = a.slot - u;
            if (t < 0) t += a.KR;
            const size_t row = ((size_t)g * a.D + t % a.D) * rows_per_class + t / a.D;
            unsigned char* base = X + row * a.RB + (size_t)s * 16 + (size_t)(u * a.n_src + q) * 2;
            *reinterpret_cast<uint16_t*>(base + (size_t)b * a.S * 16) = re;
            *reinterpret_cast<uint16_t*>(base + (size_t)(a.G + b) * a.S * 16) = im;
        }
    }
}

// ------------------------------------------------------------ tensor-core MAC
// One CTA per run of (bin group, tail K-step) units (GroupTiling), at most
// one CTA per SM.
//   warp 0     producer: bulk copies of filter tiles and ring rows into a ring
//              of pipeline stages (mbarrier complete_tx)
//   warp 1     allocates tensor memory; one lane issues two MMAs per K-step
//              (D1 = Hr X into columns [0, N), D2 = Hi X into [N, 2N) of the
//              segment's accumulator buffer) and commits each stage back to the
//              producer and each finished segment to the epilogue
//   warps 2-5  epilogue: each reads its TMEM lane quadrant (32 rows), keeps
//              the diagonal blocks, forms the complex result, writes the
//              segment's partial slot and hands the buffer back
// Every wait is bounded; a timeout raises the abort flag and the error word.
__global__ void __launch_bounds__(GRP_THREADS, 1) k_group_mac(const GroupMacArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + GRP_MAX_STAGES;
    uint64_t* accb = empty + GRP_MAX_STAGES;  // [2] segment accumulated, by buffer
    uint64_t* tfree = accb + 2;               // [2] buffer read out, by buffer
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tfree + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    unsigned char* stages = smem + GRP_HDR_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cta = blockIdx.x;
    const long long U = (long long)a.NG * a.T;
    const long long lo = (long long)cta * U / a.C, hi = (long long)(cta + 1) * U / a.C;
    const int rows_per_class = a.KR / a.D;
    const int cl = a.slot0 % a.D;

    if (tid == 0) {
        for (int i = 0; i < a.nstage; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accb + b, 1);
            mbar_init(tfree + b, 128);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // a ring class is read again only two blocks later, after ~300 MB of
            // other traffic: the ring is not kept in L2 (evict-last on the ring
            // measured slower on GB300); the filter tiles of the first keep_c
            // K-steps are, so that the next block finds them there
            const uint64_t pol_h = policy_evict_first(), pol_x = policy_evict_first();
            const uint64_t pol_keep = policy_evict_last();
            int f = 0;
            bool ok = true;
            for (long long u = lo; u < hi && ok;) {
                const int g = (int)(u / a.T);
                const long long se = min(hi, (long long)(g + 1) * a.T);
                const unsigned char* xb =
                    static_cast<const unsigned char*>(a.X) + ((size_t)g * a.D + cl) * rows_per_class * a.RB;
                const unsigned char* hb = static_cast<const unsigned char*>(a.H) + (size_t)g * a.NKS * TILE_BYTES;
                for (long long v = u; v < se; v += a.NK, ++f) {
                    const int st = f % a.nstage;
                    if (f >= a.nstage &&
                        !mbar_wait_bounded(empty + st, (uint32_t)((f / a.nstage) - 1) & 1u, abort_flag, GRP_WAIT_NS)) {
                        report(a.err, abort_flag, DEVERR_TIMEOUT_PRODUCER);
                        ok = false;
                        break;
                    }
                    const int nk = (int)min((long long)a.NK, se - v);
                    const int c = 1 + (int)(v - (long long)g * a.T);
                    unsigned char* sA = stages + (size_t)st * a.stage_bytes;
                    unsigned char* sB = sA + (size_t)a.NK * TILE_BYTES;
                    mbar_arrive_expect_tx(full + st, (uint32_t)nk * (TILE_BYTES + 2u * a.RB));
                    bulk_g2s(sA, hb + (size_t)c * TILE_BYTES, (uint32_t)nk * TILE_BYTES, full + st,
                             c < a.keep_c ? pol_keep : pol_h);
                    const int idx = ((a.slot0 + c * a.KP) % a.KR) / a.D;
                    const int rows = 2 * nk;
                    const int first = min(rows, rows_per_class - idx);
                    bulk_g2s(sB, xb + (size_t)idx * a.RB, (uint32_t)(first * a.RB), full + st, pol_x);
                    if (first < rows)
                        bulk_g2s(sB + (size_t)first * a.RB, xb, (uint32_t)((rows - first) * a.RB), full + st, pol_x);
                }
                u = se;
            }
            // leave no copy in flight: wait (bounded) for the stages issued last
            for (int j = max(0, f - a.nstage); j < f; ++j)
                mbar_wait_bounded(full + j % a.nstage, (uint32_t)(j / a.nstage) & 1u, nullptr, GRP_WAIT_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t sbase = smem_u32(stages);
            int f = 0, seg = 0;
            bool ok = true;
            for (long long u = lo; u < hi && ok; ++seg) {
                const int g = (int)(u / a.T);
                const long long se = min(hi, (long long)(g + 1) * a.T);
                const int b = seg % a.nbuf, m = seg / a.nbuf;
                if (m > 0 && !mbar_wait_bounded(tfree + b, (uint32_t)(m - 1) & 1u, abort_flag, GRP_WAIT_NS)) {
                    report(a.err, abort_flag, DEVERR_TIMEOUT_CONSUMER);
                    break;
                }
                tmem_fence_after();
                const uint32_t dacc = tbase + (uint32_t)(b * 2 * a.N);
                uint32_t acc = 0u;
                for (long long v = u; v < se; v += a.NK, ++f) {
                    const int st = f % a.nstage;
                    if (!mbar_wait_bounded(full + st, (uint32_t)(f / a.nstage) & 1u, abort_flag, GRP_WAIT_NS)) {
                        report(a.err, abort_flag, DEVERR_TIMEOUT_CONSUMER);
                        ok = false;
                        break;
                    }
                    tmem_fence_after();
                    const int nk = (int)min((long long)a.NK, se - v);
                    const uint32_t sA = sbase + (uint32_t)(st * a.stage_bytes);
                    const uint32_t sB = sA + (uint32_t)(a.NK * TILE_BYTES);
                    for (int j = 0; j < nk; ++j) {
                        const uint64_t dAr = umma_desc(sA + (uint32_t)(j * TILE_BYTES), 2048, 128);
                        const uint64_t dAi = umma_desc(sA + (uint32_t)(j * TILE_BYTES) + 4096, 2048, 128);
                        const uint64_t dB = umma_desc(sB + (uint32_t)(j * 2 * a.RB), (uint32_t)a.RB, 128);
                        umma_f16(dacc, dAr, dB, a.idesc, acc);
                        umma_f16(dacc + (uint32_t)a.N, dAi, dB, a.idesc, acc);
                        acc = 1u;
                    }
                    umma_commit(empty + st);
                }
                umma_commit(accb + b);  // arrives once every MMA of the segment has completed
                u = se;
            }
        }
    } else {
        const int quad = warp & 3;  // the TMEM lane quadrant this warp may access
        const int row = quad * 32 + lane;
        const int bq = 32 / a.n_dst;  // bins per quadrant
        const int b_lo = quad * bq;
        const int mb = row / a.n_dst, l = row - mb * a.n_dst;  // this lane's bin (in the group) and output
        const int GS = a.G * a.S;
        int seg = 0;
        for (long long u = lo; u < hi; ++seg) {
            const int g = (int)(u / a.T);
            const long long se = min(hi, (long long)(g + 1) * a.T);
            const int b = seg % a.nbuf, m = seg / a.nbuf;
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(accb + b, (uint32_t)m & 1u, abort_flag, GRP_WAIT_NS));
            if (!ok && lane == 0) report(a.err, abort_flag, DEVERR_TIMEOUT_CONSUMER);
            tmem_fence_after();
            const int j = cta - group_cta_of_unit((long long)g * a.T, U, a.C);  // this CTA's slot in group g
            const int k = g * a.G + mb;
            const float scale = __ldg(a.sH + (size_t)g * 128 + row);
            const uint32_t dl = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * 2 * a.N);
            // the quadrant's bins own columns [b_lo S, (b_lo + bq) S) of each part; read them
            // in aligned runs of 8 and let each lane keep the columns of its own bin
            const int c_lo = (b_lo * a.S) & ~7, c_hi = ((b_lo + bq) * a.S + 7) & ~7;
            for (int c = c_lo; c < c_hi; c += 8) {
                float d1r[8], d1i[8], d2r[8], d2i[8];
                if (ok) {
                    tmem_ld8(dl + (uint32_t)c, d1r);
                    tmem_ld8(dl + (uint32_t)(GS + c), d1i);
                    tmem_ld8(dl + (uint32_t)(a.N + c), d2r);
                    tmem_ld8(dl + (uint32_t)(a.N + GS + c), d2i);
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int col = c + e, bin = col / a.S, sess = col - bin * a.S;
                    if (bin != mb) continue;
                    float2 y = make_float2(0.0f, 0.0f);
                    if (ok) {
                        y = k == 0 ? make_float2(d1r[e], d2i[e]) : make_float2(d1r[e] - d2i[e], d1i[e] + d2r[e]);
                        y = cscale(y, scale);
                    }
                    a.partial[(((size_t)sess * a.SP + j) * a.n_dst + l) * a.B + k] = y;
                }
            }
            tmem_fence_before();
            mbar_arrive(tfree + b);
            u = se;
        }
    }
    tmem_fence_before();
    __syncthreads();
    __syncwarp();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(a.tmem_cols) : "memory");
}

template <int PREC>
__device__ __forceinline__ void unpack8(const uint4 w, float (&v)[8]) {
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = PREC == PREC_FP16 ? unpack_half2(u[i]) : unpack_bf162(u[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// --------------------------------------------------- head + reduction + C2R
// One CTA per (output l, session s): K-step 0 of this block (partitions
// 0 .. KP-1, the only ones that need this block's spectrum) from the filter
// tiles and ring rows, plus the fixed-order sum of the tail's SP split
// partials; then C2R, 1/B scaling, keep the last B samples (overlap-save).
template <int PREC>
__global__ void k_group_out(const GroupOutArgs a) {
    extern __shared__ float2 fsm[];
    const int B = a.B, tid = threadIdx.x, nth = blockDim.x;
    float2* P = fsm;
    float2* W = fsm + B;
    float2* tws = fsm + 2 * B;
    const int l = blockIdx.x, s = blockIdx.y;
    load_twiddles(tws, a.tw, B);
    const size_t stride = (size_t)a.n_dst * B;
    const float2* src0 = a.partial + ((size_t)s * a.SP * a.n_dst + l) * B;
    const long long U = (long long)(B / a.G) * a.T;
    const int rows_per_class = a.KR / a.D;
    const int cl = a.slot0 % a.D;
    const int idx0 = a.slot0 / a.D, idx1 = (idx0 + 1) % rows_per_class;  // ring rows t0 = slot0, t1 = slot0 + D
    const unsigned char* Hb = static_cast<const unsigned char*>(a.H);
    const unsigned char* Xb = static_cast<const unsigned char*>(a.X);
    for (int k = tid; k < B; k += nth) {
        const int g = k / a.G, b = k - g * a.G, row = b * a.n_dst + l;
        // the tail CTAs that covered group g wrote slots 0 .. n-1, summed in that order
        const int n = a.C ? group_cta_of_unit((long long)(g + 1) * a.T - 1, U, a.C) -
                                group_cta_of_unit((long long)g * a.T, U, a.C) + 1
                          : 0;
        float2 tot = make_float2(0.0f, 0.0f);
        for (int sp = 0; sp < n; ++sp) tot = cadd(tot, src0[(size_t)sp * stride + k]);
        const unsigned char* ht = Hb + (size_t)g * a.NKS * TILE_BYTES + (size_t)(row >> 3) * 128 + (size_t)(row & 7) * 16;
        const size_t cls = ((size_t)g * a.D + cl) * rows_per_class;
        float2 hd = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
            const unsigned char* xr = Xb + (cls + (kc ? idx1 : idx0)) * a.RB + (size_t)s * 16;
            float hr[8], hi[8], xre[8], xim[8];
            unpack8<PREC>(*reinterpret_cast<const uint4*>(ht + kc * 2048), hr);
            unpack8<PREC>(*reinterpret_cast<const uint4*>(ht + kc * 2048 + 4096), hi);
            unpack8<PREC>(*reinterpret_cast<const uint4*>(xr + (size_t)b * a.S * 16), xre);
            unpack8<PREC>(*reinterpret_cast<const uint4*>(xr + (size_t)(a.G + b) * a.S * 16), xim);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (k == 0) {  // packed DC and Nyquist: two real products
                    hd.x = fmaf(hr[e], xre[e], hd.x);
                    hd.y = fmaf(hi[e], xim[e], hd.y);
                } else {
                    hd.x = fmaf(hr[e], xre[e], fmaf(-hi[e], xim[e], hd.x));
                    hd.y = fmaf(hr[e], xim[e], fmaf(hi[e], xre[e], hd.y));
                }
            }
        }
        P[k] = cadd(tot, cscale(hd, __ldg(a.sH + (size_t)g * 128 + row)));
    }
    __syncthreads();
    for (int k = tid; k < B; k += nth) W[k] = c2r_pre(P, k, B, tws);
    __syncthreads();
    const float2* z = fft_smem<true>(W, P, B, a.log2B, tws, a.log2B + 1, tid, nth);
    const float invB = 1.0f / (float)B;
    float* out = a.out + ((size_t)s * a.n_dst + l) * a.out_stride;
    for (int t = tid; t < B; t += nth) {
        const int u = B + t, n = u >> 1;
        out[t] = ((u & 1) ? z[n].y : z[n].x) * invB;
    }
}

}  // namespace

// ---------------------------------------------------------------- planning

const char* plan_group(int prec, int B, int n_src, int n_dst, long long taps, int S, int num_sms, GroupPlan* out,
                       const GroupTiling& t) {
    if (prec != PREC_FP16 && prec != PREC_BF16) return "session groups store FP16 or BF16 spectra";
    if (B < 16 || B > 4096 || (B & (B - 1))) return "block must be a power of two in [16, 4096]";
    if (n_dst != 8 && n_dst != 16 && n_dst != 32) return "session groups need n_out in {8, 16, 32}";
    if (n_src != 1 && n_src != 2 && n_src != 4 && n_src != 8) return "session groups need n_in in {1, 2, 4, 8}";
    if (!(S == 1 || S == 2 || S == 4 || (S >= 8 && S % 8 == 0))) return "sessions must be 1, 2, 4 or a multiple of 8";
    if (taps < 1) return "taps must be >= 1";
    if (num_sms < 1) return "num_sms must be >= 1";
    if (t.ctas < 0) return "ctas must be >= 0";
    if (t.stage_k_steps < 0 || t.stage_k_steps > 4) return "stage_k_steps must be in [0, 4]";
    if (t.stages < 0 || t.stages == 1 || t.stages > GRP_MAX_STAGES) return "stages must be 0 or in [2, 8]";
    if (t.tail_streams < 0 || t.tail_streams > 2) return "tail_streams must be 0, 1 or 2";
    GroupPlan p{};
    p.B = B;
    p.n_src = n_src;
    p.n_dst = n_dst;
    p.S = S;
    p.G = 128 / n_dst;
    if (p.G * S > 128) return "sessions x (128 / n_out) must be <= 128";
    if (p.G * S < 8) return "sessions x (128 / n_out) must be >= 8 (MMA N >= 16)";
    const long long K = (taps + B - 1) / B;
    p.D = 8 / n_src;
    p.KP = 2 * p.D;
    const long long KR = (K + p.KP - 1) / p.KP * p.KP;
    if (KR > (1LL << 24)) return "too many partitions";
    p.K = (int)K;
    p.KR = (int)KR;
    p.NKS = p.KR / p.KP;
    p.NG = B / p.G;
    p.N = 2 * p.G * S;
    p.RB = 32 * p.G * S;
    p.nbuf = 4 * p.N <= 512 ? 2 : 1;
    p.tmem_cols = 32;
    while (p.tmem_cols < p.nbuf * 2 * p.N) p.tmem_cols *= 2;
    p.tail_streams = t.tail_streams ? t.tail_streams : 2;
    const int kb = TILE_BYTES + 2 * p.RB;
    // stages stay below ~180 KB so that the pack and output kernels of the
    // next block fit beside a MAC CTA on every SM
    const int budget = 180 * 1024 - GRP_HDR_BYTES;
    // measured on GB300 (8 and 16 sessions of the 4x16 paper set): the largest
    // stages that still give 3 in flight stream best; 1 K-step per stage starves
    // the MMA
    p.NK = t.stage_k_steps ? t.stage_k_steps : (3 * 4 * kb <= budget ? 4 : (3 * 3 * kb <= budget ? 3 : 2));
    p.nstage = t.stages ? t.stages : std::min(6, budget / (p.NK * kb));
    if (p.nstage < 2 || p.nstage * p.NK * kb > budget) return "pipeline stages do not fit in shared memory";
    p.stage_bytes = p.NK * kb;
    // at most one MAC CTA per SM: its tensor memory may be all of the SM's
    p.smem = std::max(GRP_HDR_BYTES + p.nstage * p.stage_bytes, 116 * 1024);
    p.T = p.NKS - 1;
    const long long U = (long long)p.NG * p.T;
    // default: all but 8 SMs, where the next block's pack and output kernels run
    // at once (with a MAC CTA on every SM they wait for the tail to drain)
    const int c_auto = std::max(1, num_sms > 16 ? num_sms - 8 : num_sms);
    p.C = U > 0 ? (int)std::min<long long>(U, t.ctas ? std::min(t.ctas, num_sms) : c_auto) : 0;
    p.SP = 0;
    for (int g = 0; g < p.NG && p.C; ++g) {
        const int n = group_cta_of_unit((long long)(g + 1) * p.T - 1, U, p.C) -
                      group_cta_of_unit((long long)g * p.T, U, p.C) + 1;
        p.SP = std::max(p.SP, n);
    }
    p.h_bytes = (size_t)p.NG * p.NKS * TILE_BYTES;
    p.x_bytes = (size_t)p.NG * p.KR * p.RB;
    p.partial_bytes = (size_t)S * p.SP * n_dst * B * sizeof(float2);
    *out = p;
    return nullptr;
}

const char* check_group_plan(const GroupPlan& p) {
    static thread_local char msg[256];
    if (p.G * p.n_dst != 128 || p.NG * p.G != p.B) return "group shape does not tile 128 rows / B bins";
    if (p.N % 16 || p.N < 16 || p.N > 256) return "MMA N out of range";
    if (p.nbuf < 1 || p.nbuf > 2 || p.nbuf * 2 * p.N > p.tmem_cols || p.tmem_cols > 512) return "tensor memory columns";
    if (p.RB % 16 || p.stage_bytes % 16) return "copy sizes must be multiples of 16 bytes";
    if ((size_t)p.smem > 227 * 1024) return "shared memory above the per-CTA limit";
    if (p.smem <= 114 * 1024) return "shared memory small enough for two MAC CTAs on one SM";
    if ((p.G * p.S) % 8) return "columns of a part must be a multiple of 8";
    if (p.nstage < 2 || p.nstage > GRP_MAX_STAGES) return "pipeline depth";
    if ((size_t)p.stage_bytes * p.nstage + GRP_HDR_BYTES > (size_t)p.smem) return "stages beyond shared memory";
    if (p.T != p.NKS - 1 || (p.T > 0) != (p.C > 0)) return "tail shape";
    const long long U = (long long)p.NG * p.T;
    if (p.C > U) return "more tail CTAs than units";
    const int rows_per_class = p.KR / p.D;
    long long covered = 0;
    for (int cta = 0; cta < p.C; ++cta) {
        const long long lo = (long long)cta * U / p.C, hi = (long long)(cta + 1) * U / p.C;
        if (hi <= lo) return "empty tail run";
        covered += hi - lo;
        for (long long u = lo; u < hi;) {
            const int g = (int)(u / p.T);
            const long long se = std::min(hi, (long long)(g + 1) * p.T);
            const int j = cta - group_cta_of_unit((long long)g * p.T, U, p.C);
            if (j < 0 || j >= p.SP) {
                snprintf(msg, sizeof(msg), "partial slot %d of CTA %d in group %d outside [0, %d)", j, cta, g, p.SP);
                return msg;
            }
            if (group_cta_of_unit(u, U, p.C) != cta) return "unit owner mismatch";
            for (int slot0 = 0; slot0 < std::min(p.KR, 2 * p.D + 1); ++slot0)
                for (long long v = u; v < se; v += p.NK) {
                    const int nk = (int)std::min((long long)p.NK, se - v);
                    const int c = 1 + (int)(v - (long long)g * p.T);
                    if (c < 1 || c + nk > p.NKS) return "K-step outside the tail";
                    if (((size_t)g * p.NKS + c + nk) * TILE_BYTES > p.h_bytes) return "filter copy beyond the tiles";
                    const int t0 = (slot0 + c * p.KP) % p.KR;
                    if (t0 % p.D != slot0 % p.D) return "ring class changes within a block";
                    const int idx = t0 / p.D, rows = 2 * nk;
                    const int first = std::min(rows, rows_per_class - idx);
                    const size_t cls_base = ((size_t)g * p.D + slot0 % p.D) * rows_per_class;
                    if ((cls_base + idx + first) * p.RB > p.x_bytes) return "ring copy beyond the ring";
                    if (rows - first > rows_per_class) return "ring copy wraps twice";
                    for (int jj = 0; jj < nk; ++jj) {  // the rows of K-step c are t0 and t0 + D
                        const int ta = (slot0 + (c + jj) * p.KP) % p.KR, tb = (ta + p.D) % p.KR;
                        const int ia = (idx + 2 * jj) % rows_per_class, ib = (idx + 2 * jj + 1) % rows_per_class;
                        if (ta / p.D != ia || tb / p.D != ib) {
                            snprintf(msg, sizeof(msg), "ring row order: slot0 %d K-step %d", slot0, c + jj);
                            return msg;
                        }
                    }
                }
            u = se;
        }
    }
    if (covered != U) return "tail runs do not cover every unit once";
    for (int g = 0; g < p.NG && p.C; ++g) {
        const int n = group_cta_of_unit((long long)(g + 1) * p.T - 1, U, p.C) -
                      group_cta_of_unit((long long)g * p.T, U, p.C) + 1;
        if (n < 1 || n > p.SP) return "group slot count";
    }
    if ((size_t)p.S * p.SP * p.n_dst * p.B * sizeof(float2) != p.partial_bytes) return "partial buffer size";
    return nullptr;
}

// ---------------------------------------------------------------- launchers

cudaError_t prepare_group_kernels() {
    const int fft_max = (int)fft_smem_bytes(4096);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_group_filter<PREC_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_max)))
        return e;
    if ((e = cudaFuncSetAttribute(k_group_filter<PREC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_max)))
        return e;
    if ((e = cudaFuncSetAttribute(k_group_pack<PREC_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_max)))
        return e;
    if ((e = cudaFuncSetAttribute(k_group_pack<PREC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_max)))
        return e;
    if ((e = cudaFuncSetAttribute(k_group_out<PREC_FP16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_max)))
        return e;
    if ((e = cudaFuncSetAttribute(k_group_out<PREC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_max)))
        return e;
    return cudaFuncSetAttribute(k_group_mac, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t launch_group_filter(int prec, const GroupFilterArgs& a, cudaStream_t s) {
    const long long n = (long long)a.n_dst * a.n_src * a.K;
    if (n <= 0 || n > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t sm = fft_smem_bytes(a.B);
    if (prec == PREC_FP16)
        k_group_filter<PREC_FP16><<<(unsigned)n, fft_threads(a.B), sm, s>>>(a);
    else
        k_group_filter<PREC_BF16><<<(unsigned)n, fft_threads(a.B), sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_group_pack(int prec, const GroupPackArgs& a, cudaStream_t s) {
    const dim3 grid(a.n_src, a.S);
    const size_t sm = fft_smem_bytes(a.B);
    if (prec == PREC_FP16)
        k_group_pack<PREC_FP16><<<grid, fft_threads(a.B), sm, s>>>(a);
    else
        k_group_pack<PREC_BF16><<<grid, fft_threads(a.B), sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_group_mac(const GroupPlan& p, const GroupMacArgs& a, cudaStream_t s) {
    if (p.C == 0) return cudaSuccess;
    k_group_mac<<<p.C, GRP_THREADS, p.smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_group_out(int prec, const GroupOutArgs& a, cudaStream_t s) {
    const dim3 grid(a.n_dst, a.S);
    if (prec == PREC_FP16)
        k_group_out<PREC_FP16><<<grid, out_threads(a.B), fft_smem_bytes(a.B), s>>>(a);
    else
        k_group_out<PREC_BF16><<<grid, out_threads(a.B), fft_smem_bytes(a.B), s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbconv
