// device_util.cuh - device helpers: complex arithmetic, spectrum storage types,
// mbarrier / bulk-copy (TMA) wrappers with bounded waits, and the shared-memory
// Stockham FFT used by the pack and output kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"

namespace gbconv {

// ------------------------------------------------------------------ complex

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// acc += h * x (complex)
__device__ __forceinline__ void cmac(float2& acc, float2 h, float2 x) {
    acc.x = fmaf(h.x, x.x, acc.x);
    acc.x = fmaf(-h.y, x.y, acc.x);
    acc.y = fmaf(h.x, x.y, acc.y);
    acc.y = fmaf(h.y, x.x, acc.y);
}
// Packed bin 0: (DC, Nyquist) are two independent real products.
__device__ __forceinline__ void rmac2(float2& acc, float2 h, float2 x) {
    acc.x = fmaf(h.x, x.x, acc.x);
    acc.y = fmaf(h.y, x.y, acc.y);
}

// ------------------------------------------------------------ storage types

template <int PREC>
struct Store;

// Storage of a spectrum row of BT bins.  FP32 rows interleave (re, im);
// FP16/BF16 rows are planar in chunks of four bins, [4 real parts][4
// imaginary parts] (16 bytes), so the MAC loads a thread's four bins with one
// 16-byte load and works on pairs of bins with packed FP32x2 FMAs.  `c` is the
// complex element index (row start + kl), kl the bin within the row.
template <>
struct Store<PREC_FP32> {
    static constexpr int BYTES = 8;
    static constexpr int VEC = 2;
    static constexpr bool PLANAR = false;
    __device__ __forceinline__ static void load16(const void* p, float2 (&v)[VEC]) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = make_float2(t.x, t.y);
        v[1] = make_float2(t.z, t.w);
    }
    __device__ __forceinline__ static void store1(void* base, size_t c, int kl, int BT, float2 v) {
        (void)kl;
        (void)BT;
        reinterpret_cast<float2*>(base)[c] = v;
    }
    __device__ __forceinline__ static float2 load1(const void* base, size_t c, int kl, int BT) {
        (void)kl;
        (void)BT;
        return reinterpret_cast<const float2*>(base)[c];
    }
};

// Offset (in 16-bit values) of bin kl's real part within its row; the
// imaginary part follows 4 values later.
__device__ __forceinline__ int planar_offset(int kl) { return (kl & ~3) * 2 + (kl & 3); }

__device__ __forceinline__ float2 unpack_half2(uint32_t w) {
    __half2 h2 = *reinterpret_cast<const __half2*>(&w);
    return __half22float2(h2);
}
// bfloat16 -> float is exact: the bf16 bits are the top half of the float's
__device__ __forceinline__ float2 unpack_bf162(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

template <>
struct Store<PREC_FP16> {
    static constexpr int BYTES = 4;
    static constexpr int VEC = 4;
    static constexpr bool PLANAR = true;
    __device__ __forceinline__ static float2 unpack(uint32_t w) { return unpack_half2(w); }
    __device__ __forceinline__ static void store1(void* base, size_t c, int kl, int BT, float2 v) {
        (void)BT;
        __half* h = reinterpret_cast<__half*>(base) + 2 * (c - kl) + planar_offset(kl);
        h[0] = __float2half_rn(v.x);
        h[4] = __float2half_rn(v.y);
    }
    __device__ __forceinline__ static float2 load1(const void* base, size_t c, int kl, int BT) {
        (void)BT;
        const __half* h = reinterpret_cast<const __half*>(base) + 2 * (c - kl) + planar_offset(kl);
        return make_float2(__half2float(h[0]), __half2float(h[4]));
    }
};

template <>
struct Store<PREC_BF16> {
    static constexpr int BYTES = 4;
    static constexpr int VEC = 4;
    static constexpr bool PLANAR = true;
    __device__ __forceinline__ static float2 unpack(uint32_t w) { return unpack_bf162(w); }
    __device__ __forceinline__ static void store1(void* base, size_t c, int kl, int BT, float2 v) {
        (void)BT;
        __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(base) + 2 * (c - kl) + planar_offset(kl);
        h[0] = __float2bfloat16_rn(v.x);
        h[4] = __float2bfloat16_rn(v.y);
    }
    __device__ __forceinline__ static float2 load1(const void* base, size_t c, int kl, int BT) {
        (void)BT;
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(base) + 2 * (c - kl) + planar_offset(kl);
        return make_float2(__bfloat162float(h[0]), __bfloat162float(h[4]));
    }
};

// Four planar bins (one 16-byte chunk: 8 bytes of real parts, 8 of
// imaginary parts) as floats.
template <typename St>
__device__ __forceinline__ void unpack_planar4(const uint4 t, float2 (&re)[2], float2 (&im)[2]) {
    re[0] = St::unpack(t.x);
    re[1] = St::unpack(t.y);
    im[0] = St::unpack(t.z);
    im[1] = St::unpack(t.w);
}
template <typename St>
__device__ __forceinline__ void load_planar4(const unsigned char* row, int kv, int BT, float2 (&re)[2],
                                             float2 (&im)[2]) {
    (void)BT;
    unpack_planar4<St>(*reinterpret_cast<const uint4*>(row + (size_t)kv * 16), re, im);
}

// d = a * b + c on pairs of floats.  Two scalar FMAs: measured on GB300 in
// the FP16/BF16 MAC, the packed fma.rn.f32x2 form was slower (25.5 vs 23.6 us
// per launch at the paper configuration).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}

// d = a * b on pairs of floats (two scalar multiplies, as ffma2)
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }

// Power-of-two scale for a block of values with largest magnitude `maxabs`:
// FP16 stores value/scale in [2^13, 2^14) at the top (well inside 65504),
// BF16 in [0.5, 1).  Scaling by a power of two is exact.
template <int PREC>
__device__ __forceinline__ float block_scale(float maxabs) {
    if (PREC == PREC_FP32 || !(maxabs > 1e-30f)) return 1.0f;
    int e;
    frexpf(maxabs, &e);  // maxabs = m * 2^e, m in [0.5, 1)
    return ldexpf(1.0f, PREC == PREC_FP16 ? e - 14 : e);
}

// ------------------------------------------------------- mbarrier and TMA

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Explicit shared-memory loads (ld.shared), for operands reached through
// pointers whose address space the compiler may not track.
__device__ __forceinline__ uint4 lds128(const void* p) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}
__device__ __forceinline__ float lds_f32(const float* p) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(smem_u32(p)));
    return v;
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Orders this thread's earlier generic-proxy view of global and shared memory
// before its later bulk (async-proxy) copies: data other CTAs wrote, and
// shared memory that generic code used before the copies land there.
__device__ __forceinline__ void fence_proxy_async_all() {
    asm volatile("fence.proxy.async.global;\n\tfence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after `limit_ns` of wall time or when another thread
// of the CTA has raised `abort_flag`.  Returns false on give-up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0u) {
            if (abort_flag != nullptr && *abort_flag) return false;
            if (global_timer_ns() - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void named_barrier_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ------------------------------------------------------------------- FFT
//
// Complex FFT of length N (a power of two, 16..4096) in shared memory, Stockham
// autosort formulation: stage with radix R and span Ns reads element j + r*N/R,
// multiplies by W_{Ns R}^{r (j mod Ns)}, does an R-point DFT and writes to
// (j / Ns) * Ns * R + (j mod Ns) + r * Ns.  One radix-2 stage first when log2 N
// is odd, then radix-4 stages.  Twiddles come from tw[j] = W_{2B}^j
// = exp(-i pi j / B), computed in FP64 on the host and rounded once.
// INV selects the conjugate twiddles (unscaled inverse).  Every stage ends with
// __syncthreads(); the caller synchronises before the first one.  Returns the
// buffer that holds the result (a or b).

template <bool INV>
__device__ __forceinline__ float2 tw_at(const float2* tw, int idx) {
    const float2 w = tw[idx];
    return INV ? make_float2(w.x, -w.y) : w;
}

// Copy the twiddle table W_2B^j, j in [0, 2B), into shared memory.
__device__ __forceinline__ void load_twiddles(float2* dst, const float2* __restrict__ tw, int B) {
    for (int j = threadIdx.x; j < 2 * B; j += blockDim.x) dst[j] = __ldg(tw + j);
}

// Programmatic dependent launch: let the next kernel in the stream start its
// independent prologue now / wait until the previous kernel has completed and
// its writes are visible.  Both are no-ops for ordinary launches.
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <bool INV>
__device__ float2* fft_smem(float2* a, float2* b, int N, int log2N, const float2* tw, int log2twN,
                            int tid, int nth) {
    int Ns = 1, log2Ns = 0;
    if (log2N & 1) {
        const int H = N >> 1;
        for (int j = tid; j < H; j += nth) {
            const float2 v0 = a[j], v1 = a[j + H];
            b[2 * j] = cadd(v0, v1);
            b[2 * j + 1] = csub(v0, v1);
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns = 2;
        log2Ns = 1;
    }
    while (Ns < N) {
        const int Q = N >> 2;
        const int shift = log2twN - (log2Ns + 2);  // W_{4 Ns}^m = W_{2B}^{m << shift}
        for (int j = tid; j < Q; j += nth) {
            const int k = j & (Ns - 1);
            float2 v0 = a[j], v1 = a[j + Q], v2 = a[j + 2 * Q], v3 = a[j + 3 * Q];
            if (Ns > 1) {
                const int base = k << shift;
                v1 = cmul(v1, tw_at<INV>(tw, base));
                v2 = cmul(v2, tw_at<INV>(tw, 2 * base));
                v3 = cmul(v3, tw_at<INV>(tw, 3 * base));
            }
            const float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
            const float2 s13 = cadd(v1, v3), d13 = csub(v1, v3);
            // forward: -i * d13 ; inverse: +i * d13
            const float2 rot = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
            const int o = ((j - k) << 2) + k;
            b[o] = cadd(s02, s13);
            b[o + Ns] = cadd(d02, rot);
            b[o + 2 * Ns] = csub(s02, s13);
            b[o + 3 * Ns] = csub(d02, rot);
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns <<= 2;
        log2Ns += 2;
    }
    return a;
}

// Real FFT of length 2B from the B-point complex FFT Z of z[n] = w[2n] + i w[2n+1]:
//   X[k] = E[k] + W_2B^k O[k],  E = (Z[k] + conj Z[B-k]) / 2,  O = (Z[k] - conj Z[B-k]) / 2i
// packed: X[0] = (Re Z0 + Im Z0, Re Z0 - Im Z0) = (DC, Nyquist).
__device__ __forceinline__ float2 r2c_post(const float2* Z, int k, int B, const float2* tw) {
    if (k == 0) return make_float2(Z[0].x + Z[0].y, Z[0].x - Z[0].y);
    const float2 zk = Z[k];
    const float2 zm = conjf2(Z[B - k]);
    const float2 E = cscale(cadd(zk, zm), 0.5f);
    const float2 D = cscale(csub(zk, zm), 0.5f);
    const float2 O = make_float2(D.y, -D.x);  // D / i
    return cadd(E, cmul(tw[k], O));
}

// Inverse of r2c_post: from a packed Hermitian spectrum Y to Z such that the
// unscaled inverse B-point FFT of Z, times 1/B, is z[n] = w[2n] + i w[2n+1]
// with w = IFFT_2B(Y) (scaled by 1/2B).
//   A = (Y[k] + conj Y[B-k]) / 2,  Bv = (Y[k] - conj Y[B-k]) / 2 * W_2B^-k,  Z = A + i Bv
__device__ __forceinline__ float2 c2r_pre(const float2* Y, int k, int B, const float2* tw) {
    if (k == 0) {
        const float dc = Y[0].x, ny = Y[0].y;
        return make_float2(0.5f * (dc + ny), 0.5f * (dc - ny));
    }
    const float2 yk = Y[k];
    const float2 ym = conjf2(Y[B - k]);
    const float2 A = cscale(cadd(yk, ym), 0.5f);
    const float2 Bv = cmul(cscale(csub(yk, ym), 0.5f), conjf2(tw[k]));
    return make_float2(A.x - Bv.y, A.y + Bv.x);
}

}  // namespace gbconv
