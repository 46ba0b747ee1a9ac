// kernels.cu - the engine's CUDA kernels (sm_103a) and their host launchers.
//
// Data layouts (B = n_x, block size; K partitions; R = n_src * K reduction
// indices r = p*n_src + q; BT bin-tile width, n_kt = B / BT; LT output-tile height):
//   filter spectra  H[kt][l0..][r][LTt][BT]  (for each bin tile kt and output
//                   tile starting at l0 with LTt rows, all r are contiguous)
//   FDL ring        X[kt][slot][q][BT]       (slot of partition p at block n:
//                   (p - n) mod K; ring row slot*n_src + q of reduction index r
//                   is (slot0*n_src + r) mod R, so a run of r is a run of rows
//                   with at most one wrap)
//   partials        P[split][l][B]           float2, one row per partition split
// All spectra use the packed layout described in kernels.h.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "kernels.h"
#include "spectrum_store.cuh"

namespace gbconv {

static_assert(2 * MAX_STAGES * sizeof(uint64_t) + sizeof(int) <= MAC_ARGS_OFFSET, "mbarriers overlap the staged arguments");
static_assert(MAC_ARGS_OFFSET + sizeof(MacArgs) <= MAC_RED_OFFSET, "staged MAC arguments overlap the scale maxima");
static_assert(MAC_RED_OFFSET + 16 * sizeof(float) <= MAC_HDR_BYTES, "scale maxima of 16 warps exceed the header");

namespace {

constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;  // 1 s: far beyond any legitimate wait

// Ring slot of block n's spectra (the ring's head moves back one slot per block).
__device__ __forceinline__ int ring_slot_of(long long n, int K) {
    const int m = (int)(n % K);
    return m == 0 ? 0 : K - m;
}

// ------------------------------------------------------------ pack + R2C
// One CTA per channel.  w = [previous block, in - sub]; z[n] = w[2n] + i w[2n+1];
// B-point FFT; real-FFT post-processing; push into the ring slot.
// BLK: the ring slot comes from the block number at a.blk (host-call graph);
// a separate instantiation, so that the stream path's kernels stay as they are.
template <int PREC, bool BLK = false>
__device__ __forceinline__ void pack_body(const PackArgs& a, const int c) {
    extern __shared__ float2 fsm[];
    __shared__ float red[32];
    const int B = a.B, half = B >> 1, tid = threadIdx.x, nth = blockDim.x;
    float2* bufA = fsm;
    float2* bufB = fsm + B;
    float2* tws = fsm + 2 * B;
    griddep_launch_dependents();
    load_twiddles(tws, a.tw, B);
    griddep_wait();  // input, feedback prediction and ring slot belong to earlier work
    auto slot_of = [&]() -> int { return BLK ? ring_slot_of(*a.blk, a.K) : a.slot; };  // read where used
    if (PREC == PREC_FP32 && a.save_old) {  // ordered before the push by the barriers below
        const float2* X = static_cast<const float2*>(a.X);
        const RingIndex ri{a.BT, a.n_ch, c, a.K, slot_of()};
        for (int k = tid; k < B; k += nth) {
            const int kt = k / a.BT, kl = k - kt * a.BT;
            a.save_old[((size_t)kt * a.n_ch + c) * a.BT + kl] = X[ri(k)];
        }
    }
    const float* in = a.in + (size_t)c * a.in_stride;
    const float* sub = a.sub ? a.sub + (size_t)c * B : nullptr;
    float* win = a.win + (size_t)c * B;

    for (int n = tid; n < B; n += nth) {
        float2 z;
        if (n < half) {
            z = make_float2(win[2 * n], win[2 * n + 1]);
        } else {
            const int t = 2 * n - B;
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
    float* e_out = a.e_out ? a.e_out + (size_t)c * (a.e_stride ? a.e_stride : B) : nullptr;
    for (int t = tid; t < B; t += nth) {
        const float v = sub ? in[t] - sub[t] : in[t];
        win[t] = v;
        if (e_out) e_out[t] = v;
    }
    float2* Z = fft_smem<false>(bufA, bufB, B, a.log2B, tws, a.log2B + 1, tid, nth);
    float2* Xs = (Z == bufA) ? bufB : bufA;
    for (int k = tid; k < B; k += nth) Xs[k] = r2c_post(Z, k, B, tws);
    __syncthreads();
    const float scale = store_spectrum<PREC>(Xs, B, a.BT, a.X, RingIndex{a.BT, a.n_ch, c, a.K, slot_of()}, red);
    if (PREC != PREC_FP32 && tid == 0) a.sX[(size_t)slot_of() * a.n_ch + c] = scale;
}

template <int PREC>
__global__ void k_pack_r2c(const PackArgs a) {
    pack_body<PREC>(a, blockIdx.x);
}
template <int PREC>
__global__ void k_pack_r2c_g(const PackArgs a) {
    pack_body<PREC, true>(a, blockIdx.x);
}
// the same for the closed loop (its own shared-memory carveout: see prepare_kernels)
template <int PREC>
__global__ void k_pack_r2c_cl(const PackArgs a) {
    pack_body<PREC>(a, blockIdx.x);
}
template <int PREC>
__global__ void k_pack_r2c_cl_g(const PackArgs a) {
    pack_body<PREC, true>(a, blockIdx.x);
}

// --------------------------------------------------- filter partitions R2C
// One CTA per (l, q, p): sub-filter h_lq[pB, pB+B) zero-padded to 2B, R2C,
// stored at reduction index p * n_src + q.  Reduced precision runs this twice:
// pass 0 only records each sub-filter's largest component in `maxabs`; after
// k_tile_scales has turned those into one power-of-two scale per (output
// tile, r), pass 1 stores the spectra divided by their tile's scale.
template <int PREC>
__global__ void k_filter_r2c(const FilterArgs a) {
    extern __shared__ float2 fsm[];
    __shared__ float red[32];
    const int B = a.B, half = B >> 1, tid = threadIdx.x, nth = blockDim.x;
    const int K = a.K, R = a.n_src * K;
    const int l = blockIdx.x / R;
    const int qp = blockIdx.x - l * R;
    const int q = qp / K, p = qp - q * K;
    const int r = p * a.n_src + q;
    const float* h = a.h + ((size_t)l * a.n_src + q) * (size_t)a.taps;
    const long long t0 = (long long)p * B;
    float2* bufA = fsm;
    float2* bufB = fsm + B;
    float2* tws = fsm + 2 * B;
    load_twiddles(tws, a.tw, B);
    for (int n = tid; n < B; n += nth) {
        float2 z = make_float2(0.0f, 0.0f);
        if (n < half) {
            const long long t = t0 + 2 * n;
            z.x = t < a.taps ? h[t] : 0.0f;
            z.y = t + 1 < a.taps ? h[t + 1] : 0.0f;
        }
        bufA[n] = z;
    }
    __syncthreads();
    float2* Z = fft_smem<false>(bufA, bufB, B, a.log2B, tws, a.log2B + 1, tid, nth);
    float2* Xs = (Z == bufA) ? bufB : bufA;
    for (int k = tid; k < B; k += nth) Xs[k] = r2c_post(Z, k, B, tws);
    __syncthreads();
    const int l0 = (l / a.LT) * a.LT;
    const int LTt = min(a.LT, a.n_dst - l0), ll = l - l0;
    if (PREC != PREC_FP32 && a.pass == 0) {
        const float mx = spectrum_max(Xs, B, red);
        if (tid == 0) a.maxabs[(size_t)l * R + r] = mx;
        return;
    }
    const float scale = PREC == PREC_FP32 ? 1.0f : __ldg(a.sH + (size_t)(l / a.LT) * R + r);
    const int n_lt = (a.n_dst + a.LT - 1) / a.LT;
    store_scaled<PREC>(Xs, B, a.BT, a.H, FilterIndex{a.BT, n_lt, l / a.LT, r, LTt, ll, a.tile_elems}, scale);
}

// One power-of-two scale per (output tile, reduction index): from the largest
// component over the tile's outputs (reduced precision set-up, between the two
// filter passes).
template <int PREC>
__global__ void k_tile_scales(const float* __restrict__ maxabs, float* __restrict__ sH, int n_dst, int R, int LT) {
    const int n_lt = (n_dst + LT - 1) / LT;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_lt * R) return;
    const int lt = (int)(i / R), r = (int)(i - (long long)lt * R);
    const int l0 = lt * LT, l1 = min(n_dst, l0 + LT);
    float mx = 0.0f;
    for (int l = l0; l < l1; ++l) mx = fmaxf(mx, maxabs[(size_t)l * R + r]);
    sH[i] = block_scale<PREC>(mx);
}

// Reduced-precision MAC helpers.  d.x += a.lo * b.lo, d.y += a.hi * b.hi for
// two 16-bit values packed in each word, with FP32 accumulation: the
// mixed-precision FMA forms the exact product of the two 16-bit inputs, so
// this equals converting both to FP32 and using an FP32 FMA, without the
// conversions.
template <int PREC>
__device__ __forceinline__ void mfma2(float2& d, uint32_t a, uint32_t b) {
    if constexpr (PREC == PREC_FP16)
        asm("{.reg .f16 a0, a1, b0, b1;\n\tmov.b32 {a0, a1}, %2;\n\tmov.b32 {b0, b1}, %3;\n\t"
            "fma.rn.f32.f16 %0, a0, b0, %0;\n\tfma.rn.f32.f16 %1, a1, b1, %1;}"
            : "+f"(d.x), "+f"(d.y)
            : "r"(a), "r"(b));
    else
        asm("{.reg .b16 a0, a1, b0, b1;\n\tmov.b32 {a0, a1}, %2;\n\tmov.b32 {b0, b1}, %3;\n\t"
            "fma.rn.f32.bf16 %0, a0, b0, %0;\n\tfma.rn.f32.bf16 %1, a1, b1, %1;}"
            : "+f"(d.x), "+f"(d.y)
            : "r"(a), "r"(b));
}
// (v, v) in storage precision
template <int PREC>
__device__ __forceinline__ uint32_t splat2(float v) {
    uint32_t r;
    if constexpr (PREC == PREC_FP16)
        asm("cvt.rn.f16x2.f32 %0, %1, %1;" : "=r"(r) : "f"(v));
    else
        asm("cvt.rn.bf16x2.f32 %0, %1, %1;" : "=r"(r) : "f"(v));
    return r;
}
// element-wise product of two packed pairs in storage precision
template <int PREC>
__device__ __forceinline__ uint32_t mul2(uint32_t a, uint32_t b) {
    uint32_t r;
    if constexpr (PREC == PREC_FP16)
        asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    else
        asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// ----------------------------------------------------------- FDL MAC
// Y[l][k] += sum_{r in split} H[l][r][k] * X[slot(r)][q(r)][k]   (Eq. 6 per bin)
// over r in [r_begin, R), split into S contiguous ranges per tile.
//
// One CTA per (bin tile, output tile, partition split).  Warp 8 is the
// producer: one elected lane streams the split's contiguous filter-spectrum
// range and the matching delay-line slots into an nstage-deep shared-memory
// ring with 1-D bulk copies (TMA), completion tracked by mbarriers (filters
// with an evict-first L2 policy: they are read once per block, except the
// rows below keep_r, which are kept with evict-last so that the next block
// finds them in L2; the delay line with evict-last: it is re-read by every
// output tile and by the next blocks).
// The NW consumer warps: each thread owns VEC bins x up to LPT outputs for one
// r-lane and accumulates in FP32 registers; r-lanes are combined in a fixed
// order through shared memory at the end, and the split's sums go to P[split].
//
// Stages follow a global grid over r (stage g holds r in [g*RS, (g+1)*RS)),
// and every filter tile starts on a 64 KiB boundary, so each filter copy is an
// aligned, usually power-of-two-sized chunk of HBM; a split owns an equal
// range of r, cut along the grid (its first and last stage may be partial).
//
// Reduced precision: each stored row carries a power-of-two scale (one per
// output tile and r for the filters, one per ring slot for the delay line).
// The CTA first finds the largest product of the two over its rows, s_ref;
// each row's delay-line chunk is multiplied by its own product over s_ref (a
// power of two <= 1, in storage precision: exact unless the value falls below
// the format's normal range, where it is then negligible beside the rows near
// s_ref), the sums run in mixed-precision FMAs in units of s_ref, and the
// sums are multiplied by s_ref at the end.
template <int PREC, int LPT, int NW>
__device__ __forceinline__ void mac_body(const MacArgs& a, const int tile, const int split, unsigned char* smem) {
    using St = Store<PREC>;
    constexpr int VEC = St::VEC;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + MAX_STAGES;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + MAX_STAGES);
    unsigned char* stages = smem + MAC_HDR_BYTES;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kt = tile / a.n_lt, lt = tile - kt * a.n_lt;
    const int l0 = lt * a.LT, LTt = min(a.LT, a.n_dst - l0);
    const int K = a.K, R = a.n_src * K;
    const uint64_t wait_ns = a.wait_ns ? a.wait_ns : WAIT_LIMIT_NS;
    const int gb = a.r_begin / a.RS, gt = (R + a.RS - 1) / a.RS - gb;  // stage grid
    // contiguous: split s owns the reduction indices [row0, row1), an equal
    // share of the range (so no split streams a whole stage more than another),
    // cut along the stage grid (only its first and last stage may be partial);
    // interleaved: stages gb + s + i*S, so the tile's CTAs sweep the spectra
    // side by side
    const int Rt = R - a.r_begin;
    const int row0 = a.interleave ? a.r_begin : a.r_begin + (int)((long long)split * Rt / a.S);
    const int row1 = a.interleave ? R : a.r_begin + (int)((long long)(split + 1) * Rt / a.S);
    const int g0 = a.interleave ? gb + split : row0 / a.RS;
    const int g1 = a.interleave ? gb + gt : (row1 + a.RS - 1) / a.RS;
    const int gstep = a.interleave ? a.S : 1;
    const int nit = g1 > g0 ? (g1 - g0 + gstep - 1) / gstep : 0;
    const int ring0 = (a.blk ? ring_slot_of(*a.blk + a.blk_add, K) : a.slot0) * a.n_src;  // ring row of r = 0
    const size_t hrow = (size_t)a.BT * St::BYTES;
    const size_t hr_bytes = (size_t)LTt * hrow;
    const unsigned char* Hb =
        static_cast<const unsigned char*>(a.H) + (size_t)tile * a.tile_elems * St::BYTES;
    const unsigned char* Xb = static_cast<const unsigned char*>(a.X) + (size_t)kt * R * hrow;
    auto stage_range = [&](int it, int& ra, int& rb) {
        const int g = g0 + it * gstep;
        ra = max(row0, g * a.RS);
        rb = min(row1, (g + 1) * a.RS);
    };

    if (tid == 0) {
        for (int i = 0; i < a.nstage; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], NW);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NW) {
        if (lane != 0) return;
        griddep_launch_dependents();
        const uint64_t pol_stream = policy_evict_first();
        const uint64_t pol_keep = policy_evict_last();
        // Reduced precision: the stage's per-partition scales travel with it.
        // Their runs are widened to 16-byte boundaries (the buffers carry 16
        // bytes of padding); consumers index from the run's first element.
        auto scale_runs = [&](int ra, int nr, int start, int run, int (&w)[3][2]) {
            const int fo = lt * R + ra;  // sH: one scale per (output tile, r)
            w[0][0] = fo & ~3;
            w[0][1] = (fo + nr + 3) & ~3;
            w[1][0] = start & ~3;  // sX ring rows, first run
            w[1][1] = (start + run + 3) & ~3;
            w[2][0] = 0;  // wrapped run
            w[2][1] = run < nr ? ((nr - run + 3) & ~3) : 0;
        };
        auto issue_h = [&](int it) {
            const int st = it % a.nstage;
            int ra, rb;
            stage_range(it, ra, rb);
            const int nr = rb - ra;
            unsigned char* sh = stages + (size_t)st * a.stage_bytes;
            size_t tx = (size_t)nr * (hr_bytes + hrow);
            int w[3][2];
            if (PREC != PREC_FP32) {
                int start = ring0 + ra;
                if (start >= R) start -= R;
                scale_runs(ra, nr, start, min(nr, R - start), w);
                tx += (size_t)4 * ((w[0][1] - w[0][0]) + (w[1][1] - w[1][0]) + (w[2][1] - w[2][0]));
            }
            mbar_arrive_expect_tx(&full[st], (uint32_t)tx);
            bulk_g2s(sh, Hb + (size_t)ra * hr_bytes, (uint32_t)((size_t)nr * hr_bytes), &full[st],
                     ra < a.keep_r ? pol_keep : pol_stream);
            if (PREC != PREC_FP32)
                bulk_g2s(sh + a.soff, a.sH + w[0][0], (uint32_t)(4 * (w[0][1] - w[0][0])), &full[st], pol_keep);
        };
        auto issue_x = [&](int it) {
            const int st = it % a.nstage;
            int ra, rb;
            stage_range(it, ra, rb);
            const int nr = rb - ra;
            unsigned char* sx = stages + (size_t)st * a.stage_bytes + a.xoff;
            int start = ring0 + ra;
            if (start >= R) start -= R;
            const int run = min(nr, R - start);
            bulk_g2s(sx, Xb + (size_t)start * hrow, (uint32_t)(run * hrow), &full[st], pol_keep);
            if (run < nr)
                bulk_g2s(sx + (size_t)run * hrow, Xb, (uint32_t)((nr - run) * hrow), &full[st], pol_keep);
            if (PREC != PREC_FP32) {
                int w[3][2];
                scale_runs(ra, nr, start, run, w);
                unsigned char* ss = stages + (size_t)st * a.stage_bytes + a.sxoff;
                const uint32_t b1 = 4 * (w[1][1] - w[1][0]);
                bulk_g2s(ss, a.sX + w[1][0], b1, &full[st], pol_keep);
                if (w[2][1] > 0) bulk_g2s(ss + b1, a.sX, (uint32_t)(4 * w[2][1]), &full[st], pol_keep);
            }
        };
        // the copies read data written by generic stores (earlier kernels, or
        // other CTAs of a persistent step) into shared memory generic code may
        // have used
        fence_proxy_async_all();
        // Fault-path testing: this CTA withholds its first stage (no copy, no
        // arrival on its barrier), so its consumers' bounded wait runs out.
        const bool hold = a.withhold && tile == 0 && split == 0 && nit > 0;
        // The filter spectra are constant: stream the first stages while the
        // previous kernel (the pack of this block) is still running, then wait for
        // it before touching the delay line it writes.
        const int npre = min(nit, a.nstage);
        for (int it = hold ? 1 : 0; it < npre; ++it) issue_h(it);
        griddep_wait();
        for (int it = hold ? 1 : 0; it < npre; ++it) issue_x(it);
        int issued = npre;
        bool ok = true;
        for (int it = npre; it < nit; ++it) {
            const int st = it % a.nstage;
            if (!mbar_wait_bounded(&empty[st], ((it / a.nstage) - 1) & 1, abort_flag, wait_ns)) {
                *abort_flag = 1;
                if (a.err) *(volatile int*)a.err = DEVERR_TIMEOUT_PRODUCER;
                ok = false;
                break;
            }
            issue_h(it);
            issue_x(it);
            ++issued;
        }
        if (!ok || hold) {
            // let copies already in flight land before the CTA's shared memory
            // goes away (the withheld stage has none)
            for (int it = issued > a.nstage ? issued - a.nstage : 0; it < issued; ++it)
                if (!(hold && it == 0))
                    mbar_wait_bounded(&full[it % a.nstage], (it / a.nstage) & 1, nullptr, WAIT_LIMIT_NS);
        }
        return;
    }

    // consumers
    griddep_wait();  // the split partials are still being read by the previous block's output kernel
    const int kv = tid % a.kthreads, rest = tid / a.kthreads;
    const int lg = rest % a.NLG, rl = rest / a.NLG;
    const int kglob = kt * a.BT + kv * VEC;
    const bool dc = (kglob == 0);
    float2 acc[LPT][VEC];
#pragma unroll
    for (int i = 0; i < LPT; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = make_float2(0.0f, 0.0f);

    // reduced precision: s_ref over this CTA's rows (see above); dmask clears
    // the low half (bin 0) of an operand pair in the thread holding DC/Nyquist
    float sref = 1.0f, inv_ref = 1.0f;
    uint32_t dmask = 0xffffffffu;
    if constexpr (St::PLANAR) {
        float m = 0.0f;
        for (int r = row0 + tid; r < row1; r += NW * 32) {
            int rr = ring0 + r;
            if (rr >= R) rr -= R;
            // plain load for the ring's scales: a persistent step writes them in the same launch
            m = fmaxf(m, __ldg(a.sH + (size_t)lt * R + r) * a.sX[rr]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float* sred = reinterpret_cast<float*>(smem + MAC_RED_OFFSET);
        if (lane == 0) sred[warp] = m;
        named_barrier_sync(2, NW * 32);
        m = 0.0f;
        for (int w = 0; w < NW; ++w) m = fmaxf(m, sred[w]);
        if (m > 0.0f) {
            sref = m;
            inv_ref = 1.0f / m;  // exact: a power of two
        }
        if (dc) dmask = 0xffff0000u;
    }

    bool ok = true;
    for (int it = 0; it < nit; ++it) {
        const int st = it % a.nstage;
        if (!mbar_wait_bounded(&full[st], (it / a.nstage) & 1, abort_flag, wait_ns)) {
            *abort_flag = 1;
            if (a.err) *(volatile int*)a.err = DEVERR_TIMEOUT_CONSUMER;
            ok = false;
            break;
        }
        int ra, rb;
        stage_range(it, ra, rb);
        const int nr = rb - ra;
        const unsigned char* sh = stages + (size_t)st * a.stage_bytes;
        const unsigned char* sx = sh + a.xoff;
        // reduced precision: where this stage's scales start in shared memory
        const float* ssh = reinterpret_cast<const float*>(sh + a.soff);
        const float* ssx = reinterpret_cast<const float*>(sh + a.sxoff);
        int sh0 = 0, sx0 = 0, sx2 = 0, xrun = nr;
        if (PREC != PREC_FP32) {
            const int fo = lt * R + ra;
            sh0 = fo - (fo & ~3);
            int start = ring0 + ra;
            if (start >= R) start -= R;
            xrun = min(nr, R - start);
            sx0 = start - (start & ~3);
            // the wrapped second run (ring rows 0..) lands after the first run's padded span
            sx2 = (((start + xrun + 3) & ~3) - (start & ~3)) - xrun;
        }
        // Whole output tile for this thread (every LPT output exists): a loop
        // without per-output branches, so the loads of all outputs of a row are
        // issued before their FMAs
        const bool full = lg + (LPT - 1) * a.NLG < LTt;
        if constexpr (!St::PLANAR) {
            if (full) {
                for (int j = rl; j < nr; j += a.NRL) {
                    float2 xv[VEC];
                    St::load16(sx + (size_t)j * hrow + (size_t)kv * 16, xv);
                    float2 hv[LPT][VEC];
#pragma unroll
                    for (int i = 0; i < LPT; ++i)
                        St::load16(sh + ((size_t)j * LTt + lg + i * a.NLG) * hrow + (size_t)kv * 16, hv[i]);
#pragma unroll
                    for (int i = 0; i < LPT; ++i)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            if (v == 0 && dc)
                                rmac2(acc[i][v], hv[i][v], xv[v]);
                            else
                                cmac(acc[i][v], hv[i][v], xv[v]);
                        }
                }
            } else {
            for (int j = rl; j < nr; j += a.NRL) {
                float2 xv[VEC];
                St::load16(sx + (size_t)j * hrow + (size_t)kv * 16, xv);
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    const int ll = lg + i * a.NLG;
                    if (ll < LTt) {
                        float2 hv[VEC];
                        St::load16(sh + ((size_t)j * LTt + ll) * hrow + (size_t)kv * 16, hv);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            if (v == 0 && dc)
                                rmac2(acc[i][v], hv[v], xv[v]);
                            else
                                cmac(acc[i][v], hv[v], xv[v]);
                        }
                    }
                }
            }
            }
        } else {
            // Planar rows, 4 bins per thread as two pairs; acc[i] = (re 0-1, re 2-3,
            // im 0-1, im 2-3).  Per pair: re += hr*xr + hi*(-xi), im += hr*xi + hi*xr.
            // The packed bin 0 (DC, Nyquist) needs re += hr*xr and im += hi*xi: its
            // lane of the operand pairs is set up for that once per row, outside the
            // output loop.
            if (full) {
                // Whole output tiles (the usual case): mixed-precision FMAs on the
                // stored pairs, in units of s_ref.  Software-pipelined: the next
                // row's 16-byte chunks (delay line and the LPT filter rows) load
                // while this row's FMAs run.
                auto ld_row = [&](int jj, uint4& xo, uint4 (&ho)[LPT], float& sxo, float& sho) {
                    xo = lds128(sx + (size_t)jj * hrow + (size_t)kv * 16);
#pragma unroll
                    for (int i = 0; i < LPT; ++i)
                        ho[i] = lds128(sh + ((size_t)jj * LTt + lg + i * a.NLG) * hrow + (size_t)kv * 16);
                    sxo = lds_f32(jj < xrun ? ssx + sx0 + jj : ssx + sx2 + jj);
                    sho = lds_f32(ssh + sh0 + jj);
                };
                uint4 xw = make_uint4(0u, 0u, 0u, 0u), hw[LPT];
                float sxw = 0.0f, shw = 0.0f;
#pragma unroll
                for (int i = 0; i < LPT; ++i) hw[i] = xw;
                if (rl < nr) ld_row(rl, xw, hw, sxw, shw);
                for (int j = rl; j < nr; j += a.NRL) {
                    const uint4 xc = xw;  // (re 0-1, re 2-3, im 0-1, im 2-3)
                    uint4 hc[LPT];
#pragma unroll
                    for (int i = 0; i < LPT; ++i) hc[i] = hw[i];
                    const float ratio = sxw * shw * inv_ref;
                    if (j + a.NRL < nr) ld_row(j + a.NRL, xw, hw, sxw, shw);
                    const uint32_t r2 = splat2<PREC>(ratio), nr2 = splat2<PREC>(-ratio);
                    const uint32_t xr01 = mul2<PREC>(xc.x, r2), xr23 = mul2<PREC>(xc.y, r2);
                    const uint32_t xi01 = mul2<PREC>(xc.z, r2), xi23 = mul2<PREC>(xc.w, r2);
                    const uint32_t nxi01 = mul2<PREC>(xc.z, nr2) & dmask, nxi23 = mul2<PREC>(xc.w, nr2);
                    const uint32_t xi01b = xi01 & dmask;                      // bin 0: im gets no hr*xi
                    const uint32_t xr01b = (xr01 & dmask) | (xi01 & ~dmask);  // bin 0: im += hi*xi
#pragma unroll
                    for (int i = 0; i < LPT; ++i) {
                        mfma2<PREC>(acc[i][0], hc[i].x, xr01);
                        mfma2<PREC>(acc[i][1], hc[i].y, xr23);
                        mfma2<PREC>(acc[i][2], hc[i].x, xi01b);
                        mfma2<PREC>(acc[i][3], hc[i].y, xi23);
                    }
#pragma unroll
                    for (int i = 0; i < LPT; ++i) {
                        mfma2<PREC>(acc[i][0], hc[i].z, nxi01);
                        mfma2<PREC>(acc[i][1], hc[i].w, nxi23);
                        mfma2<PREC>(acc[i][2], hc[i].z, xr01b);
                        mfma2<PREC>(acc[i][3], hc[i].w, xr23);
                    }
                }
            } else
            // ragged output tile: FP32 FMAs, both scales folded into x per row
            for (int j = rl; j < nr; j += a.NRL) {
                float2 xr[2], xi[2];
                load_planar4<St>(sx + (size_t)j * hrow, kv, a.BT, xr, xi);
                const float sc = (j < xrun ? ssx[sx0 + j] : ssx[sx2 + j]) * ssh[sh0 + j];
                const float2 sc2 = make_float2(sc, sc), nsc2 = make_float2(-sc, -sc);
                // both scales folded into x with packed multiplies; -x_i by the negated scale
                float2 nxi0 = fmul2(xi[0], nsc2);
                const float2 nxi1 = fmul2(xi[1], nsc2);
                xr[0] = fmul2(xr[0], sc2);
                xr[1] = fmul2(xr[1], sc2);
                xi[0] = fmul2(xi[0], sc2);
                xi[1] = fmul2(xi[1], sc2);
                float2 xi0 = xi[0], xr0b = xr[0];
                if (dc) {
                    nxi0.x = 0.0f;
                    xi0.x = 0.0f;
                    xr0b.x = xi[0].x;
                }
                {
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    const int ll = lg + i * a.NLG;
                    if (ll < LTt) {
                        float2 hr[2], hi[2];
                        load_planar4<St>(sh + ((size_t)j * LTt + ll) * hrow, kv, a.BT, hr, hi);
                        acc[i][0] = ffma2(hr[0], xr[0], acc[i][0]);
                        acc[i][0] = ffma2(hi[0], nxi0, acc[i][0]);
                        acc[i][1] = ffma2(hr[1], xr[1], acc[i][1]);
                        acc[i][1] = ffma2(hi[1], nxi1, acc[i][1]);
                        acc[i][2] = ffma2(hr[0], xi0, acc[i][2]);
                        acc[i][2] = ffma2(hi[0], xr0b, acc[i][2]);
                        acc[i][3] = ffma2(hr[1], xi[1], acc[i][3]);
                        acc[i][3] = ffma2(hi[1], xr[1], acc[i][3]);
                    }
                }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
    }

    if constexpr (St::PLANAR) {
        if (lg + (LPT - 1) * a.NLG < LTt)  // whole output tile: sums in units of s_ref
#pragma unroll
            for (int i = 0; i < LPT; ++i)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[i][v] = make_float2(acc[i][v].x * sref, acc[i][v].y * sref);
#pragma unroll
        for (int i = 0; i < LPT; ++i) {
            const float2 re01 = acc[i][0], re23 = acc[i][1], im01 = acc[i][2], im23 = acc[i][3];
            acc[i][0] = make_float2(re01.x, im01.x);
            acc[i][1] = make_float2(re01.y, im01.y);
            acc[i][2] = make_float2(re23.x, im23.x);
            acc[i][3] = make_float2(re23.y, im23.y);
        }
    }

    // combine r-lanes in a fixed order (stage memory is free: every stage has
    // landed).  The scratch is lane-major, [r-lane][i][v][thread of the
    // r-lane], so a warp's 32 stores of one (i, v) are consecutive 8-byte
    // words: no shared-memory bank conflicts.
    if (a.NRL > 1) {
        named_barrier_sync(1, NW * 32);
        float2* red = reinterpret_cast<float2*>(stages);
        const int T = a.NLG * a.kthreads, t = lg * a.kthreads + kv;
        if (rl > 0) {
#pragma unroll
            for (int i = 0; i < LPT; ++i) {
                const int ll = lg + i * a.NLG;
                if (ll < LTt)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) red[((size_t)((rl - 1) * LPT + i) * VEC + v) * T + t] = acc[i][v];
            }
        }
        named_barrier_sync(1, NW * 32);
        if (rl == 0) {
            for (int rr = 1; rr < a.NRL; ++rr)
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    const int ll = lg + i * a.NLG;
                    if (ll < LTt)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            acc[i][v] = cadd(acc[i][v], red[((size_t)((rr - 1) * LPT + i) * VEC + v) * T + t]);
                }
        }
    }
    if (rl != 0 || !ok || *abort_flag) return;
    float2* const part = a.blk && ((*a.blk + a.blk_add) & 1) ? a.partial_b : a.partial;
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        const int ll = lg + i * a.NLG;
        if (ll < LTt) {
            float2* dst = part + ((size_t)split * a.n_dst + l0 + ll) * a.B + kglob;
#pragma unroll
            for (int v = 0; v < VEC; ++v) dst[v] = acc[i][v];
        }
    }
}

template <int PREC, int LPT, int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) k_fdl_mac(const MacArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tile = blockIdx.x / a.S, split = blockIdx.x - tile * a.S;
    mac_body<PREC, LPT, NW>(a, tile, split, smem);
}

// Batched: CTA i runs (tile, split) of the session whose arguments are
// items[refs[i].item]; the arguments are staged in the header of shared memory.
template <int PREC, int LPT, int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) k_fdl_mac_batch(const MacArgs* __restrict__ items,
                                                                    const BatchRef* __restrict__ refs) {
    extern __shared__ __align__(1024) unsigned char smem[];
    MacArgs* sa = reinterpret_cast<MacArgs*>(smem + MAC_ARGS_OFFSET);
    const BatchRef r = refs[blockIdx.x];
    if (threadIdx.x == 0) *sa = items[r.item];
    __syncthreads();
    mac_body<PREC, LPT, NW>(*sa, r.idx, r.idx2, smem);
}

// ------------------------------------------------ FDL MAC, direct loads
// Same work and output as k_fdl_mac, without the TMA producer: every thread
// streams its own 16-byte loads straight from HBM (filter rows with the
// streaming cache hint, delay-line rows through L1, where the threads of the
// other output groups find them), U reduction indices in flight at a time.
// Several CTAs share an SM (no stage ring in shared memory), so the grid has
// more splits.  r-lanes are combined as in k_fdl_mac.
template <int PREC>
__device__ __forceinline__ void load16_global_stream(const void* p, float2 (&v)[Store<PREC>::VEC]) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    Store<PREC>::load16(&t, v);
}

template <int PREC, int LPT, int NW, int U, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_fdl_mac_ldg(const MacArgs a) {
    using St = Store<PREC>;
    constexpr int VEC = St::VEC;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x / a.S, split = blockIdx.x - tile * a.S;
    const int kt = tile / a.n_lt, lt = tile - kt * a.n_lt;
    const int l0 = lt * a.LT, LTt = min(a.LT, a.n_dst - l0);
    const int K = a.K, R = a.n_src * K, Rt = R - a.r_begin;
    const int r0 = a.r_begin + (int)((long long)split * Rt / a.S);
    const int r1 = a.r_begin + (int)((long long)(split + 1) * Rt / a.S);
    const int ring0 = (a.blk ? ring_slot_of(*a.blk + a.blk_add, K) : a.slot0) * a.n_src;
    const size_t hrow = (size_t)a.BT * St::BYTES;
    const unsigned char* Hb = static_cast<const unsigned char*>(a.H) + (size_t)tile * a.tile_elems * St::BYTES;
    const unsigned char* Xb = static_cast<const unsigned char*>(a.X) + (size_t)kt * R * hrow;
    const int kv = tid % a.kthreads, rest = tid / a.kthreads;
    const int lg = rest % a.NLG, rl = rest / a.NLG;
    const int kglob = kt * a.BT + kv * VEC;
    const bool dc = (kglob == 0);
    float2 acc[LPT][VEC];
#pragma unroll
    for (int i = 0; i < LPT; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = make_float2(0.0f, 0.0f);

    griddep_launch_dependents();
    griddep_wait();  // the delay line and the split partials belong to earlier kernels
    const int step = a.NRL * U;
    for (int rb = r0 + rl; rb < r1; rb += step) {
        float2 hv[U][LPT][VEC];
        float2 xv[U][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = rb + u * a.NRL;
            if (r < r1) {
                int row = ring0 + r;
                if (row >= R) row -= R;
                const float4 t = __ldg(reinterpret_cast<const float4*>(Xb + (size_t)row * hrow + (size_t)kv * 16));
                St::load16(&t, xv[u]);
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    const int ll = lg + i * a.NLG;
                    if (ll < LTt) load16_global_stream<PREC>(Hb + ((size_t)r * LTt + ll) * hrow + (size_t)kv * 16, hv[u][i]);
                }
                if (PREC != PREC_FP32) {
                    const float sc = __ldg(a.sX + row) * __ldg(a.sH + (size_t)lt * R + r);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) xv[u][v] = cscale(xv[u][v], sc);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (rb + u * a.NRL < r1) {
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    if (lg + i * a.NLG < LTt) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            if (v == 0 && dc)
                                rmac2(acc[i][v], hv[u][i][v], xv[u][v]);
                            else
                                cmac(acc[i][v], hv[u][i][v], xv[u][v]);
                        }
                    }
                }
            }
        }
    }

    if (a.NRL > 1) {  // lane-major scratch, as in k_fdl_mac
        float2* red = reinterpret_cast<float2*>(smem);
        const int T = a.NLG * a.kthreads, t = lg * a.kthreads + kv;
        if (rl > 0) {
#pragma unroll
            for (int i = 0; i < LPT; ++i) {
                const int ll = lg + i * a.NLG;
                if (ll < LTt)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) red[((size_t)((rl - 1) * LPT + i) * VEC + v) * T + t] = acc[i][v];
            }
        }
        __syncthreads();
        if (rl == 0) {
            for (int rr = 1; rr < a.NRL; ++rr)
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    const int ll = lg + i * a.NLG;
                    if (ll < LTt)
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            acc[i][v] = cadd(acc[i][v], red[((size_t)((rr - 1) * LPT + i) * VEC + v) * T + t]);
                }
        }
    }
    if (rl != 0) return;
    float2* const part = a.blk && ((*a.blk + a.blk_add) & 1) ? a.partial_b : a.partial;
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        const int ll = lg + i * a.NLG;
        if (ll < LTt) {
            float2* dst = part + ((size_t)split * a.n_dst + l0 + ll) * a.B + kglob;
#pragma unroll
            for (int v = 0; v < VEC; ++v) dst[v] = acc[i][v];
        }
    }
}

// --------------------------------------------- head + reduce + C2R + OLS
// One CTA per output channel l.  Per bin: the fixed-order sum of the S split
// partials (independent loads in groups of 8, pairwise within a group), then
// partition 0 of this block, sum_q H[l][q][k] * X_n[q][k] (the only term that
// needs the new input), then the C2R IFFT (1/2B) and the last B samples
// (overlap-save).
// BLK: slot and partials' parity come from the block number at a.blk
// (host-call graph; a separate instantiation, as for pack_body).
template <int PREC, bool BLK = false>
__device__ __forceinline__ void out_body(const OutArgs& a, const int l) {
    using St = Store<PREC>;
    extern __shared__ float2 fsm[];
    const int B = a.B, tid = threadIdx.x, nth = blockDim.x;
    float2* P = fsm;
    float2* W = fsm + B;
    float2* tws = fsm + 2 * B;
    griddep_launch_dependents();
    load_twiddles(tws, a.tw, B);
    const size_t stride = (size_t)a.n_dst * B;
    const int S = a.S;
    const int l0 = a.head ? (l / a.LT) * a.LT : 0;
    const int LTt = a.head ? min(a.LT, a.n_dst - l0) : 0, ll = l - l0;
    // The engine's tail partials (and the adaptive canceller's correction
    // terms) come from other streams (events the launch already waited for),
    // not from the previous kernel: sum them, and load the head's constant
    // filter spectra, while the pack kernel may still be running; then wait
    // for it before the head's delay-line row.
    const bool corr = PREC == PREC_FP32 && a.corr_G != nullptr;
    const int n_lt = (a.n_dst + a.LT - 1) / a.LT;
    float2* hs = fsm + 4 * B;  // [n_src][B] when head_pre
    // read where they are used (BLK = false: the arguments, as before)
    auto partial_of = [&]() -> const float2* { return BLK && (*a.blk & 1) ? a.partial_b : a.partial; };
    auto slot0_of = [&]() -> int { return BLK ? ring_slot_of(*a.blk, a.K) : a.slot0; };
    if (!a.early_partials) griddep_wait();
    for (int k = tid; k < B; k += nth) {
        const float2* src = partial_of() + (size_t)l * B + k;
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
        if (corr) {
            float2 c1 = make_float2(0.0f, 0.0f), c2 = make_float2(0.0f, 0.0f);
            for (int c = 0; c < a.corr_C; ++c) {
                c1 = cadd(c1, a.corr_A[(size_t)c * B + k]);
                c2 = cadd(c2, a.corr_A2[(size_t)c * B + k]);
            }
            const float2 g1 = a.corr_G[(size_t)l * B + k], g2 = a.corr_G2[(size_t)l * B + k];
            if (k == 0) {  // DC and Nyquist: real products
                rmac2(tot, g1, c1);
                rmac2(tot, g2, c2);
            } else {
                cmac(tot, g1, c1);
                cmac(tot, g2, c2);
            }
        }
        P[k] = tot;
        if (a.head && a.head_pre) {  // the same thread reads these back below
            const int kt = k / a.BT, kl = k - kt * a.BT;
            const size_t hbase = ((size_t)kt * n_lt + l / a.LT) * a.tile_elems + (size_t)ll * a.BT + kl;
            for (int q = 0; q < a.n_src; ++q) hs[(size_t)q * B + k] = St::load1(a.H, hbase + (size_t)q * LTt * a.BT, kl, a.BT);
        }
    }
    griddep_wait();
    for (int k = tid; k < B; k += nth) {
        float2 tot = P[k];
        if (a.head) {
            const int kt = k / a.BT, kl = k - kt * a.BT;
            const size_t hbase = ((size_t)kt * n_lt + l / a.LT) * a.tile_elems + (size_t)ll * a.BT + kl;
            const size_t xbase = (((size_t)kt * a.K + slot0_of()) * a.n_src) * a.BT + kl;
            float2 hd = make_float2(0.0f, 0.0f);
            for (int q = 0; q < a.n_src; ++q) {
                const float2 h = a.head_pre ? hs[(size_t)q * B + k] : St::load1(a.H, hbase + (size_t)q * LTt * a.BT, kl, a.BT);
                const float2 x = St::load1(a.X, xbase + (size_t)q * a.BT, kl, a.BT);
                float2 t = make_float2(0.0f, 0.0f);
                if (k == 0)
                    rmac2(t, h, x);
                else
                    cmac(t, h, x);
                const float sc = PREC == PREC_FP32 ? 1.0f
                                                   : __ldg(a.sH + (size_t)(l / a.LT) * a.R + q) *
                                                         a.sX[(size_t)slot0_of() * a.n_src + q];  // see k_batch_persistent
                hd.x = fmaf(sc, t.x, hd.x);
                hd.y = fmaf(sc, t.y, hd.y);
            }
            tot = cadd(tot, hd);
        }
        P[k] = tot;
    }
    __syncthreads();
    for (int k = tid; k < B; k += nth) W[k] = c2r_pre(P, k, B, tws);
    __syncthreads();
    const float2* z = fft_smem<true>(W, P, B, a.log2B, tws, a.log2B + 1, tid, nth);
    const float invB = 1.0f / (float)B;
    float* out = a.out + (size_t)l * a.out_stride;
    const float* extra = a.extra ? a.extra + (size_t)l * a.extra_stride : nullptr;
    for (int t = tid; t < B; t += nth) {
        const int u = B + t, n = u >> 1;
        const float v = ((u & 1) ? z[n].y : z[n].x) * invB;
        out[t] = extra ? v + extra[t] : v;
    }
}

template <int PREC>
__global__ void k_out_c2r(const OutArgs a) {
    out_body<PREC>(a, blockIdx.x);
}
template <int PREC>
__global__ void k_out_c2r_g(const OutArgs a) {
    out_body<PREC, true>(a, blockIdx.x);
}
template <int PREC>
__global__ void k_out_c2r_cl(const OutArgs a) {
    out_body<PREC>(a, blockIdx.x);
}
template <int PREC>
__global__ void k_out_c2r_cl_g(const OutArgs a) {
    out_body<PREC, true>(a, blockIdx.x);
}

// Output of one convolution, then the pack + R2C of the same samples into a
// second convolution's delay line (the synthesis output is the feedback
// canceller's input, Sec. 5): CTA l writes output channel l and pushes it.
// The push reads back what this CTA wrote (ordered by the barrier).
template <int PREC>
__global__ void k_out_push(const OutArgs a, const PackArgs b) {
    out_body<PREC>(a, blockIdx.x);
    __syncthreads();
    pack_body<PREC>(b, blockIdx.x);
}
template <int PREC>
__global__ void k_out_push_g(const OutArgs a, const PackArgs b) {
    out_body<PREC, true>(a, blockIdx.x);
    __syncthreads();
    pack_body<PREC, true>(b, blockIdx.x);
}

// Batched pack and output: CTA i serves channel refs[i].idx of the session
// whose arguments are items[refs[i].item] (staged in static shared memory).
template <int PREC>
__global__ void k_pack_batch(const PackArgs* __restrict__ items, const BatchRef* __restrict__ refs) {
    __shared__ PackArgs sa;
    const BatchRef r = refs[blockIdx.x];
    if (threadIdx.x == 0) sa = items[r.item];
    __syncthreads();
    pack_body<PREC>(sa, r.idx);
}

template <int PREC>
__global__ void k_out_batch(const OutArgs* __restrict__ items, const BatchRef* __restrict__ refs) {
    __shared__ OutArgs sa;
    const BatchRef r = refs[blockIdx.x];
    if (threadIdx.x == 0) {
        sa = items[r.item];
        sa.head_pre = 0;  // batched launches carry no head prefetch space
    }
    __syncthreads();
    out_body<PREC>(sa, r.idx);
}

template <int PREC>
constexpr int lpt_for() {
    return PREC == PREC_FP32 ? 8 : 4;
}

// --------------------------------------------------- persistent batch step
// One launch runs a whole batch step: every CTA claims work items in list
// order (packs, outputs, the canceller's packs and outputs, then the tail
// MACs of the next block) and runs the same device functions as the separate
// batched kernels, so the results are the same bit for bit.  An item that
// needs others' results waits (bounded) for a counter they raise: one thread
// acquires it, the CTA barrier passes the ordering on.  The writer side is a
// CTA barrier, a device-scope fence and the counter increment.  Data written
// within the launch (ring spectra and their scales, partials) is read with
// ordinary (coherent) loads or bulk copies after a proxy fence, never through
// the read-only (non-coherent) path.
template <int PREC>
__global__ void __launch_bounds__(9 * 32, 1) k_batch_persistent(const PackArgs* __restrict__ pk,
                                                                const OutArgs* __restrict__ ot,
                                                                const MacArgs* __restrict__ mc,
                                                                const PersistentWork* __restrict__ work, int n_work,
                                                                unsigned* ctr, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int s_w;
    __shared__ PackArgs s_pack;
    __shared__ OutArgs s_out;
    MacArgs* s_mac = reinterpret_cast<MacArgs*>(smem + MAC_ARGS_OFFSET);
    for (;;) {
        __syncthreads();  // the previous item is done with shared memory and s_w
        if (threadIdx.x == 0) s_w = (int)atomicAdd(ctr, 1u);
        __syncthreads();
        const int w = s_w;
        if (w >= n_work) return;
        const PersistentWork wk = work[w];
        if (threadIdx.x == 0) {
            if (wk.wait >= 0) {
                const uint64_t t0 = global_timer_ns();
                while (ld_acquire_gpu(ctr + 1 + wk.wait) < (unsigned)wk.target) {
                    if (global_timer_ns() - t0 > WAIT_LIMIT_NS) {
                        *(volatile int*)err = DEVERR_TIMEOUT_CONSUMER;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (wk.type == PW_PACK) {
                s_pack = pk[wk.item];
            } else if (wk.type == PW_OUT) {
                s_out = ot[wk.item];
                s_out.head_pre = 0;
            } else {
                *s_mac = mc[wk.item];
            }
        }
        __syncthreads();
        if (wk.type == PW_PACK) {
            pack_body<PREC>(s_pack, wk.idx);
        } else if (wk.type == PW_OUT) {
            out_body<PREC>(s_out, wk.idx);
        } else {
            mac_body<PREC, (PREC == PREC_FP32 ? 8 : 4), 8>(*s_mac, wk.idx, wk.idx2, smem);
            __syncthreads();
            if (threadIdx.x == 0) {  // the barriers' memory goes back to generic use
                uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
                for (int i = 0; i < 2 * MAX_STAGES; ++i) mbar_inval(&bars[i]);
            }
        }
        if (wk.signal >= 0) {
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(ctr + 1 + wk.signal, 1u);
            }
        }
    }
}

}  // namespace

int fft_threads(int B) {
    int t = B / 4;
    if (t < 32) t = 32;
    if (t > 256) t = 256;
    return t;
}

int out_threads(int B) {
    int t = B;
    if (t < 32) t = 32;
    if (t > 256) t = 256;
    return t;
}

// two work buffers of B complex values plus the 2B-entry twiddle table
size_t fft_smem_bytes(int B) { return (size_t)4 * B * sizeof(float2); }

namespace {

// Launch with programmatic stream serialization: the kernel may start while
// the previous kernel in the stream finishes; it orders itself with
// griddepcontrol.wait before touching anything that kernel produces.
template <typename Kern, typename Arg>
cudaError_t launch_pdl(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const Arg& arg,
                       bool pdl = true) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

}  // namespace

// The plain convolution's kernels ask for the largest shared-memory carveout,
// so an SM that ran a pack or output CTA takes a MAC CTA without first
// changing its L1/shared split (measured at the paper configuration: FP16
// steps 17.6 -> 15.7 us, FP32 unchanged).  The closed loop's pack and output
// kernels (k_*_cl, k_out_push) keep the default: there the larger carveout
// made FP16 steps longer (27.5 -> 30.8 us), FP32 within 1 %.
cudaError_t prepare_kernels(size_t mac_smem) {
    const int fft_max = (int)fft_smem_bytes(4096);
    cudaError_t e;
#define GB_ATTR_DEFAULT(kern, bytes)                                                             \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes)); \
    if (e != cudaSuccess) return e;
#define GB_ATTR(kern, bytes)                                                                              \
    GB_ATTR_DEFAULT(kern, bytes)                                                                          \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared); \
    if (e != cudaSuccess) return e;
    GB_ATTR_DEFAULT(k_out_push<PREC_FP32>, fft_max)
    GB_ATTR_DEFAULT(k_out_push<PREC_FP16>, fft_max)
    GB_ATTR_DEFAULT(k_out_push<PREC_BF16>, fft_max)
    GB_ATTR_DEFAULT(k_pack_r2c_cl<PREC_FP32>, fft_max)
    GB_ATTR_DEFAULT(k_pack_r2c_cl<PREC_FP16>, fft_max)
    GB_ATTR_DEFAULT(k_pack_r2c_cl<PREC_BF16>, fft_max)
    GB_ATTR_DEFAULT(k_out_c2r_cl<PREC_FP32>, fft_max)
    GB_ATTR_DEFAULT(k_out_c2r_cl<PREC_FP16>, fft_max)
    GB_ATTR_DEFAULT(k_out_c2r_cl<PREC_BF16>, fft_max)
    GB_ATTR_DEFAULT(k_out_push_g<PREC_FP32>, fft_max)
    GB_ATTR_DEFAULT(k_out_push_g<PREC_FP16>, fft_max)
    GB_ATTR_DEFAULT(k_out_push_g<PREC_BF16>, fft_max)
    GB_ATTR_DEFAULT(k_pack_r2c_cl_g<PREC_FP32>, fft_max)
    GB_ATTR_DEFAULT(k_pack_r2c_cl_g<PREC_FP16>, fft_max)
    GB_ATTR_DEFAULT(k_pack_r2c_cl_g<PREC_BF16>, fft_max)
    GB_ATTR_DEFAULT(k_out_c2r_cl_g<PREC_FP32>, fft_max)
    GB_ATTR_DEFAULT(k_out_c2r_cl_g<PREC_FP16>, fft_max)
    GB_ATTR_DEFAULT(k_out_c2r_cl_g<PREC_BF16>, fft_max)
    GB_ATTR(k_pack_r2c<PREC_FP32>, fft_max)
    GB_ATTR(k_pack_r2c<PREC_FP16>, fft_max)
    GB_ATTR(k_pack_r2c<PREC_BF16>, fft_max)
    GB_ATTR(k_pack_r2c_g<PREC_FP32>, fft_max)
    GB_ATTR(k_pack_r2c_g<PREC_FP16>, fft_max)
    GB_ATTR(k_pack_r2c_g<PREC_BF16>, fft_max)
    GB_ATTR(k_filter_r2c<PREC_FP32>, fft_max)
    GB_ATTR(k_filter_r2c<PREC_FP16>, fft_max)
    GB_ATTR(k_filter_r2c<PREC_BF16>, fft_max)
    GB_ATTR(k_out_c2r<PREC_FP32>, fft_max)
    GB_ATTR(k_pack_batch<PREC_FP32>, fft_max)
    GB_ATTR(k_pack_batch<PREC_FP16>, fft_max)
    GB_ATTR(k_pack_batch<PREC_BF16>, fft_max)
    GB_ATTR(k_out_batch<PREC_FP32>, fft_max)
    GB_ATTR(k_out_batch<PREC_FP16>, fft_max)
    GB_ATTR(k_out_batch<PREC_BF16>, fft_max)
    GB_ATTR((k_fdl_mac_batch<PREC_FP32, lpt_for<PREC_FP32>(), 8>), mac_smem)
    GB_ATTR((k_fdl_mac_batch<PREC_FP16, lpt_for<PREC_FP16>(), 8>), mac_smem)
    GB_ATTR((k_fdl_mac_batch<PREC_BF16, lpt_for<PREC_BF16>(), 8>), mac_smem)
    GB_ATTR(k_out_c2r<PREC_FP16>, fft_max)
    GB_ATTR(k_out_c2r<PREC_BF16>, fft_max)
    GB_ATTR(k_out_c2r_g<PREC_FP32>, fft_max)
    GB_ATTR(k_out_c2r_g<PREC_FP16>, fft_max)
    GB_ATTR(k_out_c2r_g<PREC_BF16>, fft_max)
    GB_ATTR((k_fdl_mac<PREC_FP32, lpt_for<PREC_FP32>(), 8>), mac_smem)
    GB_ATTR((k_fdl_mac<PREC_FP16, lpt_for<PREC_FP16>(), 8>), mac_smem)
    GB_ATTR((k_fdl_mac<PREC_BF16, lpt_for<PREC_BF16>(), 8>), mac_smem)
    GB_ATTR((k_fdl_mac<PREC_FP32, lpt_for<PREC_FP32>(), 16>), mac_smem)
    GB_ATTR((k_fdl_mac<PREC_FP16, lpt_for<PREC_FP16>(), 16>), mac_smem)
    GB_ATTR((k_fdl_mac<PREC_BF16, lpt_for<PREC_BF16>(), 16>), mac_smem)
    // the persistent step kernel holds a little static shared memory (its staged arguments)
    GB_ATTR(k_batch_persistent<PREC_FP32>, mac_smem - PERSISTENT_STATIC_SMEM)
    GB_ATTR(k_batch_persistent<PREC_FP16>, mac_smem - PERSISTENT_STATIC_SMEM)
    GB_ATTR(k_batch_persistent<PREC_BF16>, mac_smem - PERSISTENT_STATIC_SMEM)
    GB_ATTR((k_fdl_mac_ldg<PREC_FP32, 4, 8, 1, 3>), mac_smem)
    GB_ATTR((k_fdl_mac_ldg<PREC_FP32, 4, 8, 2, 2>), mac_smem)
#undef GB_ATTR
#undef GB_ATTR_DEFAULT
    return cudaSuccess;
}

cudaError_t launch_pack_r2c(int prec, const PackArgs& a, cudaStream_t s, bool closed_loop) {
    // one CTA per channel on the critical path: as many threads as the output
    // kernel (measured: 0.2-1.2 us shorter steps than B/4 threads)
    const dim3 grid(a.n_ch), block(out_threads(a.B));
    const size_t sm = fft_smem_bytes(a.B);
    switch (prec) {
        case PREC_FP32:
            return launch_pdl(a.blk ? (closed_loop ? k_pack_r2c_cl_g<PREC_FP32> : k_pack_r2c_g<PREC_FP32>)
                              : closed_loop ? k_pack_r2c_cl<PREC_FP32> : k_pack_r2c<PREC_FP32>,
                              grid, block, sm, s, a);
        case PREC_FP16:
            return launch_pdl(a.blk ? (closed_loop ? k_pack_r2c_cl_g<PREC_FP16> : k_pack_r2c_g<PREC_FP16>)
                              : closed_loop ? k_pack_r2c_cl<PREC_FP16> : k_pack_r2c<PREC_FP16>,
                              grid, block, sm, s, a);
        case PREC_BF16:
            return launch_pdl(a.blk ? (closed_loop ? k_pack_r2c_cl_g<PREC_BF16> : k_pack_r2c_g<PREC_BF16>)
                              : closed_loop ? k_pack_r2c_cl<PREC_BF16> : k_pack_r2c<PREC_BF16>,
                              grid, block, sm, s, a);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_filter_r2c(int prec, const FilterArgs& a, cudaStream_t s) {
    const long long n = (long long)a.n_dst * a.n_src * a.K;
    if (n <= 0 || n > 0x7fffffffLL) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)n), block(fft_threads(a.B));
    const size_t sm = fft_smem_bytes(a.B);
    switch (prec) {
        case PREC_FP32: k_filter_r2c<PREC_FP32><<<grid, block, sm, s>>>(a); break;
        case PREC_FP16: k_filter_r2c<PREC_FP16><<<grid, block, sm, s>>>(a); break;
        case PREC_BF16: k_filter_r2c<PREC_BF16><<<grid, block, sm, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_tile_scales(int prec, const float* maxabs, float* sH, int n_dst, int R, int LT, cudaStream_t s) {
    const long long n = (long long)((n_dst + LT - 1) / LT) * R;
    const unsigned grid = (unsigned)((n + 255) / 256);
    switch (prec) {
        case PREC_FP16: k_tile_scales<PREC_FP16><<<grid, 256, 0, s>>>(maxabs, sH, n_dst, R, LT); break;
        case PREC_BF16: k_tile_scales<PREC_BF16><<<grid, 256, 0, s>>>(maxabs, sH, n_dst, R, LT); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NW>
cudaError_t launch_fdl_mac_nw(int prec, const MacPlan& p, const MacArgs& a, cudaStream_t s, bool pdl) {
    const dim3 grid(p.ctas), block((NW + 1) * 32);
    switch (prec) {
        case PREC_FP32:
            return launch_pdl(k_fdl_mac<PREC_FP32, lpt_for<PREC_FP32>(), NW>, grid, block, p.smem, s, a, pdl);
        case PREC_FP16:
            return launch_pdl(k_fdl_mac<PREC_FP16, lpt_for<PREC_FP16>(), NW>, grid, block, p.smem, s, a, pdl);
        case PREC_BF16:
            return launch_pdl(k_fdl_mac<PREC_BF16, lpt_for<PREC_BF16>(), NW>, grid, block, p.smem, s, a, pdl);
        default: return cudaErrorInvalidValue;
    }
}

template <int U, int MINB>
cudaError_t launch_fdl_mac_direct_u(int prec, const MacPlan& p, const MacArgs& a, cudaStream_t s, bool pdl) {
    const dim3 grid(p.ctas), block(8 * 32);
    switch (prec) {
        case PREC_FP32: return launch_pdl(k_fdl_mac_ldg<PREC_FP32, 4, 8, U, MINB>, grid, block, p.smem, s, a, pdl);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fdl_mac_direct(int prec, const MacPlan& p, const MacArgs& a, cudaStream_t s, bool pdl) {
    return p.direct == 1 ? launch_fdl_mac_direct_u<1, 3>(prec, p, a, s, pdl)
                         : launch_fdl_mac_direct_u<2, 2>(prec, p, a, s, pdl);
}

cudaError_t launch_fdl_mac(int prec, const MacPlan& p, const MacArgs& a, cudaStream_t s, bool pdl) {
    if (p.direct) return launch_fdl_mac_direct(prec, p, a, s, pdl);
    switch (p.nw) {
        case 8: return launch_fdl_mac_nw<8>(prec, p, a, s, pdl);
        case 16: return launch_fdl_mac_nw<16>(prec, p, a, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

size_t out_head_smem(int n_src, int B) {
    // keep the output CTA small enough to share an SM with a tail MAC CTA
    const size_t extra = (size_t)n_src * B * sizeof(float2);
    return fft_smem_bytes(B) + extra <= 64 * 1024 ? extra : 0;
}

cudaError_t launch_out_c2r(int prec, const OutArgs& a, cudaStream_t s, bool closed_loop) {
    const dim3 grid(a.n_dst), block(out_threads(a.B));
    const size_t sm = fft_smem_bytes(a.B) + (a.head && a.head_pre ? (size_t)a.n_src * a.B * sizeof(float2) : 0);
    switch (prec) {
        case PREC_FP32:
            return launch_pdl(a.blk ? (closed_loop ? k_out_c2r_cl_g<PREC_FP32> : k_out_c2r_g<PREC_FP32>)
                              : closed_loop ? k_out_c2r_cl<PREC_FP32> : k_out_c2r<PREC_FP32>,
                              grid, block, sm, s, a);
        case PREC_FP16:
            return launch_pdl(a.blk ? (closed_loop ? k_out_c2r_cl_g<PREC_FP16> : k_out_c2r_g<PREC_FP16>)
                              : closed_loop ? k_out_c2r_cl<PREC_FP16> : k_out_c2r<PREC_FP16>,
                              grid, block, sm, s, a);
        case PREC_BF16:
            return launch_pdl(a.blk ? (closed_loop ? k_out_c2r_cl_g<PREC_BF16> : k_out_c2r_g<PREC_BF16>)
                              : closed_loop ? k_out_c2r_cl<PREC_BF16> : k_out_c2r<PREC_BF16>,
                              grid, block, sm, s, a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename Kern, typename... Args>
cudaError_t launch_pdl_n(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
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

cudaError_t launch_out_push(int prec, const OutArgs& a, const PackArgs& b, cudaStream_t s) {
    if (a.n_dst != b.n_ch || a.B != b.B || !a.blk != !b.blk) return cudaErrorInvalidValue;
    const dim3 grid(a.n_dst), block(out_threads(a.B));
    const size_t sm = fft_smem_bytes(a.B) + (a.head && a.head_pre ? (size_t)a.n_src * a.B * sizeof(float2) : 0);
    switch (prec) {
        case PREC_FP32:
            return launch_pdl_n(a.blk ? k_out_push_g<PREC_FP32> : k_out_push<PREC_FP32>, grid, block, sm, s, a, b);
        case PREC_FP16:
            return launch_pdl_n(a.blk ? k_out_push_g<PREC_FP16> : k_out_push<PREC_FP16>, grid, block, sm, s, a, b);
        case PREC_BF16:
            return launch_pdl_n(a.blk ? k_out_push_g<PREC_BF16> : k_out_push<PREC_BF16>, grid, block, sm, s, a, b);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pack_batch(int prec, const PackArgs* items, const BatchRef* refs, int n, int Bmax,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 grid(n), block(fft_threads(Bmax));
    const size_t sm = fft_smem_bytes(Bmax);
    switch (prec) {
        case PREC_FP32: return launch_pdl_n(k_pack_batch<PREC_FP32>, grid, block, sm, s, items, refs);
        case PREC_FP16: return launch_pdl_n(k_pack_batch<PREC_FP16>, grid, block, sm, s, items, refs);
        case PREC_BF16: return launch_pdl_n(k_pack_batch<PREC_BF16>, grid, block, sm, s, items, refs);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_out_batch(int prec, const OutArgs* items, const BatchRef* refs, int n, int Bmax, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 grid(n), block(out_threads(Bmax));
    const size_t sm = fft_smem_bytes(Bmax);
    switch (prec) {
        case PREC_FP32: return launch_pdl_n(k_out_batch<PREC_FP32>, grid, block, sm, s, items, refs);
        case PREC_FP16: return launch_pdl_n(k_out_batch<PREC_FP16>, grid, block, sm, s, items, refs);
        case PREC_BF16: return launch_pdl_n(k_out_batch<PREC_BF16>, grid, block, sm, s, items, refs);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mac_batch(int prec, const MacArgs* items, const BatchRef* refs, int n, size_t smem,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const dim3 grid(n), block((8 + 1) * 32);
    switch (prec) {
        case PREC_FP32:
            return launch_pdl_n(k_fdl_mac_batch<PREC_FP32, lpt_for<PREC_FP32>(), 8>, grid, block, smem, s, items, refs);
        case PREC_FP16:
            return launch_pdl_n(k_fdl_mac_batch<PREC_FP16, lpt_for<PREC_FP16>(), 8>, grid, block, smem, s, items, refs);
        case PREC_BF16:
            return launch_pdl_n(k_fdl_mac_batch<PREC_BF16, lpt_for<PREC_BF16>(), 8>, grid, block, smem, s, items, refs);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_persistent(int prec, const PackArgs* pk, const OutArgs* ot, const MacArgs* mc,
                                    const PersistentWork* work, int n_work, unsigned* ctr, int* err, int ctas,
                                    size_t smem, cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    if (ctas < 1 || smem > MAC_SMEM_LIMIT - PERSISTENT_STATIC_SMEM) return cudaErrorInvalidValue;
    const dim3 grid(ctas), block(9 * 32);
    switch (prec) {
        case PREC_FP32: k_batch_persistent<PREC_FP32><<<grid, block, smem, s>>>(pk, ot, mc, work, n_work, ctr, err); break;
        case PREC_FP16: k_batch_persistent<PREC_FP16><<<grid, block, smem, s>>>(pk, ot, mc, work, n_work, ctr, err); break;
        case PREC_BF16: k_batch_persistent<PREC_BF16><<<grid, block, smem, s>>>(pk, ot, mc, work, n_work, ctr, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gbconv
