// engine.cu - the streaming convolution engine behind the C ABI of conv.h.
//
// One engine = one auralization stream on one GPU: the synthesis convolution
// (n_in inputs -> n_out outputs, Sec. 3.1 Eq. 2) and optionally the feedback
// canceller (n_out loudspeakers -> n_in microphones, Eq. 3), each a uniformly
// partitioned overlap-save convolution with a frequency-domain delay line
// (Sec. 4).  All state (filter spectra, delay lines, sliding windows, pending
// feedback prediction) stays resident in device memory; per block only the
// n_in x B input samples and n_out x B output samples cross to the host.
//
// Split-phase schedule.  Partitions 1..K-1 of block n+1 only need input
// spectra of blocks <= n, so their MAC (the "tail": all but 1/K of the bytes)
// is enqueued on a low-priority background stream as soon as block n's
// spectrum is in the delay line.  When block n+1 arrives, the caller's stream
// runs only the pack/R2C of the new block and one output kernel that adds
// partition 0 (the "head") to the tail's split partials and transforms back.
// Tail partials are double-buffered by block parity, and the tails alternate
// between two background streams so that, when blocks come back to back, the
// tail of block n+1 takes over each SM as the tail of block n leaves it (no
// drain and ramp of the HBM stream between blocks):
//   caller stream:      pack(n) -> [rec packed] -> [wait tail(n)] -> out(n)
//   background n+1 & 1: [wait packed(n)] -> tail(n+1) -> [rec tail(n+1 & 1)]
// pack(n+1) overwrites the ring slot of block n+1-K, which tail(n) (already
// waited for by out(n)) was the last to read; tail(n+1) never reads it.
// tail(n+2) reuses the partials out(n) read; it waits for pack(n+1), which
// the caller stream runs after out(n).
//
// With the feedback canceller the caller stream runs three kernels per block:
// the microphone pack (e = m - c), the synthesis output fused with the push
// of l_n into the canceller's ring, and the canceller's output (c_n).  The
// canceller's tails alternate over a second pair of background streams.  The
// adaptive canceller adds the NLMS step on a high-priority stream beside the
// synthesis output and a deferred step fused into the canceller's tail (see
// nlms.h and enqueue_afc_synthesis / enqueue_afc_prediction).
//
// Host-call graphs.  A paced blocking host call (conv_process_block, or
// afc_process_block with the static canceller) enqueues the same kernels as
// one CUDA graph launch instead: the stream schedule above, captured once,
// with the kernels reading the block number from device memory (HostGraph
// below).  Back-to-back calls keep the stream schedule, whose next pack does
// not wait for the previous tail.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "conv.h"
#include "host_util.h"
#include "kernels.h"
#include "nlms.h"

using namespace gbconv;

namespace {

thread_local std::string g_err;

int set_err(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call) GB_CK(call)

inline int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int pow2_ceil(int v) {
    int r = 1;
    while (r < v) r <<= 1;
    return r;
}

// Tiling fields a caller (the autotuner) may fix; 0 leaves a field to the planner.
struct TileOverride {
    int kernel = 0, bin_tile = 0, stages = 0, stage_kib = 0, splits = 0, warps = 0, order = 0;
};

TileOverride from_api(const conv_tiling* t) {
    TileOverride o;
    if (t) {
        o.kernel = t->kernel;
        o.bin_tile = t->bin_tile;
        o.stages = t->stages;
        o.stage_kib = t->stage_kib;
        o.splits = t->splits;
        o.warps = t->warps;
        o.order = t->order;
    }
    return o;
}

const char* check_override(const TileOverride& o) {
    if (o.kernel < CONV_KERNEL_AUTO || o.kernel > CONV_KERNEL_DIRECT2) return "unknown kernel";
    if (o.bin_tile < 0 || (o.bin_tile && (o.bin_tile < 16 || o.bin_tile > 256 || (o.bin_tile & (o.bin_tile - 1)))))
        return "bin_tile must be 0 or a power of two in [16, 256]";
    if (o.stages < 0 || (o.stages && (o.stages < 2 || o.stages > MAX_STAGES))) return "stages must be 0 or in [2, 8]";
    if (o.stage_kib < 0 || o.stage_kib > 96) return "stage_kib must be in [0, 96]";
    if (o.splits < 0) return "splits must be >= 0";
    if (o.warps != 0 && o.warps != 8 && o.warps != 16) return "warps must be 0, 8 or 16";
    if (o.order < 0 || o.order > 2) return "order must be 0, 1 or 2";
    return nullptr;
}

inline bool is_pow2(size_t v) { return v && !(v & (v - 1)); }
inline size_t pow2_floor(size_t v) {
    size_t r = 1;
    while (r * 2 <= v) r *= 2;
    return r;
}

// Tiling of one FDL MAC.  Chooses bin/output tiles, the consumer thread layout,
// the pipeline stage size and depth, and the number of partition splits so
// that the grid covers every SM once (no second wave) while each CTA still
// streams at least a few stages.
MacPlan plan_mac(int prec, int B, int n_src, int n_dst, int K, int num_sms, int r_begin,
                 const TileOverride& o = TileOverride()) {
    MacPlan p{};
    p.B = B;
    p.n_src = n_src;
    p.n_dst = n_dst;
    p.K = K;
    p.R = n_src * K;
    p.r_begin = r_begin;
    const int Rt = p.R - r_begin;
    p.es = prec == PREC_FP32 ? 8 : 4;
    p.VEC = 16 / p.es;
    // the direct-load MAC reads interleaved FP32 rows only; reduced precision uses the TMA MAC
    p.direct = prec != PREC_FP32 ? 0 : (o.kernel == CONV_KERNEL_DIRECT1 ? 1 : (o.kernel == CONV_KERNEL_DIRECT2 ? 2 : 0));
    p.LPT = (prec == PREC_FP32 && !p.direct) ? 8 : 4;
    p.nw = p.direct ? 8 : (o.warps ? o.warps : MAC_CONSUMER_WARPS);
    p.interleave = (!p.direct && o.order == CONV_ORDER_INTERLEAVED) ? 1 : 0;
    p.LT = std::min(n_dst, 16);
    p.n_lt = (n_dst + p.LT - 1) / p.LT;
    // Bin tiles: enough (bin tile x output tile) pairs that ~16-20 partition
    // splits per tile cover the SMs.  Few splits keep the split partials (which
    // the output kernel must read back) a small fraction of the streamed bytes.
    int want_kt = std::max(1, num_sms / (16 * p.n_lt));
    int n_kt = 1;
    while (n_kt * 2 <= want_kt) n_kt *= 2;
    p.BT = std::max(16, std::min(256, B / n_kt));
    if (o.bin_tile) p.BT = std::max(16, std::min(256, o.bin_tile));
    if (p.BT > B) p.BT = B;
    p.n_kt = B / p.BT;
    p.kthreads = p.BT / p.VEC;
    const int rest = (p.nw * 32) / p.kthreads;
    p.NLG = pow2_ceil((p.LT + p.LPT - 1) / p.LPT);
    if (p.NLG > rest) p.NLG = rest;
    if (p.LT > p.LPT * p.NLG) {  // too few threads per bin for the tile: shorter output tiles
        p.LT = p.LPT * p.NLG;
        p.n_lt = (n_dst + p.LT - 1) / p.LT;
    }
    p.NRL = rest / p.NLG;
    // Stage pitch: filter copies of a power-of-two size (64 KiB by default),
    // which, with 64 KiB-aligned tiles and a global stage grid, keeps every
    // copy aligned to its size across the HBM channel interleave (measured:
    // 32/64 KiB copies stream faster than 40-60 KiB ones).
    const size_t per_r_h = (size_t)p.LT * p.BT * p.es;
    const size_t per_r = per_r_h + (size_t)p.BT * p.es;
    const size_t stage_target = o.stage_kib ? (size_t)o.stage_kib * 1024 : 65536;
    int rs;
    if (is_pow2(per_r_h) && per_r_h <= stage_target)
        rs = (int)(pow2_floor(stage_target) / per_r_h);
    else
        rs = (int)std::max<size_t>(1, (stage_target + per_r / 2) / per_r);
    p.RS = std::max(1, std::min(rs, std::max(1, p.R)));
    const size_t budget = MAC_SMEM_LIMIT - MAC_HDR_BYTES;
    const bool scaled = prec != PREC_FP32;
    // scale parts: a run widened to 16-byte boundaries at both ends (+ a wrapped second run for sX)
    auto sh_part = [&](int RS) { return scaled ? align_up(((size_t)RS + 8) * 4, 128) : 0; };
    auto sx_part = [&](int RS) { return scaled ? align_up(((size_t)RS + 12) * 4, 128) : 0; };
    auto stage_size = [&](int RS) {
        return align_up((size_t)RS * p.LT * p.BT * p.es, 128) + align_up((size_t)RS * p.BT * p.es, 128) +
               sh_part(RS) + sx_part(RS);
    };
    while (p.RS > 1 && 2 * stage_size(p.RS) > budget) p.RS = is_pow2(per_r_h) ? p.RS / 2 : p.RS - 1;
    const size_t hpart = align_up((size_t)p.RS * p.LT * p.BT * p.es, 128);
    p.xoff = (unsigned)hpart;
    p.soff = (unsigned)(hpart + align_up((size_t)p.RS * p.BT * p.es, 128));
    p.sxoff = (unsigned)(p.soff + sh_part(p.RS));
    p.stage_bytes = (unsigned)stage_size(p.RS);
    const int fit = (int)std::max<size_t>(2, budget / p.stage_bytes);
    // measured on the back-to-back step: two large stages for every precision
    // (they leave room on each SM for the next block's pack and output CTAs)
    p.nstage = std::min(2, fit);
    if (o.stages) p.nstage = std::max(2, std::min(o.stages, fit));
    // scratch for combining r-lanes reuses (and if needed extends) the stage ring
    const size_t red = (size_t)(p.NRL - 1) * p.LPT * p.NLG * p.BT * sizeof(float2);  // lane-major r-lane scratch
    p.smem = MAC_HDR_BYTES + std::max((size_t)p.nstage * p.stage_bytes, align_up(red, 128));
    const int tiles = p.n_kt * p.n_lt;
    int gt = Rt > 0 ? (p.R + p.RS - 1) / p.RS - r_begin / p.RS : 0;  // stages on the grid
    int by_work = std::max(1, gt / 2);
    // never a second wave: the grid fits the SMs at the occupancy shared memory allows
    int per_sm = (int)std::max<size_t>(1, SM_SMEM_BYTES / (p.smem + CTA_SMEM_RESERVED));
    if (p.direct) {
        // no stage ring: shared memory only holds the r-lane scratch; the
        // register budget sets the CTAs per SM (3 or 2)
        p.nstage = 0;
        p.stage_bytes = 0;
        p.smem = std::max<size_t>(16, align_up(red, 128));
        per_sm = std::min(p.direct == 1 ? 3 : 2, (int)(SM_SMEM_BYTES / (p.smem + CTA_SMEM_RESERVED)));
        gt = Rt;  // splits are plain ranges of reduction indices
        by_work = std::max(1, Rt / (p.NRL * 4));
    }
    // all but 8 SMs: the next block's pack and output kernels run there at once
    // (measured on the back-to-back step: 6-20 % shorter than a grid on every SM)
    const int sms = (!p.direct && num_sms > 16) ? num_sms - 8 : num_sms;
    int S = std::max(1, sms * per_sm / tiles);
    S = std::min(S, by_work);
    if (o.splits) S = o.splits;
    S = std::min(S, gt);
    p.S = Rt > 0 ? std::max(1, S) : 0;
    p.ctas = tiles * p.S;
    p.tile_elems = align_up((size_t)p.R * p.LT * p.BT * p.es, 65536) / p.es;
    p.h_bytes = (size_t)tiles * p.tile_elems * p.es;
    p.x_bytes = (size_t)p.R * B * p.es;
    p.partial_bytes = std::max<size_t>(16, (size_t)p.S * n_dst * B * sizeof(float2));
    return p;
}

// Host replay for the direct-load MAC: every thread's filter and delay-line
// rows, the r-lane scratch and the partial rows, against the buffer sizes.
int check_direct_plan(const MacPlan& p, std::string* why) {
    char buf[256];
    auto bad = [&](const char* what) {
        snprintf(buf, sizeof(buf), "plan check failed (direct): %s (B=%d n_src=%d n_dst=%d K=%d)", what, p.B, p.n_src,
                 p.n_dst, p.K);
        *why = buf;
        return -1;
    };
    const int Rt = p.R - p.r_begin;
    if (p.nw != 8 || p.LPT != 4) return bad("thread shape");
    if (p.kthreads * p.VEC != p.BT || p.kthreads > 256) return bad("bin threads");
    const int rest = 256 / p.kthreads;
    if (p.kthreads * rest != 256 || p.NLG * p.NRL != rest) return bad("thread layout");
    if ((p.LT + p.NLG - 1) / p.NLG > p.LPT) return bad("outputs per thread above LPT");
    if (p.S < 1 || p.S > Rt) return bad("split count");
    if ((size_t)(p.NRL - 1) * p.LPT * p.NLG * p.BT * 8 > p.smem) return bad("r-lane scratch");
    if (p.smem > MAC_SMEM_LIMIT) return bad("shared memory");
    const size_t hrow = (size_t)p.BT * p.es;
    if ((size_t)p.R * p.LT * p.BT > p.tile_elems) return bad("tile pitch below a tile");
    if ((size_t)p.n_kt * p.n_lt * p.tile_elems * p.es > p.h_bytes) return bad("tile pitch");
    for (int tile = 0; tile < p.n_kt * p.n_lt; ++tile) {
        const int kt = tile / p.n_lt, lt = tile % p.n_lt;
        const int l0 = lt * p.LT, LTt = std::min(p.LT, p.n_dst - l0);
        if (LTt < 1) return bad("empty output tile");
        // last row of the last r of the tile, last 16 bytes
        const size_t hend = (size_t)tile * p.tile_elems * p.es + ((size_t)(p.R - 1) * LTt + LTt - 1) * hrow + hrow;
        if (hend > p.h_bytes) return bad("filter row past the spectra");
        if ((size_t)kt * p.R * hrow + (size_t)p.R * hrow > p.x_bytes) return bad("delay-line row past the ring");
        for (int split = 0; split < p.S; ++split) {
            const int r0 = p.r_begin + (int)((long long)split * Rt / p.S);
            const int r1 = p.r_begin + (int)((long long)(split + 1) * Rt / p.S);
            if (r1 <= r0) return bad("empty split");
            const size_t last = (((size_t)split * p.n_dst + l0 + LTt - 1) * p.B + (size_t)kt * p.BT + p.BT);
            if (last * sizeof(float2) > p.partial_bytes) return bad("partial write past the buffer");
        }
    }
    return 0;
}

// Host replay of the address arithmetic of one FDL MAC launch (producer bulk
// copies, consumer shared-memory reads, r-lane scratch, partial writes) against
// the buffer and shared-memory sizes of the plan, for every CTA and stage.
// Returns 0 or a description of the first violation in `why`.
int check_plan(const MacPlan& p, std::string* why) {
    char buf[256];
    auto bad = [&](const char* what) {
        snprintf(buf, sizeof(buf), "plan check failed: %s (B=%d n_src=%d n_dst=%d K=%d)", what, p.B, p.n_src, p.n_dst,
                 p.K);
        *why = buf;
        return -1;
    };
    const int Rt = p.R - p.r_begin;
    if (Rt < 0 || p.r_begin < 0) return bad("reduction range");
    if (Rt == 0) return p.S == 0 ? 0 : bad("splits over an empty range");
    if (p.direct) return check_direct_plan(p, why);
    if (p.nstage < 1 || p.nstage > MAX_STAGES) return bad("stage count");
    if (p.smem > MAC_SMEM_LIMIT) return bad("shared memory above the kernel's limit");
    if (p.nw != 8 && p.nw != 16) return bad("consumer warps");
    if (p.kthreads * p.VEC != p.BT || p.kthreads > p.nw * 32) return bad("bin threads");
    const int rest = (p.nw * 32) / p.kthreads;
    if (p.kthreads * rest != p.nw * 32 || p.NLG * p.NRL != rest) return bad("thread layout");
    if ((p.LT + p.NLG - 1) / p.NLG > p.LPT) return bad("outputs per thread above LPT");
    const int gb = p.r_begin / p.RS, gt = (p.R + p.RS - 1) / p.RS - gb;
    if (p.S < 1 || p.S > gt) return bad("split count");
    if ((size_t)p.n_kt * p.n_lt * p.tile_elems * p.es > p.h_bytes) return bad("tile pitch");
    if ((size_t)p.R * p.LT * p.BT > p.tile_elems) return bad("tile pitch below a tile");
    if (p.B % p.BT) return bad("bin tile");
    const size_t hrow = (size_t)p.BT * p.es;
    if (hrow % 16) return bad("row not a multiple of 16 bytes");
    if (p.stage_bytes % 16 || p.xoff % 16) return bad("stage alignment");
    if ((size_t)(p.NRL - 1) * p.LPT * p.NLG * p.BT * 8 > p.smem - MAC_HDR_BYTES) return bad("r-lane scratch");
    if ((size_t)p.nstage * p.stage_bytes > p.smem - MAC_HDR_BYTES) return bad("stage ring");
    for (int cta = 0; cta < p.ctas; ++cta) {
        const int tile = cta / p.S, split = cta % p.S;
        const int kt = tile / p.n_lt, lt = tile % p.n_lt;
        if (kt >= p.n_kt) return bad("tile index");
        const int l0 = lt * p.LT, LTt = std::min(p.LT, p.n_dst - l0);
        if (LTt < 1) return bad("empty output tile");
        // the kernel's split ranges: equal shares of the reduction range cut
        // along the stage grid (contiguous), or every S-th stage (interleaved)
        const int row0 = p.interleave ? p.r_begin : p.r_begin + (int)((long long)split * Rt / p.S);
        const int row1 = p.interleave ? p.R : p.r_begin + (int)((long long)(split + 1) * Rt / p.S);
        const int g0 = p.interleave ? gb + split : row0 / p.RS;
        const int g1 = p.interleave ? gb + gt : (row1 + p.RS - 1) / p.RS;
        const int gstep = p.interleave ? p.S : 1;
        if (g1 <= g0 || row1 <= row0) return bad("empty split");
        if ((g1 - g0 + gstep - 1) / gstep < 1) return bad("split without a stage");
        const size_t hr = (size_t)LTt * hrow;
        const size_t hb = (size_t)tile * p.tile_elems * p.es;
        const size_t xb = (size_t)kt * p.R * hrow;
        for (int g = g0; g < g1; g += gstep) {
            const int ra = std::max(row0, g * p.RS), rb = std::min(row1, (g + 1) * p.RS), nr = rb - ra;
            if (nr < 1) return bad("empty stage");
            if (nr > p.RS) return bad("stage above its pitch");
            const size_t tx = (size_t)nr * (hr + hrow);
            if (tx >= (1u << 20)) return bad("transaction bytes");
            if ((size_t)rb * hr > (size_t)p.tile_elems * p.es) return bad("filter copy past its tile");
            if (hb + (size_t)rb * hr > p.h_bytes) return bad("filter copy past the spectra");
            if ((size_t)nr * hr > p.xoff) return bad("filter copy past its stage part");
            if (p.xoff + (size_t)nr * hrow > p.stage_bytes) return bad("delay-line copy past its stage");
            if (p.es == 4) {
                const int fo = lt * p.R + ra;
                const int a0 = fo & ~3, a1 = (fo + nr + 3) & ~3;
                if ((size_t)a1 > (size_t)p.n_lt * p.R + 4) return bad("filter scales past their buffer");
                if (p.soff + 4 * (size_t)(a1 - a0) > p.sxoff) return bad("filter scales past their stage part");
                for (int slot0 = 0; slot0 < p.K; slot0 += std::max(1, p.K / 7)) {
                    const int start = (slot0 * p.n_src + ra) % p.R;
                    const int run = std::min(nr, p.R - start);
                    const int b0 = start & ~3, b1 = (start + run + 3) & ~3;
                    const int c1 = run < nr ? ((nr - run + 3) & ~3) : 0;
                    if ((size_t)b1 > (size_t)p.R + 4 || (size_t)c1 > (size_t)p.R + 4) return bad("slot scales past their buffer");
                    if (p.sxoff + 4 * (size_t)((b1 - b0) + c1) > p.stage_bytes) return bad("slot scales past their stage part");
                    if (tx + 4 * (size_t)((a1 - a0) + (b1 - b0) + c1) >= (1u << 20)) return bad("transaction bytes");
                }
            }
            for (int slot0 = 0; slot0 < p.K; slot0 += std::max(1, p.K / 7)) {
                int start = slot0 * p.n_src + ra;
                start %= p.R;
                const int run = std::min(nr, p.R - start);
                if (run < 1) return bad("empty delay-line run");
                if (xb + (size_t)(start + run) * hrow > p.x_bytes) return bad("delay-line copy past the ring");
                if (run < nr && xb + (size_t)(nr - run) * hrow > p.x_bytes) return bad("wrapped copy past the ring");
            }
        }
        const size_t last = (((size_t)split * p.n_dst + l0 + LTt - 1) * p.B + (size_t)kt * p.BT + p.BT);
        if (last * sizeof(float2) > p.partial_bytes) return bad("partial write past the buffer");
    }
    return 0;
}

// One partitioned convolution: spectra, delay line, window and split partials.
struct Part {
    int n_src = 0, n_dst = 0, K = 0;
    long long taps = 0;
    MacPlan plan{};
    void* H = nullptr;
    float* sH = nullptr;
    void* X = nullptr;
    float* sX = nullptr;
    float* win = nullptr;
    float2* partial[2] = {nullptr, nullptr};  // tail partials, by block parity
    size_t win_floats = 0;                    // the input window's history samples, all channels
    cudaEvent_t ev_packed = nullptr;           // this block's spectrum is in the ring
    cudaEvent_t ev_tail[2] = {nullptr, nullptr};  // tail partials of the block of that parity are ready
    bool allocated = false;
    bool ready = false;
};

size_t part_bytes(const MacPlan& p, int prec, size_t win_floats) {
    size_t b = p.h_bytes + p.x_bytes + 2 * p.partial_bytes + win_floats * sizeof(float);
    if (prec != PREC_FP32) b += ((size_t)p.n_lt * p.R + (size_t)p.R + 8) * sizeof(float);
    return b;
}

}  // namespace

void gbconv::set_last_error_message(const char* msg) { g_err = msg ? msg : ""; }

// The blocking host calls as CUDA graphs.  conv_process_block's graph holds
// the pack of block n, its output (programmatic edge, as on a stream) and an
// event recorded after the output, with block n+1's tail MAC beside the
// output.  afc_process_block's adds the closed loop: the output also pushes
// into the canceller's ring, then come the prediction c_n = F_hat * l_n and the
// canceller's tail for block n+1.  Both end with a node that advances the
// block number in device memory.  They are captured once from the same
// launchers as the stream path.  The kernels take ring slots and the
// partials' parity from that device word, so the nodes' arguments stay the
// same from block to block and a call is one graph launch.  A launch starts
// after the whole previous one, tails included, which orders block n+1's
// outputs after its tails.
struct HostGraphKey {  // launch shapes a captured graph depends on
    int prec = -1, B = 0, head_pre = 0;
    int n_src = 0, n_dst = 0, ctas = 0, nw = 0, direct = 0, S = 0;  // the synthesis MAC
    size_t smem = 0;
    int f_src = 0, f_dst = 0, f_ctas = 0, f_nw = 0, f_direct = 0, f_S = 0;  // the canceller's (closed loop)
    size_t f_smem = 0;
    bool operator==(const HostGraphKey& o) const {
        return prec == o.prec && B == o.B && head_pre == o.head_pre && n_src == o.n_src && n_dst == o.n_dst &&
               ctas == o.ctas && nw == o.nw && direct == o.direct && S == o.S && smem == o.smem &&
               f_src == o.f_src && f_dst == o.f_dst && f_ctas == o.f_ctas && f_nw == o.f_nw &&
               f_direct == o.f_direct && f_S == o.f_S && f_smem == o.f_smem;
    }
};

enum { GN_PACK, GN_OUT, GN_TAIL, GN_FOUT, GN_FTAIL, GN_COUNT };  // kernel nodes of a graph

struct HostGraphForm {  // one captured graph
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    cudaGraphNode_t node[GN_COUNT] = {};
    cudaKernelNodeParams prm[GN_COUNT] = {};
    HostGraphKey key;
    // the nodes' current arguments: pack, output (and the push into the
    // canceller's ring), tail; the canceller's output and tail
    PackArgs pa{}, pb{};
    OutArgs oa{}, of{};
    MacArgs ma{}, mf{};
};

struct HostGraph {
    int mode = 1;  // 0 off, 1 when the previous tail has finished, 2 always
    bool live = false;  // the engine's last block went through a graph (its tails are not in the ev_tail events)
    HostGraphForm plain, loop;  // conv_process_block's, afc_process_block's
    cudaStream_t cs[3] = {nullptr, nullptr, nullptr};  // capture streams
    cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr}, ev_out = nullptr;
    long long blocks = 0;  // blocks that went through a graph
    bool called = false;   // a host call ran before (last_call is set)
    std::chrono::steady_clock::time_point last_call{};  // start of the previous host call
};

struct conv_engine {
    int dev = 0;
    double fs = 48000.0;
    int B = 0, log2B = 0, n_in = 0, n_out = 0;
    long long taps = 0;
    int prec = CONV_FP32;
    int num_sms = 0;
    cudaStream_t stream = nullptr;     // the engine's own stream for host-buffer calls
    // low-priority streams for the tail MACs, by block parity: [0], [1] the
    // synthesis, [2], [3] the canceller (so a canceller tail never queues
    // behind the much longer synthesis tail of the same block)
    cudaStream_t bg[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_done = nullptr;     // output of the current host-buffer call is on the host
    cudaEvent_t ev_handoff = nullptr;  // orders a block after the previous one enqueued on another stream
    cudaStream_t last_stream = nullptr;
    bool has_last = false;
    float2* tw = nullptr;
    float2* tw_lo = nullptr;  // tw's residuals W_2B^j - tw[j] (float-float FFT of the NLMS step)
    // n_f = 3 n_x form (afc_set_spectrum_reuse): every spectrum has 3B/2 bins,
    // the synthesis keeps two blocks of history, and its output spectrum is
    // pushed into the canceller's delay line as it is; tw3[j] = W_3B^j
    bool reuse = false;
    float2* tw3 = nullptr;
    float *d_e = nullptr, *d_c = nullptr;
    float *h_in = nullptr, *h_out = nullptr, *h_e = nullptr;
    float *m_in = nullptr, *m_out = nullptr, *m_e = nullptr;  // device addresses of h_in / h_out / h_e (mapped pinned memory)
    int* h_err = nullptr;
    int* d_err = nullptr;
    TileOverride tiling;  // applies to the synthesis convolution
    Part syn, fb;
    long long nblk = 0;
    double guard = 0.0;
    bool prof = false;
    std::vector<cudaEvent_t> ev0, ev1;
    void* flush_buf = nullptr;  // conv_profile_flush_l2: read before each timed tail
    // conv_set_l2_keep: bytes of tail filter spectra streamed with the L2
    // evict-last policy, so the next block finds them in L2 (measured at the
    // paper configuration: 52-60 MB gives the shortest steps, FP32 and FP16)
    long long l2_keep = 56LL * 1000 * 1000;
    size_t flush_bytes = 0;
    size_t ev_used = 0;
    size_t dev_bytes = 0;
    // adaptive canceller (afc_set_adaptation)
    bool adapt = false;
    float mu = 0.0f, lam = 0.0f, delta = 0.0f;
    cudaStream_t as = nullptr;     // high-priority stream of the NLMS step (critical path)
    cudaEvent_t ev_prep = nullptr;    // this block's step G is ready (the power sum has read the ring)
    cudaEvent_t ev_corr = nullptr;    // the next block's correlation chunks are written
    float2* d_pow = nullptr;     // [2][B] packed power estimates, by block parity
    float2* d_G = nullptr;       // [3][n_in][B] step-scaled error spectra, by block mod 3
    float2* d_A = nullptr;       // [2][2][9][B] correlation chunks + their sum (block parity, lag one/two)
    unsigned* d_ticket = nullptr;  // [B] completion counters of the correlation kernel
    float2* d_side = nullptr;    // [2][n_kt][n_out][BT] ring slots the pushes overwrote, by block parity
    bool upd_pending = false;    // the previous block's step is not yet in the tail partitions
    int fb_S_full = 0;           // the canceller's default splits (the adaptive pass; its partials' size)
    int in_batches = 0;          // batches holding this session
    // non-uniform partitioning (conv_set_far_block): taps [0, far_B) in this
    // engine's own partitions of `block`, taps [far_B, taps) in a nested engine
    // of block far_B driven once every far_B / block blocks
    conv_engine* far = nullptr;
    int far_B = 0;
    long long taps_total = 0;
    float* d_acc = nullptr;             // [n_in][far_B] input of the far engine's next block
    float* d_far_out[2] = {nullptr, nullptr};  // [n_out][far_B] far outputs, by far-block parity
    const float* addend = nullptr;      // added by this block's output kernel, or null
    int addend_stride = 0;
    int e_stride = 0;                   // row pitch of the pack's e_out for this block (0: block)
    // conv_process_blocks: row pitches of the synthesis input and output (0: block)
    int io_in_stride = 0, io_out_stride = 0;
    float *d_cin = nullptr, *d_cout = nullptr;  // its device chunk buffers
    long long chunk_cap = 0;                    // blocks they hold
    cudaEvent_t ev_join = nullptr;  // conv_join_async: marks each of the engine's streams
    // fault-path testing (conv_inject_wait_timeout): the next synthesis tail
    // MAC withholds one stage and bounds its waits by inject_ns
    bool inject = false;
    unsigned long long inject_ns = 0;
    HostGraph hg;     // conv_process_block's graph (conv_set_host_graph)
    long long* d_blk = nullptr;  // its block number (the next block the graph processes)
    conv_stats st{};  // counters of conv_get_stats
};

namespace {

// The host-call graph's block number in device memory.
__global__ void k_blk_set(long long* blk, long long n) { *blk = n; }
__global__ void k_blk_advance(long long* blk) { *blk += 1; }

// Reads n 16-byte words (kernel timing's L2 flush: clean lines of this buffer
// replace whatever the cache held, with no write-back left for the next
// kernel).  The buffer is zero, so the store that keeps the loads is never
// taken.
__global__ void k_l2_flush_read(const uint4* __restrict__ p, size_t n, unsigned* sink) {
    unsigned acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = p[i];
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9e3779b9u) *sink = acc;
}

template <typename T>
int dev_alloc(conv_engine* e, T** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t r = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (r != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_err(r == cudaErrorMemoryAllocation ? CONV_E_NOMEM : CONV_E_CUDA, "cudaMalloc(%zu): %s", bytes,
                       cudaGetErrorString(r));
    }
    e->dev_bytes += bytes;
    return CONV_OK;
}

template <typename T>
void dev_free(conv_engine* e, T** p, size_t bytes) {
    if (*p) {
        cudaFree(*p);
        e->dev_bytes -= bytes ? bytes : 16;
    }
    *p = nullptr;
}

void part_free(conv_engine* e, Part& P) {
    if (!P.allocated) return;
    const MacPlan& p = P.plan;
    dev_free(e, &P.H, p.h_bytes);
    dev_free(e, &P.X, p.x_bytes);
    dev_free(e, &P.partial[0], p.partial_bytes);
    dev_free(e, &P.partial[1], p.partial_bytes);
    dev_free(e, &P.win, P.win_floats * sizeof(float));
    if (P.sH) dev_free(e, &P.sH, ((size_t)p.n_lt * p.R + 4) * sizeof(float));
    if (P.sX) dev_free(e, &P.sX, ((size_t)p.R + 4) * sizeof(float));
    P.allocated = false;
    P.ready = false;
}

int check_fits(size_t need) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const size_t margin = 64ull << 20;
    if (need + margin > free_b)
        return set_err(CONV_E_NOMEM, "device footprint %zu bytes does not fit in %zu free bytes", need, free_b);
    return CONV_OK;
}

// Packed bins per spectrum row (n_f / 2) and history samples per channel of
// the input window (n_f - n_x): n_f = 2 n_x, or 3 n_x in the reuse form.
inline int bins_of(const conv_engine* e) { return e->reuse ? 3 * (e->B / 2) : e->B; }
inline int hist_of(const conv_engine* e) { return e->reuse ? 2 * e->B : e->B; }

// Bin tile of the reuse form (3B/2 bins, not a power of two) when none is
// given: the planner's rule, rounded down to a power of two dividing the bins.
TileOverride reuse_tiling(const conv_engine* e, const TileOverride& o, int n_dst) {
    TileOverride r = o;
    if (!e->reuse || o.bin_tile) return r;
    const int bins = bins_of(e);
    const int LT = std::min(n_dst, 16), n_lt = (n_dst + LT - 1) / LT;
    int n_kt = 1;
    while (n_kt * 2 <= std::max(1, e->num_sms / (16 * n_lt))) n_kt *= 2;
    int bt = (int)pow2_floor((size_t)std::max(1, bins / n_kt));
    while (bt > 16 && bins % bt) bt /= 2;
    r.bin_tile = std::max(16, std::min(256, bt));
    return r;
}

int part_alloc(conv_engine* e, Part& P, int n_src, int n_dst, long long taps,
               const TileOverride& o = TileOverride()) {
    part_free(e, P);
    P.n_src = n_src;
    P.n_dst = n_dst;
    P.taps = taps;
    const long long K = (taps + e->B - 1) / e->B;
    if (K <= 0 || (long long)n_src * K > 0x7fffffffLL / 2)
        return set_err(CONV_E_INVAL, "taps %lld gives too many partitions", taps);
    P.K = (int)K;
    P.plan = plan_mac(e->prec, bins_of(e), n_src, n_dst, P.K, e->num_sms, n_src, reuse_tiling(e, o, n_dst));
    const MacPlan& p = P.plan;
    std::string why;
    if (check_plan(p, &why)) return set_err(CONV_E_INVAL, "%s", why.c_str());
    int rc = check_fits(part_bytes(p, e->prec, (size_t)n_src * hist_of(e)));
    if (rc) return rc;
    P.allocated = true;  // partial allocations are released by part_free
    if ((rc = dev_alloc(e, &P.H, p.h_bytes))) return rc;
    if ((rc = dev_alloc(e, &P.X, p.x_bytes))) return rc;
    if ((rc = dev_alloc(e, &P.partial[0], p.partial_bytes))) return rc;
    if ((rc = dev_alloc(e, &P.partial[1], p.partial_bytes))) return rc;
    if (!P.ev_packed) CK(cudaEventCreateWithFlags(&P.ev_packed, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i)
        if (!P.ev_tail[i]) CK(cudaEventCreateWithFlags(&P.ev_tail[i], cudaEventDisableTiming));
    P.win_floats = (size_t)n_src * hist_of(e);
    if ((rc = dev_alloc(e, &P.win, P.win_floats * sizeof(float)))) return rc;
    if (e->prec != PREC_FP32) {
        // +4 floats: scale runs are read widened to 16-byte boundaries
        if ((rc = dev_alloc(e, &P.sH, ((size_t)p.n_lt * p.R + 4) * sizeof(float)))) return rc;
        if ((rc = dev_alloc(e, &P.sX, ((size_t)p.R + 4) * sizeof(float)))) return rc;
        CK(cudaMemsetAsync(P.sH, 0, ((size_t)p.n_lt * p.R + 4) * sizeof(float), e->stream));
    }
    CK(cudaMemsetAsync(P.H, 0, p.h_bytes, e->stream));
    return CONV_OK;
}

int part_reset(conv_engine* e, Part& P) {
    if (!P.allocated) return CONV_OK;
    CK(cudaMemsetAsync(P.X, 0, P.plan.x_bytes, e->stream));
    CK(cudaMemsetAsync(P.win, 0, P.win_floats * sizeof(float), e->stream));
    if (P.sX) CK(cudaMemsetAsync(P.sX, 0, ((size_t)P.plan.R + 4) * sizeof(float), e->stream));
    CK(cudaMemsetAsync(P.partial[0], 0, P.plan.partial_bytes, e->stream));
    CK(cudaMemsetAsync(P.partial[1], 0, P.plan.partial_bytes, e->stream));
    CK(cudaEventRecord(P.ev_tail[0], e->stream));  // block 0's tail: zero partials
    CK(cudaEventRecord(P.ev_tail[1], e->stream));
    return CONV_OK;
}

// Upload time-domain filters [n_dst][n_src][taps] and build their spectra.
int part_set_filters(conv_engine* e, Part& P, const float* h) {
    const size_t bytes = (size_t)P.n_dst * P.n_src * (size_t)P.taps * sizeof(float);
    const size_t mbytes = e->prec != PREC_FP32 ? (size_t)P.n_dst * P.plan.R * sizeof(float) : 0;
    float* d_h = nullptr;
    float* d_max = nullptr;
    int rc = dev_alloc(e, &d_h, bytes);
    if (rc) return rc;
    if (mbytes && (rc = dev_alloc(e, &d_max, mbytes))) {
        dev_free(e, &d_h, bytes);
        return rc;
    }
    cudaError_t r = cudaMemcpyAsync(d_h, h, bytes, cudaMemcpyHostToDevice, e->stream);
    FilterArgs a{};
    a.h = d_h;
    a.taps = P.taps;
    a.n_dst = P.n_dst;
    a.n_src = P.n_src;
    a.K = P.K;
    a.B = e->B;
    a.log2B = e->log2B;
    a.BT = P.plan.BT;
    a.LT = P.plan.LT;
    a.H = P.H;
    a.sH = P.sH;
    a.maxabs = d_max;
    a.tile_elems = P.plan.tile_elems;
    a.tw = e->reuse ? e->tw3 : e->tw;
    auto launch = [&](const FilterArgs& fa) {
        return e->reuse ? launch_filter3(e->prec, fa, e->stream) : launch_filter_r2c(e->prec, fa, e->stream);
    };
    if (e->prec != PREC_FP32) {
        // pass 0: per-sub-filter maxima; one scale per (output tile, r); pass 1: store
        a.pass = 0;
        if (r == cudaSuccess) r = launch(a);
        if (r == cudaSuccess)
            r = launch_tile_scales(e->prec, d_max, P.sH, P.n_dst, P.plan.R, P.plan.LT, e->stream);
    }
    a.pass = 1;
    if (r == cudaSuccess) r = launch(a);
    if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
    dev_free(e, &d_h, bytes);
    if (d_max) dev_free(e, &d_max, mbytes);
    if (r != cudaSuccess) return set_err(CONV_E_CUDA, "filter spectra: %s", cudaGetErrorString(r));
    P.ready = true;
    return CONV_OK;
}

inline int slot0_for(long long n, int K) {
    const int m = (int)(n % K);
    return m == 0 ? 0 : K - m;
}

// Argument blocks of one block of one partitioned convolution (shared by the
// single-engine launches and the batched ones).
PackArgs pack_args(conv_engine* e, Part& P, long long blk, const float* src, int stride, const float* sub,
                   float* e_out) {
    PackArgs a{};
    a.in = src;
    a.in_stride = stride;
    a.sub = sub;
    a.e_out = e_out;
    a.e_stride = e_out && &P == &e->syn ? e->e_stride : 0;
    a.win = P.win;
    a.X = P.X;
    a.sX = P.sX;
    a.B = e->B;
    a.log2B = e->log2B;
    a.BT = P.plan.BT;
    a.n_ch = P.n_src;
    a.K = P.K;
    a.slot = slot0_for(blk, P.K);
    a.tw = e->reuse ? e->tw3 : e->tw;
    return a;
}

// First reduction index past the tail filter rows kept in L2 (MacArgs.keep_r):
// the canceller's spectra (small, read every block) take the budget first,
// the synthesis gets the rest; a row r holds every output's and bin's value.
int keep_r_of(const conv_engine* e, const Part& P) {
    const MacPlan& p = P.plan;
    const long long row = (long long)p.n_dst * p.B * p.es;
    long long budget = e->l2_keep;
    if (&P == &e->syn && e->fb.allocated) {
        const MacPlan& f = e->fb.plan;
        budget -= std::min(budget, (long long)(f.R - f.r_begin) * f.n_dst * f.B * f.es);
    }
    const long long rows = row > 0 ? std::min<long long>(p.R - p.r_begin, budget / row) : 0;
    return p.r_begin + (int)rows;
}

MacArgs tail_args(conv_engine* e, Part& P, long long blk) {
    const MacPlan& p = P.plan;
    MacArgs a{};
    a.H = P.H;
    a.X = P.X;
    a.sH = P.sH;
    a.sX = P.sX;
    a.partial = P.partial[blk & 1];
    a.B = p.B;
    a.BT = p.BT;
    a.n_kt = p.n_kt;
    a.n_dst = p.n_dst;
    a.LT = p.LT;
    a.n_lt = p.n_lt;
    a.n_src = p.n_src;
    a.K = p.K;
    a.S = p.S;
    a.RS = p.RS;
    a.nstage = p.nstage;
    a.r_begin = p.r_begin;
    a.interleave = p.interleave;
    a.kthreads = p.kthreads;
    a.NLG = p.NLG;
    a.NRL = p.NRL;
    a.slot0 = slot0_for(blk, P.K);
    a.stage_bytes = p.stage_bytes;
    a.xoff = p.xoff;
    a.soff = p.soff;
    a.sxoff = p.sxoff;
    a.tile_elems = p.tile_elems;
    a.err = e->d_err;
    a.keep_r = keep_r_of(e, P);
    if (e->inject && &P == &e->syn) {
        a.withhold = 1;
        a.wait_ns = e->inject_ns;
        e->inject = false;
    }
    return a;
}

OutArgs out_args(conv_engine* e, Part& P, long long blk, float* out) {
    const MacPlan& p = P.plan;
    OutArgs a{};
    a.partial = P.partial[blk & 1];
    a.S = p.S;
    a.n_dst = P.n_dst;
    a.B = e->B;
    a.log2B = e->log2B;
    a.tw = e->reuse ? e->tw3 : e->tw;
    a.out = out;
    a.out_stride = (&P == &e->syn && e->io_out_stride) ? e->io_out_stride : e->B;
    a.head = 1;
    a.H = P.H;
    a.X = P.X;
    a.sH = P.sH;
    a.sX = P.sX;
    a.n_src = P.n_src;
    a.K = P.K;
    a.R = p.R;
    a.BT = p.BT;
    a.LT = p.LT;
    a.slot0 = slot0_for(blk, P.K);
    a.tile_elems = p.tile_elems;
    if (&P == &e->syn && e->addend) {
        a.extra = e->addend;
        a.extra_stride = e->addend_stride;
    }
    a.early_partials = 1;  // every schedule waits for the tail's event before the output launch
    a.head_pre = (!e->reuse && out_head_smem(P.n_src, e->B) > 0) ? 1 : 0;
    return a;
}

int enqueue_pack(conv_engine* e, Part& P, const float* src, int stride, const float* sub, float* e_out,
                 cudaStream_t s, bool closed_loop = false) {
    const PackArgs a = pack_args(e, P, e->nblk, src, stride, sub, e_out);
    CK(e->reuse ? launch_pack3(e->prec, a, s) : launch_pack_r2c(e->prec, a, s, closed_loop));
    return CONV_OK;
}

// Tail MAC for block `blk`: partitions 1..K-1, into the partial buffer of the
// block's parity.
int enqueue_tail(conv_engine* e, Part& P, long long blk, cudaStream_t s, bool timed, bool pdl = true) {
    const MacPlan& p = P.plan;
    if (p.S == 0) return CONV_OK;  // K = 1: no tail
    const bool rec = timed && e->prof && e->ev_used < e->ev0.size();
    if (rec && e->flush_bytes) {
        k_l2_flush_read<<<e->num_sms * 4, 256, 0, s>>>(static_cast<const uint4*>(e->flush_buf),
                                                        e->flush_bytes / sizeof(uint4),
                                                        static_cast<unsigned*>(e->flush_buf));
        CK(cudaGetLastError());
    }
    if (rec) CK(cudaEventRecord(e->ev0[e->ev_used], s));
    CK(launch_fdl_mac(e->prec, p, tail_args(e, P, blk), s, pdl));
    if (rec) {
        CK(cudaEventRecord(e->ev1[e->ev_used], s));
        ++e->ev_used;
    }
    return CONV_OK;
}

// Output of block `blk`: head (partition 0) + tail partials + C2R + OLS.
int enqueue_out(conv_engine* e, Part& P, long long blk, float* out, cudaStream_t s) {
    const OutArgs a = out_args(e, P, blk, out);
    CK(e->reuse ? launch_out3(e->prec, a, PackArgs{}, s) : launch_out_c2r(e->prec, a, s));
    return CONV_OK;
}

// One block of one partitioned convolution on stream s (see the schedule at
// the top of this file).
int enqueue_conv(conv_engine* e, Part& P, const float* src, const float* sub, float* e_out, float* out,
                 cudaStream_t s, bool timed) {
    int rc;
    const long long n = e->nblk;
    const int in_stride = (&P == &e->syn && e->io_in_stride) ? e->io_in_stride : e->B;
    if ((rc = enqueue_pack(e, P, src, in_stride, sub, e_out, s))) return rc;
    CK(cudaEventRecord(P.ev_packed, s));
    CK(cudaStreamWaitEvent(s, P.ev_tail[n & 1], 0));
    if ((rc = enqueue_out(e, P, n, out, s))) return rc;
    cudaStream_t bg = e->bg[(&P == &e->fb ? 2 : 0) + ((n + 1) & 1)];
    CK(cudaStreamWaitEvent(bg, P.ev_packed, 0));
    // kernel timing needs each tail alone on the GPU: then tails run one after another
    if (timed && e->prof) CK(cudaStreamWaitEvent(bg, P.ev_tail[n & 1], 0));
    if ((rc = enqueue_tail(e, P, n + 1, bg, timed))) return rc;
    CK(cudaEventRecord(P.ev_tail[(n + 1) & 1], bg));
    return CONV_OK;
}

int check_dev_err(conv_engine* e) {
    if (e->far) {
        const int rc = check_dev_err(e->far);
        if (rc) return rc;
    }
    const int v = *(volatile int*)e->h_err;
    if (v != DEVERR_NONE) {
        *(volatile int*)e->h_err = DEVERR_NONE;
        ++e->st.device_errors;
        return set_err(CONV_E_TIMEOUT, "device-side wait gave up (code %d); results of the block are invalid", v);
    }
    return CONV_OK;
}

// Latency record of one blocking host-buffer call that started at t0.
void record_call(conv_engine* e, std::chrono::steady_clock::time_point t0) {
    const double us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    conv_stats& st = e->st;
    ++st.timed_calls;
    st.sum_latency_us += us;
    if (us > st.max_latency_us) st.max_latency_us = us;
    if (us > (double)e->B / e->fs * 1e6) ++st.deadline_misses;
    int b = 0;
    while (b < CONV_STATS_BUCKETS - 1 && us >= (double)(2ll << b)) ++b;
    ++st.latency_hist[b];
}

// Makes stream s wait for everything the engine has enqueued on its own
// streams (background tails, the NLMS step stream, the host-call stream, the
// stream of the last block) and on its far engine's.
int join_streams(conv_engine* e, cudaStream_t s) {
    if (e->far) {
        const int rc = join_streams(e->far, s);
        if (rc) return rc;
    }
    cudaStream_t src[7] = {e->bg[0], e->bg[1], e->bg[2], e->bg[3], e->as, e->stream,
                           e->has_last ? e->last_stream : e->stream};
    for (int i = 0; i < 7; ++i) {
        if (!src[i] || src[i] == s) continue;
        CK(cudaEventRecord(e->ev_join, src[i]));
        CK(cudaStreamWaitEvent(s, e->ev_join, 0));
    }
    return CONV_OK;
}

int flush_nlms_update(conv_engine* e);

int engine_reset(conv_engine* e) {
    int rc;
    if (e->has_last) CK(cudaStreamSynchronize(e->last_stream));  // blocks enqueued on a caller's stream
    for (int i = 0; i < 4; ++i) CK(cudaStreamSynchronize(e->bg[i]));
    if (e->as) CK(cudaStreamSynchronize(e->as));
    CK(cudaStreamSynchronize(e->stream));
    // the adapted spectra are kept: apply the step still pending on them
    if ((rc = flush_nlms_update(e))) return rc;
    if ((rc = part_reset(e, e->syn))) return rc;
    if ((rc = part_reset(e, e->fb))) return rc;
    if (e->d_c) CK(cudaMemsetAsync(e->d_c, 0, (size_t)e->n_in * e->B * sizeof(float), e->stream));
    if (e->d_pow) CK(cudaMemsetAsync(e->d_pow, 0, 2 * (size_t)e->B * sizeof(float2), e->stream));
    if (e->d_G) {  // zero ring: no step pending, correlations and saved entries zero
        CK(cudaMemsetAsync(e->d_G, 0, 3 * (size_t)e->n_in * e->B * sizeof(float2), e->stream));
        CK(cudaMemsetAsync(e->d_A, 0, 36 * (size_t)e->B * sizeof(float2), e->stream));
        CK(cudaMemsetAsync(e->d_side, 0, 2 * (size_t)e->n_out * e->B * sizeof(float2), e->stream));
    }
    e->upd_pending = false;
    if (e->far) {
        if ((rc = engine_reset(e->far))) return rc;
        CK(cudaMemsetAsync(e->d_acc, 0, (size_t)e->n_in * e->far_B * sizeof(float), e->stream));
        for (int i = 0; i < 2; ++i)
            CK(cudaMemsetAsync(e->d_far_out[i], 0, (size_t)e->n_out * e->far_B * sizeof(float), e->stream));
    }
    CK(cudaStreamSynchronize(e->stream));
    e->nblk = 0;
    e->has_last = false;
    e->hg.live = false;  // part_reset recorded the zero partials' events
    return CONV_OK;
}

int enqueue_block(conv_engine* e, const float* d_in, float* d_out, cudaStream_t s);

// Non-uniform partitioning around block n of the near part.  Far block k
// (input samples [k F, (k+1) F), F = far block) convolved with h[F:] lands on
// samples [(k+1) F, (k+2) F), i.e. on near blocks (k+1) m .. (k+2) m - 1
// (m = F / B): near block n adds slice n mod m of far block n / m - 1, which
// the far engine finished at the end of near block (n / m) m - 1.  Then this
// block's input (the error signal when the canceller runs) is appended to the
// far engine's next input, and after the m-th block the far engine runs.
void far_before(conv_engine* e) {
    if (!e->far) return;
    const int m = e->far_B / e->B;
    const long long k = e->nblk / m;
    const int j = (int)(e->nblk % m);
    e->addend = e->d_far_out[(k + 1) & 1] + (size_t)j * e->B;  // far block k - 1 (zeros before the first)
    e->addend_stride = e->far_B;
}

int far_after(conv_engine* e, const float* src, cudaStream_t s) {
    if (!e->far) return CONV_OK;
    e->addend = nullptr;
    const int m = e->far_B / e->B;
    const long long k = e->nblk / m;
    const int j = (int)(e->nblk % m);
    if (src)  // else the pack wrote the block into the far input already
        CK(cudaMemcpy2DAsync(e->d_acc + (size_t)j * e->B, (size_t)e->far_B * sizeof(float), src,
                             (size_t)e->B * sizeof(float), (size_t)e->B * sizeof(float), (size_t)e->n_in,
                             cudaMemcpyDeviceToDevice, s));
    if (j == m - 1) return enqueue_block(e->far, e->d_acc, e->d_far_out[k & 1], s);
    return CONV_OK;
}

// Blocks of one engine are a chain (window, ring, partials): a block enqueued on
// another stream than the previous one first waits for everything the
// previous stream holds.
int stream_handoff(conv_engine* e, cudaStream_t s) {
    if (e->has_last && s != e->last_stream) {
        CK(cudaEventRecord(e->ev_handoff, e->last_stream));
        CK(cudaStreamWaitEvent(s, e->ev_handoff, 0));
    }
    e->last_stream = s;
    e->has_last = true;
    return CONV_OK;
}

int host_graph_settle(conv_engine* e);

int enqueue_block(conv_engine* e, const float* d_in, float* d_out, cudaStream_t s) {
    if (int rc = host_graph_settle(e)) return rc;
    if (int rc = stream_handoff(e, s)) return rc;
    far_before(e);
    float* acc = nullptr;
    if (e->far) {  // the pack appends the input block to the far engine's next input directly
        acc = e->d_acc + (size_t)(e->nblk % (e->far_B / e->B)) * e->B;
        e->e_stride = e->far_B;
    }
    int rc = enqueue_conv(e, e->syn, d_in, nullptr, acc, d_out, s, true);
    e->e_stride = 0;
    if (!rc) rc = far_after(e, nullptr, s);
    if (rc) return rc;
    ++e->nblk;
    ++e->st.blocks;
    return CONV_OK;
}

void host_graph_free(HostGraphForm& F) {
    if (F.x) cudaGraphExecDestroy(F.x);
    if (F.g) cudaGraphDestroy(F.g);
    F = HostGraphForm{};
}

void host_graph_destroy(HostGraph& G) {
    host_graph_free(G.plain);
    host_graph_free(G.loop);
    for (int i = 0; i < 3; ++i)
        if (G.cs[i]) cudaStreamDestroy(G.cs[i]);
    for (int i = 0; i < 2; ++i) {
        if (G.ev_fork[i]) cudaEventDestroy(G.ev_fork[i]);
        if (G.ev_join[i]) cudaEventDestroy(G.ev_join[i]);
    }
    if (G.ev_out) cudaEventDestroy(G.ev_out);
    const int mode = G.mode;
    G = HostGraph{};
    G.mode = mode;
}

// Before a block goes through a stream again: the last graph's tails (block
// nblk's) are complete once the engine's stream has passed that graph launch.
int host_graph_settle(conv_engine* e) {
    if (!e->hg.live) return CONV_OK;
    CK(cudaEventRecord(e->syn.ev_tail[e->nblk & 1], e->stream));
    if (e->fb.allocated) CK(cudaEventRecord(e->fb.ev_tail[e->nblk & 1], e->stream));
    e->hg.live = false;
    return CONV_OK;
}

// loop: afc_process_block's graph (the static canceller), else conv_process_block's.
bool host_graph_eligible(const conv_engine* e, bool loop) {
    return e->hg.mode > 0 && !e->reuse && !e->far && !e->prof && !e->adapt && !e->inject && e->in_batches == 0 &&
           !e->io_in_stride && !e->io_out_stride && (!loop || e->fb.ready);
}

// The graph pays off when the previous block's tail has finished, as in
// real-time use (one call per block period).  Back to back, the stream path
// starts the pack while that tail still runs, which the graph would wait for
// (measured, paper 4x16, block 256, FP32: 27.4 us per call on the stream path
// against 32.2 us through the graph).  Mode 1 tells the two uses apart by the
// host clock: asking the device (an event or stream query) cost about 2 us per
// call, most of what the graph saves.  The choice never changes the result.
bool host_graph_now(conv_engine* e, std::chrono::steady_clock::time_point t0) {
    HostGraph& G = e->hg;
    const double gap_s = std::chrono::duration<double>(t0 - G.last_call).count();
    G.last_call = t0;
    const bool first = !G.called;
    G.called = true;
    return G.mode == 2 || first || gap_s >= 0.5 * (double)e->B / e->fs;
}

HostGraphKey host_graph_key(const conv_engine* e, bool loop) {
    const MacPlan& p = e->syn.plan;
    HostGraphKey k;
    k.prec = e->prec;
    k.B = e->B;
    k.head_pre = out_head_smem(e->syn.n_src, e->B) > 0 ? 1 : 0;
    k.n_src = e->syn.n_src;
    k.n_dst = e->syn.n_dst;
    k.ctas = p.ctas;
    k.nw = p.nw;
    k.direct = p.direct;
    k.S = p.S;
    k.smem = p.smem;
    if (loop) {
        const MacPlan& f = e->fb.plan;
        k.f_src = e->fb.n_src;
        k.f_dst = e->fb.n_dst;
        k.f_ctas = f.ctas;
        k.f_nw = f.nw;
        k.f_direct = f.direct;
        k.f_S = f.S;
        k.f_smem = f.smem;
    }
    return k;
}

// The node that the last launch captured on stream s added to the graph.
int captured_node(cudaStream_t s, cudaGraphNode_t* node) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd));
    if (st != cudaStreamCaptureStatusActive || nd != 1) return set_err(CONV_E_CUDA, "graph capture lost its node");
    *node = deps[0];
    return CONV_OK;
}

// Stream `to` continues after what stream `from` has captured so far.
int capture_fork(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
    CK(cudaEventRecord(ev, from));
    CK(cudaStreamWaitEvent(to, ev, 0));
    return CONV_OK;
}

// Captures one block of the form's work on the capture streams, with the
// form's stored arguments.
int host_graph_capture(conv_engine* e, bool loop, HostGraphForm& F) {
    HostGraph& G = e->hg;
    cudaStream_t c0 = G.cs[0], c1 = G.cs[1], c2 = G.cs[2];
    int rc;
    CK(launch_pack_r2c(e->prec, F.pa, c0, loop));
    if ((rc = captured_node(c0, &F.node[GN_PACK]))) return rc;
    if ((rc = capture_fork(c0, c1, G.ev_fork[0]))) return rc;
    if (e->syn.plan.S > 0) {  // else K = 1: no tail
        CK(launch_fdl_mac(e->prec, e->syn.plan, F.ma, c1, false));
        if ((rc = captured_node(c1, &F.node[GN_TAIL]))) return rc;
    }
    CK(loop ? launch_out_push(e->prec, F.oa, F.pb, c0) : launch_out_c2r(e->prec, F.oa, c0));
    if ((rc = captured_node(c0, &F.node[GN_OUT]))) return rc;
    CK(cudaEventRecordWithFlags(G.ev_out, c0, cudaEventRecordExternal));  // the call waits for this
    if (loop) {
        if ((rc = capture_fork(c0, c2, G.ev_fork[1]))) return rc;
        if (e->fb.plan.S > 0) {
            CK(launch_fdl_mac(e->prec, e->fb.plan, F.mf, c2, false));
            if ((rc = captured_node(c2, &F.node[GN_FTAIL]))) return rc;
        }
        CK(launch_out_c2r(e->prec, F.of, c0, true));
        if ((rc = captured_node(c0, &F.node[GN_FOUT]))) return rc;
        if ((rc = capture_fork(c2, c0, G.ev_join[1]))) return rc;
    }
    if ((rc = capture_fork(c1, c0, G.ev_join[0]))) return rc;
    k_blk_advance<<<1, 1, 0, c0>>>(e->d_blk);  // after the outputs and the tails have read it
    CK(cudaGetLastError());
    return CONV_OK;
}

void copy_args(HostGraphForm& to, const HostGraphForm& from) {
    std::memcpy(&to.pa, &from.pa, sizeof to.pa);
    std::memcpy(&to.pb, &from.pb, sizeof to.pb);
    std::memcpy(&to.oa, &from.oa, sizeof to.oa);
    std::memcpy(&to.of, &from.of, sizeof to.of);
    std::memcpy(&to.ma, &from.ma, sizeof to.ma);
    std::memcpy(&to.mf, &from.mf, sizeof to.mf);
}

int host_graph_build(conv_engine* e, bool loop, HostGraphForm& F, const HostGraphForm& now) {
    HostGraph& G = e->hg;
    host_graph_free(F);
    if (!G.cs[0]) {
        for (int i = 0; i < 3; ++i) CK(cudaStreamCreateWithFlags(&G.cs[i], cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            CK(cudaEventCreateWithFlags(&G.ev_fork[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&G.ev_join[i], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&G.ev_out, cudaEventDisableTiming));
    }
    copy_args(F, now);
    CK(cudaStreamBeginCapture(G.cs[0], cudaStreamCaptureModeThreadLocal));
    const int rc = host_graph_capture(e, loop, F);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(G.cs[0], &g);
    if (rc || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        host_graph_free(F);
        cudaGetLastError();
        return rc ? rc : set_err(CONV_E_CUDA, "graph capture: %s", cudaGetErrorString(ec));
    }
    F.g = g;
    CK(cudaGraphInstantiate(&F.x, F.g, 0));
    for (int i = 0; i < GN_COUNT; ++i)
        if (F.node[i]) CK(cudaGraphKernelNodeGetParams(F.node[i], &F.prm[i]));
    F.key = host_graph_key(e, loop);  // last: a failed build leaves no key that matches
    return CONV_OK;
}

int set_node_args(HostGraphForm& F, int i, void* a0, void* a1 = nullptr) {
    void* argv[2] = {a0, a1};
    F.prm[i].kernelParams = argv;
    const cudaError_t r = cudaGraphExecKernelNodeSetParams(F.x, F.node[i], &F.prm[i]);
    F.prm[i].kernelParams = nullptr;
    CK(r);
    return CONV_OK;
}

// Copies an argument block into the node's stored one and reports whether it
// changed (compared byte for byte: a difference in padding only costs an
// unneeded update).
template <typename T>
bool args_changed(T& stored, const T& now) {
    if (std::memcmp(&stored, &now, sizeof(T)) == 0) return false;
    std::memcpy(&stored, &now, sizeof(T));
    return true;
}

// The arguments of block 0, with the block number read from d_blk instead.
void host_graph_args(conv_engine* e, bool loop, HostGraphForm& a) {
    Part& P = e->syn;
    Part& Q = e->fb;
    long long* blk = e->d_blk;
    a.pa = pack_args(e, P, 0, e->m_in, e->B, loop ? e->d_c : nullptr, loop ? e->m_e : nullptr);
    a.pa.blk = blk;
    a.oa = out_args(e, P, 0, e->m_out);
    a.oa.blk = blk;
    a.oa.partial_b = P.partial[1];
    if (P.plan.S > 0) {
        a.ma = tail_args(e, P, 0);
        a.ma.blk = blk;
        a.ma.blk_add = 1;  // the tail of the next block
        a.ma.partial_b = P.partial[1];
    }
    if (!loop) return;
    a.pb = pack_args(e, Q, 0, e->m_out, e->B, nullptr, nullptr);  // the output pushed into the canceller's ring
    a.pb.blk = blk;
    a.of = out_args(e, Q, 0, e->d_c);  // the prediction for the next block
    a.of.blk = blk;
    a.of.partial_b = Q.partial[1];
    if (Q.plan.S > 0) {
        a.mf = tail_args(e, Q, 0);
        a.mf.blk = blk;
        a.mf.blk_add = 1;
        a.mf.partial_b = Q.partial[1];
    }
}

// One block of conv_process_block (loop = false) or afc_process_block
// (loop = true) through its graph; the stream paths are enqueue_block and
// enqueue_afc_synthesis + enqueue_afc_prediction with the mapped host buffers.
int host_graph_block(conv_engine* e, bool loop) {
    HostGraph& G = e->hg;
    HostGraphForm& F = loop ? G.loop : G.plain;
    const long long n = e->nblk;
    int rc;
    if (!e->d_blk && (rc = dev_alloc(e, &e->d_blk, sizeof(long long)))) return rc;
    HostGraphForm now;
    host_graph_args(e, loop, now);
    if (!F.x || !(F.key == host_graph_key(e, loop))) {
        if ((rc = host_graph_build(e, loop, F, now))) return rc;
    } else {  // a new L2 budget, new buffers after a replan, ...
        const bool out_new = args_changed(F.oa, now.oa) | args_changed(F.pb, now.pb);
        if (args_changed(F.pa, now.pa) && (rc = set_node_args(F, GN_PACK, &F.pa))) return rc;
        if (out_new && (rc = set_node_args(F, GN_OUT, &F.oa, loop ? &F.pb : nullptr))) return rc;
        if (F.node[GN_TAIL] && args_changed(F.ma, now.ma) && (rc = set_node_args(F, GN_TAIL, &F.ma))) return rc;
        if (F.node[GN_FOUT] && args_changed(F.of, now.of) && (rc = set_node_args(F, GN_FOUT, &F.of))) return rc;
        if (F.node[GN_FTAIL] && args_changed(F.mf, now.mf) && (rc = set_node_args(F, GN_FTAIL, &F.mf))) return rc;
    }
    if ((rc = stream_handoff(e, e->stream))) return rc;
    if (!G.live) {
        // block n's tails ran on background streams (or are the reset's zero
        // partials), and the host kept the block number
        CK(cudaStreamWaitEvent(e->stream, e->syn.ev_tail[n & 1], 0));
        if (loop) CK(cudaStreamWaitEvent(e->stream, e->fb.ev_tail[n & 1], 0));
        k_blk_set<<<1, 1, 0, e->stream>>>(e->d_blk, n);
        CK(cudaGetLastError());
    }
    CK(cudaGraphLaunch(F.x, e->stream));
    G.live = true;
    ++G.blocks;
    ++e->nblk;
    ++e->st.blocks;
    return CONV_OK;
}

// Ring slot of block m's spectra (m may be negative: zeros before the first block).
inline int slot_of(long long m, int K) {
    const int r = (int)((-m) % K);
    return r < 0 ? r + K : r;
}

// Three step buffers: block m+2's step kernel may run while block m's step is
// still being applied to the tail partitions.
float2* G_of(conv_engine* e, long long m) { return e->d_G + (size_t)(((m % 3) + 3) % 3) * e->n_in * e->B; }
float2* side_of(conv_engine* e, long long m) { return e->d_side + (size_t)(m & 1) * e->n_out * e->B; }
// Correlation chunks of block m (index 0..7) and their sum (index 8).
float2* A_of(conv_engine* e, long long m, int lag, int idx = 0) {
    return e->d_A + (((size_t)(m & 1) * 2 + (lag - 1)) * 9 + idx) * e->B;
}

// Adaptive canceller (deferred update, see nlms.h), block n.
// On the high-priority stream e->as once e_n is written: the step G_n
// (nlms_prep: R2C of e_n, the power recursion over the newest delay-line
// entry, block n-1) and its application to partition 0.
int enqueue_nlms_prep(conv_engine* e, const float* d_err_block) {
    Part& F = e->fb;
    const MacPlan& p = F.plan;
    const long long n = e->nblk;
    CK(cudaStreamWaitEvent(e->as, e->syn.ev_packed, 0));  // e_n is written
    NlmsPrepArgs a{};
    a.e = d_err_block;
    a.U = static_cast<const float2*>(F.X);
    a.slot0 = slot_of(n - 1, F.K);
    a.pow_in = e->d_pow + (size_t)(n & 1) * e->B;
    a.pow_out = e->d_pow + (size_t)((n + 1) & 1) * e->B;
    a.G = G_of(e, n);
    a.B = e->B;
    a.log2B = e->log2B;
    a.BT = p.BT;
    a.L = F.n_src;
    a.K = F.K;
    a.mu = e->mu;
    a.lam = e->lam;
    a.delta = e->delta;
    a.tw = e->tw;
    a.tw_lo = e->tw_lo;
    a.F = static_cast<float2*>(F.H);
    a.LT = p.LT;
    a.n_lt = p.n_lt;
    a.tile_elems = p.tile_elems;
    CK(launch_nlms_prep(a, F.n_dst, e->as));
    CK(cudaEventRecord(e->ev_prep, e->as));
    return CONV_OK;
}

// Arguments of block m's step on the tail partitions (entries j = 1..K-1,
// blocks m-2 .. m-1-K).  after_push: block m+1's push is done, so blocks m-K
// and m+1-K come from the saved slots; else only block m-K.
NlmsUpdateArgs update_args(conv_engine* e, long long m, bool after_push) {
    Part& F = e->fb;
    const MacPlan& p = F.plan;
    NlmsUpdateArgs u{};
    u.F = static_cast<float2*>(F.H);
    u.U = static_cast<const float2*>(F.X);
    u.G = G_of(e, m);
    u.B = e->B;
    u.BT = p.BT;
    u.n_kt = p.n_kt;
    u.LT = p.LT;
    u.n_lt = p.n_lt;
    u.P = F.n_dst;
    u.L = F.n_src;
    u.K = F.K;
    u.slot0 = slot_of(m - 1, F.K);  // entry 0 = block m-1
    u.r_begin = F.n_src;
    // few rows per CTA: every thread's read-modify-writes of F_hat are in flight at once
    const long long rows = (long long)(p.R - u.r_begin) * p.n_kt * p.n_lt;
    u.rows_per_cta = (int)std::max<long long>(1, std::min<long long>(4, (rows + 16LL * e->num_sms - 1) /
                                                                             (16LL * e->num_sms)));
    u.tile_elems = p.tile_elems;
    u.U_old[0] = side_of(e, m);
    u.U_old[1] = after_push ? side_of(e, m + 1) : nullptr;
    return u;
}

// Block m's step on the tail partitions on its own (before block m+1's push).
int enqueue_nlms_update(conv_engine* e, long long m, cudaStream_t s) {
    if (m < 0 || e->fb.K < 2) return CONV_OK;
    CK(launch_nlms_update(update_args(e, m, false), s));
    return CONV_OK;
}

// After block m+1's push: block m's step on the tail partitions (if `step`)
// in one pass with the tail MAC of block m+2 (which needs F_m).
int enqueue_nlms_update_mac(conv_engine* e, long long m, bool step, cudaStream_t s) {
    Part& F = e->fb;
    if (F.K < 2 || e->fb_S_full == 0) return CONV_OK;
    NlmsUpdateMacArgs a{};
    a.u = update_args(e, m, true);
    if (!step || m < 0) a.u.G = nullptr;
    a.partial = static_cast<float2*>(F.partial[(m + 2) & 1]);
    a.S = e->fb_S_full;
    a.mac_slot0 = slot_of(m + 2, F.K);
    CK(launch_nlms_update_mac(a, s));
    return CONV_OK;
}

// Correlation chunks for block m+1 from the delay line after block m's push.
int enqueue_nlms_corr(conv_engine* e, long long m, cudaStream_t s) {
    Part& F = e->fb;
    NlmsCorrArgs c{};
    c.C = nlms_corr_chunks(F.K);
    if (c.C == 0) return CONV_OK;
    c.U = static_cast<const float2*>(F.X);
    c.oldest = side_of(e, m);
    c.A1 = A_of(e, m + 1, 1);
    c.A2 = A_of(e, m + 1, 2);
    c.A1f = A_of(e, m + 1, 1, 8);
    c.A2f = A_of(e, m + 1, 2, 8);
    c.ticket = e->d_ticket;
    c.B = e->B;
    c.BT = F.plan.BT;
    c.L = F.n_src;
    c.K = F.K;
    c.slot_m = slot_of(m, F.K);
    CK(launch_nlms_corr(c, s));
    return CONV_OK;
}

// Applies a pending step now, before the next push (reading the spectra back,
// or leaving the adaptive schedule).
int flush_nlms_update(conv_engine* e) {
    if (!e->upd_pending) return CONV_OK;
    e->upd_pending = false;
    int rc = enqueue_nlms_update(e, e->nblk - 1, e->stream);
    if (rc) return rc;
    CK(cudaStreamSynchronize(e->stream));
    return CONV_OK;
}

// Synthesis with feedback cancellation (Sec. 5): e = mic - c_prev, l = H^T * e
// (first half), then c = F_hat * l, kept for the next block (second half).
// The synthesis output kernel also pushes l_n into the canceller's delay line
// (one kernel less on the block's critical path).  The host-buffer call
// copies l and e out between the halves.
int enqueue_afc_synthesis(conv_engine* e, const float* d_mic, float* d_out, float* d_e, cudaStream_t s) {
    if (int rc = host_graph_settle(e)) return rc;
    if (int rc = stream_handoff(e, s)) return rc;
    Part& P = e->syn;
    Part& F = e->fb;
    const long long n = e->nblk;
    // the far engine's input and the NLMS step's input are the error signal
    float* eb = d_e ? d_e : ((e->far || e->adapt) ? e->d_e : nullptr);
    int rc;
    far_before(e);
    if ((rc = enqueue_pack(e, P, d_mic, e->B, e->d_c, eb, s, true))) return rc;
    CK(cudaEventRecord(P.ev_packed, s));
    if (e->adapt && (rc = enqueue_nlms_prep(e, eb))) return rc;
    CK(cudaStreamWaitEvent(s, P.ev_tail[n & 1], 0));
    PackArgs pa = pack_args(e, F, n, d_out, e->B, nullptr, nullptr);
    if (e->adapt) {
        // The push keeps the entry it overwrites (block n-K) for the deferred
        // step; the previous block's background work has read the slots
        // involved; with K = 1 the step kernel reads the overwritten slot.
        pa.save_old = side_of(e, n);
        CK(cudaStreamWaitEvent(s, F.ev_tail[n & 1], 0));
        CK(cudaStreamWaitEvent(s, e->ev_corr, 0));
        if (F.K == 1) CK(cudaStreamWaitEvent(s, e->ev_prep, 0));
    }
    // n_f = 3 n_x: the synthesis output spectrum itself goes into the
    // canceller's ring; else the output samples are packed and transformed
    CK(e->reuse ? launch_out3(e->prec, out_args(e, P, n, d_out), pa, s)
                : launch_out_push(e->prec, out_args(e, P, n, d_out), pa, s));
    CK(cudaEventRecord(F.ev_packed, s));
    cudaStream_t bg = e->bg[(n + 1) & 1];
    CK(cudaStreamWaitEvent(bg, P.ev_packed, 0));
    if (e->prof) CK(cudaStreamWaitEvent(bg, P.ev_tail[n & 1], 0));
    if ((rc = enqueue_tail(e, P, n + 1, bg, true))) return rc;
    CK(cudaEventRecord(P.ev_tail[(n + 1) & 1], bg));
    return far_after(e, eb, s);
}

int enqueue_afc_prediction(conv_engine* e, cudaStream_t s) {
    Part& F = e->fb;
    const long long n = e->nblk;
    int rc;
    CK(cudaStreamWaitEvent(s, F.ev_tail[n & 1], 0));
    OutArgs oa = out_args(e, F, n, e->d_c);
    if (e->adapt && F.K >= 2) oa.S = e->fb_S_full;  // the adaptive pass's partials
    if (e->adapt) {
        // G_n and the step on partition 0 are done; the tail of this block
        // holds F_{n-2}: add the two steps it lacks
        CK(cudaStreamWaitEvent(s, e->ev_prep, 0));
        oa.corr_G = G_of(e, n);
        oa.corr_G2 = G_of(e, n - 1);
        oa.corr_A = A_of(e, n, 1, 8);
        oa.corr_A2 = A_of(e, n, 2, 8);
        oa.corr_C = F.K >= 2 ? 1 : 0;
    }
    CK(e->reuse ? launch_out3(e->prec, oa, PackArgs{}, s) : launch_out_c2r(e->prec, oa, s, true));
    if (!e->adapt) {
        cudaStream_t bg = e->bg[2 + ((n + 1) & 1)];
        CK(cudaStreamWaitEvent(bg, F.ev_packed, 0));
        if ((rc = enqueue_tail(e, F, n + 1, bg, false))) return rc;
        CK(cudaEventRecord(F.ev_tail[(n + 1) & 1], bg));
    } else {
        // background, a block ahead: the correlations of block n+1, and
        // block n-1's step on the tail partitions fused with block n+1's tail
        // (in order on one stream: each pass follows the one that read the
        // spectra before it)
        cudaStream_t bg = e->bg[2], bc = e->bg[3];
        CK(cudaStreamWaitEvent(bc, F.ev_packed, 0));
        if ((rc = enqueue_nlms_corr(e, n, bc))) return rc;
        CK(cudaEventRecord(e->ev_corr, bc));
        CK(cudaStreamWaitEvent(bg, F.ev_packed, 0));
        if ((rc = enqueue_nlms_update_mac(e, n - 1, e->upd_pending, bg))) return rc;
        e->upd_pending = true;
        CK(cudaEventRecord(F.ev_tail[(n + 1) & 1], bg));
    }
    ++e->nblk;
    ++e->st.blocks;
    return CONV_OK;
}

void engine_free(conv_engine* e) {
    if (!e) return;
    DeviceGuard g(e->dev);
    if (e->far) {
        engine_free(e->far);
        e->far = nullptr;
    }
    dev_free(e, &e->d_cin, 0);
    dev_free(e, &e->d_cout, 0);
    dev_free(e, &e->d_acc, 0);
    dev_free(e, &e->d_far_out[0], 0);
    dev_free(e, &e->d_far_out[1], 0);
    if (e->stream) cudaStreamSynchronize(e->stream);
    for (int i = 0; i < 4; ++i)
        if (e->bg[i]) cudaStreamSynchronize(e->bg[i]);
    if (e->as) cudaStreamSynchronize(e->as);
    for (Part* P : {&e->syn, &e->fb}) {
        if (P->ev_packed) cudaEventDestroy(P->ev_packed);
        for (int i = 0; i < 2; ++i)
            if (P->ev_tail[i]) cudaEventDestroy(P->ev_tail[i]);
    }
    part_free(e, e->syn);
    part_free(e, e->fb);
    dev_free(e, &e->tw, 0);
    dev_free(e, &e->tw_lo, 0);
    dev_free(e, &e->tw3, 0);
    if (e->flush_buf) {
        cudaFree(e->flush_buf);
        e->flush_buf = nullptr;
    }
    dev_free(e, &e->d_e, 0);
    dev_free(e, &e->d_c, 0);
    dev_free(e, &e->d_pow, 0);
    dev_free(e, &e->d_G, 0);
    dev_free(e, &e->d_A, 0);
    dev_free(e, &e->d_ticket, 0);
    dev_free(e, &e->d_side, 0);
    if (e->ev_prep) cudaEventDestroy(e->ev_prep);
    if (e->ev_corr) cudaEventDestroy(e->ev_corr);
    if (e->as) cudaStreamDestroy(e->as);
    if (e->h_in) cudaFreeHost(e->h_in);
    if (e->h_out) cudaFreeHost(e->h_out);
    if (e->h_e) cudaFreeHost(e->h_e);
    if (e->h_err) cudaFreeHost(e->h_err);
    for (auto ev : e->ev0) cudaEventDestroy(ev);
    for (auto ev : e->ev1) cudaEventDestroy(ev);
    host_graph_destroy(e->hg);
    dev_free(e, &e->d_blk, sizeof(long long));
    if (e->ev_done) cudaEventDestroy(e->ev_done);
    if (e->ev_handoff) cudaEventDestroy(e->ev_handoff);
    if (e->ev_join) cudaEventDestroy(e->ev_join);
    for (int i = 0; i < 4; ++i)
        if (e->bg[i]) cudaStreamDestroy(e->bg[i]);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

int create_impl(conv_engine* e, double fs, int block, int n_in, int n_out, long long taps) {
    if (!(fs > 0.0) || !std::isfinite(fs)) return set_err(CONV_E_INVAL, "fs must be positive");
    if (block < 16 || block > 4096 || (block & (block - 1)))
        return set_err(CONV_E_INVAL, "block %d must be a power of two in [16, 4096]", block);
    if (n_in < 1 || n_in > 1024 || n_out < 1 || n_out > 1024)
        return set_err(CONV_E_INVAL, "n_in %d / n_out %d must be in [1, 1024]", n_in, n_out);
    if (taps < 1) return set_err(CONV_E_INVAL, "taps must be >= 1");
    e->fs = fs;
    e->B = block;
    e->log2B = ilog2(block);
    e->n_in = n_in;
    e->n_out = n_out;
    e->taps = taps;
    e->taps_total = taps;
    CK(cudaGetDevice(&e->dev));
    cudaDeviceProp prop{};
    CK(cudaGetDeviceProperties(&prop, e->dev));
    e->num_sms = prop.multiProcessorCount;
    CK(prepare_kernels(MAC_SMEM_LIMIT));
    int prio_low = 0, prio_high = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    CK(cudaStreamCreateWithPriority(&e->stream, cudaStreamNonBlocking, prio_high));
    for (int i = 0; i < 4; ++i) CK(cudaStreamCreateWithPriority(&e->bg[i], cudaStreamNonBlocking, prio_low));
    // spin-wait on completion: a blocking wait would add the host's wake-up latency to every block
    CK(cudaEventCreateWithFlags(&e->ev_done, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&e->ev_handoff, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&e->ev_join, cudaEventDisableTiming));
    // twiddles W_2B^j = exp(-i pi j / B), FP64 on the host, rounded once to FP32
    std::vector<float2> tw(2 * (size_t)block);
    const double pi = 3.14159265358979323846264338327950288;
    for (int j = 0; j < 2 * block; ++j) {
        const double ang = -pi * (double)j / (double)block;
        tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    std::vector<float2> tw_lo(2 * (size_t)block);
    for (int j = 0; j < 2 * block; ++j) {
        const double ang = -pi * (double)j / (double)block;
        tw_lo[j] = make_float2((float)(std::cos(ang) - (double)tw[j].x), (float)(std::sin(ang) - (double)tw[j].y));
    }
    int rc;
    if ((rc = dev_alloc(e, &e->tw, tw.size() * sizeof(float2)))) return rc;
    CK(cudaMemcpy(e->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    if ((rc = dev_alloc(e, &e->tw_lo, tw_lo.size() * sizeof(float2)))) return rc;
    CK(cudaMemcpy(e->tw_lo, tw_lo.data(), tw_lo.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaHostAlloc(reinterpret_cast<void**>(&e->h_in), (size_t)n_in * block * sizeof(float), cudaHostAllocMapped));
    CK(cudaHostAlloc(reinterpret_cast<void**>(&e->h_out), (size_t)n_out * block * sizeof(float), cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->m_in), e->h_in, 0));
    CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->m_out), e->h_out, 0));
    CK(cudaHostAlloc(reinterpret_cast<void**>(&e->h_e), (size_t)n_in * block * sizeof(float), cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->m_e), e->h_e, 0));
    CK(cudaHostAlloc(reinterpret_cast<void**>(&e->h_err), sizeof(int), cudaHostAllocMapped));
    *e->h_err = 0;
    CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->d_err), e->h_err, 0));
    if ((rc = part_alloc(e, e->syn, n_in, n_out, taps))) return rc;
    return engine_reset(e);
}

}  // namespace

extern "C" {

conv_engine* conv_create(double fs, int block, int n_in, int n_out, long long taps) {
    conv_engine* e = new (std::nothrow) conv_engine();
    if (!e) {
        set_err(CONV_E_NOMEM, "out of host memory");
        return nullptr;
    }
    if (create_impl(e, fs, block, n_in, n_out, taps) != CONV_OK) {
        const std::string msg = g_err;
        engine_free(e);
        g_err = msg;
        return nullptr;
    }
    g_err.clear();
    return e;
}

int conv_set_precision(conv_engine* e, int mode) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (mode != CONV_FP32 && mode != CONV_FP16 && mode != CONV_BF16)
        return set_err(CONV_E_INVAL, "unknown precision %d", mode);
    if (e->syn.ready || e->fb.allocated)
        return set_err(CONV_E_STATE, "precision must be set before conv_set_filters / afc_set_paths");
    if (mode == e->prec) return CONV_OK;
    DeviceGuard g(e->dev);
    int rc;
    if (e->far && (rc = conv_set_precision(e->far, mode))) return rc;
    e->prec = mode;
    rc = part_alloc(e, e->syn, e->n_in, e->n_out, e->taps, e->tiling);
    if (rc) return rc;
    return engine_reset(e);
}

int afc_set_spectrum_reuse(conv_engine* e, int on) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (on != 0 && on != 1) return set_err(CONV_E_INVAL, "on must be 0 or 1");
    if (e->syn.ready || e->fb.allocated)
        return set_err(CONV_E_STATE, "the FFT size must be set before conv_set_filters / afc_set_paths");
    if (on && e->B < 32) return set_err(CONV_E_INVAL, "the n_f = 3 n_x form needs block >= 32 (block %d)", e->B);
    if (on && e->far) return set_err(CONV_E_STATE, "a far block is not combined with the n_f = 3 n_x form");
    if (on && e->adapt) return set_err(CONV_E_STATE, "the adaptive canceller is not combined with the n_f = 3 n_x form");
    if (e->in_batches > 0) return set_err(CONV_E_STATE, "session is in a batch");
    if ((on != 0) == e->reuse) return CONV_OK;
    DeviceGuard g(e->dev);
    int rc;
    if (on && !e->tw3) {
        CK(prepare_reuse_kernels());
        // twiddles W_3B^j = exp(-2 pi i j / 3B), FP64 on the host, rounded once to FP32
        const int n = 3 * e->B;
        std::vector<float2> tw(n);
        const double pi = 3.14159265358979323846264338327950288;
        for (int j = 0; j < n; ++j) {
            const double ang = -2.0 * pi * (double)j / (double)n;
            tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        }
        if ((rc = dev_alloc(e, &e->tw3, tw.size() * sizeof(float2)))) return rc;
        CK(cudaMemcpy(e->tw3, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    e->reuse = on != 0;
    if ((rc = part_alloc(e, e->syn, e->n_in, e->n_out, e->taps, e->tiling))) {
        const std::string msg = g_err;
        e->reuse = !e->reuse;
        if (part_alloc(e, e->syn, e->n_in, e->n_out, e->taps, e->tiling) == CONV_OK) engine_reset(e);
        g_err = msg;
        return rc;
    }
    return engine_reset(e);
}

int conv_set_tiling(conv_engine* e, const conv_tiling* t) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (e->syn.ready || e->fb.allocated)
        return set_err(CONV_E_STATE, "tiling must be set before conv_set_filters / afc_set_paths");
    const TileOverride o = from_api(t);
    if (const char* msg = check_override(o)) return set_err(CONV_E_INVAL, "%s", msg);
    DeviceGuard g(e->dev);
    const TileOverride old = e->tiling;
    e->tiling = o;
    int rc = part_alloc(e, e->syn, e->n_in, e->n_out, e->taps, e->tiling);
    if (rc) {
        e->tiling = old;
        const std::string msg = g_err;
        if (part_alloc(e, e->syn, e->n_in, e->n_out, e->taps, e->tiling) == CONV_OK) engine_reset(e);
        g_err = msg;
        return rc;
    }
    return engine_reset(e);
}

int conv_set_filters(conv_engine* e, const float* h) {
    if (!e || !h) return set_err(CONV_E_INVAL, "null argument");
    DeviceGuard g(e->dev);
    int rc;
    if (!e->far) {
        if ((rc = part_set_filters(e, e->syn, h))) return rc;
        return engine_reset(e);
    }
    // h[l][q][0 .. far_B) to this engine, h[l][q][far_B .. taps) to the far engine
    const size_t pairs = (size_t)e->n_out * e->n_in, T = (size_t)e->taps_total, F = (size_t)e->far_B;
    std::vector<float> near(pairs * F), farh(pairs * (T - F));
    for (size_t i = 0; i < pairs; ++i) {
        std::memcpy(near.data() + i * F, h + i * T, F * sizeof(float));
        std::memcpy(farh.data() + i * (T - F), h + i * T + F, (T - F) * sizeof(float));
    }
    if ((rc = part_set_filters(e, e->syn, near.data()))) return rc;
    if ((rc = conv_set_filters(e->far, farh.data()))) return rc;
    return engine_reset(e);
}

int conv_set_far_block(conv_engine* e, int far_block) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (e->syn.ready || e->fb.allocated)
        return set_err(CONV_E_STATE, "the far block must be set before conv_set_filters / afc_set_paths");
    if (e->in_batches > 0) return set_err(CONV_E_STATE, "session is in a batch");
    if (far_block != 0) {
        if (far_block <= e->B || far_block > 4096 || (far_block & (far_block - 1)))
            return set_err(CONV_E_INVAL, "far block %d must be 0 or a power of two in (block, 4096]", far_block);
        if (e->taps_total <= far_block)
            return set_err(CONV_E_INVAL, "taps %lld must exceed the far block %d", e->taps_total, far_block);
        if (e->reuse) return set_err(CONV_E_STATE, "a far block is not combined with the n_f = 3 n_x form");
    }
    DeviceGuard g(e->dev);
    if (e->far) {
        engine_free(e->far);
        e->far = nullptr;
    }
    dev_free(e, &e->d_acc, (size_t)e->n_in * e->far_B * sizeof(float));
    for (int i = 0; i < 2; ++i) dev_free(e, &e->d_far_out[i], (size_t)e->n_out * e->far_B * sizeof(float));
    e->far_B = 0;
    e->taps = e->taps_total;
    int rc;
    if (far_block != 0) {
        conv_engine* f = new (std::nothrow) conv_engine();
        if (!f) return set_err(CONV_E_NOMEM, "out of host memory");
        if ((rc = create_impl(f, e->fs, far_block, e->n_in, e->n_out, e->taps_total - far_block)) ||
            (rc = conv_set_precision(f, e->prec))) {
            const std::string msg = g_err;
            engine_free(f);
            g_err = msg;
            part_alloc(e, e->syn, e->n_in, e->n_out, e->taps, e->tiling);
            return rc;
        }
        f->l2_keep = e->l2_keep;
        e->far = f;
        e->far_B = far_block;
        e->taps = far_block;
        if ((rc = dev_alloc(e, &e->d_acc, (size_t)e->n_in * far_block * sizeof(float)))) return rc;
        for (int i = 0; i < 2; ++i)
            if ((rc = dev_alloc(e, &e->d_far_out[i], (size_t)e->n_out * far_block * sizeof(float)))) return rc;
    }
    if ((rc = part_alloc(e, e->syn, e->n_in, e->n_out, e->taps, e->tiling))) return rc;
    return engine_reset(e);
}

conv_engine* conv_far_engine(conv_engine* e) { return e ? e->far : nullptr; }

// With the feedback canceller, the synthesis tail runs on two thirds of its
// default grid (2/3 of the partition splits; the filter layout does not
// depend on them) and leaves the rest of the SMs to the canceller's tail
// (measured on the paper's 4 x 16 set with a 0.5 s canceller, B = 256:
// 37.3 -> 34.2 us per block; the plain engine is fastest on the full grid).
// An explicit split count from conv_set_tiling is kept.
void plan_syn_beside_canceller(conv_engine* e) {
    Part& P = e->syn;
    if (!P.allocated || e->tiling.splits != 0) return;
    const TileOverride base = reuse_tiling(e, e->tiling, P.n_dst);
    const MacPlan full = plan_mac(e->prec, bins_of(e), P.n_src, P.n_dst, P.K, e->num_sms, P.n_src, base);
    if (full.S < 3) return;
    TileOverride o = base;
    o.splits = (2 * full.S) / 3;
    MacPlan q = plan_mac(e->prec, bins_of(e), P.n_src, P.n_dst, P.K, e->num_sms, P.n_src, o);
    if (q.h_bytes != P.plan.h_bytes || q.x_bytes != P.plan.x_bytes || q.tile_elems != P.plan.tile_elems ||
        q.partial_bytes > P.plan.partial_bytes)
        return;
    q.partial_bytes = P.plan.partial_bytes;  // the buffers keep their size
    std::string why;
    if (check_plan(q, &why)) return;
    P.plan = q;
}

// The canceller's own tail runs on 2 splits per tile (16 CTAs at the paper
// config) beside that: 34.2 -> 32.7 us per block.  Its partials keep the size
// of the default plan, whose split count the adaptive pass uses.
void plan_fb_beside_synthesis(conv_engine* e) {
    Part& F = e->fb;
    e->fb_S_full = F.plan.S;
    if (!F.allocated || F.plan.S <= 2) return;
    TileOverride o = reuse_tiling(e, TileOverride(), F.n_dst);
    o.splits = 2;
    MacPlan q = plan_mac(e->prec, bins_of(e), F.n_src, F.n_dst, F.K, e->num_sms, F.n_src, o);
    if (q.h_bytes != F.plan.h_bytes || q.x_bytes != F.plan.x_bytes || q.tile_elems != F.plan.tile_elems ||
        q.partial_bytes > F.plan.partial_bytes)
        return;
    q.partial_bytes = F.plan.partial_bytes;
    std::string why;
    if (check_plan(q, &why)) return;
    F.plan = q;
}

int afc_set_paths(conv_engine* e, const float* f, long long taps_fb) {
    if (!e || !f) return set_err(CONV_E_INVAL, "null argument");
    if (taps_fb < 1) return set_err(CONV_E_INVAL, "taps_fb must be >= 1");
    DeviceGuard g(e->dev);
    int rc;
    e->upd_pending = false;  // the estimate is replaced: a pending step of the old one is dropped
    if ((rc = part_alloc(e, e->fb, e->n_out, e->n_in, taps_fb))) return rc;
    if (!e->d_c && (rc = dev_alloc(e, &e->d_c, (size_t)e->n_in * e->B * sizeof(float)))) return rc;
    if (!e->d_e && (rc = dev_alloc(e, &e->d_e, (size_t)e->n_in * e->B * sizeof(float)))) return rc;
    if ((rc = part_set_filters(e, e->fb, f))) return rc;
    plan_syn_beside_canceller(e);
    plan_fb_beside_synthesis(e);
    return engine_reset(e);
}

int conv_process_block_async(conv_engine* e, const float* d_in, float* d_out, void* cuda_stream) {
    if (!e || !d_in || !d_out) return set_err(CONV_E_INVAL, "null argument");
    if (!e->syn.ready) return set_err(CONV_E_STATE, "filters not set");
    if (e->adapt) return set_err(CONV_E_STATE, "the adaptive canceller needs every block through afc_process_block");
    DeviceGuard g(e->dev);
    return enqueue_block(e, d_in, d_out, static_cast<cudaStream_t>(cuda_stream));
}

int conv_process_block(conv_engine* e, const float* in, float* out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!e || !in || !out) return set_err(CONV_E_INVAL, "null argument");
    if (!e->syn.ready) return set_err(CONV_E_STATE, "filters not set");
    if (e->adapt) return set_err(CONV_E_STATE, "the adaptive canceller needs every block through afc_process_block");
    DeviceGuard g(e->dev);
    const size_t ib = (size_t)e->n_in * e->B * sizeof(float), ob = (size_t)e->n_out * e->B * sizeof(float);
    std::memcpy(e->h_in, in, ib);
    // the pack kernel reads the block from mapped pinned host memory and the
    // output kernel writes there (over the coherent CPU-GPU link): no copy
    // launches per block (measured: p50 call latency 38.8 -> 34.7 us)
    int rc;
    if (host_graph_eligible(e, false) && host_graph_now(e, t0)) {
        // one graph launch instead of three launches and five event calls
        if ((rc = host_graph_block(e, false))) return rc;
        CK(cudaEventSynchronize(e->hg.ev_out));  // the next block's tail keeps running
    } else {
        if ((rc = enqueue_block(e, e->m_in, e->m_out, e->stream))) return rc;
        CK(cudaEventRecord(e->ev_done, e->stream));
        CK(cudaEventSynchronize(e->ev_done));  // the next block's tail keeps running
    }
    if ((rc = check_dev_err(e))) return rc;
    std::memcpy(out, e->h_out, ob);
    record_call(e, t0);
    return CONV_OK;
}

int conv_process_blocks(conv_engine* e, const float* in, float* out, long long n_blocks) {
    if (!e || !in || !out) return set_err(CONV_E_INVAL, "null argument");
    if (n_blocks < 1) return set_err(CONV_E_INVAL, "n_blocks must be >= 1");
    if (!e->syn.ready) return set_err(CONV_E_STATE, "filters not set");
    if (e->adapt) return set_err(CONV_E_STATE, "the adaptive canceller needs every block through afc_process_block");
    DeviceGuard g(e->dev);
    const long long C = std::min<long long>(n_blocks, 256);  // blocks per chunk
    int rc = CONV_OK;
    if (C > e->chunk_cap) {
        CK(cudaStreamSynchronize(e->stream));
        dev_free(e, &e->d_cin, (size_t)e->n_in * e->chunk_cap * e->B * sizeof(float));
        dev_free(e, &e->d_cout, (size_t)e->n_out * e->chunk_cap * e->B * sizeof(float));
        e->chunk_cap = 0;
        if ((rc = dev_alloc(e, &e->d_cin, (size_t)e->n_in * C * e->B * sizeof(float)))) return rc;
        if ((rc = dev_alloc(e, &e->d_cout, (size_t)e->n_out * C * e->B * sizeof(float)))) return rc;
        e->chunk_cap = C;
    }
    const size_t T = (size_t)n_blocks * e->B, fs = sizeof(float);
    for (long long b0 = 0; b0 < n_blocks; b0 += C) {
        const long long nb = std::min(C, n_blocks - b0);
        const size_t w = (size_t)nb * e->B;
        CK(cudaMemcpy2DAsync(e->d_cin, (size_t)C * e->B * fs, in + (size_t)b0 * e->B, T * fs, w * fs, e->n_in,
                             cudaMemcpyHostToDevice, e->stream));
        e->io_in_stride = (int)(C * e->B);
        e->io_out_stride = (int)(C * e->B);
        for (long long b = 0; b < nb && !rc; ++b)
            rc = enqueue_block(e, e->d_cin + (size_t)b * e->B, e->d_cout + (size_t)b * e->B, e->stream);
        e->io_in_stride = e->io_out_stride = 0;
        if (rc) return rc;
        CK(cudaMemcpy2DAsync(out + (size_t)b0 * e->B, T * fs, e->d_cout, (size_t)C * e->B * fs, w * fs, e->n_out,
                             cudaMemcpyDeviceToHost, e->stream));
    }
    CK(cudaEventRecord(e->ev_done, e->stream));
    CK(cudaEventSynchronize(e->ev_done));
    return check_dev_err(e);
}

int afc_process_block_async(conv_engine* e, const float* d_mic, float* d_out, float* d_e, void* cuda_stream) {
    if (!e || !d_mic || !d_out) return set_err(CONV_E_INVAL, "null argument");
    if (!e->syn.ready || !e->fb.ready) return set_err(CONV_E_STATE, "filters or feedback paths not set");
    DeviceGuard g(e->dev);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc = enqueue_afc_synthesis(e, d_mic, d_out, d_e, s);
    if (rc) return rc;
    return enqueue_afc_prediction(e, s);
}

int afc_process_block(conv_engine* e, const float* mic, float* out, float* e_or_null) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!e || !mic || !out) return set_err(CONV_E_INVAL, "null argument");
    if (!e->syn.ready || !e->fb.ready) return set_err(CONV_E_STATE, "filters or feedback paths not set");
    DeviceGuard g(e->dev);
    const size_t ib = (size_t)e->n_in * e->B * sizeof(float), ob = (size_t)e->n_out * e->B * sizeof(float);
    const bool want_e = e_or_null != nullptr || e->guard > 0.0;
    std::memcpy(e->h_in, mic, ib);
    int rc;
    if (host_graph_eligible(e, true) && host_graph_now(e, t0)) {
        // one graph launch; the pack writes e straight into h_e
        if ((rc = host_graph_block(e, true))) return rc;
        CK(cudaEventSynchronize(e->hg.ev_out));  // the prediction and the tails keep running
    } else {
        // microphone block in and loudspeaker block out through mapped pinned host memory
        if ((rc = enqueue_afc_synthesis(e, e->m_in, e->m_out, e->d_e, e->stream))) return rc;
        if (want_e) CK(cudaMemcpyAsync(e->h_e, e->d_e, ib, cudaMemcpyDeviceToHost, e->stream));
        CK(cudaEventRecord(e->ev_done, e->stream));
        // the prediction for the next block runs while this block's output is read on the host
        if ((rc = enqueue_afc_prediction(e, e->stream))) return rc;
        CK(cudaEventSynchronize(e->ev_done));
    }
    if ((rc = check_dev_err(e))) return rc;
    if (e->guard > 0.0) {
        double ss = 0.0;
        const size_t n = (size_t)e->n_in * e->B;
        for (size_t i = 0; i < n; ++i) ss += (double)e->h_e[i] * e->h_e[i];
        const double rms = std::sqrt(ss / (double)n);
        if (!(rms <= e->guard)) {
            engine_reset(e);
            ++e->st.guard_trips;
            return set_err(CONV_E_UNSTABLE, "closed-loop guard: rms(e) = %g exceeds %g; loop state reset", rms,
                           e->guard);
        }
    }
    std::memcpy(out, e->h_out, ob);
    if (e_or_null) std::memcpy(e_or_null, e->h_e, ib);
    record_call(e, t0);
    return CONV_OK;
}

int afc_set_guard(conv_engine* e, double max_rms) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (!(max_rms >= 0.0)) return set_err(CONV_E_INVAL, "guard must be >= 0");
    e->guard = max_rms;
    return CONV_OK;
}

int afc_set_adaptation(conv_engine* e, double mu, double lambda, double delta) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (!(mu >= 0.0 && mu < 2.0)) return set_err(CONV_E_INVAL, "mu must be in [0, 2)");
    if (!(lambda >= 0.0 && lambda < 1.0)) return set_err(CONV_E_INVAL, "lambda must be in [0, 1)");
    if (!(delta >= 0.0) || !std::isfinite(delta)) return set_err(CONV_E_INVAL, "delta must be finite and >= 0");
    if (mu > 0.0 && !(delta > 0.0)) return set_err(CONV_E_INVAL, "delta must be > 0 when mu > 0");
    if (!e->fb.ready) return set_err(CONV_E_STATE, "feedback paths not set");
    if (e->prec != CONV_FP32) return set_err(CONV_E_STATE, "the adaptive canceller needs FP32 spectra");
    if (e->far) return set_err(CONV_E_STATE, "the adaptive canceller is not combined with a far block");
    if (e->reuse && mu > 0.0)
        return set_err(CONV_E_STATE, "the adaptive canceller is not combined with the n_f = 3 n_x form");
    if (e->in_batches > 0) return set_err(CONV_E_STATE, "session is in a batch");
    DeviceGuard g(e->dev);
    int rc;
    if (!e->as) {
        int prio_low = 0, prio_high = 0;
        CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
        CK(cudaStreamCreateWithPriority(&e->as, cudaStreamNonBlocking, prio_high));
        CK(cudaEventCreateWithFlags(&e->ev_prep, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&e->ev_corr, cudaEventDisableTiming));
    }
    if (!e->d_pow) {
        if ((rc = dev_alloc(e, &e->d_pow, 2 * (size_t)e->B * sizeof(float2)))) return rc;
        CK(cudaMemsetAsync(e->d_pow, 0, 2 * (size_t)e->B * sizeof(float2), e->stream));
    }
    if (!e->d_G && (rc = dev_alloc(e, &e->d_G, 3 * (size_t)e->n_in * e->B * sizeof(float2)))) return rc;
    if (!e->d_A && (rc = dev_alloc(e, &e->d_A, 36 * (size_t)e->B * sizeof(float2)))) return rc;
    if (!e->d_ticket) {
        if ((rc = dev_alloc(e, &e->d_ticket, (size_t)e->B * sizeof(unsigned)))) return rc;
        CK(cudaMemsetAsync(e->d_ticket, 0, (size_t)e->B * sizeof(unsigned), e->stream));
    }
    if (!e->d_side && (rc = dev_alloc(e, &e->d_side, 2 * (size_t)e->n_out * e->B * sizeof(float2)))) return rc;
    if (e->has_last) CK(cudaStreamSynchronize(e->last_stream));
    for (int i = 0; i < 4; ++i) CK(cudaStreamSynchronize(e->bg[i]));
    CK(cudaStreamSynchronize(e->as));
    CK(cudaStreamSynchronize(e->stream));
    const bool was = e->adapt;
    const bool now = mu > 0.0;
    if (was && !now) {
        // the static schedule expects the stored spectra complete and this
        // block's tail computed with them
        if ((rc = flush_nlms_update(e))) return rc;
        if ((rc = enqueue_tail(e, e->fb, e->nblk, e->stream, false))) return rc;
        CK(cudaEventRecord(e->fb.ev_tail[e->nblk & 1], e->stream));
    }
    if (!was && now) {
        // the static tail of this block holds the current spectra; no step
        // before this block (G of the previous block zero), and this block's
        // correlations from the delay line as it is
        CK(cudaMemsetAsync(e->d_G, 0, 3 * (size_t)e->n_in * e->B * sizeof(float2), e->stream));
        CK(cudaMemsetAsync(e->d_A, 0, 36 * (size_t)e->B * sizeof(float2), e->stream));
        CK(cudaMemsetAsync(e->d_side, 0, 2 * (size_t)e->n_out * e->B * sizeof(float2), e->stream));
        if (e->nblk > 0 && (rc = enqueue_nlms_corr(e, e->nblk - 1, e->stream))) return rc;
        // this block's canceller tail again, in the split count of the
        // adaptive pass, whose partials the adaptive output reads
        if ((rc = enqueue_nlms_update_mac(e, e->nblk - 2, false, e->stream))) return rc;
        CK(cudaEventRecord(e->fb.ev_tail[e->nblk & 1], e->stream));
        e->upd_pending = false;
    }
    CK(cudaStreamSynchronize(e->stream));
    e->adapt = now;
    e->mu = (float)mu;
    e->lam = (float)lambda;
    e->delta = (float)delta;
    return CONV_OK;
}

int afc_get_path_spectra(conv_engine* e, float* f_spec) {
    if (!e || !f_spec) return set_err(CONV_E_INVAL, "null argument");
    if (!e->fb.ready) return set_err(CONV_E_STATE, "feedback paths not set");
    if (e->prec != CONV_FP32) return set_err(CONV_E_STATE, "path spectra are read back from FP32 engines only");
    if (e->reuse) return set_err(CONV_E_STATE, "path spectra are read back in the n_f = 2 n_x form only");
    DeviceGuard g(e->dev);
    if (e->has_last) CK(cudaStreamSynchronize(e->last_stream));
    for (int i = 0; i < 4; ++i) CK(cudaStreamSynchronize(e->bg[i]));
    if (e->as) CK(cudaStreamSynchronize(e->as));
    CK(cudaStreamSynchronize(e->stream));
    int rc;
    if ((rc = flush_nlms_update(e))) return rc;  // the last block's step on the tail partitions
    const Part& F = e->fb;
    const MacPlan& p = F.plan;
    std::vector<float2> tiles(p.h_bytes / sizeof(float2));
    CK(cudaMemcpy(tiles.data(), F.H, p.h_bytes, cudaMemcpyDeviceToHost));
    // tiles (kt, lt) at (kt*n_lt + lt)*tile_elems, then [r][LTt][BT]; r = j*L + l
    float2* out = reinterpret_cast<float2*>(f_spec);
    const int P = F.n_dst, L = F.n_src, K = F.K, B = e->B;
    for (int kt = 0; kt < p.n_kt; ++kt)
        for (int lt = 0; lt < p.n_lt; ++lt) {
            const int LTt = std::min(p.LT, P - lt * p.LT);
            const float2* t = tiles.data() + ((size_t)kt * p.n_lt + lt) * p.tile_elems;
            for (int r = 0; r < p.R; ++r)
                for (int ll = 0; ll < LTt; ++ll)
                    for (int kl = 0; kl < p.BT; ++kl) {
                        const int pm = lt * p.LT + ll, l = r % L, j = r / L, k = kt * p.BT + kl;
                        out[(((size_t)pm * L + l) * K + j) * B + k] = t[((size_t)r * LTt + ll) * p.BT + kl];
                    }
        }
    return CONV_OK;
}

int conv_reset(conv_engine* e) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    DeviceGuard g(e->dev);
    return engine_reset(e);
}

int conv_join_async(conv_engine* e, void* cuda_stream) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    DeviceGuard g(e->dev);
    return join_streams(e, static_cast<cudaStream_t>(cuda_stream));
}

int conv_get_stats(const conv_engine* e, conv_stats* out) {
    if (!e || !out) return set_err(CONV_E_INVAL, "null argument");
    *out = e->st;
    return CONV_OK;
}

int conv_set_host_graph(conv_engine* e, int mode) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (mode < 0 || mode > 2) return set_err(CONV_E_INVAL, "mode %d must be 0, 1 or 2", mode);
    DeviceGuard g(e->dev);
    e->hg.mode = mode;
    if (mode == 0) {
        int rc;
        if ((rc = host_graph_settle(e))) return rc;
        CK(cudaStreamSynchronize(e->stream));
        host_graph_free(e->hg.plain);
        host_graph_free(e->hg.loop);
    }
    return CONV_OK;
}

int conv_get_host_graph(const conv_engine* e, int* mode, long long* graph_blocks) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (mode) *mode = e->hg.mode;
    if (graph_blocks) *graph_blocks = e->hg.blocks;
    return CONV_OK;
}

int conv_reset_stats(conv_engine* e) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    e->st = conv_stats{};
    return CONV_OK;
}

int conv_inject_wait_timeout(conv_engine* e, long long wait_ns) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (wait_ns < 1000 || wait_ns > 1000000000ll) return set_err(CONV_E_INVAL, "wait_ns must be in [1e3, 1e9]");
    if (!e->syn.ready) return set_err(CONV_E_STATE, "filters not set");
    if (e->syn.plan.S == 0) return set_err(CONV_E_STATE, "one partition: the engine runs no tail MAC");
    if (e->syn.plan.direct) return set_err(CONV_E_STATE, "the direct-load MAC has no pipeline waits");
    e->inject = true;
    e->inject_ns = (unsigned long long)wait_ns;
    return CONV_OK;
}

int conv_synchronize(conv_engine* e) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    DeviceGuard g(e->dev);
    if (e->far) {
        const int rc = conv_synchronize(e->far);
        if (rc) return rc;
    }
    for (int i = 0; i < 4; ++i) CK(cudaStreamSynchronize(e->bg[i]));
    if (e->as) CK(cudaStreamSynchronize(e->as));
    CK(cudaStreamSynchronize(e->stream));
    CK(cudaDeviceSynchronize());
    return check_dev_err(e);
}

int conv_get_info(const conv_engine* e, conv_info* out) {
    if (!e || !out) return set_err(CONV_E_INVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    const MacPlan& p = e->syn.plan;
    out->block = e->B;
    out->n_in = e->n_in;
    out->n_out = e->n_out;
    out->taps = e->taps_total;
    out->K = e->syn.K;
    out->taps_fb = e->fb.allocated ? e->fb.taps : 0;
    out->K_fb = e->fb.allocated ? e->fb.K : 0;
    out->precision = e->prec;
    // algorithmic bytes of one tail MAC launch: partitions 1..K-1 of every
    // filter spectrum plus the matching delay-line rows, each read once
    auto tail_bytes = [](const MacPlan& q) {
        const size_t Rt = (size_t)(q.R - q.r_begin);
        return (long long)(((size_t)q.n_dst + 1) * Rt * q.B * q.es);
    };
    out->mac_bytes = tail_bytes(p);
    out->mac_fb_bytes = e->fb.allocated ? tail_bytes(e->fb.plan) : 0;
    out->mac_ctas = p.ctas;
    out->mac_splits = p.S;
    out->mac_smem = (long long)p.smem;
    out->mac_bin_tile = p.BT;
    out->mac_stages = p.nstage;
    out->mac_stage_bytes = p.stage_bytes;
    out->mac_warps = p.nw;
    out->mac_kernel = p.direct == 0 ? CONV_KERNEL_TMA : (p.direct == 1 ? CONV_KERNEL_DIRECT1 : CONV_KERNEL_DIRECT2);
    out->device_bytes = (long long)e->dev_bytes;
    out->kernels_per_block = 3;
    // pack, output (+ the canceller's push) and tail of the synthesis, output
    // and tail of the canceller; adaptive: NLMS step, update and the
    // correlation chunks (K_fb >= 2)
    out->kernels_per_afc_block = 5 + (e->adapt ? 2 + (e->fb.K >= 2 ? 1 : 0) : 0);
    out->afc_adaptive = e->adapt ? 1 : 0;
    out->far_block = e->far_B;
    out->K_far = e->far ? e->far->syn.K : 0;
    out->mac_far_bytes = e->far ? tail_bytes(e->far->syn.plan) : 0;
    out->fft_size = e->reuse ? 3LL * e->B : 2LL * e->B;
    out->l2_keep_bytes = e->l2_keep;
    return CONV_OK;
}

int conv_profile_enable(conv_engine* e, int enable) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    DeviceGuard g(e->dev);
    e->prof = enable > 0;
    if (e->prof) {
        const size_t want = enable > 1 ? (size_t)enable : 4096;
        while (e->ev0.size() < want) {
            cudaEvent_t a, b;
            CK(cudaEventCreate(&a));
            CK(cudaEventCreate(&b));
            e->ev0.push_back(a);
            e->ev1.push_back(b);
        }
    }
    e->ev_used = 0;
    return CONV_OK;
}

int conv_set_l2_keep(conv_engine* e, long long bytes) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (bytes < 0) return set_err(CONV_E_INVAL, "bytes must be >= 0");
    e->l2_keep = bytes;
    if (e->far) e->far->l2_keep = bytes;
    return CONV_OK;
}

int conv_profile_flush_l2(conv_engine* e, long long bytes) {
    if (!e) return set_err(CONV_E_INVAL, "null handle");
    if (bytes < 0) return set_err(CONV_E_INVAL, "bytes must be >= 0");
    DeviceGuard g(e->dev);
    if ((size_t)bytes > e->flush_bytes || bytes == 0) {
        if (e->flush_buf) CK(cudaFree(e->flush_buf));
        e->flush_buf = nullptr;
        e->flush_bytes = 0;
        if (bytes > 0) {
            if (cudaMalloc(&e->flush_buf, (size_t)bytes) != cudaSuccess) {
                cudaGetLastError();
                return set_err(CONV_E_NOMEM, "L2 flush buffer of %lld bytes", bytes);
            }
            CK(cudaMemset(e->flush_buf, 0, (size_t)bytes));
        }
    }
    e->flush_bytes = (size_t)bytes;
    return CONV_OK;
}

int conv_profile_read(conv_engine* e, double* mac_ms_total, long long* launches) {
    if (!e || !mac_ms_total || !launches) return set_err(CONV_E_INVAL, "null argument");
    DeviceGuard g(e->dev);
    double tot = 0.0;
    for (size_t i = 0; i < e->ev_used; ++i) {
        CK(cudaEventSynchronize(e->ev1[i]));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e->ev0[i], e->ev1[i]));
        tot += ms;
    }
    *mac_ms_total = tot;
    *launches = (long long)e->ev_used;
    e->ev_used = 0;
    return CONV_OK;
}

long long conv_footprint(int precision, int block, int n_in, int n_out, long long taps, long long taps_fb,
                         int num_sms) {
    if (precision < CONV_FP32 || precision > CONV_BF16 || block < 16 || block > 4096 || (block & (block - 1)) ||
        n_in < 1 || n_out < 1 || taps < 1 || taps_fb < 0 || num_sms < 1) {
        set_err(CONV_E_INVAL, "invalid footprint arguments");
        return -1;
    }
    auto part = [&](int n_src, int n_dst, long long t) -> long long {
        const long long K = (t + block - 1) / block;
        if ((long long)n_src * K > 0x7fffffffLL / 2) return -1;
        const MacPlan p = plan_mac(precision, block, n_src, n_dst, (int)K, num_sms, n_src);
        // part buffers: spectra, ring, two partial buffers, window, scales
        return (long long)part_bytes(p, precision, (size_t)n_src * block) + (long long)p.partial_bytes;
    };
    long long b = part(n_in, n_out, taps);
    if (b < 0) return set_err(CONV_E_INVAL, "too many partitions"), -1;
    if (taps_fb > 0) {
        const long long f = part(n_out, n_in, taps_fb);
        if (f < 0) return set_err(CONV_E_INVAL, "too many partitions"), -1;
        b += f + 2LL * n_in * block * (long long)sizeof(float);  // prediction and error buffers
    }
    // twiddles and their residuals, staging, error word
    b += 4LL * block * (long long)sizeof(float2) + (long long)(n_in + n_out) * block * (long long)sizeof(float);
    return b;
}

int conv_plan_check(int precision, int block, int n_src, int n_dst, long long taps, int num_sms,
                    const conv_tiling* t) {
    if (precision < CONV_FP32 || precision > CONV_BF16 || block < 16 || block > 4096 || (block & (block - 1)) ||
        n_src < 1 || n_dst < 1 || taps < 1 || num_sms < 1)
        return set_err(CONV_E_INVAL, "invalid plan arguments");
    const TileOverride o = from_api(t);
    if (const char* msg = check_override(o)) return set_err(CONV_E_INVAL, "%s", msg);
    const long long K = (taps + block - 1) / block;
    if ((long long)n_src * K > 0x7fffffffLL / 2) return set_err(CONV_E_INVAL, "too many partitions");
    const MacPlan p = plan_mac(precision, block, n_src, n_dst, (int)K, num_sms, n_src, o);
    std::string why;
    if (check_plan(p, &why)) return set_err(CONV_E_INVAL, "%s", why.c_str());
    return CONV_OK;
}

// ------------------------------------------------------------- batches
//
// A batch runs one block of every member session per step with three kernel
// launches in total (batched pack, batched output, batched tail MAC), each CTA
// reading its session's arguments from a descriptor table that the step
// uploads in one copy.  Sessions keep their own state (rings, windows,
// partials, block counters); the split-phase schedule is the single engine's,
// across the whole batch.

}  // extern "C"

struct conv_batch {
    int dev = 0;
    int prec = CONV_FP32;
    std::vector<conv_engine*> sessions;
    cudaStream_t stream = nullptr;
    cudaStream_t bg[2] = {nullptr, nullptr};
    cudaEvent_t ev_packed = nullptr, ev_tail[2] = {nullptr, nullptr}, ev_staged[2] = {nullptr, nullptr};
    std::vector<int> all_idx;
    // descriptor tables, double-buffered by step parity: host staging (pinned) and device
    unsigned char* h_tab[2] = {nullptr, nullptr};
    unsigned char* d_tab[2] = {nullptr, nullptr};
    size_t tab_cap = 0;
    long long step = 0;
    // persistent mode (conv_batch_set_persistent): one launch per step
    bool persistent = false;
    bool graph = false;         // replay the step (copy, counter reset, launch) from a CUDA graph
    int num_sms = 0;
    unsigned* d_ctr = nullptr;  // claim counter + two counters per item, zeroed before each step
    size_t ctr_cap = 0;         // unsigned values it holds
    cudaStream_t cap = nullptr;  // capture stream of the step graphs
    // one graph per table parity, and what it was captured for
    struct GraphKey {
        size_t bytes = 0, smem = 0, nctr = 0;
        int n_work = 0, ctas = 0;
        const void *d = nullptr, *h = nullptr, *ctr = nullptr, *err = nullptr;
        bool operator==(const GraphKey& o) const {
            return bytes == o.bytes && smem == o.smem && nctr == o.nctr && n_work == o.n_work && ctas == o.ctas &&
                   d == o.d && h == o.h && ctr == o.ctr && err == o.err;
        }
    } gkey[2];
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
};

namespace {

void batch_free_graphs(conv_batch* b) {
    for (int i = 0; i < 2; ++i) {
        if (b->gexec[i]) cudaGraphExecDestroy(b->gexec[i]);
        b->gexec[i] = nullptr;
        b->gkey[i] = conv_batch::GraphKey();
    }
}

void batch_free_tables(conv_batch* b) {
    batch_free_graphs(b);  // the graphs name the tables
    for (int i = 0; i < 2; ++i) {
        if (b->h_tab[i]) cudaFreeHost(b->h_tab[i]);
        if (b->d_tab[i]) cudaFree(b->d_tab[i]);
        b->h_tab[i] = b->d_tab[i] = nullptr;
    }
    b->tab_cap = 0;
}

int batch_sync(conv_batch* b) {
    CK(cudaStreamSynchronize(b->bg[0]));
    CK(cudaStreamSynchronize(b->bg[1]));
    CK(cudaStreamSynchronize(b->stream));
    return CONV_OK;
}

size_t align16(size_t v) { return (v + 15) / 16 * 16; }

// The persistent form of a batch step: the argument tables are built (h), the
// work list is appended in dependency order, and one launch runs it all.
// Counters: 2 i = packs of argument item i done, 2 i + 1 = its outputs done.
int batch_step_persistent(conv_batch* b, int count, const int* idx, unsigned char* h, unsigned char* d, size_t o_pack,
                          size_t o_out, size_t o_mac, size_t o_work, int n_work, int n_items, size_t mac_smem, int Bmax,
                          size_t bytes, int par, cudaStream_t s) {
    PersistentWork* wk = reinterpret_cast<PersistentWork*>(h + o_work);
    std::vector<int> fb_item(count, -1);
    for (int j = 0, ia = count; j < count; ++j)
        if (b->sessions[idx[j]]->fb.allocated) fb_item[j] = ia++;
    int w = 0;
    auto add = [&](int type, int item, int i1, int i2, int wait, int target, int signal) {
        wk[w++] = PersistentWork{type, item, i1, i2, wait, target, signal};
    };
    for (int j = 0; j < count; ++j)  // synthesis packs (e = mic - c_prev for canceller sessions)
        for (int c = 0; c < b->sessions[idx[j]]->syn.n_src; ++c) add(PW_PACK, j, c, 0, -1, 0, 2 * j);
    for (int j = 0; j < count; ++j) {  // synthesis outputs: head + tail partials + C2R
        const Part& P = b->sessions[idx[j]]->syn;
        for (int l = 0; l < P.n_dst; ++l) add(PW_OUT, j, l, 0, 2 * j, P.n_src, 2 * j + 1);
    }
    for (int j = 0; j < count; ++j)  // the canceller's packs of the loudspeaker blocks
        if (fb_item[j] >= 0) {
            const conv_engine* e = b->sessions[idx[j]];
            for (int c = 0; c < e->fb.n_src; ++c) add(PW_PACK, fb_item[j], c, 0, 2 * j + 1, e->syn.n_dst, 2 * fb_item[j]);
        }
    for (int j = 0; j < count; ++j)  // the canceller's outputs (the prediction for the next block)
        if (fb_item[j] >= 0) {
            const Part& F = b->sessions[idx[j]]->fb;
            for (int p = 0; p < F.n_dst; ++p) add(PW_OUT, fb_item[j], p, 0, 2 * fb_item[j], F.n_src, -1);
        }
    for (int j = 0; j < count; ++j) {  // tail MACs of the next block, both convolutions
        const conv_engine* e = b->sessions[idx[j]];
        const MacPlan& p = e->syn.plan;
        if (p.S)
            for (int cta = 0; cta < p.ctas; ++cta) add(PW_MAC, j, cta / p.S, cta % p.S, 2 * j, e->syn.n_src, -1);
        if (fb_item[j] >= 0 && e->fb.plan.S) {
            const MacPlan& q = e->fb.plan;
            for (int cta = 0; cta < q.ctas; ++cta)
                add(PW_MAC, fb_item[j], cta / q.S, cta % q.S, 2 * fb_item[j], e->fb.n_src, -1);
        }
    }
    if (w != n_work) return set_err(CONV_E_STATE, "persistent work list: %d items, %d expected", w, n_work);
    const size_t nctr = 1 + 2 * (size_t)n_items;
    if (nctr > b->ctr_cap) {
        int rc;
        if ((rc = batch_sync(b))) return rc;
        batch_free_graphs(b);
        if (b->d_ctr) cudaFree(b->d_ctr);
        b->d_ctr = nullptr;
        b->ctr_cap = 0;
        CK(cudaMalloc(reinterpret_cast<void**>(&b->d_ctr), 2 * nctr * sizeof(unsigned)));
        b->ctr_cap = 2 * nctr;
    }
    const size_t smem = std::max(mac_smem, fft_smem_bytes(Bmax));
    if (smem > MAC_SMEM_LIMIT - PERSISTENT_STATIC_SMEM)
        return set_err(CONV_E_INVAL, "persistent step: %zu bytes of shared memory above the kernel's limit", smem);
    const int ctas = std::max(1, std::min(n_work, b->num_sms));
    int* err = b->sessions[idx[0]]->d_err;
    // the step's three operations: table copy, counter reset, the launch
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t r = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, q);
        if (r == cudaSuccess) r = cudaMemsetAsync(b->d_ctr, 0, nctr * sizeof(unsigned), q);
        if (r == cudaSuccess)
            r = launch_batch_persistent(b->prec, reinterpret_cast<const PackArgs*>(d + o_pack),
                                        reinterpret_cast<const OutArgs*>(d + o_out),
                                        reinterpret_cast<const MacArgs*>(d + o_mac),
                                        reinterpret_cast<const PersistentWork*>(d + o_work), n_work, b->d_ctr, err, ctas,
                                        smem, q);
        return r;
    };
    // tails of earlier steps in the other mode ran on the background streams
    CK(cudaStreamWaitEvent(s, b->ev_tail[0], 0));
    CK(cudaStreamWaitEvent(s, b->ev_tail[1], 0));
    if (b->graph) {
        // the graph's copy reads the pinned table when it runs, so a replay
        // carries this step's arguments; a new layout is captured again
        conv_batch::GraphKey k;
        k.bytes = bytes;
        k.smem = smem;
        k.nctr = nctr;
        k.n_work = n_work;
        k.ctas = ctas;
        k.d = d;
        k.h = h;
        k.ctr = b->d_ctr;
        k.err = err;
        if (!b->gexec[par] || !(b->gkey[par] == k)) {
            if (b->gexec[par]) CK(cudaGraphExecDestroy(b->gexec[par]));
            b->gexec[par] = nullptr;
            if (!b->cap) CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
            CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            const cudaError_t r = enqueue(b->cap);
            cudaGraph_t graph = nullptr;
            const cudaError_t r2 = cudaStreamEndCapture(b->cap, &graph);
            if (r != cudaSuccess || r2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return set_err(CONV_E_CUDA, "capturing the persistent step: %s",
                               cudaGetErrorString(r != cudaSuccess ? r : r2));
            }
            const cudaError_t r3 = cudaGraphInstantiate(&b->gexec[par], graph, 0);
            cudaGraphDestroy(graph);
            if (r3 != cudaSuccess) {
                b->gexec[par] = nullptr;
                return set_err(CONV_E_CUDA, "instantiating the persistent step: %s", cudaGetErrorString(r3));
            }
            b->gkey[par] = k;
        }
        CK(cudaGraphLaunch(b->gexec[par], s));
    } else {
        CK(enqueue(s));
    }
    CK(cudaEventRecord(b->ev_staged[par], s));
    // the step's tails are done when the launch is: the join and the next
    // step's waits see them through the tail event
    cudaStream_t bg = b->bg[par ^ 1];
    CK(cudaEventRecord(b->ev_packed, s));
    CK(cudaStreamWaitEvent(bg, b->ev_packed, 0));
    CK(cudaEventRecord(b->ev_tail[par ^ 1], bg));
    for (int j = 0; j < count; ++j) {
        ++b->sessions[idx[j]]->nblk;
        ++b->sessions[idx[j]]->st.blocks;
    }
    ++b->step;
    return CONV_OK;
}

}  // namespace

extern "C" {

conv_batch* conv_batch_create(int precision) {
    if (precision < CONV_FP32 || precision > CONV_BF16) {
        set_err(CONV_E_INVAL, "unknown precision %d", precision);
        return nullptr;
    }
    conv_batch* b = new (std::nothrow) conv_batch();
    if (!b) {
        set_err(CONV_E_NOMEM, "out of host memory");
        return nullptr;
    }
    b->prec = precision;
    auto fail = [&](cudaError_t r, const char* what) {
        set_err(CONV_E_CUDA, "%s: %s", what, cudaGetErrorString(r));
        conv_batch_destroy(b);
        return nullptr;
    };
    cudaError_t r = cudaGetDevice(&b->dev);
    if (r != cudaSuccess) return fail(r, "cudaGetDevice");
    int lo = 0, hi = 0;
    if ((r = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess) return fail(r, "priorities");
    if ((r = cudaStreamCreateWithPriority(&b->stream, cudaStreamNonBlocking, hi)) != cudaSuccess) return fail(r, "stream");
    for (int i = 0; i < 2; ++i) {
        if ((r = cudaStreamCreateWithPriority(&b->bg[i], cudaStreamNonBlocking, lo)) != cudaSuccess) return fail(r, "stream");
        if ((r = cudaEventCreateWithFlags(&b->ev_tail[i], cudaEventDisableTiming)) != cudaSuccess) return fail(r, "event");
        if ((r = cudaEventCreateWithFlags(&b->ev_staged[i], cudaEventDisableTiming)) != cudaSuccess)
            return fail(r, "event");
        if ((r = cudaEventRecord(b->ev_tail[i], b->stream)) != cudaSuccess) return fail(r, "event");
        if ((r = cudaEventRecord(b->ev_staged[i], b->stream)) != cudaSuccess) return fail(r, "event");
    }
    if ((r = cudaEventCreateWithFlags(&b->ev_packed, cudaEventDisableTiming)) != cudaSuccess) return fail(r, "event");
    g_err.clear();
    return b;
}

int conv_batch_add(conv_batch* b, conv_engine* e) {
    if (!b || !e) return set_err(CONV_E_INVAL, "null argument");
    if (e->prec != b->prec) return set_err(CONV_E_INVAL, "session precision differs from the batch's");
    if (e->dev != b->dev) return set_err(CONV_E_INVAL, "session lives on another device");
    if (!e->syn.ready) return set_err(CONV_E_STATE, "filters not set");
    if (e->fb.allocated && !e->fb.ready) return set_err(CONV_E_STATE, "feedback paths not set");
    if (e->syn.plan.direct || e->syn.plan.nw != 8 || (e->fb.allocated && (e->fb.plan.direct || e->fb.plan.nw != 8)))
        return set_err(CONV_E_INVAL, "batched sessions use the TMA MAC with 8 consumer warps");
    if (e->adapt) return set_err(CONV_E_STATE, "sessions with an adaptive canceller are not batched");
    if (e->far) return set_err(CONV_E_STATE, "sessions with a far block are not batched");
    if (e->reuse) return set_err(CONV_E_STATE, "sessions in the n_f = 3 n_x form are not batched");
    for (conv_engine* x : b->sessions)
        if (x == e) return set_err(CONV_E_INVAL, "session already in the batch");
    DeviceGuard g(b->dev);
    int rc;
    if ((rc = batch_sync(b))) return rc;
    // the session's own streams may still run its last tail: let it finish
    for (int i = 0; i < 4; ++i) CK(cudaStreamSynchronize(e->bg[i]));
    CK(cudaStreamSynchronize(e->stream));
    e->hg.live = false;  // the batch runs the session's tails from here
    b->sessions.push_back(e);
    ++e->in_batches;
    return CONV_OK;
}

int conv_batch_remove(conv_batch* b, conv_engine* e) {
    if (!b || !e) return set_err(CONV_E_INVAL, "null argument");
    auto it = std::find(b->sessions.begin(), b->sessions.end(), e);
    if (it == b->sessions.end()) return set_err(CONV_E_INVAL, "session not in the batch");
    DeviceGuard g(b->dev);
    int rc;
    if ((rc = batch_sync(b))) return rc;
    b->sessions.erase(it);
    --e->in_batches;
    // its next block's tail partials are complete: mark them ready for its own streams
    CK(cudaEventRecord(e->syn.ev_tail[e->nblk & 1], e->stream));
    if (e->fb.allocated) CK(cudaEventRecord(e->fb.ev_tail[e->nblk & 1], e->stream));
    return CONV_OK;
}

int conv_batch_size(const conv_batch* b) { return b ? (int)b->sessions.size() : 0; }

int conv_batch_process_async(conv_batch* b, const float* const* d_in, float* const* d_out, void* cuda_stream) {
    if (!b) return set_err(CONV_E_INVAL, "null handle");
    const int n = (int)b->sessions.size();
    b->all_idx.resize(n);
    for (int i = 0; i < n; ++i) b->all_idx[i] = i;
    return conv_batch_process_some_async(b, n, b->all_idx.data(), d_in, d_out, cuda_stream);
}

int conv_batch_process_some_async(conv_batch* b, int count, const int* idx, const float* const* d_in,
                                  float* const* d_out, void* cuda_stream) {
    if (!b || (count > 0 && (!idx || !d_in || !d_out))) return set_err(CONV_E_INVAL, "null argument");
    const int nses = (int)b->sessions.size();
    if (count < 0 || count > nses) return set_err(CONV_E_INVAL, "count %d outside [0, %d]", count, nses);
    if (count == 0) return CONV_OK;
    std::vector<char> seen(nses, 0);
    for (int j = 0; j < count; ++j) {
        if (idx[j] < 0 || idx[j] >= nses || seen[idx[j]]) return set_err(CONV_E_INVAL, "bad session index %d", idx[j]);
        seen[idx[j]] = 1;
        if (!d_in[j] || !d_out[j]) return set_err(CONV_E_INVAL, "null buffer for session %d", idx[j]);
    }
    DeviceGuard g(b->dev);
    cudaStream_t s = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : b->stream;
    // count the CTAs of each launch (synthesis, feedback canceller)
    int n_pack = 0, n_out = 0, n_fpack = 0, n_fout = 0, n_mac = 0, n_afc = 0, Bmax = 16;
    size_t mac_smem = 0;
    for (int j = 0; j < count; ++j) {
        conv_engine* e = b->sessions[idx[j]];
        n_pack += e->syn.n_src;
        n_out += e->syn.n_dst;
        n_mac += e->syn.plan.S ? e->syn.plan.ctas : 0;
        Bmax = std::max(Bmax, e->B);
        if (e->syn.plan.S) mac_smem = std::max(mac_smem, e->syn.plan.smem);
        if (e->fb.allocated) {
            ++n_afc;
            n_fpack += e->fb.n_src;
            n_fout += e->fb.n_dst;
            n_mac += e->fb.plan.S ? e->fb.plan.ctas : 0;
            if (e->fb.plan.S) mac_smem = std::max(mac_smem, e->fb.plan.smem);
        }
    }
    const int n_items = count + n_afc;  // synthesis items first, then the canceller's
    const size_t o_pack = 0;
    const size_t o_out = align16(o_pack + (size_t)n_items * sizeof(PackArgs));
    const size_t o_mac = align16(o_out + (size_t)n_items * sizeof(OutArgs));
    const size_t o_rp = align16(o_mac + (size_t)n_items * sizeof(MacArgs));
    const size_t o_ro = align16(o_rp + (size_t)(n_pack + n_fpack) * sizeof(BatchRef));
    const size_t o_rm = align16(o_ro + (size_t)(n_out + n_fout) * sizeof(BatchRef));
    const int n_work = b->persistent ? n_pack + n_out + n_fpack + n_fout + n_mac : 0;
    const size_t o_work = align16(o_rm + (size_t)n_mac * sizeof(BatchRef));
    const size_t bytes = align16(o_work + (size_t)n_work * sizeof(PersistentWork));
    if (bytes > b->tab_cap) {
        int rc;
        if ((rc = batch_sync(b))) return rc;
        batch_free_tables(b);
        const size_t cap = bytes * 2;
        for (int i = 0; i < 2; ++i) {
            CK(cudaHostAlloc(reinterpret_cast<void**>(&b->h_tab[i]), cap, cudaHostAllocDefault));
            CK(cudaMalloc(reinterpret_cast<void**>(&b->d_tab[i]), cap));
        }
        b->tab_cap = cap;
    }
    const int par = (int)(b->step & 1);
    CK(cudaEventSynchronize(b->ev_staged[par]));  // the copy that last read this staging buffer is done
    unsigned char* h = b->h_tab[par];
    unsigned char* d = b->d_tab[par];
    PackArgs* pk = reinterpret_cast<PackArgs*>(h + o_pack);
    OutArgs* ot = reinterpret_cast<OutArgs*>(h + o_out);
    MacArgs* mc = reinterpret_cast<MacArgs*>(h + o_mac);
    BatchRef* rp = reinterpret_cast<BatchRef*>(h + o_rp);
    BatchRef* ro = reinterpret_cast<BatchRef*>(h + o_ro);
    BatchRef* rm = reinterpret_cast<BatchRef*>(h + o_rm);
    int ip = 0, io = 0, im = 0, ifp = n_pack, ifo = n_out, ia = count;
    for (int j = 0; j < count; ++j) {
        conv_engine* e = b->sessions[idx[j]];
        Part& P = e->syn;
        const long long blk = e->nblk;
        const bool afc = e->fb.allocated;
        // synthesis: e = mic - c_prev for canceller sessions (Sec. 5)
        pk[j] = pack_args(e, P, blk, d_in[j], e->B, afc ? e->d_c : nullptr, nullptr);
        ot[j] = out_args(e, P, blk, d_out[j]);
        ot[j].head_pre = 0;
        mc[j] = tail_args(e, P, blk + 1);
        mc[j].keep_r = 0;  // a batch's spectra together far exceed L2: all evict-first
        for (int c = 0; c < P.n_src; ++c) rp[ip++] = BatchRef{j, c, 0};
        for (int l = 0; l < P.n_dst; ++l) ro[io++] = BatchRef{j, l, 0};
        if (P.plan.S)
            for (int cta = 0; cta < P.plan.ctas; ++cta) rm[im++] = BatchRef{j, cta / P.plan.S, cta % P.plan.S};
        if (afc) {
            // canceller: c = F_hat * out, kept for the next block
            Part& F = e->fb;
            pk[ia] = pack_args(e, F, blk, d_out[j], e->B, nullptr, nullptr);
            ot[ia] = out_args(e, F, blk, e->d_c);
            ot[ia].head_pre = 0;
            mc[ia] = tail_args(e, F, blk + 1);
            mc[ia].keep_r = 0;
            for (int c = 0; c < F.n_src; ++c) rp[ifp++] = BatchRef{ia, c, 0};
            for (int l = 0; l < F.n_dst; ++l) ro[ifo++] = BatchRef{ia, l, 0};
            if (F.plan.S)
                for (int cta = 0; cta < F.plan.ctas; ++cta) rm[im++] = BatchRef{ia, cta / F.plan.S, cta % F.plan.S};
            ++ia;
        }
    }
    if (b->persistent) return batch_step_persistent(b, count, idx, h, d, o_pack, o_out, o_mac, o_work, n_work, n_items,
                                                    mac_smem, Bmax, bytes, par, s);
    CK(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(b->ev_staged[par], s));
    const PackArgs* d_pk = reinterpret_cast<const PackArgs*>(d + o_pack);
    const OutArgs* d_ot = reinterpret_cast<const OutArgs*>(d + o_out);
    const MacArgs* d_mc = reinterpret_cast<const MacArgs*>(d + o_mac);
    const BatchRef* d_rp = reinterpret_cast<const BatchRef*>(d + o_rp);
    const BatchRef* d_ro = reinterpret_cast<const BatchRef*>(d + o_ro);
    const BatchRef* d_rm = reinterpret_cast<const BatchRef*>(d + o_rm);
    // caller stream: pack all -> [wait outstanding tails] -> outputs; then the
    // canceller's pack and outputs.  A session that skipped steps computed its
    // tail in an earlier launch: waiting on both tail streams covers it.
    CK(launch_pack_batch(b->prec, d_pk, d_rp, n_pack, Bmax, s));
    if (!n_afc) CK(cudaEventRecord(b->ev_packed, s));
    CK(cudaStreamWaitEvent(s, b->ev_tail[0], 0));
    CK(cudaStreamWaitEvent(s, b->ev_tail[1], 0));
    CK(launch_out_batch(b->prec, d_ot, d_ro, n_out, Bmax, s));
    if (n_afc) {
        CK(launch_pack_batch(b->prec, d_pk, d_rp + n_pack, n_fpack, Bmax, s));
        CK(cudaEventRecord(b->ev_packed, s));
        CK(launch_out_batch(b->prec, d_ot, d_ro + n_out, n_fout, Bmax, s));
    }
    // background: the next block's tails of every processed session (both
    // convolutions) in one launch
    cudaStream_t bg = b->bg[par ^ 1];
    CK(cudaStreamWaitEvent(bg, b->ev_packed, 0));
    CK(launch_mac_batch(b->prec, d_mc, d_rm, n_mac, mac_smem, bg));
    CK(cudaEventRecord(b->ev_tail[par ^ 1], bg));
    for (int j = 0; j < count; ++j) {
        ++b->sessions[idx[j]]->nblk;
        ++b->sessions[idx[j]]->st.blocks;
    }
    ++b->step;
    return CONV_OK;
}

int conv_batch_set_persistent(conv_batch* b, int mode) {
    if (!b) return set_err(CONV_E_INVAL, "null handle");
    if (mode < 0 || mode > 2) return set_err(CONV_E_INVAL, "mode must be 0, 1 or 2");
    DeviceGuard g(b->dev);
    if (!b->num_sms) CK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev));
    b->persistent = mode != 0;
    b->graph = mode == 2;
    return CONV_OK;
}

int conv_batch_join_async(conv_batch* b, void* cuda_stream) {
    if (!b) return set_err(CONV_E_INVAL, "null handle");
    DeviceGuard g(b->dev);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the latest tail launch of each parity (every tail of the batch runs on one of the two)
    CK(cudaStreamWaitEvent(s, b->ev_tail[0], 0));
    CK(cudaStreamWaitEvent(s, b->ev_tail[1], 0));
    return CONV_OK;
}

int conv_batch_synchronize(conv_batch* b) {
    if (!b) return set_err(CONV_E_INVAL, "null handle");
    DeviceGuard g(b->dev);
    int rc = batch_sync(b);
    if (rc) return rc;
    for (conv_engine* e : b->sessions)
        if ((rc = check_dev_err(e))) return rc;
    return CONV_OK;
}

long long conv_batch_step_bytes(const conv_batch* b) {
    if (!b) return 0;
    long long t = 0;
    auto tail = [](const MacPlan& p) { return (long long)(((size_t)p.n_dst + 1) * (size_t)(p.R - p.r_begin) * p.B * p.es); };
    for (conv_engine* e : b->sessions) {
        t += tail(e->syn.plan);
        if (e->fb.allocated) t += tail(e->fb.plan);
    }
    return t;
}

void conv_batch_destroy(conv_batch* b) {
    if (!b) return;
    DeviceGuard g(b->dev);
    if (b->stream) batch_sync(b);
    for (conv_engine* e : b->sessions) {
        --e->in_batches;
        cudaEventRecord(e->syn.ev_tail[e->nblk & 1], e->stream);
        if (e->fb.allocated) cudaEventRecord(e->fb.ev_tail[e->nblk & 1], e->stream);
    }
    batch_free_tables(b);
    if (b->d_ctr) cudaFree(b->d_ctr);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ev_packed) cudaEventDestroy(b->ev_packed);
    for (int i = 0; i < 2; ++i) {
        if (b->ev_tail[i]) cudaEventDestroy(b->ev_tail[i]);
        if (b->ev_staged[i]) cudaEventDestroy(b->ev_staged[i]);
        if (b->bg[i]) cudaStreamDestroy(b->bg[i]);
    }
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

void conv_destroy(conv_engine* e) { engine_free(e); }

const char* conv_last_error(void) { return g_err.c_str(); }

}  // extern "C"
