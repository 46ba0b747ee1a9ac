// kernels.h - argument blocks and host launchers of the engine's CUDA kernels.
//
// Kernels (all hand-written for sm_103a, FP32 arithmetic):
//   pack_r2c    input packing + 2B-point R2C FFT + FDL push   (Sec. 4, stage 1)
//   filter_r2c  sub-filter zero-padding + R2C FFT            (Sec. 4, initialisation)
//   fdl_mac     FDL complex multiply-accumulate over a range of partitions of
//               all input->output pairs, split over partition ranges (Sec. 4,
//               stage 2; Eq. 6).  The engine runs it over partitions 1..K-1 of
//               the NEXT block as soon as the current block's spectrum is in
//               the delay line (they only need past input).
//   out_c2r     partition 0 of this block (the only part that needs the new
//               input) + fixed-order reduction of the split partials, C2R IFFT
//               and overlap-save discard                      (Sec. 4, stage 3)
//
// Spectra are "packed": bins 0..B-1 of the 2B-point real FFT, with the real
// Nyquist bin B stored in the imaginary slot of bin 0 (both are real for a
// real signal), so every row is B complex values.
//
// Reduction index: r = p * n_src + q (partition-major), so partition 0 of all
// inputs is r in [0, n_src) and partitions 1..K-1 are one contiguous range.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace gbconv {

enum Prec { PREC_FP32 = 0, PREC_FP16 = 1, PREC_BF16 = 2 };

// Device error codes written to the engine's host-mapped error word.
enum DevErr { DEVERR_NONE = 0, DEVERR_TIMEOUT_PRODUCER = 1, DEVERR_TIMEOUT_CONSUMER = 2 };

constexpr int MAC_CONSUMER_WARPS = 8;  // default consumer warps (8 or 16), plus one producer warp
constexpr int MAC_HDR_BYTES = 1024;                          // mbarriers + flags
constexpr int MAX_STAGES = 8;
constexpr size_t MAC_SMEM_LIMIT = 227 * 1024;  // dynamic shared memory the MAC may use (sm_100 family maximum)
constexpr size_t SM_SMEM_BYTES = 228 * 1024;   // shared memory per SM
constexpr size_t CTA_SMEM_RESERVED = 1024;     // per-CTA system reservation

// Tiling of one FDL MAC (one partitioned convolution with n_src inputs, n_dst
// outputs and K partitions) over the reduction range [r_begin, R).  Spectra of
// a (bin tile, output tile) pair are stored contiguously over r, so each CTA
// streams one contiguous range.
struct MacPlan {
    int B, n_src, n_dst, K, R;
    int r_begin;   // first reduction index the MAC covers
    int es;        // bytes per stored complex value (8 fp32, 4 fp16/bf16)
    int VEC;       // complex values per 16-byte load
    int LPT;       // max outputs per consumer thread
    int BT, n_kt;  // bin tile width, number of bin tiles
    int LT, n_lt;  // output tile height, number of output tiles
    int nw;        // consumer warps (8 or 16)
    int interleave;  // TMA MAC: 1 = split s takes stages s, s+S, ... (else contiguous ranges)
    int direct;    // direct-load MAC (no TMA ring, 8 warps): 1 = one partition in flight per
                   // thread, 3 CTAs/SM; 2 = two in flight, 2 CTAs/SM; 0 = TMA pipeline
    int kthreads, NLG, NRL;  // consumer thread layout: bins x output groups x r-lanes
    int RS;        // reduction indices per pipeline stage (the stage grid's pitch)
    int nstage;    // pipeline depth
    int S;         // partition splits per tile (0: empty range, no MAC launch)
    unsigned stage_bytes, xoff;
    unsigned soff, sxoff;  // reduced precision: filter / delay-line scale parts of a stage
    size_t smem;   // dynamic shared memory per CTA
    int ctas;
    size_t tile_elems;  // filter tile pitch in stored values (64 KiB aligned)
    size_t h_bytes, x_bytes, partial_bytes;
};

struct MacArgs {
    const void* H;    // filter spectra: tile (kt, lt) at (kt*n_lt + lt)*tile_elems, then [r][LTt][BT]
    const void* X;    // FDL ring [kt][slot][q][BT]
    const float* sH;  // [lt tile][r] per-partition scales (reduced precision), else null
    const float* sX;  // [K][n_src] per-slot scales (reduced precision), else null
    float2* partial;  // [S][n_dst][B]
    int B, BT, n_kt, n_dst, LT, n_lt, n_src, K, S, RS, nstage;
    int r_begin;
    int interleave;
    int kthreads, NLG, NRL;
    int slot0;  // ring slot of partition 0 for the block this MAC serves
    unsigned stage_bytes, xoff, soff, sxoff;
    size_t tile_elems;
    int* err;   // device-visible error word (host-mapped), or null
    // bound of the pipeline's barrier waits in ns (0: the default, 1 s)
    unsigned long long wait_ns;
    // fault-path testing (TMA kernel): 1 = the producer of tile 0 / split 0
    // withholds its first stage, so that CTA's consumers wait on a barrier
    // nothing completes and give up after wait_ns (error word, abort flag)
    int withhold;
    // filter-spectrum rows r < keep_r are streamed with the L2 evict-last
    // policy (kept in L2 from one block to the next), the others evict-first
    int keep_r;
    // non-null (the host-call graph, whose arguments stay the same from block
    // to block): this MAC serves block *blk + blk_add, whose partition-0 slot
    // replaces slot0 and whose parity picks partial (even) or partial_b (odd)
    const long long* blk;
    float2* partial_b;
    int blk_add;
};

struct PackArgs {
    const float* in;  // [n_ch][in_stride], first B samples of each row used
    int in_stride;
    const float* sub;  // [n_ch][B] subtracted from `in` (feedback prediction), or null
    float* e_out;      // [n_ch][e_stride] receives in - sub, or null
    int e_stride;      // row pitch of e_out (0: B)
    float* win;        // [n_ch][B] previous block (sliding-window state)
    void* X;           // FDL ring [n_kt][K][n_ch][BT] (storage type)
    float* sX;         // [K][n_ch] slot scales (reduced precision), else null
    int B, log2B, BT, n_ch, K, slot;
    const float2* tw;  // W_2B^j = exp(-i pi j / B), j in [0, 2B)
    // FP32 rings only: receives the slot's previous spectra, [n_kt][n_ch][BT],
    // before the push overwrites them (null: not kept)
    float2* save_old;
    // non-null (host-call graph): the block number, whose ring slot replaces
    // slot (launch_pack_r2c then launches the kernel's variant that reads it)
    const long long* blk;
};

struct FilterArgs {
    const float* h;  // [n_dst][n_src][taps]
    long long taps;
    int n_dst, n_src, K, B, log2B, BT, LT;
    void* H;    // tiled spectra
    const float* sH;  // [lt tile][r] scales (reduced precision pass 1), else null
    float* maxabs;    // [n_dst][R] largest components (reduced precision pass 0)
    int pass;         // reduced precision: 0 = record maxabs, 1 = store scaled
    size_t tile_elems;
    const float2* tw;
};

struct OutArgs {
    const float2* partial;  // [S][n_dst][B] (S may be 0)
    int S, n_dst, B, log2B;
    const float2* tw;
    float* out;  // [n_dst][out_stride]
    int out_stride;
    // partition 0 of this block, added after the split partials (head = 0: none)
    int head;
    const void* H;
    const void* X;
    const float* sH;
    const float* sX;
    int n_src, K, R, BT, LT, slot0;
    size_t tile_elems;
    // added to the output after the overlap-save discard ([n_dst][extra_stride]), or null
    const float* extra;
    int extra_stride;
    // 1: the partials come from another stream, complete before this launch, so
    // they are summed before waiting for the previous kernel in the stream;
    // 0: the previous kernel may be writing them
    int early_partials;
    // FP32 only (corr_G null: none).  Adds corr_G[l][k] * sum_c corr_A[c][k] +
    // corr_G2[l][k] * sum_c corr_A2[c][k] to bin k: the effect of the two
    // NLMS steps that the tail's filter spectra do not hold yet (see nlms.h)
    const float2* corr_G;   // [n_dst][B] this block's step
    const float2* corr_G2;  // [n_dst][B] the previous block's step
    const float2* corr_A;   // [corr_C][B] lag-one correlation chunks
    const float2* corr_A2;  // [corr_C][B] lag-two correlation chunks
    int corr_C;
    // 1: the launch adds n_src*B float2 of shared memory in which the head's
    // filter spectra (constant) are loaded before waiting for the previous
    // kernel (out_head_smem)
    int head_pre;
    // non-null (host-call graph): the block number, whose slot replaces slot0
    // and whose parity picks partial (even) or partial_b (odd) (launch_out_c2r
    // then launches the kernel's variant that reads it)
    const long long* blk;
    const float2* partial_b;
};

// Extra shared memory of an output launch that prefetches its head spectra
// (0 when n_src x B is too large to keep the CTA small).
size_t out_head_smem(int n_src, int B);

// One CTA of a batched launch: which session's arguments (items[item]), and
// the channel (pack/output) or the tile and split (MAC) it serves.
struct BatchRef {
    int item, idx, idx2;
};

// The batched MAC stages its arguments in the shared-memory header after the
// mbarriers and the abort flag.
constexpr int MAC_ARGS_OFFSET = 256;
// ... and keeps the reduced-precision MAC's per-warp scale maxima there.
constexpr int MAC_RED_OFFSET = 768;

// One work item of a persistent batch step (launch_batch_persistent).  The
// CTAs claim items in list order; an item may wait for a counter that items
// earlier in the list raise, so the lowest unfinished item never waits on an
// unclaimed one and the step cannot deadlock.
enum PersistentWorkType { PW_PACK = 0, PW_OUT = 1, PW_MAC = 2 };
// Shared memory the persistent step kernel keeps for its static variables;
// its dynamic part is limited to MAC_SMEM_LIMIT minus this.
constexpr size_t PERSISTENT_STATIC_SMEM = 2048;
struct PersistentWork {
    int type;    // PersistentWorkType
    int item;    // index into the pack / output / MAC argument tables
    int idx, idx2;  // channel (pack, output) or tile and split (MAC)
    int wait;    // counter to wait for (-1: none) ...
    int target;  // ... until it reaches this value
    int signal;  // counter raised when the item is done (-1: none)
};

int fft_threads(int B);
int out_threads(int B);
size_t fft_smem_bytes(int B);

// Sets the message conv_last_error() returns on the calling thread.
void set_last_error_message(const char* msg);

cudaError_t prepare_kernels(size_t mac_smem);
// closed_loop: the canceller's schedule (kernels with the default shared-memory carveout)
cudaError_t launch_pack_r2c(int prec, const PackArgs& a, cudaStream_t s, bool closed_loop = false);
cudaError_t launch_filter_r2c(int prec, const FilterArgs& a, cudaStream_t s);
cudaError_t launch_tile_scales(int prec, const float* maxabs, float* sH, int n_dst, int R, int LT, cudaStream_t s);
// pdl: programmatic dependent launch after the previous kernel in the stream.
// The MAC streams its first filter stages before waiting for that kernel, so
// pass false when the previous kernel writes the filter spectra.
cudaError_t launch_fdl_mac(int prec, const MacPlan& p, const MacArgs& a, cudaStream_t s, bool pdl = true);
cudaError_t launch_out_c2r(int prec, const OutArgs& a, cudaStream_t s, bool closed_loop = false);
// Output (a) fused with the push of each output channel into another ring (b,
// b.in = a.out, b.n_ch = a.n_dst).  a.blk and b.blk are both set (the
// variant that reads the block number) or both null.
// Pack, output and push launch their block-number variants (the host-call
// graphs) when the arguments' blk is set, closed loop or not.
cudaError_t launch_out_push(int prec, const OutArgs& a, const PackArgs& b, cudaStream_t s);
cudaError_t launch_pack_batch(int prec, const PackArgs* items, const BatchRef* refs, int n, int Bmax, cudaStream_t s);
cudaError_t launch_out_batch(int prec, const OutArgs* items, const BatchRef* refs, int n, int Bmax, cudaStream_t s);
cudaError_t launch_mac_batch(int prec, const MacArgs* items, const BatchRef* refs, int n, size_t smem, cudaStream_t s);
// One batch step as a single launch of `ctas` persistent CTAs working through
// `work` (device, n_work items).  ctr: device counters, [0] the claim counter
// and [1 + i] counter i, all zero at launch.  err: device error word (a
// bounded dependency wait that gave up).  smem: the larger of the MAC's and
// the FFT kernels' dynamic shared memory.
// The n_f = 3 n_x form (reuse.cu; block in [32, 4096]).  PackArgs.win holds
// [n_ch][2 B]; the twiddle table (PackArgs / OutArgs / FilterArgs .tw) is
// W_3B^j, j in [0, 3B); every spectrum row has 3B/2 packed bins and the MAC
// is planned over them.  launch_out3 pushes each output channel's
// accumulated spectrum into push's ring when push.X is set (push.n_ch =
// a.n_dst).
size_t fft3_smem_bytes(int B);
cudaError_t prepare_reuse_kernels();
cudaError_t launch_pack3(int prec, const PackArgs& a, cudaStream_t s);
cudaError_t launch_filter3(int prec, const FilterArgs& a, cudaStream_t s);
cudaError_t launch_out3(int prec, const OutArgs& a, const PackArgs& push, cudaStream_t s);
cudaError_t launch_batch_persistent(int prec, const PackArgs* pk, const OutArgs* ot, const MacArgs* mc,
                                    const PersistentWork* work, int n_work, unsigned* ctr, int* err, int ctas,
                                    size_t smem, cudaStream_t s);

}  // namespace gbconv
