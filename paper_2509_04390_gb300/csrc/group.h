// group.h - shared-filter session groups: plan, argument blocks, launchers.
//
// S sessions that use the same filter set H (n_out x n_in x taps, block B) and
// run in lock-step turn the FDL MAC of Sec. 4 (Eq. 6) into one small complex
// GEMM per bin:  Y_k[l][s] = sum_r H_k[l][r] X_k[r][s],  r = p*n_src + q.
// The kernels run it on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16, FP32 accumulators in tensor memory):
//
//   rows (M = 128)    G = 128 / n_out bins x n_out outputs of one bin group
//   columns (N)       2 parts (re, im) x G bins x S sessions
//   reduction (K=16)  16 consecutive r of one K-step
//
// Every bin of a group meets every bin's delay line, so only the G diagonal
// blocks of the M x N product are kept (the rest is the price of batching G
// small GEMMs into one instruction; tensor throughput is far above the
// HBM-bound rate).  The real and imaginary filter parts are two A operands
// (D1 = Hr X, D2 = Hi X); the epilogue forms Yr = D1[re] - D2[im],
// Yi = D1[im] + D2[re], and for the packed bin 0 (DC, Nyquist) the two real
// products D1[re], D2[im].
//
// Operands are stored in HBM exactly as the canonical no-swizzle K-major
// shared-memory layout wants them (core matrices of 8 rows x 16 bytes), so
// each pipeline stage is two or three plain bulk copies:
//
//   filter tiles  per (group g, K-step c): [Hr 4 KiB][Hi 4 KiB]; core matrix
//                 (row group rg, K half kc) at kc*2048 + rg*128
//   delay line    ring rows of RB = 32*G*S bytes; ring row t holds slots
//                 t .. t+D-1 (mod KR) of every (part, bin, session) as one
//                 16-byte core-matrix row [slot u][input q] (D = 8 / n_src), so
//                 every slot is written D times by the pack and read once by
//                 the MAC; rows are stored by class t mod D so that the rows
//                 a run of K-steps needs are consecutive
//
// Storage FP16 or BF16 (both operands the same type).  Filter rows carry a
// power-of-two scale per (bin, output), applied in the epilogue; the delay
// line is unscaled (FP16 holds spectra up to 65504, i.e. |x| <= 1 at any
// block size; larger values saturate).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace gbconv {

constexpr int GRP_HDR_BYTES = 1024;
constexpr int GRP_MAX_STAGES = 8;
constexpr int GRP_THREADS = 192;  // producer warp, MMA warp, 4 epilogue warps

// Tiling fields a caller may fix (0 leaves a field to the planner).
struct GroupTiling {
    int ctas = 0;           // MAC CTAs (at most one per SM)
    int stage_k_steps = 0;  // K-steps per pipeline stage (1..4)
    int stages = 0;         // pipeline depth (2..8)
    int tail_streams = 0;   // background streams the tails alternate over (1 or 2)
};

// Work split of the tail MAC: the NG * T units (bin group g, tail K-step c =
// 1 + u - g*T) are cut into C equal runs, run i = [i*U/C, (i+1)*U/C), one per
// CTA; a run that crosses a group boundary finishes one accumulator and starts
// the next.  The CTAs that share a group write partials to consecutive slots.
__host__ __device__ inline int group_cta_of_unit(long long u, long long U, int C) {
    long long i = u * C / U;
    while (i + 1 < C && (i + 1) * U / C <= u) ++i;
    while (i > 0 && i * U / C > u) --i;
    return (int)i;
}

struct GroupPlan {
    int B, n_src, n_dst, S, K;
    int G;         // bins per group = 128 / n_dst
    int NG;        // groups = B / G
    int D;         // slots per ring row = 8 / n_src
    int KP;        // partitions per K-step = 2 D
    int KR;        // ring slots = K rounded up to KP
    int NKS;       // K-steps per block = KR / KP
    int N;         // MMA N = 2 G S
    int RB;        // ring row bytes = 32 G S
    int T;         // tail K-steps per group, NKS - 1
    int C;         // tail MAC CTAs (0: no tail)
    int SP;        // partial slots per group: most CTAs that share one group
    int NK;        // K-steps per pipeline stage
    int nstage;
    int stage_bytes;  // NK * (8192 + 2 RB)
    int smem;         // dynamic shared memory per CTA
    int nbuf;      // TMEM accumulator buffers (2: the next group's MMAs overlap the epilogue)
    int tail_streams;
    int tmem_cols;    // power of two >= nbuf * 2 N
    size_t h_bytes, x_bytes, partial_bytes;  // partial_bytes: one block parity
};

struct GroupMacArgs {
    const void* H;       // filter tiles
    const void* X;       // ring
    const float* sH;     // [NG][128] row scales
    float2* partial;     // [S][SP][n_dst][B]
    int B, n_dst, S, G, NG, D, KP, KR, NKS, N, RB, T, C, SP, NK, nstage, stage_bytes, slot0, tmem_cols, nbuf;
    uint32_t idesc;
    int* err;
    // K-steps c < keep_c of every bin group are streamed with the L2
    // evict-last policy (kept in L2 from one block to the next)
    int keep_c;
};

struct GroupPackArgs {
    const float* in;  // [S][n_src][in_stride], first B samples of each row used
    int in_stride;
    float* win;       // [S][n_src][B]
    void* X;
    int B, log2B, n_src, S, G, D, KR, RB, slot;
    const float2* tw;
};

struct GroupFilterArgs {
    const float* h;  // [n_dst][n_src][taps]
    long long taps;
    int n_dst, n_src, K, B, log2B, G, KP, NKS, pass;
    unsigned* maxbits;  // [B][n_dst] largest |component| (float bits), pass 0
    float* sH;          // [NG][128] written in pass 1
    void* H;
    const float2* tw;
};

struct GroupOutArgs {
    const float2* partial;
    float* out;  // [S][n_dst][out_stride], first B samples of each row written
    int out_stride;
    int B, log2B, n_dst, T, C, SP;
    const float2* tw;
    // head: K-step 0 (partitions 0 .. KP-1) of this block, on CUDA cores
    const void* H;
    const void* X;
    const float* sH;
    int G, D, KR, NKS, RB, S, slot0;
};

// Plans a group; returns nullptr or a message naming the unsupported parameter.
const char* plan_group(int prec, int B, int n_src, int n_dst, long long taps, int S, int num_sms, GroupPlan* p,
                       const GroupTiling& t = GroupTiling());
// Replays every copy and store address of one block against the buffer and
// shared-memory sizes (host only); nullptr or a message.
const char* check_group_plan(const GroupPlan& p);

cudaError_t prepare_group_kernels();
cudaError_t launch_group_filter(int prec, const GroupFilterArgs& a, cudaStream_t s);
cudaError_t launch_group_pack(int prec, const GroupPackArgs& a, cudaStream_t s);
cudaError_t launch_group_mac(const GroupPlan& p, const GroupMacArgs& a, cudaStream_t s);
cudaError_t launch_group_out(int prec, const GroupOutArgs& a, cudaStream_t s);

}  // namespace gbconv
