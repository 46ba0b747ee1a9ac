// group_engine.cu - the conv_group_* entry points of conv.h: shared-filter
// session groups whose FDL MAC runs on the tensor cores (group.h).
//
// Split-phase schedule, as for a single engine.  K-steps 1.. of block n+1
// (partitions KP.., which need only spectra of blocks <= n+1-KP) are the
// "tail": the tensor-core MAC runs them on a low-priority background stream
// as soon as block n's spectra are in the ring, into split partials of block
// n+1's parity.  When block n+1 arrives, the caller's stream runs the pack +
// R2C of every session and one output kernel per (session, output) that adds
// K-step 0 (the "head", on CUDA cores) to the tail's partials and transforms
// back.  Tails alternate between two background streams:
//   caller stream:      pack(n) -> [rec packed] -> [wait tail(n)] -> out(n)
//   background n+1 & 1: [wait packed(n)] -> tail(n+1) -> [rec tail(n+1 & 1)]
// pack(n+1) overwrites the slot of block n+1-KR, which only tail(n) read (and
// out(n) waited for it); the ring rows pack(n+1) writes are never rows that
// tail(n+1) reads (they hold slot0(n+1) at position 0 only in K-step 0's row).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "conv.h"
#include "group.h"
#include "host_util.h"

// Filter tiles a group keeps in L2 between blocks by default (conv_group_set_l2_keep)
constexpr long long GROUP_L2_KEEP_DEFAULT = 60LL * 1000 * 1000;
#include "kernels.h"

using namespace gbconv;

struct conv_group {
    int dev = 0;
    int prec = CONV_FP16;
    int B = 0, log2B = 0, n_in = 0, n_out = 0, S = 0;
    long long taps = 0;
    int num_sms = 0;
    GroupPlan plan{};
    uint32_t idesc = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t bg[2] = {nullptr, nullptr};
    cudaEvent_t ev_done = nullptr;
    cudaEvent_t ev_packed = nullptr;
    cudaEvent_t ev_handoff = nullptr;  // orders a block after the previous one enqueued on another stream
    cudaStream_t last_stream = nullptr;
    bool has_last = false;
    cudaEvent_t ev_tail[2] = {nullptr, nullptr};
    void* H = nullptr;
    void* X = nullptr;
    float* sH = nullptr;
    float* win = nullptr;
    float2* partial[2] = {nullptr, nullptr};  // tail partials by block parity
    float2* tw = nullptr;
    float *h_in = nullptr, *h_out = nullptr;  // mapped pinned host staging of conv_group_process
    float *m_in = nullptr, *m_out = nullptr;  // their device addresses
    float *d_cin = nullptr, *d_cout = nullptr;  // conv_group_process_blocks chunk buffers
    long long chunk_cap = 0;
    int io_stride = 0;  // row pitch of the input and output of the block being enqueued (0: block)
    int *h_err = nullptr, *d_err = nullptr;
    long long nblk = 0;
    bool ready = false;
    bool prof = false;
    // conv_group_set_l2_keep: bytes of filter tiles streamed evict-last
    long long l2_keep = GROUP_L2_KEEP_DEFAULT;
    std::vector<cudaEvent_t> ev0, ev1;
    size_t ev_used = 0;
    size_t dev_bytes = 0;
};

namespace {

template <typename T>
int galloc(conv_group* g, T** p, size_t bytes) {
    cudaError_t r = cudaMalloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
    if (r != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(r == cudaErrorMemoryAllocation ? CONV_E_NOMEM : CONV_E_CUDA, "cudaMalloc(%zu): %s", bytes,
                    cudaGetErrorString(r));
    }
    g->dev_bytes += bytes ? bytes : 16;
    return CONV_OK;
}

void group_free(conv_group* g) {
    if (!g) return;
    DeviceGuard d(g->dev);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (int i = 0; i < 2; ++i)
        if (g->bg[i]) cudaStreamSynchronize(g->bg[i]);
    for (void* p : {g->H, g->X, (void*)g->sH, (void*)g->win, (void*)g->partial[0], (void*)g->partial[1], (void*)g->tw,
                    (void*)g->d_cin, (void*)g->d_cout})
        if (p) cudaFree(p);
    if (g->h_in) cudaFreeHost(g->h_in);
    if (g->h_out) cudaFreeHost(g->h_out);
    if (g->h_err) cudaFreeHost(g->h_err);
    for (auto ev : g->ev0) cudaEventDestroy(ev);
    for (auto ev : g->ev1) cudaEventDestroy(ev);
    if (g->ev_done) cudaEventDestroy(g->ev_done);
    if (g->ev_packed) cudaEventDestroy(g->ev_packed);
    if (g->ev_handoff) cudaEventDestroy(g->ev_handoff);
    for (int i = 0; i < 2; ++i) {
        if (g->ev_tail[i]) cudaEventDestroy(g->ev_tail[i]);
        if (g->bg[i]) cudaStreamDestroy(g->bg[i]);
    }
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

int to_prec(int precision) {
    return precision == CONV_FP16 ? PREC_FP16 : (precision == CONV_BF16 ? PREC_BF16 : (precision == CONV_FP32 ? PREC_FP32 : -1));
}

int sync_all(conv_group* g) {
    for (int i = 0; i < 2; ++i) GB_CK(cudaStreamSynchronize(g->bg[i]));
    GB_CK(cudaStreamSynchronize(g->stream));
    return CONV_OK;
}

int group_reset_impl(conv_group* g) {
    int rc;
    if (g->has_last) GB_CK(cudaStreamSynchronize(g->last_stream));  // blocks enqueued on a caller's stream
    if ((rc = sync_all(g))) return rc;
    const GroupPlan& p = g->plan;
    GB_CK(cudaMemsetAsync(g->X, 0, p.x_bytes, g->stream));
    GB_CK(cudaMemsetAsync(g->win, 0, (size_t)g->S * g->n_in * g->B * sizeof(float), g->stream));
    for (int i = 0; i < 2; ++i) {
        GB_CK(cudaMemsetAsync(g->partial[i], 0, p.partial_bytes, g->stream));
        GB_CK(cudaEventRecord(g->ev_tail[i], g->stream));  // block 0's tail: zero partials
    }
    GB_CK(cudaStreamSynchronize(g->stream));
    g->nblk = 0;
    g->has_last = false;
    return CONV_OK;
}

GroupTiling from_api(const conv_group_tiling* t) {
    GroupTiling o;
    if (t) {
        o.ctas = t->ctas;
        o.stage_k_steps = t->stage_k_steps;
        o.stages = t->stages;
        o.tail_streams = t->tail_streams;
    }
    return o;
}

int create_impl(conv_group* g, int precision, int block, int n_in, int n_out, long long taps, int sessions,
                const conv_group_tiling* tiling) {
    const int prec = to_prec(precision);
    if (prec < 0) return fail(CONV_E_INVAL, "unknown precision %d", precision);
    GB_CK(cudaGetDevice(&g->dev));
    cudaDeviceProp prop{};
    GB_CK(cudaGetDeviceProperties(&prop, g->dev));
    g->num_sms = prop.multiProcessorCount;
    if (const char* why = plan_group(prec, block, n_in, n_out, taps, sessions, g->num_sms, &g->plan, from_api(tiling)))
        return fail(CONV_E_INVAL, "%s", why);
    if (const char* why = check_group_plan(g->plan)) return fail(CONV_E_INVAL, "%s", why);
    g->prec = precision;
    g->B = block;
    g->log2B = 0;
    while ((1 << g->log2B) < block) ++g->log2B;
    g->n_in = n_in;
    g->n_out = n_out;
    g->S = sessions;
    g->taps = taps;
    const GroupPlan& p = g->plan;
    const uint32_t t = prec == PREC_BF16 ? 1u : 0u;
    // kind::f16: D F32, A and B of the same 16-bit type, both K-major, N, M = 128
    g->idesc = (1u << 4) | (t << 7) | (t << 10) | ((uint32_t)(p.N >> 3) << 17) | ((128u >> 4) << 24);
    size_t free_b = 0, total_b = 0;
    GB_CK(cudaMemGetInfo(&free_b, &total_b));
    const size_t need = p.h_bytes + p.x_bytes + 2 * p.partial_bytes + (size_t)p.NG * 128 * sizeof(float) +
                        (size_t)sessions * (n_in + n_out) * block * sizeof(float) * 2;
    if (need + (64ull << 20) > free_b)
        return fail(CONV_E_NOMEM, "device footprint %zu bytes does not fit in %zu free bytes", need, free_b);
    GB_CK(prepare_group_kernels());
    int rc;
    if ((rc = galloc(g, &g->H, p.h_bytes))) return rc;
    if ((rc = galloc(g, &g->X, p.x_bytes))) return rc;
    if ((rc = galloc(g, &g->sH, (size_t)p.NG * 128 * sizeof(float)))) return rc;
    if ((rc = galloc(g, &g->win, (size_t)sessions * n_in * block * sizeof(float)))) return rc;
    if ((rc = galloc(g, &g->partial[0], p.partial_bytes))) return rc;
    if ((rc = galloc(g, &g->partial[1], p.partial_bytes))) return rc;
    if ((rc = galloc(g, &g->tw, 2 * (size_t)block * sizeof(float2)))) return rc;
    GB_CK(cudaHostAlloc(reinterpret_cast<void**>(&g->h_in), (size_t)sessions * n_in * block * sizeof(float),
                        cudaHostAllocMapped));
    GB_CK(cudaHostAlloc(reinterpret_cast<void**>(&g->h_out), (size_t)sessions * n_out * block * sizeof(float),
                        cudaHostAllocMapped));
    GB_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&g->m_in), g->h_in, 0));
    GB_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&g->m_out), g->h_out, 0));
    GB_CK(cudaHostAlloc(reinterpret_cast<void**>(&g->h_err), sizeof(int), cudaHostAllocMapped));
    *g->h_err = 0;
    GB_CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&g->d_err), g->h_err, 0));
    int lo = 0, hi = 0;
    GB_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    GB_CK(cudaStreamCreateWithPriority(&g->stream, cudaStreamNonBlocking, hi));
    for (int i = 0; i < 2; ++i) {
        GB_CK(cudaStreamCreateWithPriority(&g->bg[i], cudaStreamNonBlocking, lo));
        GB_CK(cudaEventCreateWithFlags(&g->ev_tail[i], cudaEventDisableTiming));
    }
    GB_CK(cudaEventCreateWithFlags(&g->ev_packed, cudaEventDisableTiming));
    GB_CK(cudaEventCreateWithFlags(&g->ev_handoff, cudaEventDisableTiming));
    GB_CK(cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming));
    // twiddles W_2B^j = exp(-i pi j / B), FP64 on the host, rounded once
    std::vector<float2> tw(2 * (size_t)block);
    const double pi = 3.14159265358979323846264338327950288;
    for (int j = 0; j < 2 * block; ++j) {
        const double ang = -pi * (double)j / (double)block;
        tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    GB_CK(cudaMemcpy(g->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    GB_CK(cudaMemset(g->H, 0, p.h_bytes));
    GB_CK(cudaMemset(g->sH, 0, (size_t)p.NG * 128 * sizeof(float)));
    return group_reset_impl(g);
}

inline int slot0_of(long long n, int KR) {
    const int m = (int)(n % KR);
    return m == 0 ? 0 : KR - m;  // slot of partition 0 at block n: (0 - n) mod KR
}

// Tail MAC of block `blk` (K-steps 1..NKS-1) into the partials of its parity.
int enqueue_tail(conv_group* g, long long blk, cudaStream_t s) {
    const GroupPlan& p = g->plan;
    if (p.C == 0) return CONV_OK;
    GroupMacArgs a{};
    a.H = g->H;
    a.X = g->X;
    a.sH = g->sH;
    a.partial = g->partial[blk & 1];
    a.B = g->B;
    a.n_dst = g->n_out;
    a.S = g->S;
    a.G = p.G;
    a.NG = p.NG;
    a.D = p.D;
    a.KP = p.KP;
    a.KR = p.KR;
    a.NKS = p.NKS;
    a.N = p.N;
    a.RB = p.RB;
    a.T = p.T;
    a.C = p.C;
    a.SP = p.SP;
    a.nbuf = p.nbuf;
    a.NK = p.NK;
    a.nstage = p.nstage;
    a.stage_bytes = p.stage_bytes;
    a.slot0 = slot0_of(blk, p.KR);
    a.tmem_cols = p.tmem_cols;
    a.idesc = g->idesc;
    a.err = g->d_err;
    // one K-step of every bin group is NG filter tiles of 8 KiB
    a.keep_c = (int)std::min<long long>(p.NKS, g->l2_keep / ((long long)p.NG * 8192));
    const bool rec = g->prof && g->ev_used < g->ev0.size();
    if (rec) GB_CK(cudaEventRecord(g->ev0[g->ev_used], s));
    GB_CK(launch_group_mac(p, a, s));
    if (rec) {
        GB_CK(cudaEventRecord(g->ev1[g->ev_used], s));
        ++g->ev_used;
    }
    return CONV_OK;
}

int enqueue_group(conv_group* g, const float* d_in, float* d_out, cudaStream_t s) {
    // blocks of a group are a chain: a block on another stream than the
    // previous one first waits for that stream
    if (g->has_last && s != g->last_stream) {
        GB_CK(cudaEventRecord(g->ev_handoff, g->last_stream));
        GB_CK(cudaStreamWaitEvent(s, g->ev_handoff, 0));
    }
    g->last_stream = s;
    g->has_last = true;
    const GroupPlan& p = g->plan;
    const long long n = g->nblk;
    const int slot0 = slot0_of(n, p.KR);
    const int prec = to_prec(g->prec);
    GroupPackArgs pk{};
    pk.in = d_in;
    pk.in_stride = g->io_stride ? g->io_stride : g->B;
    pk.win = g->win;
    pk.X = g->X;
    pk.B = g->B;
    pk.log2B = g->log2B;
    pk.n_src = g->n_in;
    pk.S = g->S;
    pk.G = p.G;
    pk.D = p.D;
    pk.KR = p.KR;
    pk.RB = p.RB;
    pk.slot = slot0;
    pk.tw = g->tw;
    GB_CK(launch_group_pack(prec, pk, s));
    GB_CK(cudaEventRecord(g->ev_packed, s));
    GB_CK(cudaStreamWaitEvent(s, g->ev_tail[n & 1], 0));
    GroupOutArgs o{};
    o.partial = g->partial[n & 1];
    o.out = d_out;
    o.out_stride = g->io_stride ? g->io_stride : g->B;
    o.B = g->B;
    o.log2B = g->log2B;
    o.n_dst = g->n_out;
    o.T = p.T;
    o.C = p.C;
    o.SP = p.SP;
    o.tw = g->tw;
    o.H = g->H;
    o.X = g->X;
    o.sH = g->sH;
    o.G = p.G;
    o.D = p.D;
    o.KR = p.KR;
    o.NKS = p.NKS;
    o.RB = p.RB;
    o.S = g->S;
    o.slot0 = slot0;
    GB_CK(launch_group_out(prec, o, s));
    cudaStream_t bg = g->bg[p.tail_streams == 2 ? (n + 1) & 1 : 0];
    GB_CK(cudaStreamWaitEvent(bg, g->ev_packed, 0));
    // kernel timing needs each tail alone on the GPU: then tails run one after another
    if (g->prof) GB_CK(cudaStreamWaitEvent(bg, g->ev_tail[n & 1], 0));
    int rc = enqueue_tail(g, n + 1, bg);
    if (rc) return rc;
    GB_CK(cudaEventRecord(g->ev_tail[(n + 1) & 1], bg));
    ++g->nblk;
    return CONV_OK;
}

int check_err(conv_group* g) {
    const int v = *(volatile int*)g->h_err;
    if (v != 0) {
        *(volatile int*)g->h_err = 0;
        return fail(CONV_E_TIMEOUT, "device-side wait gave up (code %d); results of the block are invalid", v);
    }
    return CONV_OK;
}

}  // namespace

extern "C" {

conv_group* conv_group_create(int precision, int block, int n_in, int n_out, long long taps, int sessions) {
    return conv_group_create_tiled(precision, block, n_in, n_out, taps, sessions, nullptr);
}

conv_group* conv_group_create_tiled(int precision, int block, int n_in, int n_out, long long taps, int sessions,
                                    const conv_group_tiling* tiling) {
    conv_group* g = new (std::nothrow) conv_group();
    if (!g) {
        fail(CONV_E_NOMEM, "out of host memory");
        return nullptr;
    }
    if (create_impl(g, precision, block, n_in, n_out, taps, sessions, tiling) != CONV_OK) {
        const std::string msg = conv_last_error();
        group_free(g);
        set_last_error_message(msg.c_str());
        return nullptr;
    }
    set_last_error_message("");
    return g;
}

int conv_group_set_filters(conv_group* g, const float* h) {
    if (!g || !h) return fail(CONV_E_INVAL, "null argument");
    DeviceGuard d(g->dev);
    const GroupPlan& p = g->plan;
    const size_t bytes = (size_t)g->n_out * g->n_in * (size_t)g->taps * sizeof(float);
    const size_t mbytes = (size_t)g->B * g->n_out * sizeof(unsigned);
    float* d_h = nullptr;
    unsigned* d_max = nullptr;
    int rc;
    if ((rc = galloc(g, &d_h, bytes))) return rc;
    if ((rc = galloc(g, &d_max, mbytes))) {
        cudaFree(d_h);
        g->dev_bytes -= bytes;
        return rc;
    }
    cudaError_t r = cudaMemcpyAsync(d_h, h, bytes, cudaMemcpyHostToDevice, g->stream);
    if (r == cudaSuccess) r = cudaMemsetAsync(d_max, 0, mbytes, g->stream);
    if (r == cudaSuccess) r = cudaMemsetAsync(g->H, 0, p.h_bytes, g->stream);
    GroupFilterArgs a{};
    a.h = d_h;
    a.taps = g->taps;
    a.n_dst = g->n_out;
    a.n_src = g->n_in;
    a.K = p.K;
    a.B = g->B;
    a.log2B = g->log2B;
    a.G = p.G;
    a.KP = p.KP;
    a.NKS = p.NKS;
    a.maxbits = d_max;
    a.sH = g->sH;
    a.H = g->H;
    a.tw = g->tw;
    const int prec = to_prec(g->prec);
    for (int pass = 0; pass < 2 && r == cudaSuccess; ++pass) {
        a.pass = pass;
        r = launch_group_filter(prec, a, g->stream);
    }
    if (r == cudaSuccess) r = cudaStreamSynchronize(g->stream);
    cudaFree(d_h);
    cudaFree(d_max);
    g->dev_bytes -= bytes + mbytes;
    if (r != cudaSuccess) return fail(CONV_E_CUDA, "group filter tiles: %s", cudaGetErrorString(r));
    g->ready = true;
    return group_reset_impl(g);
}

int conv_group_process_async(conv_group* g, const float* d_in, float* d_out, void* cuda_stream) {
    if (!g || !d_in || !d_out) return fail(CONV_E_INVAL, "null argument");
    if (!g->ready) return fail(CONV_E_STATE, "filters not set");
    DeviceGuard d(g->dev);
    return enqueue_group(g, d_in, d_out, static_cast<cudaStream_t>(cuda_stream));
}

int conv_group_process(conv_group* g, const float* in, float* out) {
    if (!g || !in || !out) return fail(CONV_E_INVAL, "null argument");
    if (!g->ready) return fail(CONV_E_STATE, "filters not set");
    DeviceGuard d(g->dev);
    const size_t ib = (size_t)g->S * g->n_in * g->B * sizeof(float);
    const size_t ob = (size_t)g->S * g->n_out * g->B * sizeof(float);
    std::memcpy(g->h_in, in, ib);
    // blocks in and out through mapped pinned host memory: no copy launches per block
    int rc = enqueue_group(g, g->m_in, g->m_out, g->stream);
    if (rc) return rc;
    GB_CK(cudaEventRecord(g->ev_done, g->stream));
    GB_CK(cudaEventSynchronize(g->ev_done));  // the next block's tail keeps running
    if ((rc = check_err(g))) return rc;
    std::memcpy(out, g->h_out, ob);
    return CONV_OK;
}

int conv_group_process_blocks(conv_group* g, const float* in, float* out, long long n_blocks) {
    if (!g || !in || !out) return fail(CONV_E_INVAL, "null argument");
    if (n_blocks < 1) return fail(CONV_E_INVAL, "n_blocks must be >= 1");
    if (!g->ready) return fail(CONV_E_STATE, "filters not set");
    DeviceGuard d(g->dev);
    const long long C = std::min<long long>(n_blocks, 256);  // blocks per chunk
    const size_t rows_in = (size_t)g->S * g->n_in, rows_out = (size_t)g->S * g->n_out, fs = sizeof(float);
    int rc = CONV_OK;
    if (C > g->chunk_cap) {
        if ((rc = sync_all(g))) return rc;
        for (float** p : {&g->d_cin, &g->d_cout})
            if (*p) {
                cudaFree(*p);
                *p = nullptr;
            }
        g->dev_bytes -= (rows_in + rows_out) * (size_t)g->chunk_cap * g->B * fs;
        g->chunk_cap = 0;
        if ((rc = galloc(g, &g->d_cin, rows_in * (size_t)C * g->B * fs))) return rc;
        if ((rc = galloc(g, &g->d_cout, rows_out * (size_t)C * g->B * fs))) return rc;
        g->chunk_cap = C;
    }
    const size_t T = (size_t)n_blocks * g->B;
    for (long long b0 = 0; b0 < n_blocks; b0 += C) {
        const long long nb = std::min(C, n_blocks - b0);
        const size_t w = (size_t)nb * g->B;
        GB_CK(cudaMemcpy2DAsync(g->d_cin, (size_t)C * g->B * fs, in + (size_t)b0 * g->B, T * fs, w * fs, rows_in,
                              cudaMemcpyHostToDevice, g->stream));
        g->io_stride = (int)(C * g->B);
        for (long long b = 0; b < nb && !rc; ++b)
            rc = enqueue_group(g, g->d_cin + (size_t)b * g->B, g->d_cout + (size_t)b * g->B, g->stream);
        g->io_stride = 0;
        if (rc) return rc;
        GB_CK(cudaMemcpy2DAsync(out + (size_t)b0 * g->B, T * fs, g->d_cout, (size_t)C * g->B * fs, w * fs, rows_out,
                              cudaMemcpyDeviceToHost, g->stream));
    }
    GB_CK(cudaEventRecord(g->ev_done, g->stream));
    GB_CK(cudaEventSynchronize(g->ev_done));
    return check_err(g);
}

int conv_group_reset(conv_group* g) {
    if (!g) return fail(CONV_E_INVAL, "null handle");
    DeviceGuard d(g->dev);
    return group_reset_impl(g);
}

int conv_group_join_async(conv_group* g, void* cuda_stream) {
    if (!g) return fail(CONV_E_INVAL, "null handle");
    DeviceGuard d(g->dev);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the latest tail of each parity (with one tail stream both name its latest tails)
    GB_CK(cudaStreamWaitEvent(s, g->ev_tail[0], 0));
    GB_CK(cudaStreamWaitEvent(s, g->ev_tail[1], 0));
    return CONV_OK;
}

int conv_group_synchronize(conv_group* g) {
    if (!g) return fail(CONV_E_INVAL, "null handle");
    DeviceGuard d(g->dev);
    int rc;
    if ((rc = sync_all(g))) return rc;
    GB_CK(cudaDeviceSynchronize());
    return check_err(g);
}

int conv_group_get_info(const conv_group* g, conv_group_info* out) {
    if (!g || !out) return fail(CONV_E_INVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    const GroupPlan& p = g->plan;
    out->block = g->B;
    out->n_in = g->n_in;
    out->n_out = g->n_out;
    out->taps = g->taps;
    out->sessions = g->S;
    out->precision = g->prec;
    out->K = p.K;
    out->ring_slots = p.KR;
    out->bins_per_group = p.G;
    out->groups = p.NG;
    out->splits = p.SP;
    out->tail_ctas = p.C;
    out->acc_buffers = p.nbuf;
    out->k_steps = p.NKS;
    out->stage_k_steps = p.NK;
    out->stages = p.nstage;
    out->mac_ctas = p.C;
    out->mac_smem = p.smem;
    out->tmem_cols = p.tmem_cols;
    // tail launch: every filter tile and every delay-line slot of every
    // session of K-steps 1..NKS-1, read once
    out->mac_bytes = (long long)(g->n_out + g->S) * g->n_in * (long long)(p.KR - p.KP) * g->B * 4;
    out->device_bytes = (long long)g->dev_bytes;
    out->kernels_per_block = 3;
    out->tail_streams = p.tail_streams;
    return CONV_OK;
}

int conv_group_plan_check(int precision, int block, int n_in, int n_out, long long taps, int sessions, int num_sms,
                          const conv_group_tiling* tiling) {
    const int prec = to_prec(precision);
    if (prec < 0) return fail(CONV_E_INVAL, "unknown precision %d", precision);
    GroupPlan p{};
    if (const char* why = plan_group(prec, block, n_in, n_out, taps, sessions, num_sms, &p, from_api(tiling)))
        return fail(CONV_E_INVAL, "%s", why);
    if (const char* why = check_group_plan(p)) return fail(CONV_E_INVAL, "%s", why);
    return CONV_OK;
}

int conv_group_set_l2_keep(conv_group* g, long long bytes) {
    if (!g) return fail(CONV_E_INVAL, "null handle");
    if (bytes < 0) return fail(CONV_E_INVAL, "bytes must be >= 0");
    g->l2_keep = bytes;
    return CONV_OK;
}

int conv_group_profile_enable(conv_group* g, int enable) {
    if (!g) return fail(CONV_E_INVAL, "null handle");
    DeviceGuard d(g->dev);
    g->prof = enable > 0;
    if (g->prof) {
        const size_t want = enable > 1 ? (size_t)enable : 4096;
        while (g->ev0.size() < want) {
            cudaEvent_t a, b;
            GB_CK(cudaEventCreate(&a));
            GB_CK(cudaEventCreate(&b));
            g->ev0.push_back(a);
            g->ev1.push_back(b);
        }
    }
    g->ev_used = 0;
    return CONV_OK;
}

int conv_group_profile_read(conv_group* g, double* total_ms, long long* launches) {
    if (!g || !total_ms || !launches) return fail(CONV_E_INVAL, "null argument");
    DeviceGuard d(g->dev);
    int rc;
    if ((rc = sync_all(g))) return rc;
    double tot = 0.0;
    for (size_t i = 0; i < g->ev_used; ++i) {
        float ms = 0.0f;
        GB_CK(cudaEventElapsedTime(&ms, g->ev0[i], g->ev1[i]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = (long long)g->ev_used;
    g->ev_used = 0;
    return CONV_OK;
}

void conv_group_destroy(conv_group* g) { group_free(g); }

}  // extern "C"
