// noalloc.cu - an FDL MAC + output transform entry point that allocates nothing.
//
// For callers that must not allocate device memory: a real-time audio callback
// (an allocation can block for an unbounded time, which breaks the block
// deadline), code running while a host framework owns every device buffer, or
// a plugin that only receives pointers from its host.  They pass their own
// spectra and output buffer; the partition-split partials, which the regular
// engine keeps in a buffer it allocates, live here in a fixed file-scope
// device array instead, and the twiddle tables in a second one.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "conv.h"
#include "kernels.h"

using namespace gbconv;

namespace {

// Scratch for the split partials: [S][n_out][block] complex float.  Every GPU
// that loads this library holds these bytes until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = 2u << 20;  // 2 MiB
constexpr int NOALLOC_MAX_BLOCK = 256;
constexpr int NOALLOC_MAX_OUT = 16;
constexpr int NOALLOC_MAX_DEVICES = 64;
// twiddle tables W_2B^j, j < 2B, for B = 16, 32, 64, 128, 256, back to back
constexpr int NOALLOC_TW_ENTRIES = 2 * (16 + 32 + 64 + 128 + 256);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) float2 g_noalloc_tw[NOALLOC_TW_ENTRIES];
// DEVERR_* of a bounded wait that gave up, kept until conv_fdl_mac_noalloc_status
static __device__ __align__(16) int g_noalloc_err;

struct DeviceSlot {
    bool ready = false;
    float2* scratch = nullptr;  // device address of g_noalloc_scratch on this device
    float2* tw = nullptr;       // device address of g_noalloc_tw on this device
    int* err = nullptr;         // device address of g_noalloc_err on this device
};

std::mutex g_mu;
DeviceSlot g_dev[NOALLOC_MAX_DEVICES];

int fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[384];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "conv_fdl_mac_noalloc: %s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "conv_fdl_mac_noalloc: %s", msg);
    set_last_error_message(buf);
    return code;
}

int tw_offset(int B) {
    int off = 0;
    for (int b = 16; b < B; b <<= 1) off += 2 * b;
    return off;
}

// Once per device, with that device current: resolve the arrays' device
// addresses (host code only has stand-ins for them) and fill the twiddles.
int setup_device(int dev, DeviceSlot** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSlot& d = g_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(CONV_E_CUDA, "cudaGetSymbolAddress(scratch)", e);
        d.scratch = static_cast<float2*>(p);
        e = cudaGetSymbolAddress(&p, g_noalloc_tw);
        if (e != cudaSuccess) return fail(CONV_E_CUDA, "cudaGetSymbolAddress(twiddles)", e);
        d.tw = static_cast<float2*>(p);
        e = cudaGetSymbolAddress(&p, g_noalloc_err);
        if (e != cudaSuccess) return fail(CONV_E_CUDA, "cudaGetSymbolAddress(error word)", e);
        d.err = static_cast<int*>(p);
        float2 host[NOALLOC_TW_ENTRIES];
        const double pi = 3.14159265358979323846264338327950288;
        for (int B = 16; B <= NOALLOC_MAX_BLOCK; B <<= 1)
            for (int j = 0; j < 2 * B; ++j) {
                const double ang = -pi * (double)j / (double)B;
                host[tw_offset(B) + j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            }
        e = cudaMemcpyToSymbol(g_noalloc_tw, host, sizeof(host));
        if (e != cudaSuccess) return fail(CONV_E_CUDA, "twiddle upload", e);
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_noalloc_err, &zero, sizeof(zero));
        if (e != cudaSuccess) return fail(CONV_E_CUDA, "error word", e);
        e = prepare_kernels(MAC_SMEM_LIMIT);
        if (e != cudaSuccess) return fail(CONV_E_CUDA, "kernel attributes", e);
        d.ready = true;
    }
    *out = &d;
    return CONV_OK;
}

}  // namespace

extern "C" int conv_fdl_mac_noalloc(const float* d_H, const float* d_X, int block, int n_in, int n_out, long long K,
                                    long long slot0, float* d_y, void* cuda_stream) {
    if (!d_H || !d_X || !d_y) return fail(CONV_E_INVAL, "null pointer");
    // the MAC streams d_H and d_X with bulk copies, which need 16-byte aligned sources
    if (((uintptr_t)d_H | (uintptr_t)d_X) & 15u) return fail(CONV_E_INVAL, "d_H and d_X must be 16-byte aligned");
    if ((uintptr_t)d_y & 3u) return fail(CONV_E_INVAL, "d_y must be 4-byte aligned");
    if (block < 16 || block > NOALLOC_MAX_BLOCK || (block & (block - 1)))
        return fail(CONV_E_INVAL, "block must be a power of two in [16, 256]");
    if (n_out < 1 || n_out > NOALLOC_MAX_OUT) return fail(CONV_E_INVAL, "n_out must be in [1, 16]");
    if (n_in < 1 || K < 1 || (long long)n_in * K > (1ll << 30)) return fail(CONV_E_INVAL, "n_in * K out of range");
    if (slot0 < 0 || slot0 >= K) return fail(CONV_E_INVAL, "slot0 must be in [0, K)");
    const size_t row = (size_t)n_out * block * sizeof(float2);
    if (row > NOALLOC_SCRATCH_BYTES) return fail(CONV_E_INVAL, "one partial row exceeds the 2 MiB scratch");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(CONV_E_INVAL, "device index above 63");
    DeviceSlot* d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc) return rc;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "SM count", e);

    // One tile covering every bin and every output: the engine's tiled filter
    // layout then reduces to H[p][q][l][k], and its ring to X[slot][q][k].
    MacPlan p{};
    p.B = block;
    p.n_src = n_in;
    p.n_dst = n_out;
    p.K = (int)K;
    p.R = n_in * (int)K;
    p.r_begin = 0;
    p.es = 8;
    p.VEC = 2;
    p.LPT = 8;
    p.BT = block;
    p.n_kt = 1;
    p.LT = n_out;
    p.n_lt = 1;
    p.nw = MAC_CONSUMER_WARPS;
    p.kthreads = block / 2;
    const int rest = (p.nw * 32) / p.kthreads;
    p.NLG = n_out > 8 ? 2 : 1;
    p.NRL = rest / p.NLG;
    const size_t per_r = (size_t)(p.LT + 1) * p.BT * p.es;
    int rs = (int)((32768 + per_r / 2) / per_r);
    if (rs < 1) rs = 1;
    rs = (rs + p.NRL - 1) / p.NRL * p.NRL;
    p.RS = rs < p.R ? rs : p.R;
    const size_t hpart = ((size_t)p.RS * p.LT * p.BT * p.es + 127) / 128 * 128;
    const size_t xpart = ((size_t)p.RS * p.BT * p.es + 127) / 128 * 128;
    p.xoff = (unsigned)hpart;
    p.stage_bytes = (unsigned)(hpart + xpart);
    size_t nst = (200 * 1024 - MAC_HDR_BYTES) / p.stage_bytes;
    p.nstage = (int)(nst < 2 ? 2 : (nst > MAX_STAGES ? MAX_STAGES : nst));
    const size_t red = (size_t)(p.NRL - 1) * p.LPT * p.NLG * p.BT * sizeof(float2);  // lane-major r-lane scratch
    const size_t ring = (size_t)p.nstage * p.stage_bytes;
    p.smem = MAC_HDR_BYTES + (ring > red ? ring : (red + 127) / 128 * 128);
    if (p.smem > 200 * 1024) return fail(CONV_E_INVAL, "tiling needs more shared memory than planned");
    const long long grid_stages = (p.R + p.RS - 1) / p.RS;  // stage grid from r = 0
    long long S = sms;
    const long long fit = (long long)(NOALLOC_SCRATCH_BYTES / row);
    if (S > fit) S = fit;
    if (S > grid_stages) S = grid_stages;
    if (S < 1) S = 1;
    p.S = (int)S;
    p.ctas = p.S;
    p.tile_elems = (size_t)n_out * p.R * block;  // one tile: the caller's layout, no padding
    p.h_bytes = (size_t)n_out * p.R * block * p.es;
    p.x_bytes = (size_t)p.R * block * p.es;
    p.partial_bytes = (size_t)p.S * row;

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    MacArgs a{};
    a.H = d_H;
    a.X = d_X;
    a.sH = nullptr;
    a.sX = nullptr;
    a.partial = d->scratch;
    a.B = block;
    a.BT = p.BT;
    a.n_kt = 1;
    a.n_dst = n_out;
    a.LT = p.LT;
    a.n_lt = 1;
    a.n_src = n_in;
    a.K = p.K;
    a.S = p.S;
    a.RS = p.RS;
    a.nstage = p.nstage;
    a.kthreads = p.kthreads;
    a.NLG = p.NLG;
    a.NRL = p.NRL;
    a.r_begin = 0;
    a.slot0 = (int)slot0;
    a.stage_bytes = p.stage_bytes;
    a.xoff = p.xoff;
    a.tile_elems = p.tile_elems;
    a.err = d->err;
    // no early start: the caller's previous kernel may be writing d_H
    e = launch_fdl_mac(PREC_FP32, p, a, s, false);
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "MAC launch", e);

    int log2B = 0;
    while ((1 << log2B) < block) ++log2B;
    OutArgs r{};
    r.partial = d->scratch;
    r.S = p.S;
    r.n_dst = n_out;
    r.B = block;
    r.log2B = log2B;
    r.tw = d->tw + tw_offset(block);
    r.out = d_y;
    r.out_stride = block;
    r.head = 0;
    e = launch_out_c2r(PREC_FP32, r, s);
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "output-transform launch", e);
    return CONV_OK;
}

extern "C" int conv_fdl_mac_noalloc_status(void* cuda_stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(CONV_E_INVAL, "device index above 63");
    DeviceSlot* d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "stream synchronize", e);
    int v = 0;
    e = cudaMemcpy(&v, d->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "error word read", e);
    if (v == DEVERR_NONE) return CONV_OK;
    e = cudaMemset(d->err, 0, sizeof(int));
    if (e != cudaSuccess) return fail(CONV_E_CUDA, "error word clear", e);
    char buf[160];
    snprintf(buf, sizeof(buf), "conv_fdl_mac_noalloc: a device-side wait gave up (code %d); that call's output is invalid", v);
    set_last_error_message(buf);
    return CONV_E_TIMEOUT;
}
