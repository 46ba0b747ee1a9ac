// host_util.h - host-side helpers shared by the C entry points: error
// reporting into conv_last_error(), CUDA-call checking, device scoping.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>

#include "conv.h"
#include "kernels.h"

namespace gbconv {

// Formats the calling thread's conv_last_error() message; returns `code`.
inline int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error_message(buf);
    return code;
}

// Makes `dev` the current device for the scope and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace gbconv

// Returns CONV_E_CUDA (with the call, the CUDA message and the source line) from
// the enclosing function when a CUDA runtime call fails.
#define GB_CK(call)                                                                                        \
    do {                                                                                                   \
        cudaError_t gb_e_ = (call);                                                                        \
        if (gb_e_ != cudaSuccess)                                                                          \
            return ::gbconv::fail(CONV_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(gb_e_), __FILE__, \
                                  __LINE__);                                                               \
    } while (0)
