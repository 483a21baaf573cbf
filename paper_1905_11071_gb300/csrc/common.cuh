// Internal helpers shared by the library's translation units: status
// reporting, argument checks and launch utilities.  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>

#include "../../include/slista.h"

namespace slista {

// Last-error message of the calling host thread (slista_last_error()).
void set_error(const char *fmt, ...);
void clear_error();

// Records `code` with a formatted message and returns it.
int fail(int code, const char *fmt, ...);

// Maps the pending CUDA error (if any) of the last launch to SLISTA_ERR_CUDA.
int check_launch(const char *what);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Pads the code length m to the multiple of 32 the SIMT kernels are built for.
inline int pad32(int m) { return ((m + 31) / 32) * 32; }

// Number of streaming multiprocessors of the current device (cached).
int num_sms();

// Whether `kernel` was already opted in to `bytes` of dynamic shared memory
// on the current device (smem_known), and the record of an opt-in.
bool smem_known(const void *kernel, size_t bytes);
void smem_record(const void *kernel, size_t bytes);

// Dynamic shared memory opt-in for a kernel.  Done once per kernel and
// device, so that calls made later under stream capture issue no attribute
// change.
template <class K>
inline cudaError_t allow_smem(K kernel, size_t bytes)
{
    const void *fn = reinterpret_cast<const void *>(kernel);
    if (smem_known(fn, bytes)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) smem_record(fn, bytes);
    return e;
}

}  // namespace slista

// Argument-check helpers: return from the calling entry point on failure.
#define SLISTA_REQUIRE(cond, code, ...)                           \
    do {                                                          \
        if (!(cond)) return ::slista::fail((code), __VA_ARGS__);  \
    } while (0)

#define SLISTA_CUDA_TRY(call)                                                        \
    do {                                                                             \
        cudaError_t _e = (call);                                                     \
        if (_e != cudaSuccess)                                                       \
            return ::slista::fail(SLISTA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
    } while (0)
