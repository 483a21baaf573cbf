// tcgen05 (sm_103a tensor-core) layer kernels.  Placeholder until the
// tensor-core path lands: reports the tensor-core precisions as unsupported.
#include "common.cuh"
#include "kernels.h"

namespace slista {

__device__ int g_device_flag = 0;

int read_and_clear_device_flag(cudaStream_t st)
{
    int h = 0;
    SLISTA_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_device_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        SLISTA_CUDA_TRY(cudaMemcpyToSymbolAsync(g_device_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
        return fail(SLISTA_ERR_TIMEOUT, "a kernel's bounded wait expired (device flag %d)", h);
    }
    return SLISTA_OK;
}

namespace tc {
bool supported(int) { return false; }
size_t forward_ws_bytes(int) { return 0; }
int launch_forward(const PgdArgs &, int, void *, cudaStream_t)
{
    return fail(SLISTA_ERR_UNSUPPORTED, "tensor-core path not built");
}
}  // namespace tc
}  // namespace slista
