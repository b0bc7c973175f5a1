// rate.cu -- the generator's own throughput on this device (sg_philox_rate): how many
// Philox4x32-10 blocks per second the SMs produce when drawing is all they do.  The
// Metropolis draws of one word of 32 replicas take two blocks (App. D.1 / D.2 sweeps),
// so 16 times this rate bounds the attempt rate of the sweeps' integer work: the
// measured counterpart of the multiply-pipe roof.
#include <stdint.h>

#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr uint32_t kRateDomain = 7;  // a counter domain no draw of the method uses

// Two independent blocks per step, as a sweep thread draws its planes.  The XOR of all
// outputs is stored only when it equals one fixed word, so the work cannot be dropped
// and practically nothing is written.
__global__ void __launch_bounds__(256) philox_rate_kernel(uint32_t n, uint32_t k0, uint32_t k1, uint32_t* sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint32_t c = 0; c < n; c += 2) {
        const Philox4 a = philox4x32_10(t, c, 0u, kRateDomain, k0, k1);
        const Philox4 b = philox4x32_10(t, c + 1u, 0u, kRateDomain, k0, k1);
        acc ^= a.v[0] ^ a.v[1] ^ a.v[2] ^ a.v[3] ^ b.v[0] ^ b.v[1] ^ b.v[2] ^ b.v[3];
    }
    if (acc == 0x9E3779B9u) sink[t] = acc;
}

}  // namespace
}  // namespace sg

extern "C" int32_t sg_philox_rate(int32_t blocks_per_thread, double* blocks_per_second, void* stream)
{
    using namespace sg;
    clear_error();
    if (!blocks_per_second || blocks_per_thread < 2 || (blocks_per_thread & 1)) {
        set_error("blocks_per_thread must be even and at least 2 (got %d), output non-NULL", blocks_per_thread);
        return SG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    SG_TRY_CUDA(cudaGetDevice(&dev));
    SG_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = 8 * sms;  // eight resident blocks per SM
    uint32_t* sink = nullptr;
    SG_TRY_CUDA(cudaMallocAsync(&sink, sizeof(uint32_t) * (size_t)threads * blocks, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int32_t rc = SG_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SG_ECUDA;
    if (rc == SG_OK) {
        philox_rate_kernel<<<blocks, threads, 0, st>>>(64u, 1u, 2u, sink);  // warm-up
        cudaEventRecord(e0, st);
        philox_rate_kernel<<<blocks, threads, 0, st>>>((uint32_t)blocks_per_thread, 1u, 2u, sink);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
            rc = SG_ECUDA;
    }
    if (rc != SG_OK) set_error("generator rate measurement failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (rc == SG_OK) *blocks_per_second = (double)threads * blocks * (double)blocks_per_thread / (ms * 1e-3);
    return rc;
}
