// noalloc.cu -- energy evaluation that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: a serving loop that owns the
// whole device-memory budget through its own pool, or a latency-critical path where
// an allocation (which may synchronise the device or fail under fragmentation) is
// not allowed.  sg_energy_noalloc serves them: the caller passes device inputs and a
// device output, and every piece of scratch the computation needs comes from one
// fixed array declared below, which every GPU that loads this library keeps until
// the process exits.
#include <mutex>

#include "sg_internal.h"

namespace sg {
namespace {

// The scratch.  Host code must not take this name as a device address: its device
// address comes from cudaGetSymbolAddress with the device current (scratch_on_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The first call on a device
// is the set-up: the lookup (which also loads this library's device code there) and the
// cache entry.  Later calls repeat the lookup, which is cheap once the code is loaded, and
// refresh the entry if the address moved -- after cudaDeviceReset, or under another
// context -- so a stale address is never handed to a kernel.
int32_t scratch_on_device(unsigned char** out)
{
    int dev = 0;
    SG_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return SG_EINVAL;
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    *out = g_scratch_ptr[dev];
    return SG_OK;
}

// Stores the coupling-record pointer the energy kernel reads from device memory
// (a kernel argument, so no host buffer is involved).
__global__ void store_pointer(const uint2** slot, const uint2* value) { *slot = value; }

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" int32_t sg_energy_noalloc(int32_t L, const int8_t* J3_dev, const int8_t* spins_dev,
                                     int32_t n_configs, int64_t* E_dev, void* stream)
{
    clear_error();
    if (!J3_dev || !spins_dev || !E_dev || n_configs < 1 || L < 2 || L > SG_LMAX || (L & 1)) {
        set_error("sg_energy_noalloc: bad arguments (L even in [2, %d], n_configs >= 1, "
                  "non-NULL device pointers)", SG_LMAX);
        return SG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)L * L * L;
    const int Wn = words_for(n_configs), Rp = 32 * Wn;
    // scratch layout: [E sums: 8 * Rp][status: 16][j6 pointer: 16][coupling records: 8 * N]
    //                 [sign bytes: N][packed spins: N * Wn 32-bit words]
    const size_t off_E = 0;
    const size_t off_bad = round_up(off_E + 8 * (size_t)Rp, 256);
    const size_t off_ptr = off_bad + 16;
    const size_t off_j6 = round_up(off_ptr + 16, 256);
    const size_t off_j1 = round_up(off_j6 + 8 * N, 256);
    const size_t off_sp = round_up(off_j1 + N, 256);
    const size_t need = off_sp + N * (size_t)Wn * 4;
    if (need > (size_t)SG_NOALLOC_SCRATCH_BYTES) {
        set_error("sg_energy_noalloc: L=%d with %d configurations needs %zu bytes of scratch, "
                  "more than the fixed %u", L, n_configs, need, (unsigned)SG_NOALLOC_SCRATCH_BYTES);
        return SG_EINVAL;
    }
    unsigned char* base = nullptr;
    int32_t rc = scratch_on_device(&base);
    if (rc != SG_OK) return rc;
    unsigned long long* E64 = reinterpret_cast<unsigned long long*>(base + off_E);
    int* bad = reinterpret_cast<int*>(base + off_bad);
    const uint2** j6_ptr = reinterpret_cast<const uint2**>(base + off_ptr);
    uint2* j6 = reinterpret_cast<uint2*>(base + off_j6);
    uint8_t* j1 = base + off_j1;
    int8_t* packed = reinterpret_cast<int8_t*>(base + off_sp);

    // the array keeps the previous call's contents: clear the sums and the status word
    SG_TRY_CUDA(cudaMemsetAsync(E64, 0, 8 * (size_t)Rp, st));
    SG_TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    store_pointer<<<1, 1, 0, st>>>(j6_ptr, j6);
    SG_TRY_CUDA(cudaGetLastError());
    rc = launch_prepare_j6(J3_dev, j6, j1, L, st);
    if (rc != SG_OK) return rc;
    rc = launch_pack_spins(spins_dev, packed, L, Rp, n_configs, bad, st);
    if (rc != SG_OK) return rc;
    rc = launch_energy(packed, j6_ptr, 1, L, Wn, E64, st);
    if (rc != SG_OK) return rc;
    rc = launch_copy_energies(E64, E_dev, n_configs, st);
    if (rc != SG_OK) return rc;
    int hbad = 0;
    SG_TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaStreamSynchronize(st));
    if (hbad) {
        set_error("%d spin values are not -1 or +1", hbad);
        return SG_EINVAL;
    }
    return SG_OK;
}
