// kernels.cu -- device kernels of the Metropolis path (sm_103a) other than the sweep itself
// (sweep.cu): couplings, initial spins, energies (Eq. 1), PT bookkeeping, layout changes.
//
// Device layout.  Spins of a run are bit-packed: [I][N][Wn] 32-bit words -- instance,
// site in storage order (see storage_of: colour-split rows), word -- with Wn =
// ceil(R / 32); bit b of word w is replica 32w + b, a set bit meaning spin -1.  Padding
// replicas (32w + b >= R) stay +1 and never flip.  Couplings of a site are one 8-byte
// record: byte q holds the int8 coupling to the neighbour in direction q (+x, -x, +y,
// -y, +z, -z); a second byte per site holds their sign bits (read when every |J| = 1).
#include <stdio.h>

#include <algorithm>

#include "exchange.cuh"
#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------------- couplings

__global__ void prepare_j6_kernel(const int8_t* __restrict__ J3, uint2* __restrict__ j6,
                                  uint8_t* __restrict__ j1, int L)
{
    const int64_t N = (int64_t)L * L * L;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((int64_t)L * L));
        const int64_t LL = (int64_t)L * L;
        const int64_t bx = (x == 0 ? L - 1 : x - 1) + (int64_t)L * y + LL * z;
        const int64_t by = x + (int64_t)L * (y == 0 ? L - 1 : y - 1) + LL * z;
        const int64_t bz = x + (int64_t)L * y + LL * (z == 0 ? L - 1 : z - 1);
        const uint32_t b0 = (uint8_t)J3[3 * i + 0], b1 = (uint8_t)J3[3 * bx + 0];
        const uint32_t b2 = (uint8_t)J3[3 * i + 1], b3 = (uint8_t)J3[3 * by + 1];
        const uint32_t b4 = (uint8_t)J3[3 * i + 2], b5 = (uint8_t)J3[3 * bz + 2];
        j6[i] = make_uint2(b0 | (b1 << 8) | (b2 << 16) | (b3 << 24), b4 | (b5 << 8));
        // bit q: coupling q is negative (used only when every coupling is +-1)
        j1[i] = (uint8_t)((b0 >> 7) | ((b1 >> 7) << 1) | ((b2 >> 7) << 2) | ((b3 >> 7) << 3) |
                          ((b4 >> 7) << 4) | ((b5 >> 7) << 5));
    }
}

// ---------------------------------------------------------------- initial state

// Replica r of site i starts at -1 when bit 31 of word r % 4 of
// Philox(i, kSweepInit, r / 4, 0) is set: eight calls fill one 32-replica word.
__global__ void init_spins_kernel(uint32_t* __restrict__ spins, const RunKeys* __restrict__ keys,
                                  int L, int Wn, int R)
{
    const int inst = blockIdx.y;
    const RunKeys key = keys[inst];
    const int64_t N = (int64_t)L * L * L;
    const int64_t items = N * Wn;
    uint32_t* s = spins + (int64_t)inst * items;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(t % Wn);
        const int64_t i = logical_of(L, t / Wn);
        uint32_t word = 0;
        for (int q = 0; q < 8; ++q) {
            if (32 * w + 4 * q >= R) break;
            const Philox4 r = philox4x32_10((uint32_t)i, kSweepInit, (uint32_t)(8 * w + q), kDomainMetropolis,
                                            key.k0, key.k1);
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (32 * w + 4 * q + m < R && (r.v[m] >> 31)) word |= 1u << (4 * q + m);
        }
        s[t] = word;
    }
}

// ---------------------------------------------------------------- energy (Eq. 1)

// H = sum over edges of J_ij s_i s_j, every edge counted once as a forward bond (+x, +y,
// +z) of its lower site.  One warp per (row, word) item; lane b sums replica 32w + b
// along the row from broadcast loads of the row's words, and adds the row's total to
// E_out[inst][32w + b].
__global__ void __launch_bounds__(kBlock)
energy_bits_kernel(const uint32_t* __restrict__ spins, const uint2* const* __restrict__ j6_ptrs, int L, int Wn,
                   unsigned long long* __restrict__ E_out)
{
    const int inst = blockIdx.y;
    const int LL = L * L, H = L >> 1;
    const uint2* __restrict__ j6 = j6_ptrs[inst];
    const uint32_t* __restrict__ s = spins + (size_t)inst * (size_t)LL * L * Wn;
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const int64_t items = (int64_t)LL * Wn;
    unsigned long long* Ei = E_out + (size_t)inst * 32 * Wn;
    for (int64_t t = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); t < items; t += (int64_t)gridDim.x * warps) {
        const int r = (int)(t / Wn), w = (int)(t % Wn);
        const int z = r / L, y = r - z * L;
        const int ryp = z * L + (y + 1 == L ? 0 : y + 1);
        const int rzp = (z + 1 == L ? 0 : z + 1) * L + y;
        const uint32_t* __restrict__ row = s + (size_t)r * L * Wn + w;
        const uint32_t* __restrict__ rowy = s + (size_t)ryp * L * Wn + w;
        const uint32_t* __restrict__ rowz = s + (size_t)rzp * L * Wn + w;
        long long e = 0;
        for (int x = 0; x < L; ++x) {
            const int pos = (x & 1) * H + (x >> 1);
            const int xp = x + 1 == L ? 0 : x + 1;
            const int posx = (xp & 1) * H + (xp >> 1);
            const uint2 rec = j6[r * L + x];
            const int J[3] = {(int)(int8_t)(rec.x & 0xFFu), (int)(int8_t)((rec.x >> 16) & 0xFFu),
                              (int)(int8_t)(rec.y & 0xFFu)};
            const uint32_t me = row[(size_t)pos * Wn];
            const uint32_t nb[3] = {row[(size_t)posx * Wn], rowy[(size_t)pos * Wn], rowz[(size_t)pos * Wn]};
#pragma unroll
            for (int d = 0; d < 3; ++d) e += J[d] * (1 - 2 * (int)(((me ^ nb[d]) >> lane) & 1u));
        }
        if (e) atomicAdd(&Ei[32 * w + lane], (unsigned long long)e);
    }
}

// All |J| = 1: H = 3N - 2 * (satisfied forward bonds), a bond being satisfied when its
// term J s_i s_j is -1.  Each warp takes one word w and each of its threads a set of
// sites; a thread adds the bit-sliced count (0..3) of its sites' satisfied forward bonds
// into vertical counters, and the warp reduces them through a 32 x 32 bit transpose.
constexpr int kEBits = 24;  // counter planes: up to 2^24 - 1 per thread

__global__ void __launch_bounds__(kBlock)
energy_unit_kernel(const uint32_t* __restrict__ spins, const uint8_t* const* __restrict__ j1_ptrs, int L, int Wn,
                   unsigned long long* __restrict__ E_out)
{
    const int inst = blockIdx.y;
    const int64_t N = (int64_t)L * L * L;
    const int H = L >> 1;
    const uint8_t* __restrict__ j1 = j1_ptrs[inst];
    const uint32_t* __restrict__ s = spins + (size_t)inst * (size_t)N * Wn;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // warp index in the instance's grid
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int wpw = nw / Wn;  // warps per word
    if (gw >= wpw * Wn) return;  // whole warps only
    const int w = gw % Wn;
    const int64_t chunk = (int64_t)(gw / Wn) * 32 + lane, nchunks = (int64_t)wpw * 32;
    uint32_t V[kEBits];
#pragma unroll
    for (int k = 0; k < kEBits; ++k) V[k] = 0;
    int64_t nsites = 0;
    for (int64_t is = chunk; is < N; is += nchunks) {  // storage position
        const int row = (int)(is / L), pos = (int)(is - (int64_t)row * L);
        const int z = row / L, y = row - z * L;
        const int par = pos >= H ? 1 : 0, j = pos - par * H, x = 2 * j + par;
        const int xp = x + 1 == L ? 0 : x + 1;
        const int posx = (xp & 1) * H + (xp >> 1);
        const int rowy = z * L + (y + 1 == L ? 0 : y + 1), rowz = (z + 1 == L ? 0 : z + 1) * L + y;
        const uint32_t me = s[is * Wn + w];
        const uint32_t nx = s[((int64_t)row * L + posx) * Wn + w];
        const uint32_t ny = s[((int64_t)rowy * L + pos) * Wn + w];
        const uint32_t nz = s[((int64_t)rowz * L + pos) * Wn + w];
        const uint32_t sb = j1[(int64_t)row * L + x];
        // satisfied: the spins differ under J > 0, agree under J < 0 (bits 0, 2, 4: +x, +y, +z)
        const uint32_t a = me ^ nx ^ (0u - (sb & 1u));
        const uint32_t b = me ^ ny ^ (0u - ((sb >> 2) & 1u));
        const uint32_t c = me ^ nz ^ (0u - ((sb >> 4) & 1u));
        const uint32_t c0 = a ^ b ^ c, c1 = mp::maj3(a, b, c);  // the count: planes of weight 1, 2
        // V += (c1 c0), the carry rippled up until it is gone
        uint32_t carry = V[0] & c0;
        V[0] ^= c0;
        {
            const uint32_t t = V[1] ^ c1 ^ carry;
            carry = mp::maj3(V[1], c1, carry);
            V[1] = t;
        }
#pragma unroll
        for (int k = 2; k < kEBits; ++k) {
            if (!carry) break;
            const uint32_t t = V[k] & carry;
            V[k] ^= carry;
            carry = t;
        }
        ++nsites;
    }
    // lane r of the transposed planes holds replica r of every lane's counter
    uint32_t T[kEBits];
#pragma unroll
    for (int k = 0; k < kEBits; ++k) T[k] = mp::warp_transpose(V[k], lane);
    long long sat = 0;
#pragma unroll
    for (int k = 0; k < kEBits; ++k) sat += (long long)__popc(T[k]) << k;
    long long sites = nsites;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sites += __shfl_xor_sync(0xFFFFFFFFu, sites, o);
    const long long e = 3 * sites - 2 * sat;
    if (e) atomicAdd(&E_out[(size_t)inst * 32 * Wn + 32 * w + lane], (unsigned long long)e);
}

// ---------------------------------------------------------------- parallel tempering

__global__ void pt_setup_kernel(const unsigned long long* __restrict__ E64, int32_t* __restrict__ E,
                                uint8_t* __restrict__ rung_of_slot, uint8_t* __restrict__ slot_of_rung,
                                unsigned long long* __restrict__ accepts, int32_t* __restrict__ minE,
                                int Rp, int K)
{
    const int inst = blockIdx.x;
    __shared__ int32_t s_min;
    if (threadIdx.x == 0) s_min = 0x7FFFFFFF;
    __syncthreads();
    for (int r = threadIdx.x; r < Rp; r += blockDim.x) {
        const int32_t e = (int32_t)(long long)E64[(int64_t)inst * Rp + r];
        E[(int64_t)inst * Rp + r] = e;
        rung_of_slot[(int64_t)inst * Rp + r] = (uint8_t)(r < K ? r : 0);
        if (r < K) {
            slot_of_rung[(int64_t)inst * K + r] = (uint8_t)r;
            atomicMin(&s_min, e);
        }
        if (r + 1 < K) accepts[(int64_t)inst * (K - 1) + r] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) minE[inst] = s_min;
}

// Exchange attempts after sweep `sweep` (see exchange.cuh), one block per instance.
__global__ void pt_exchange_kernel(const ExchangeArgs x, uint32_t sweep)
{
    __shared__ int32_t s_min;
    const uint32_t s = sweep + (x.sweep_base ? *x.sweep_base : 0u);
    pt_exchange_block(x, blockIdx.x, s, threadIdx.x, blockDim.x, &s_min);
}

// ---------------------------------------------------------------- checks and layout

__global__ void narrow_energy_kernel(const unsigned long long* __restrict__ E64,
                                     int32_t* __restrict__ E, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        E[q] = (int32_t)(long long)E64[q];
}

__global__ void check_energy_kernel(const unsigned long long* __restrict__ E64,
                                    const int32_t* __restrict__ E, int Rp, int R, int I,
                                    int* __restrict__ mismatch)
{
    const int64_t n = (int64_t)I * Rp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q % Rp);
        if (r < R && (long long)E64[q] != (long long)E[q]) atomicAdd(mismatch, 1);
    }
}

__global__ void unpack_spins_kernel(const uint32_t* __restrict__ words, int8_t* __restrict__ out, int L, int Wn,
                                    int R)
{
    const int64_t N = (int64_t)L * L * L;
    const int64_t n = (int64_t)R * N;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / N);
        const int64_t i = q % N;
        const uint32_t word = words[storage_of(L, i) * Wn + (r >> 5)];
        out[q] = ((word >> (r & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

// in: [R][N] int8 spins of +-1 in logical site order; words: [N][Wn] packed (padding
// replicas +1).  Values other than +-1 are counted in *bad and stored as +1.
__global__ void pack_spins_kernel(const int8_t* __restrict__ in, uint32_t* __restrict__ words, int L, int Wn,
                                  int R, int* __restrict__ bad)
{
    const int64_t N = (int64_t)L * L * L;
    const int64_t n = (int64_t)Wn * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = logical_of(L, t / Wn);
        const int w = (int)(t % Wn);
        uint32_t word = 0;
        int nbad = 0;
        for (int b = 0; b < 32; ++b) {
            const int r = 32 * w + b;
            if (r >= R) break;
            const int8_t v = in[(int64_t)r * N + i];
            if (v == -1) word |= 1u << b;
            else if (v != 1) ++nbad;
        }
        if (nbad) atomicAdd(bad, nbad);
        words[t] = word;
    }
}

int grid_for(int64_t items, int multiple_of = 1, int cap = 1 << 20)
{
    int64_t b = (items + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    b = (b + multiple_of - 1) / multiple_of * multiple_of;
    return (int)b;
}

int32_t check_launch(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s launch failed: %s", what, cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace

int32_t launch_prepare_j6(const int8_t* J3_dev, uint2* j6_dev, uint8_t* j1_dev, int L,
                          cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    prepare_j6_kernel<<<grid_for(N, 1, 4096), kBlock, 0, st>>>(J3_dev, j6_dev, j1_dev, L);
    return check_launch("prepare_j6");
}

int32_t launch_init_spins(int8_t* spins, const RunKeys* keys_dev, int I, int L, int Wn, int R,
                          cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    dim3 grid(grid_for(N * Wn, 1, 8192), I);
    init_spins_kernel<<<grid, kBlock, 0, st>>>((uint32_t*)spins, keys_dev, L, Wn, R);
    return check_launch("init_spins");
}

int32_t launch_energy(const int8_t* spins, const uint2* const* j6_ptrs, int I, int L, int Wn,
                      unsigned long long* E_out, cudaStream_t st, const uint8_t* const* j1_ptrs)
{
    if (j1_ptrs) {  // all |J| = 1: the bit-sliced kernel, at least two warps per word
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t N = (int64_t)L * L * L;
        const int64_t want_warps = std::max<int64_t>(2 * Wn, (8LL * sms * (kBlock / 32) + I - 1) / I);
        const int64_t max_warps = std::max<int64_t>(Wn, (N * Wn + 31) / 32);  // a site per lane at most
        const int64_t warps = (std::min(want_warps, max_warps) + Wn - 1) / Wn * Wn;  // a multiple of Wn
        const int gx = (int)std::min<int64_t>((warps * 32 + kBlock - 1) / kBlock, 1 << 20);
        energy_unit_kernel<<<dim3(gx, I), kBlock, 0, st>>>((const uint32_t*)spins, j1_ptrs, L, Wn, E_out);
        return check_launch("energy_unit");
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t items = (int64_t)L * L * Wn;
    const int64_t want = (8LL * sms + I - 1) / I;  // about eight blocks per SM over all instances
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((items + 7) / 8, want));
    dim3 grid(gx, I);
    energy_bits_kernel<<<grid, kBlock, 0, st>>>((const uint32_t*)spins, j6_ptrs, L, Wn, E_out);
    return check_launch("energy");
}

int32_t launch_half_sweep_sa(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_row, int32_t* /*E*/, int* status, bool unit_j, int I,
                             int L, int Wn, int R, uint32_t sweep, int colour, cudaStream_t st)
{
    return launch_sweep_rows_sa(spins, j6_ptrs, j1_ptrs, keys, thr_row, unit_j, I, L, Wn, R, sweep, colour, st,
                                nullptr, status);
}

int32_t launch_half_sweep_pt(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_rungs, const uint8_t* rung_of_slot, int32_t* E,
                             int* status, bool unit_j, int I, int L, int Wn, int K, uint32_t sweep,
                             int colour, const ExchangeArgs* xch, unsigned* done, bool* fused,
                             cudaStream_t st)
{
    if (fused) *fused = false;
    return launch_sweep_rows_pt(spins, j6_ptrs, j1_ptrs, keys, thr_rungs, rung_of_slot, E, unit_j, I, L, Wn, K,
                                sweep, colour, xch, done, fused, st, nullptr, status);
}

int32_t launch_pt_setup(const unsigned long long* E64, int32_t* E, uint8_t* rung_of_slot,
                        uint8_t* slot_of_rung, unsigned long long* accepts, int32_t* minE, int I,
                        int Rp, int K, cudaStream_t st)
{
    pt_setup_kernel<<<I, kBlock, 0, st>>>(E64, E, rung_of_slot, slot_of_rung, accepts, minE, Rp, K);
    return check_launch("pt_setup");
}

int32_t launch_pt_exchange(const ExchangeArgs& x, int I, uint32_t sweep, cudaStream_t st)
{
    pt_exchange_kernel<<<I, 128, 0, st>>>(x, sweep);
    return check_launch("pt_exchange");
}

int32_t launch_check_energy(const unsigned long long* E64, const int32_t* E, int I, int Rp, int R,
                            int* mismatch, cudaStream_t st)
{
    check_energy_kernel<<<grid_for((int64_t)I * Rp, 1, 1024), kBlock, 0, st>>>(E64, E, Rp, R, I,
                                                                                mismatch);
    return check_launch("check_energy");
}

namespace {
__global__ void copy_energies_kernel(const unsigned long long* __restrict__ E64,
                                     int64_t* __restrict__ E, int n)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        E[q] = (int64_t)(long long)E64[q];
}
}  // namespace

int32_t launch_copy_energies(const unsigned long long* E64, int64_t* E, int n, cudaStream_t st)
{
    copy_energies_kernel<<<grid_for(n, 1, 1024), kBlock, 0, st>>>(E64, E, n);
    return check_launch("copy_energies");
}

int32_t launch_narrow_energy(const unsigned long long* E64, int32_t* E, int64_t n, cudaStream_t st)
{
    narrow_energy_kernel<<<grid_for(n, 1, 1024), kBlock, 0, st>>>(E64, E, n);
    return check_launch("narrow_energy");
}

int32_t launch_unpack_spins(const int8_t* spins, int8_t* out, int L, int Rp, int R, int I_index,
                            cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    const int Wn = Rp / 32;
    unpack_spins_kernel<<<grid_for((int64_t)R * N, 1, 8192), kBlock, 0, st>>>(
        reinterpret_cast<const uint32_t*>(spins) + (int64_t)I_index * N * Wn, out, L, Wn, R);
    return check_launch("unpack_spins");
}

int32_t launch_pack_spins(const int8_t* in, int8_t* spins, int L, int Rp, int R, int* bad,
                          cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    const int Wn = Rp / 32;
    pack_spins_kernel<<<grid_for((int64_t)Wn * N, 1, 8192), kBlock, 0, st>>>(in, reinterpret_cast<uint32_t*>(spins),
                                                                            L, Wn, R, bad);
    return check_launch("pack_spins");
}

}  // namespace sg
