// tile.cu -- Metropolis half sweep streamed through shared memory (the hot path for
// lattices whose rows are a multiple of 16 bytes).
//
// A block owns one instance, a tile of TY consecutive rows y0..y0+TY-1 of every slab,
// and a range of ZC slabs z0..z0+ZC-1.  It walks z: to update slab z it needs slabs
// z-1, z, z+1 restricted to rows y0-1..y0+TY (one halo row on each side).  Such a
// "slab tile" is TY+2 contiguous rows of L*Rp bytes, each fetched by one bulk
// asynchronous copy (cp.async.bulk) that completes on an mbarrier; periodic wrap in
// y is just the row index of each copy.  Four tile buffers form a ring: while slab z
// is being updated, slab z+2 is already in flight.  Updated words of the colour
// being swept go straight back to global memory; the shared copies are only read,
// since a half sweep never reads the sites it writes.
//
// Every wait on an mbarrier is bounded.  A wait that runs out sets the run's status
// word, the block stops computing, waits (bounded again) for its own copies still in
// flight, and returns.
#include <stdint.h>
#include <stdlib.h>

#include "async_copy.cuh"
#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kThrStrideT = 17;
constexpr int kRing = 4;
constexpr int kMaxLaneSteps = 10;  // site updates a thread may add to its 8-bit energy lanes
using ac::bulk_g2s;
using ac::mbar_expect_tx;
using ac::mbar_init;
using ac::mbar_wait;

struct TileArgs {
    uint32_t* spins;               // [I][N][Wn] words
    const uint2* const* j6_ptrs;
    const uint8_t* const* j1_ptrs;
    const RunKeys* keys;
    const uint32_t* thr;           // SA: one row; PT: [K][kThrRow]
    const uint8_t* rung_of_slot;   // PT: [I][Rp]
    int32_t* E;                    // PT: [I][Rp]
    int* status;                   // set to SG_ETIMEOUT when a wait gives up
    int L, Wn, Rvalid, G, TY, ZC, ytiles, zchunks;
    uint32_t sweep;
    int colour;
};

template <bool PT, bool UNITJ, int WG, int CH, bool PAD = true>
__global__ void __launch_bounds__(256, 2) sweep_tile_kernel(const TileArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kRing];
    __shared__ uint32_t s_thr[PT ? 256 * kThrStrideT : kThrRow];
    __shared__ uint4 s_lead[PT ? 64 : 1];  // PT: leading threshold bytes per word (unit couplings)
    __shared__ int s_dE[PT ? 256 : 1];
    __shared__ int s_abort;

    const int L = a.L, Wn = a.Wn, G = a.G, TY = a.TY, ZC = a.ZC;
    const int Rp = 4 * Wn;
    const int LL = L * L;
    const uint32_t row_bytes = (uint32_t)L * (uint32_t)Rp;
    const uint32_t tile_bytes = row_bytes * (uint32_t)(TY + 2);
    const int unit = blockIdx.x;
    const int inst = unit / (a.ytiles * a.zchunks);
    const int rem = unit - inst * a.ytiles * a.zchunks;
    const int y0 = (rem / a.zchunks) * TY;
    const int z0 = (rem % a.zchunks) * ZC;
    const RunKeys key = a.keys[inst];
    uint32_t* __restrict__ s = a.spins + (size_t)inst * (size_t)LL * L * Wn;
    const unsigned char* __restrict__ gbytes = reinterpret_cast<const unsigned char*>(s);
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;

    if (tid == 0) {
        for (int b = 0; b < kRing; ++b) mbar_init(&bars[b], 1);
        ac::mbar_fence_init();
        s_abort = 0;
    }
    if (PT) {
        for (int q = tid; q < Rp * kThrRow; q += nthreads) {
            const int slot = q / kThrRow, k = q % kThrRow;
            s_thr[slot * kThrStrideT + k] = a.thr[a.rung_of_slot[(size_t)inst * Rp + slot] * kThrRow + k];
        }
        for (int q = tid; q < Rp; q += nthreads) s_dE[q] = 0;
    } else {
        for (int q = tid; q < kThrRow; q += nthreads) s_thr[q] = a.thr[q];
    }
    __syncthreads();
    uint4 lead_sa = make_uint4(0, 0, 0, 0);  // SA: one record for every word
    if (UNITJ) {
        if (PT) {
            for (int q = tid; q < Wn; q += nthreads) {
                const uint32_t* t0 = s_thr + 4 * q * kThrStrideT;
                s_lead[q] = mp::lead_record(t0, t0 + kThrStrideT, t0 + 2 * kThrStrideT, t0 + 3 * kThrStrideT);
            }
            __syncthreads();
        } else {
            lead_sa = mp::lead_record(s_thr, s_thr, s_thr, s_thr);
        }
    }

    // slab k (k = -1 .. ZC) of the unit lives in ring buffer (k+1) % kRing, as that
    // buffer's ((k+1)/kRing)-th fill
    auto issue = [&](int k) {
        const int b = (k + 1) % kRing;
        unsigned char* dst = smem + (size_t)b * tile_bytes;
        const int z = (z0 + k + L) % L;
        mbar_expect_tx(&bars[b], tile_bytes);
        for (int r = 0; r < TY + 2; ++r) {
            const int y = (y0 - 1 + r + L) % L;
            bulk_g2s(dst + (size_t)r * row_bytes, gbytes + ((size_t)z * L + y) * row_bytes, row_bytes,
                     &bars[b]);
        }
    };
    auto wait_slab = [&](int k) -> bool {
        return mbar_wait(&bars[(k + 1) % kRing], (uint32_t)(((k + 1) / kRing) & 1));
    };
    if (tid == 0)
        for (int k = -1; k <= 1 && k <= ZC; ++k) issue(k);

    const int g = threadIdx.x % G;
    const int j0 = threadIdx.x / G;
    const int JX = blockDim.x / G;
    const int H = L >> 1;
    const int r = threadIdx.y;  // tile row handled by this thread (0 .. TY-1)
    const int wbase = g * CH * WG;

    uint32_t vmask[CH][WG];
    uint32_t acc[CH][WG];
#pragma unroll
    for (int ch = 0; ch < CH; ++ch)
#pragma unroll
        for (int wi = 0; wi < WG; ++wi) {
            uint32_t m = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (4 * (wbase + ch * WG + wi) + b < a.Rvalid) m |= 0x80u << (8 * b);
            vmask[ch][wi] = PAD ? m : 0x80808080u;
            acc[ch][wi] = 0;
        }


    // Folds the 8-bit energy lanes into the block's per-slot sums (called by every
    // thread at a converged point, at most every kMaxLaneSteps site updates).
    auto flush = [&]() {
        const int lane = tid & 31;
        const bool full = nthreads - (tid & ~31) >= 32;
        const bool full_warp_same = full && (G == 1);
        const bool shuffle_same = full && G < 32 && (32 % G) == 0;
#pragma unroll
        for (int ch = 0; ch < CH; ++ch)
#pragma unroll
            for (int wi = 0; wi < WG; ++wi) {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int slot = 4 * (wbase + ch * WG + wi) + b;
                    int d = 2 * mp::lane_sum(acc[ch][wi], b);
                    if (full_warp_same) {
                        d = __reduce_add_sync(0xFFFFFFFFu, d);
                        if (lane == 0 && d) atomicAdd(&s_dE[slot], d);
                    } else if (shuffle_same) {
                        for (int off = G; off < 32; off <<= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, off);
                        if (lane < G && d) atomicAdd(&s_dE[slot], d);
                    } else if (d) {
                        atomicAdd(&s_dE[slot], d);
                    }
                }
                acc[ch][wi] = 0;
            }
    };

    bool ok = true;
    if (!wait_slab(-1) || !wait_slab(0)) ok = false;
    int issued_to = 1;  // highest slab index issued so far
    for (int t = 0; t < ZC; ++t) {
        if (tid == 0 && t + 2 <= ZC && ok) {
            // buffer of slab t+2 held slab t-2, whose last reader finished at step t-1
            ac::fence_proxy_async();
            issue(t + 2);
            issued_to = t + 2;
        }
        if (ok && !wait_slab(t + 1)) ok = false;
        if (!ok) s_abort = 1;
        if (ok && r < TY) {
            const int z = (z0 + t) % L;
            const int y = (y0 + r) % L;
            const int par = (y + z + a.colour) & 1;
            const uint32_t* bm = reinterpret_cast<const uint32_t*>(smem + (size_t)(t % kRing) * tile_bytes);
            const uint32_t* b0 = reinterpret_cast<const uint32_t*>(smem + (size_t)((t + 1) % kRing) * tile_bytes);
            const uint32_t* bp = reinterpret_cast<const uint32_t*>(smem + (size_t)((t + 2) % kRing) * tile_bytes);
            const int rowW = L * Wn;  // words per row
            const uint32_t* own_row = b0 + (size_t)(r + 1) * rowW;
            for (int j = j0; j < H; j += JX) {
                const int x = 2 * j + par;
                const int i = (z * L + y) * L + x;  // logical site (counters, couplings)
                // storage positions in a row (colour-split): this site is entry j of half
                // `par`, its x neighbours entries j + par and j + par - 1 of the other half
                const int px = par * H + j;
                const int jp = j + par == H ? 0 : j + par, jm = j + par == 0 ? H - 1 : j + par - 1;
                const int xp = (1 - par) * H + jp, xm = (1 - par) * H + jm;
                const mp::Couplings cp = UNITJ ? mp::decode_unit(a.j1_ptrs[inst][i])
                                               : mp::decode_general(a.j6_ptrs[inst][i]);
                const uint32_t* nbp[6] = {own_row + xp * Wn, own_row + xm * Wn,
                                          b0 + (size_t)(r + 2) * rowW + px * Wn,
                                          b0 + (size_t)r * rowW + px * Wn,
                                          bp + (size_t)(r + 1) * rowW + px * Wn,
                                          bm + (size_t)(r + 1) * rowW + px * Wn};
#pragma unroll
                for (int ch = 0; ch < CH; ++ch) {
                    const int w0 = wbase + ch * WG;
                    uint32_t self[WG], P[WG];
                    mp::load_words<WG>(own_row + px * Wn + w0, self);
#pragma unroll
                    for (int wi = 0; wi < WG; ++wi) P[wi] = 0;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        uint32_t n[WG];
                        mp::load_words<WG>(nbp[q] + w0, n);
#pragma unroll
                        for (int wi = 0; wi < WG; ++wi) P[wi] += mp::bond_term(n[wi], cp, q);
                    }
                    const uint32_t* thr = PT ? s_thr + 4 * w0 * kThrStrideT : s_thr;
                    if (mp::update_words<PT, UNITJ, WG, kThrStrideT>(self, P, vmask[ch], cp.msum, (uint32_t)i,
                                                                     a.sweep, (uint32_t)w0, key, thr,
                                                                     PT ? s_lead + w0 : &lead_sa, acc[ch]))
                        mp::store_words<WG>(s + ((size_t)(z * L + y) * L + px) * Wn + w0, self);
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
        if (PT && (t + 1) % kMaxLaneSteps == 0 && t + 1 < ZC) flush();
    }

    if (s_abort) {
        if (tid == 0) {
            atomicExch(a.status, SG_ETIMEOUT);
            // let the copies still in flight (at most the last three slabs issued) land
            // before the block's shared memory is released; each wait is bounded
            for (int k = issued_to - 2; k <= issued_to; ++k)
                if (k >= -1) wait_slab(k);
        }
        return;
    }

    if (PT) {
        flush();
        __syncthreads();
        int32_t* Ei = a.E + (size_t)inst * Rp;
        for (int q = tid; q < Rp; q += nthreads)
            if (s_dE[q]) atomicAdd(&Ei[q], s_dE[q]);
    }
}

struct TileShape {
    int TY, ZC, G, CH, WG;
    dim3 block;
    size_t smem;
    int units;
};

int env_int(const char* name, int dflt)
{
    const char* e = getenv(name);
    return e ? atoi(e) : dflt;
}

bool tile_shape(int I, int L, int Wn, TileShape* sh)
{
    sh->WG = (Wn % 4 == 0) ? 4 : (Wn % 2 == 0) ? 2 : 1;
    sh->CH = (sh->WG == 4 && (Wn / 4) % 2 == 0) ? 2 : 1;
    sh->G = Wn / (sh->WG * sh->CH);
    const int Rp = 4 * Wn;
    const long row_bytes = (long)L * Rp;
    if (L < 16 || row_bytes % 16 != 0 || sh->G > 32) return false;
    const int TX = (L / 2) * sh->G;
    if (TX > 256) return false;
    // rows per tile: the largest divisor of L with TX * TY <= 256 and the ring <= 160 KB
    int TY = env_int("SG_TILE_TY", 0);
    if (TY <= 0 || L % TY != 0 || TX * TY > 256) {
        TY = 0;
        for (int t = 1; t <= L; ++t)
            if (L % t == 0 && TX * t <= 256 && (long)kRing * (t + 2) * row_bytes <= 160 * 1024) TY = t;
    }
    if (TY == 0 || (TX * TY) % 32 != 0) return false;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // slabs per unit: the largest divisor of L leaving at least ~3 waves of 2 blocks per SM
    int ZC = env_int("SG_TILE_ZC", 0);
    if (ZC <= 0 || L % ZC != 0) {
        ZC = 1;
        for (int t = 1; t <= L; ++t)
            if (L % t == 0 && (long)I * (L / TY) * (L / t) >= 6L * sms) ZC = t;
    }
    sh->TY = TY;
    sh->ZC = ZC;
    sh->block = dim3(TX, TY, 1);
    sh->smem = (size_t)kRing * (TY + 2) * row_bytes;
    sh->units = I * (L / TY) * (L / ZC);
    return true;
}

template <bool PT, bool UNITJ, int WG, int CH>
int32_t launch_tile_variant(const TileShape& sh, const TileArgs& a, cudaStream_t st)
{
    static bool attr_set = false;  // per instantiation: allow > 48 KB of dynamic shared memory
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_tile_kernel<PT, UNITJ, WG, CH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024);
        if (e != cudaSuccess) {
            set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            return SG_ECUDA;
        }
        attr_set = true;
    }
    sweep_tile_kernel<PT, UNITJ, WG, CH><<<sh.units, sh.block, sh.smem, st>>>(a);
    return SG_OK;
}

template <bool PT, bool UNITJ>
int32_t launch_tile_shape(const TileShape& sh, const TileArgs& a, cudaStream_t st)
{
    if (sh.WG == 4 && sh.CH == 2) return launch_tile_variant<PT, UNITJ, 4, 2>(sh, a, st);
    if (sh.WG == 4) return launch_tile_variant<PT, UNITJ, 4, 1>(sh, a, st);
    if (sh.WG == 2) return launch_tile_variant<PT, UNITJ, 2, 1>(sh, a, st);
    return launch_tile_variant<PT, UNITJ, 1, 1>(sh, a, st);
}

}  // namespace

bool tile_kernel_supports(int I, int L, int Wn)
{
    // tuning knob SG_SWEEP_KERNEL: 2 selects this kernel where it applies; the default
    // (and 1) is the row kernel, which measures faster on the workloads timed so far
    if (env_int("SG_SWEEP_KERNEL", 1) != 2) return false;
    TileShape sh;
    return tile_shape(I, L, Wn, &sh);
}

int32_t launch_sweep_tile(int8_t* spins, const uint2* const* j6_ptrs, const uint8_t* const* j1_ptrs,
                          const RunKeys* keys, const uint32_t* thr, const uint8_t* rung_of_slot,
                          int32_t* E, int* status, bool pt, bool unit_j, int I, int L, int Wn,
                          int Rvalid, uint32_t sweep, int colour, cudaStream_t st)
{
    TileShape sh;
    if (!tile_shape(I, L, Wn, &sh)) {
        set_error("tile sweep does not support L=%d, Wn=%d", L, Wn);
        return SG_EINVAL;
    }
    TileArgs a{};
    a.spins = reinterpret_cast<uint32_t*>(spins);
    a.j6_ptrs = j6_ptrs;
    a.j1_ptrs = j1_ptrs;
    a.keys = keys;
    a.thr = thr;
    a.rung_of_slot = rung_of_slot;
    a.E = E;
    a.status = status;
    a.L = L;
    a.Wn = Wn;
    a.Rvalid = Rvalid;
    a.G = sh.G;
    a.TY = sh.TY;
    a.ZC = sh.ZC;
    a.ytiles = L / sh.TY;
    a.zchunks = L / sh.ZC;
    a.sweep = sweep;
    a.colour = colour;
    int32_t rc;
    if (pt)
        rc = unit_j ? launch_tile_shape<true, true>(sh, a, st) : launch_tile_shape<true, false>(sh, a, st);
    else
        rc = unit_j ? launch_tile_shape<false, true>(sh, a, st) : launch_tile_shape<false, false>(sh, a, st);
    if (rc != SG_OK) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("tile sweep launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace sg
