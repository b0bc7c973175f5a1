// ptslab.cuh -- the per-block machinery of the parallel-tempering kernels that keep part
// of a lattice in shared memory for many sweeps (App. D.2): ptcluster.cu (z-slabs of a
// thread-block cluster) and ptcoop.cu (row blocks of a cooperative grid).  K <= 32: one
// 32-bit word of 32 slots per site, all couplings +-1.
//
// A block holds its slots' thresholds (per slot rows for ties, and the bit planes of the
// word the bit-sliced compare reads), updates words (metropolis.cuh) with a per-warp queue
// of tied draws decided later, and, in a colour-1 half sweep, sums every slot's energy
// (6 - 2c per site, c the satisfied count after the update) in bit-sliced counters.  The
// kernels supply the geometry: which words a thread updates and where their neighbours lie.
#pragma once
#include <stdint.h>

#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace pts {

constexpr int kThreads = 512;    // 128 registers, no spills (768 or 1024 threads measured slower)
constexpr int kWarps = kThreads / 32;
constexpr int kTieCap = 48;  // queued tie entries per warp
// A warp decides its queue once it holds this many entries -- about one pass of its 32
// lanes when it is checked every second item (a warp-item adds 1 to 2 on average, at most
// 32; a full queue decides the overflowing ties on the spot).  24 measured 4 % faster than
// 16 at L = 64 (20 to 28 and checks every 2, 4 or 8 items all within 1 %).
constexpr int kTieResolve = 24;
constexpr int kCheckEvery = 2;  // items a thread updates between checks of its warp's queue
constexpr int kThrStride = 17;   // per-slot threshold row stride (bank spread)
constexpr int kVBits = 8;        // energy counters: up to 42 items of at most 6 before a fold
constexpr int kFoldItems = 42;
constexpr size_t kTieBytes = (size_t)kWarps * kTieCap * 2 * sizeof(uint4);

// Shared state of one block.
struct Shared {
    uint32_t thr[32 * kThrStride];  // per slot: thresholds of its rung, k = 0 .. 15
    uint4 tp4[8];                   // threshold-byte plane j of k = 2, 4, 6 (bit b: slot b)
    uint4 lz;                       // slots whose threshold of k = 2, 4, 6 has nonzero low 24 bits
    uint32_t rthr[32 * kThrRow];    // per rung: its threshold row
    int E[32];                      // the block's energy sums of a colour-1 half sweep
    uint32_t acc[32];               // accepted swaps of rung pairs in this launch
    uint8_t rung[32], slot[32];     // slot -> rung, rung -> slot
    int tie_n[kWarps];
    int min;                        // lowest energy seen
};

// The same update with the threshold planes read from shared memory where they are used:
// tp4[j] = {plane j of k = 2, of k = 4, of k = 6, -} (j = 0 .. 7, least significant first),
// and the coupling signs taken from the sign byte one bond at a time, so that few of the
// word's values are live at once.
__device__ __forceinline__ void update_word_unit_smem(uint32_t self, const uint32_t (&n)[6], uint32_t sbits,
                                                      uint32_t valid, const uint4* tp4, const uint32_t (&A)[8],
                                                      uint32_t* flip, uint32_t* tie, uint32_t* c0, uint32_t* c1,
                                                      uint32_t* c2)
{
    uint32_t a[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) a[q] = self ^ n[q] ^ (0u - ((sbits >> q) & 1u));
    const uint32_t s1 = a[0] ^ a[1] ^ a[2], k1 = mp::maj3(a[0], a[1], a[2]);
    const uint32_t s2 = a[3] ^ a[4] ^ a[5], k2 = mp::maj3(a[3], a[4], a[5]);
    *c0 = s1 ^ s2;
    const uint32_t t = s1 & s2;
    *c1 = k1 ^ k2 ^ t;
    *c2 = mp::maj3(k1, k2, t);
    const uint32_t need = *c2 & valid;
    const uint32_t free = ~*c2 & valid;
    uint32_t lt = 0, eq = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint4 p = tp4[j];
        const uint32_t T = (*c1 & p.z) | (~*c1 & ((*c0 & p.y) | (~*c0 & p.x)));
        lt = mp::maj3(~A[j], T, lt);
        eq &= ~(A[j] ^ T);
    }
    *flip = free | (need & lt);
    *tie = need & eq;
}

__device__ __forceinline__ uint32_t valid_bits(int K) { return K >= 32 ? 0xFFFFFFFFu : (1u << K) - 1u; }

// Loads the slot map and thresholds of an instance; every thread of the block calls it.
__device__ __forceinline__ void load_state(Shared& sh, const uint8_t* rung_of_slot, const uint8_t* slot_of_rung,
                                           const uint32_t* thr, int K, int32_t minE, int tid)
{
    if (tid < 32) {
        sh.rung[tid] = rung_of_slot[tid];
        if (tid < K) sh.slot[tid] = slot_of_rung[tid];
        sh.E[tid] = 0;
        sh.acc[tid] = 0;
    }
    for (int q = tid; q < K * kThrRow; q += kThreads) sh.rthr[q] = thr[q];
    if (tid < kWarps) sh.tie_n[tid] = 0;
    if (tid == 0) sh.min = minE;
}

// The slot-to-rung map gives every slot its thresholds; called by every thread, the first
// warp does the work (a __syncthreads must follow before the tables are read).
__device__ __forceinline__ void build_thresholds(Shared& sh, int warp, int lane)
{
    if (warp != 0) return;
    const uint32_t* row = sh.rthr + (int)sh.rung[lane] * kThrRow;
#pragma unroll
    for (int k = 0; k < kThrRow; ++k) sh.thr[lane * kThrStride + k] = row[k];
    const uint32_t t2 = row[2], t4 = row[4], t6 = row[6];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t p2 = __ballot_sync(0xFFFFFFFFu, mp::threshold_plane_bit(t2, j) != 0u);
        const uint32_t p4 = __ballot_sync(0xFFFFFFFFu, mp::threshold_plane_bit(t4, j) != 0u);
        const uint32_t p6 = __ballot_sync(0xFFFFFFFFu, mp::threshold_plane_bit(t6, j) != 0u);
        if (lane == 0) sh.tp4[j] = make_uint4(p2, p4, p6, 0u);
    }
    const uint32_t l2 = __ballot_sync(0xFFFFFFFFu, (t2 & 0xFFFFFFu) != 0u);
    const uint32_t l4 = __ballot_sync(0xFFFFFFFFu, (t4 & 0xFFFFFFu) != 0u);
    const uint32_t l6 = __ballot_sync(0xFFFFFFFFu, (t6 & 0xFFFFFFu) != 0u);
    if (lane == 0) sh.lz = make_uint4(l2, l4, l6, 0u);
}

// One word to update: its logical site i (draw counters, sign byte), its index `is` in the
// block's word array, its word and its six neighbours' words, its coupling sign bits and
// its eight leading-byte draw planes.
struct Work {
    uint32_t i;
    int is;
    uint32_t self, n[6], sbits, A[8];
};

// The updates of one thread during one half sweep.
struct Updater {
    Shared& sh;
    uint32_t* words;  // the block's word array (Work::is indexes it)
    uint4* ties;      // this warp's queue: {i, is, -, tie}, {c0, c1, stored word, -}
    RunKeys key;
    uint32_t valid, sweep;
    int warp, lane;
    bool energy;
    uint32_t V[kVBits];
    int nitems;

    __device__ __forceinline__ Updater(Shared& s, uint32_t* w, uint4* all_ties, RunKeys k, uint32_t v, uint32_t sw,
                                       int tid, bool e)
        : sh(s), words(w), ties(all_ties + (tid >> 5) * kTieCap * 2), key(k), valid(v), sweep(sw), warp(tid >> 5),
          lane(tid & 31), energy(e), nitems(0)
    {
#pragma unroll
        for (int j = 0; j < kVBits; ++j) V[j] = 0;
    }

    __device__ __forceinline__ void draws(Work& w) const { mp::lead_planes(w.i, sweep, 0u, key, w.A); }

    // this thread's counters into the block's sums (only when they would overflow)
    __device__ __forceinline__ void fold()
    {
        for (int b = 0; b < 32; ++b) {
            const int e = 6 * nitems - 2 * mp::vcount(V, b);
            if (e) atomicAdd(&sh.E[b], e);
        }
#pragma unroll
        for (int j = 0; j < kVBits; ++j) V[j] = 0;
        nitems = 0;
    }

    // Decides this warp's queued ties (every lane of the warp calls it): a blind store of
    // the word its owner stored -- a word has at most one entry and nobody else writes it --
    // and, in a colour-1 half sweep, 2k added to the slot's energy for each late flip.
    __device__ __forceinline__ void resolve()
    {
        __syncwarp();
        const int n = min(sh.tie_n[warp], kTieCap);
        for (int e = lane; e < n; e += 32) {
            const uint4 t = ties[2 * e], u = ties[2 * e + 1];
            const uint32_t acc =
                mp::resolve_tie_bits(t.w, u.x, u.y, sh.thr, kThrStride, t.x, sweep, 0u, key.k0, key.k1);
            if (acc) {
                words[t.y] = u.z ^ acc;
                if (energy)
                    for (uint32_t m = acc; m; m &= m - 1u) {
                        const int b = __ffs(m) - 1;
                        const int c = 4 + (int)((u.x >> b) & 1u) + 2 * (int)((u.y >> b) & 1u);
                        atomicAdd(&sh.E[b], 2 * (2 * c - 6));
                    }
            }
        }
        __syncwarp();
        if (lane == 0) sh.tie_n[warp] = 0;
        __syncwarp();
    }

    // the periodic check: every lane of the warp calls it after the same number of updates
    __device__ __forceinline__ void maybe_resolve()
    {
        __syncwarp();
        if (sh.tie_n[warp] >= kTieResolve) resolve();
    }

    __device__ __forceinline__ void update(const Work& w)
    {
        uint32_t flip, tie, c0, c1, c2;
        update_word_unit_smem(w.self, w.n, w.sbits, valid, sh.tp4, w.A, &flip, &tie, &c0, &c1, &c2);
        {
            const uint4 z = sh.lz;
            tie &= (c1 & z.z) | (~c1 & ((c0 & z.y) | (~c0 & z.x)));  // the others reject
        }
        if (tie) {
            const int p = atomicAdd(&sh.tie_n[warp], 1);
            if (p < kTieCap) {
                ties[2 * p] = make_uint4(w.i, (uint32_t)w.is, 0u, tie);
                ties[2 * p + 1] = make_uint4(c0, c1, w.self ^ flip, 0u);
            } else {  // queue full: decide here
                flip |= mp::resolve_tie_bits(tie, c0, c1, sh.thr, kThrStride, w.i, sweep, 0u, key.k0, key.k1);
            }
        }
        if (energy) {
            mp::count_after_flip(flip, c0, c1, c2);
            mp::vadd3(V, c0, c1, c2);
            if (++nitems == kFoldItems) fold();
        }
        words[w.is] = w.self ^ flip;  // unconditional: cheaper than the branch
    }

    // End of a colour-1 half sweep (every thread of the block, after its last resolve):
    // lane b collects slot b of every lane through a bit transpose per plane and adds the
    // warp's sum to the block's.  A __syncthreads must follow before sh.E is read.
    __device__ __forceinline__ void energy_to_block()
    {
        uint32_t T[kVBits];
#pragma unroll
        for (int jb = 0; jb < kVBits; ++jb) T[jb] = mp::warp_transpose(V[jb], lane);
        const int n = __reduce_add_sync(0xFFFFFFFFu, nitems);
        int cnt = 0;
#pragma unroll
        for (int jb = 0; jb < kVBits; ++jb) cnt += __popc(T[jb]) << jb;
        const int e = 6 * n - 2 * cnt;
        if (e) atomicAdd(&sh.E[lane], e);
    }
};

// The exchange after sweep `sweep` (App. D.2), decided by the first warp of a block from
// the instance's slot energies E (lane b: slot b): pairs (k, k+1) with k = sweep mod 2,
// accepted when d = E_a - E_b <= 0 or the draw u < T_k(d).  Updates the block's slot map,
// its accepted-swap counts (when `count`) and its running minimum.  Called by the first
// warp only; a build_thresholds and a __syncthreads must follow.
__device__ __forceinline__ void exchange(Shared& sh, int Eq, uint32_t sweep, int K, RunKeys key, const uint32_t* xtab,
                                         const uint32_t* xoff, const uint32_t* xlen, const uint32_t* xtail,
                                         bool count, int lane)
{
    const int k = 2 * lane + (int)(sweep & 1u);
    const bool pair = k + 1 < K;
    const int sa = pair ? sh.slot[k] : 0, sb = pair ? sh.slot[k + 1] : 0;
    const int Ea = __shfl_sync(0xFFFFFFFFu, Eq, sa), Eb = __shfl_sync(0xFFFFFFFFu, Eq, sb);
    if (pair) {
        const int64_t d = (int64_t)Ea - (int64_t)Eb;
        bool accept = d <= 0;
        if (!accept) {
            const uint32_t u = philox4x32_10((uint32_t)k, sweep, 0u, kDomainExchange, key.k0, key.k1).v[0];
            const uint32_t T = d <= (int64_t)xlen[k] ? xtab[xoff[k] + (uint32_t)(d - 1)] : xtail[k];
            accept = u < T;
        }
        if (accept) {
            sh.rung[sa] = (uint8_t)(k + 1);
            sh.rung[sb] = (uint8_t)k;
            sh.slot[k] = (uint8_t)sb;
            sh.slot[k + 1] = (uint8_t)sa;
            if (count) sh.acc[k] += 1u;
        }
    }
    int m = lane < K ? Eq : 0x7FFFFFFF;
    m = __reduce_min_sync(0xFFFFFFFFu, m);
    if (lane == 0 && m < sh.min) sh.min = m;
    __syncwarp();
}

// Writes an instance's slot map, swap counts and minimum back (first warp of one block).
__device__ __forceinline__ void store_state(const Shared& sh, uint8_t* rung_of_slot, uint8_t* slot_of_rung,
                                            unsigned long long* accepts, int32_t* minE, int K, int lane)
{
    rung_of_slot[lane] = sh.rung[lane];
    if (lane < K) slot_of_rung[lane] = sh.slot[lane];
    if (lane + 1 < K) accepts[lane] += (unsigned long long)sh.acc[lane];
    if (lane == 0) *minE = sh.min;
}

}  // namespace pts
}  // namespace sg
