// sweep.cu -- the Metropolis half-sweep kernel: the hot path (App. D.1, App. D.2).
//
// One launch updates every site of one checkerboard colour, for every replica of a
// group of instances.  Thread mapping (no division except one multiply-high per row):
//   blockIdx.y        instance
//   blockIdx.x, ty    rows (y, z) of the lattice, dealt out grid-stride: thread (bx, ty)
//                     takes rows (c * gridDim.x + bx) * blockDim.y + ty, c < rows_per_thread
//   tx = j * G + g    site j of the colour inside the row, word group g
// A word holds four replicas (one byte each).  Thread g of a site owns CH chunks of
// WG consecutive words, so it updates 4*WG*CH replicas with one decode of the site's
// couplings, and one Philox4x32-10 call per word (the counter (site, sweep, word, 0)
// names exactly that word's four replicas).
//
// Per word (bit layout in kernels.cu):
//   P  = sum_q ((n_q ^ S_q) & M_q)                 2|J| for each negative bond term
//   W  = s_i == +1 ? P : 2*sum|J| - P                2 * (weight of unsatisfied bonds)
//   k  = W - sum|J|  (= -x; flipping raises E by 2k)
// Bytes with k <= 0 flip unconditionally; the others flip when their Philox word is
// below thr[k].  "k > 0" is found for four bytes by one borrow-free subtraction; the
// draws are taken only when some lane of the warp needs one (a warp-uniform branch,
// so the WG Philox chains of a chunk interleave), and the byte decisions are
// branch-free.  For parallel tempering the energy change of every slot is summed in
// 8-bit lanes (at most 10 updates per thread, each adding <= 24) and reduced once per
// thread with warp reductions.
#include <stdlib.h>

#include "exchange.cuh"
#include "async_copy.cuh"
#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kThrStride = 17;   // per-slot threshold row stride in shared memory (bank spread)
constexpr int kTieCap = 32;      // queued tied draws per warp

// Words of the staged PT variant's threshold table in dynamic shared memory (Rp slots),
// rounded so that the row buffers after it stay 128-byte aligned.
__host__ __device__ constexpr int staged_thr_words(int Rp) { return (Rp * kThrStride + 31) & ~31; }

struct SweepArgs {
    uint32_t* spins;
    const uint2* const* j6_ptrs;     // per instance: [N] records of the six int8 couplings
    const uint8_t* const* j1_ptrs;   // per instance: [N] sign bits (used when all |J| = 1)
    const RunKeys* keys;
    const uint32_t* thr;          // SA: one row of kThrRow ([S][kThrRow] with sweep_base); PT: [K][kThrRow]
    const uint8_t* rung_of_slot;  // PT: [I][Rp]
    int32_t* E;                   // PT: [I][Rp] energies, updated
    int L, Wn, Rvalid, G, rows_per_thread;
    uint32_t Lmagic;              // ceil(2^32 / L): row / L by multiply-high
    uint32_t sweep;
    int colour;
    ExchangeArgs x;               // PT exchange performed by the last block of each instance
    unsigned* done;               // [I] blocks finished in this launch (reset by the last one)
    const uint32_t* sweep_base;   // if set, the sweep index is *sweep_base + sweep
    int* status;                  // staged variant: set to SG_ETIMEOUT when a copy wait gives up
    int segw;                     // staged variant: words of one half row, (L/2) * Wn
};

// NST > 0: the staged variant.  Each warp owns one row at a time (blockDim.x == 32, one
// site per thread) and keeps NST rows in flight: for row (y, z) the six half rows it
// reads -- its own sites, their x neighbours, and the matching halves of rows y+-1 and
// z+-1 -- arrive in shared memory by bulk asynchronous copies that complete on the
// warp's mbarrier for that ring slot, issued NST rows ahead of use.  The updated spins
// go straight back to global memory; a half sweep never reads what it writes.
template <bool PT, bool UNITJ, int WG, int CH, bool PAD, int MINB = 2, bool DRAW = false,
          bool XCH = false, int NST = 0>
__global__ void __launch_bounds__(256, MINB) sweep_rows_kernel(const SweepArgs a)
{
    // staged PT: the slot thresholds live at the start of the dynamic array, sized to Rp
    __shared__ uint32_t s_thr_fixed[PT ? (NST > 0 ? 1 : 256 * kThrStride) : kThrRow];
    __shared__ int s_dE[PT ? 256 : 1];
    extern __shared__ __align__(128) uint32_t s_stage[];  // NST > 0: [thr][TY][NST][6][segw]
    __shared__ uint64_t s_bar[NST > 0 ? 8 * NST : 1];
    __shared__ uint4 s_lead[PT ? 64 : 1];  // PT: leading threshold bytes per word (unit couplings)
    __shared__ uint4 s_ties[8 * kTieCap];  // per warp: draws whose leading byte tied
    __shared__ int s_tie_n[8];

    const int inst = blockIdx.y;
    const int L = a.L, Wn = a.Wn, G = a.G;
    const int Rp = 4 * Wn;
    const int H = L >> 1;
    const int LL = L * L;
    const RunKeys key = a.keys[inst];
    const uint32_t sweep = a.sweep + (a.sweep_base ? *a.sweep_base : 0u);
    uint32_t* __restrict__ s = a.spins + (size_t)inst * (size_t)LL * L * Wn;
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    uint32_t* s_thr = (PT && NST > 0) ? s_stage : s_thr_fixed;
    const int thr_words = (PT && NST > 0) ? staged_thr_words(Rp) : 0;

    if (PT) {
        for (int q = tid; q < Rp * kThrRow; q += nthreads) {
            const int slot = q / kThrRow, k = q % kThrRow;
            s_thr[slot * kThrStride + k] = a.thr[a.rung_of_slot[(size_t)inst * Rp + slot] * kThrRow + k];
        }
        for (int q = tid; q < Rp; q += nthreads) s_dE[q] = 0;
    } else {
        // with a device sweep index, thr is the run's [S][kThrRow] schedule table
        const uint32_t* row = a.sweep_base ? a.thr + (size_t)sweep * kThrRow : a.thr;
        for (int q = tid; q < kThrRow; q += nthreads) s_thr[q] = row[q];
    }
    if constexpr (NST > 0) {
        if (threadIdx.x == 0) {
            for (int k = 0; k < NST; ++k) ac::mbar_init(&s_bar[threadIdx.y * NST + k], 1);
            ac::mbar_fence_init();
        }
    }
    if (tid < 8) s_tie_n[tid] = 0;
    __syncthreads();
    uint4 lead_sa = make_uint4(0, 0, 0, 0);  // SA: one record for every word
    if (UNITJ) {
        if (PT) {
            for (int q = tid; q < Wn; q += nthreads) {
                const uint32_t* t0 = s_thr + 4 * q * kThrStride;
                s_lead[q] = mp::lead_record(t0, t0 + kThrStride, t0 + 2 * kThrStride, t0 + 3 * kThrStride);
            }
            __syncthreads();
        } else {
            lead_sa = mp::lead_record(s_thr, s_thr, s_thr, s_thr);
        }
    }

    const int g = threadIdx.x % G;
    const int j0 = threadIdx.x / G;
    const int JX = blockDim.x / G;
    const int wbase = g * CH * WG;  // first word owned by this thread

    uint32_t vmask[CH][WG];  // bit 7 of each byte that is a real replica (not padding)
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

    constexpr int KMAX = UNITJ ? 6 : 12;  // largest |k| of one flip
    // Folds the 8-bit energy lanes into the block's per-slot sums.  Called by whole
    // warps at the same point of the row loop.
    auto flush = [&]() {
        const int lane = tid & 31;
        const bool full = __activemask() == 0xFFFFFFFFu;
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
    int items = 0;  // site updates folded into the 8-bit lanes since the last flush

    // Deferred ties of this thread's warp.  resolve_list() is called by every live lane of
    // the warp at a convergent point: the lanes share the queued entries, decide each from
    // the low 24 bits of its draws, and flip the accepted bytes in global memory (the
    // warp's own earlier stores to those words are ordered before by __syncwarp).
    const int warp = tid >> 5, lane32 = tid & 31;
    const mp::TieList ties{s_ties + warp * kTieCap, &s_tie_n[warp], kTieCap};
    const int warp_lanes = min(32, nthreads - 32 * warp);  // the block's last warp may be partial
    const unsigned wm = warp_lanes == 32 ? 0xFFFFFFFFu : (1u << warp_lanes) - 1u;
    auto resolve_list = [&]() {
        __syncwarp(wm);
        const int n = min(*ties.count, kTieCap);
        const int lanes = __popc(wm), rank = __popc(wm & ((1u << lane32) - 1u));
        for (int e = rank; e < n; e += lanes) {
            const uint4 t = ties.entries[e];
            const uint32_t w = t.z & 0xFFFFu, nib = t.z >> 16;
            const uint32_t tie = ((nib & 1u) << 7) | ((nib & 2u) << 14) | ((nib & 4u) << 21) | ((nib & 8u) << 28);
            const uint32_t* row = PT ? s_thr + 4 * w * kThrStride : s_thr;
            const uint32_t acc_t = mp::resolve_ties(tie, t.w, row, PT ? kThrStride : 0, t.x, sweep, w, key.k0, key.k1);
            if (acc_t) {
                const uint32_t ff = mp::prmt(acc_t, 0u, 0xBA98u);
                s[(size_t)t.y * Wn + w] ^= ff & 0xFEFEFEFEu;
                if (PT)
                    for (int b = 0; b < 4; ++b)
                        if ((acc_t >> (8 * b + 7)) & 1u) atomicAdd(&s_dE[4 * w + b], 2 * (int)((t.w >> (8 * b)) & 0xFFu));
            }
        }
        __syncwarp(wm);
        if (rank == 0) *ties.count = 0;
        __syncwarp(wm);
    };

    if constexpr (NST > 0) {
        // rows c = 0, 1, ... of this warp: (c * gridDim.x + blockIdx.x) * blockDim.y + threadIdx.y
        const int segw = a.segw;
        const uint32_t seg_bytes = (uint32_t)segw * 4u;
        uint32_t* ring = s_stage + thr_words + (size_t)threadIdx.y * NST * 6 * segw;
        uint64_t* bars = s_bar + threadIdx.y * NST;
        const int lane = threadIdx.x;
        auto row_of = [&](int c) { return (c * (int)gridDim.x + (int)blockIdx.x) * (int)blockDim.y + (int)threadIdx.y; };
        // lane 0: the six half rows of row c into ring slot c % NST
        // the whole warp: the six half rows of row c into ring slot c % NST, lane k < 6
        // issuing copy k after lane 0 has announced the bytes
        auto issue = [&](int c) {
            uint64_t* bar = &bars[c % NST];
            if (lane == 0) ac::mbar_expect_tx(bar, 6u * seg_bytes);
            __syncwarp();
            if (lane < 6) {
                const int row = row_of(c);
                const int z = (int)__umulhi((uint32_t)row, a.Lmagic);
                const int y = row - z * L;
                const int par = (y + z + a.colour) & 1;
                const int src = lane < 2    ? row
                                : lane == 2 ? row + (y + 1 == L ? 1 - L : 1)
                                : lane == 3 ? row + (y == 0 ? L - 1 : -1)
                                : lane == 4 ? row + (z + 1 == L ? 1 - L : 1) * L
                                            : row + (z == 0 ? L - 1 : -1) * L;
                const int half = lane == 1 ? 1 - par : par;  // x neighbours sit in the other half
                ac::fence_proxy_async();  // this slot's earlier reads come before the refill
                ac::bulk_g2s(ring + (size_t)(c % NST) * 6 * segw + (size_t)lane * segw,
                             s + ((size_t)src * L + (size_t)half * H) * Wn, seg_bytes, bar);
            }
        };
        for (int c = 0; c < NST && c < a.rows_per_thread; ++c)
            if (row_of(c) < LL) issue(c);
        bool ok = true;
        int c = 0;
        for (; c < a.rows_per_thread; ++c) {
            const int row = row_of(c);
            if (row >= LL) break;
            ok = __all_sync(0xFFFFFFFFu, ac::mbar_wait(&bars[c % NST], (uint32_t)((c / NST) & 1)));
            if (!ok) break;
            const int z = (int)__umulhi((uint32_t)row, a.Lmagic);
            const int y = row - z * L;
            const int par = (y + z + a.colour) & 1;
            const int rowoff = row * L;
            const int j = j0;  // one site per thread: blockDim.x == G * H
            const int i = rowoff + 2 * j + par;  // logical site (counters, couplings)
            const int is = rowoff + par * H + j;  // storage position
            const int jp = j + par == H ? 0 : j + par, jm = j + par == 0 ? H - 1 : j + par - 1;
            const uint32_t* buf = ring + (size_t)(c % NST) * 6 * segw;
            const mp::Couplings cp = UNITJ ? mp::decode_unit(a.j1_ptrs[inst][i])
                                           : mp::decode_general(a.j6_ptrs[inst][i]);
#pragma unroll
            for (int ch = 0; ch < CH; ++ch) {
                const int w0 = wbase + ch * WG;
                uint32_t self[WG], P[WG];
                mp::load_words<WG>(buf + j * Wn + w0, self);
#pragma unroll
                for (int wi = 0; wi < WG; ++wi) P[wi] = 0;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    // q = +x, -x, +y, -y, +z, -z: half row 1 (at jp, jm), then rows 2..5 at j
                    const int at = q == 0 ? segw + jp * Wn : q == 1 ? segw + jm * Wn : (q) * segw + j * Wn;
                    uint32_t n[WG];
                    mp::load_words<WG>(buf + at + w0, n);
#pragma unroll
                    for (int wi = 0; wi < WG; ++wi) P[wi] += mp::bond_term(n[wi], cp, q);
                }
                const uint32_t* thr = PT ? s_thr + 4 * w0 * kThrStride : s_thr;
                if (mp::update_words<PT, UNITJ, WG, kThrStride, true>(self, P, vmask[ch], cp.msum, (uint32_t)i,
                                                                     sweep, (uint32_t)w0, key, thr,
                                                                     PT ? s_lead + w0 : &lead_sa, acc[ch],
                                                                     &ties, (uint32_t)is))
                    mp::store_words<WG>(s + (size_t)is * Wn + w0, self);
            }
            if (PT && ++items == mp::kLaneCapacity<KMAX>) {
                flush();
                items = 0;
            }
            __syncwarp();  // every lane is done with slot c % NST
            if (*ties.count >= kTieCap / 2) resolve_list();
            if (c + NST < a.rows_per_thread && row_of(c + NST) < LL) issue(c + NST);
        }
        if (!ok) {
            // a copy did not arrive: report it, then wait (bounded) for the copies this
            // warp still has in flight before the block may exit
            if (lane == 0 && a.status) atomicExch(a.status, SG_ETIMEOUT);
            for (int k = c; k < c + NST && k < a.rows_per_thread; ++k)
                if (row_of(k) < LL) ac::mbar_wait(&bars[k % NST], (uint32_t)((k / NST) & 1));
        }
    } else {
        // rows are dealt out grid-stride, so the blocks of an instance advance together
        // through the lattice and the +-z neighbour rows they read are still in L2
        for (int c = 0; c < a.rows_per_thread; ++c) {
            const int row = (c * gridDim.x + blockIdx.x) * blockDim.y + threadIdx.y;
            if (row >= LL) break;
            const int z = (int)__umulhi((uint32_t)row, a.Lmagic);
            const int y = row - z * L;
            const int par = (y + z + a.colour) & 1;
            const int dyp = (y + 1 == L ? 1 - L : 1) * L, dym = (y == 0 ? L - 1 : -1) * L;
            const int dzp = (z + 1 == L ? 1 - L : 1) * LL, dzm = (z == 0 ? L - 1 : -1) * LL;
            const int rowoff = row * L;
            for (int j = j0; j < H; j += JX) {
                const int x = 2 * j + par;
                const int i = rowoff + x;  // logical site (counters, couplings)
                // storage positions (colour-split rows): this site is entry j of half `par`;
                // its x neighbours are entries j + par and j + par - 1 of the other half
                const int is = rowoff + par * H + j;
                const int ho = rowoff + (1 - par) * H;
                const int jp = j + par == H ? 0 : j + par, jm = j + par == 0 ? H - 1 : j + par - 1;
                const int nb[6] = {ho + jp, ho + jm, is + dyp, is + dym, is + dzp, is + dzm};
                const mp::Couplings cp = UNITJ ? mp::decode_unit(a.j1_ptrs[inst][i])
                                               : mp::decode_general(a.j6_ptrs[inst][i]);
    #pragma unroll
                for (int ch = 0; ch < CH; ++ch) {
                    const int w0 = wbase + ch * WG;
                    uint32_t self[WG], P[WG];
                    mp::load_words<WG>(s + (size_t)is * Wn + w0, self);
    #pragma unroll
                    for (int wi = 0; wi < WG; ++wi) P[wi] = 0;
    #pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        uint32_t n[WG];
                        mp::load_words<WG>(s + (size_t)nb[q] * Wn + w0, n);
    #pragma unroll
                        for (int wi = 0; wi < WG; ++wi) P[wi] += mp::bond_term(n[wi], cp, q);
                    }
                    const uint32_t* thr = PT ? s_thr + 4 * w0 * kThrStride : s_thr;
                    if (mp::update_words<PT, UNITJ, WG, kThrStride, true>(self, P, vmask[ch], cp.msum,
                                                                         (uint32_t)i, sweep, (uint32_t)w0, key,
                                                                         thr, PT ? s_lead + w0 : &lead_sa,
                                                                         acc[ch], &ties, (uint32_t)is))
                        mp::store_words<WG>(s + (size_t)is * Wn + w0, self);
                }
                if (PT && ++items == mp::kLaneCapacity<KMAX>) {
                    flush();
                    items = 0;
                }
            }
        }

    }

    resolve_list();
    if (PT) {
        flush();
        __syncthreads();
        int32_t* Ei = a.E + (size_t)inst * Rp;
        for (int q = tid; q < Rp; q += nthreads)
            if (s_dE[q]) atomicAdd(&Ei[q], s_dE[q]);
        if (XCH) {
            // The block that finishes last for this instance performs the exchange: every
            // block publishes its energy sums, then counts itself done; no block waits.
            __shared__ int s_last;
            __shared__ int32_t s_min;
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = atomicAdd(&a.done[inst], 1u) == gridDim.x - 1;
            __syncthreads();
            if (s_last) {
                __threadfence();
                pt_exchange_block(a.x, inst, sweep, tid, nthreads, &s_min);
                if (tid == 0) a.done[inst] = 0;
            }
        }
    }
}

// Tuning knob SG_DRAW_ALWAYS (default 1): compute the draws unconditionally in the
// padding-free variants (0: only when some lane of the warp needs one).
bool draw_always()
{
    static const bool v = [] {
        const char* e = getenv("SG_DRAW_ALWAYS");
        return !(e && atoi(e) == 0);
    }();
    return v;
}

struct SweepShape {
    dim3 block, grid;
    int G, CH, WG, rows_per_thread;
    int nst = 0;      // staged variant: rows in flight per warp (0: plain loads)
    size_t smem = 0;  // staged variant: dynamic shared memory per block
};

// Tuning knob SG_ROWS_STAGE: rows in flight per warp in the staged variant, 2 (default)
// or 3; 0 turns the staged variant off.  Read at every launch.
int stage_depth()
{
    const char* e = getenv("SG_ROWS_STAGE");
    const int d = e ? atoi(e) : 2;
    return (d == 0 || d == 3) ? d : 2;
}

// Tuning knob: largest number of 4-word chunks per thread (1 or 2), from the
// environment variable SG_SWEEP_MAX_CH (default 2).
int max_chunks()
{
    static const int v = [] {
        const char* e = getenv("SG_SWEEP_MAX_CH");
        return (e && atoi(e) == 1) ? 1 : 2;
    }();
    return v;
}

// Tuning knob SG_ROWS_MINB (2, 3 or 4): resident blocks per SM the register budget is
// cut for, for the padding-free four-word variants.
int rows_min_blocks()
{
    static const int v = [] {
        const char* e = getenv("SG_ROWS_MINB");
        const int m = e ? atoi(e) : 0;
        return (m == 3 || m == 4) ? m : 2;
    }();
    return v;
}

SweepShape sweep_shape(int I, int L, int Wn, bool pt, bool pad)
{
    SweepShape sh;
    sh.WG = (Wn % 4 == 0) ? 4 : (Wn % 2 == 0) ? 2 : 1;
    sh.CH = (sh.WG == 4 && (Wn / 4) % 2 == 0 && max_chunks() == 2) ? 2 : 1;
    sh.G = Wn / (sh.WG * sh.CH);
    const int H = L / 2;
    int JX = 256 / sh.G;
    if (JX < 1) JX = 1;
    if (JX > H) JX = H;
    const int TX = sh.G * JX;
    int TY = 256 / TX;
    if (TY < 1) TY = 1;
    const int LL = L * L;
    if (TY > LL) TY = LL;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long bps = rows_min_blocks();
    // staged variant: one warp per row (a half row is exactly 32 threads' sites), rows
    // whose halves are whole 16-byte units, and room for the ring in shared memory
    if (stage_depth() > 0 && !pad && sh.WG == 4 && TX == 32 && sh.G * H == 32 && (H * Wn) % 4 == 0 &&
        rows_min_blocks() == 2 && draw_always()) {
        int per_sm = 0, per_block = 0;
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const int nst = stage_depth();
        const size_t ring = (size_t)TY * nst * 6 * (size_t)(H * Wn) * 4;
        const size_t thr = pt ? (size_t)staged_thr_words(4 * Wn) * 4 : 0;
        const size_t fixed = (pt ? 256 * 4 + 64 * 16 : kThrRow * 4 + 16) + 8 * 8 * 3 + 8 * kTieCap * 16 + 32 + 64;
        const size_t need = ring + thr;
        const long long fit = (long long)per_sm / (long long)(need + fixed + 1024);
        if ((long long)need <= per_block && fit >= 1) {
            sh.nst = nst;
            sh.smem = need;
            bps = fit < 2 ? fit : 2;
        }
    }
    // rows per thread: enough blocks for about two per SM, so that each block fills
    // its threshold table and reduces its energies once for many rows
    long long rpt = ((long long)LL * I + (long long)TY * bps * sms - 1) / ((long long)TY * bps * sms);
    if (rpt < 1) rpt = 1;
    const char* e = getenv("SG_ROWS_RPT");  // tuning knob: rows per thread
    if (e && atoi(e) >= 1) rpt = atoi(e);
    sh.rows_per_thread = (int)rpt;
    sh.block = dim3(TX, TY, 1);
    sh.grid = dim3((LL + TY * (int)rpt - 1) / (TY * (int)rpt), I, 1);
    return sh;
}

// Launches one instantiation with the shape's dynamic shared memory (raising the
// kernel's limit when the staged ring needs more than the default 48 KB).
template <typename K>
void launch_with_smem(K kernel, const SweepShape& sh, const SweepArgs& a, cudaStream_t st)
{
    if (sh.smem > 48 * 1024)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    kernel<<<sh.grid, sh.block, sh.smem, st>>>(a);
}

template <bool PT, bool UNITJ, int CH>
void launch_nopad(const SweepShape& sh, const SweepArgs& a, bool xch, cudaStream_t st)
{
    if (sh.nst == 2 || sh.nst == 3) {
        if (PT && xch)
            launch_with_smem(sh.nst == 2 ? sweep_rows_kernel<PT, UNITJ, 4, CH, false, 2, true, true, 2>
                                         : sweep_rows_kernel<PT, UNITJ, 4, CH, false, 2, true, true, 3>,
                             sh, a, st);
        else
            launch_with_smem(sh.nst == 2 ? sweep_rows_kernel<PT, UNITJ, 4, CH, false, 2, true, false, 2>
                                         : sweep_rows_kernel<PT, UNITJ, 4, CH, false, 2, true, false, 3>,
                             sh, a, st);
        return;
    }
    if (draw_always() && rows_min_blocks() == 2) {
        if (PT && xch)
            sweep_rows_kernel<PT, UNITJ, 4, CH, false, 2, true, true><<<sh.grid, sh.block, 0, st>>>(a);
        else
            sweep_rows_kernel<PT, UNITJ, 4, CH, false, 2, true><<<sh.grid, sh.block, 0, st>>>(a);
        return;
    }
    switch (rows_min_blocks()) {
    case 4:
        sweep_rows_kernel<PT, UNITJ, 4, CH, false, 4><<<sh.grid, sh.block, 0, st>>>(a);
        break;
    case 3:
        sweep_rows_kernel<PT, UNITJ, 4, CH, false, 3><<<sh.grid, sh.block, 0, st>>>(a);
        break;
    default:
        sweep_rows_kernel<PT, UNITJ, 4, CH, false, 2><<<sh.grid, sh.block, 0, st>>>(a);
    }
}

// Launches the variant for the shape; returns true when it also performed the exchange.
template <bool PT, bool UNITJ>
bool launch_variant(const SweepShape& sh, const SweepArgs& a, bool pad, bool xch, cudaStream_t st)
{
    const bool fused = xch && !pad && draw_always() && rows_min_blocks() == 2 && sh.WG == 4;
    if (sh.WG == 4 && sh.CH == 2) {
        if (pad)
            sweep_rows_kernel<PT, UNITJ, 4, 2, true><<<sh.grid, sh.block, 0, st>>>(a);
        else
            launch_nopad<PT, UNITJ, 2>(sh, a, fused, st);
    } else if (sh.WG == 4) {
        if (pad)
            sweep_rows_kernel<PT, UNITJ, 4, 1, true><<<sh.grid, sh.block, 0, st>>>(a);
        else
            launch_nopad<PT, UNITJ, 1>(sh, a, fused, st);
    } else if (sh.WG == 2) {
        sweep_rows_kernel<PT, UNITJ, 2, 1, true><<<sh.grid, sh.block, 0, st>>>(a);
    } else {
        sweep_rows_kernel<PT, UNITJ, 1, 1, true><<<sh.grid, sh.block, 0, st>>>(a);
    }
    return fused;
}

template <bool PT>
int32_t launch_rows(SweepArgs a, int I, bool unit_j, bool xch, bool* fused, cudaStream_t st)
{
    const bool pad = a.Rvalid != 4 * a.Wn;  // padding replicas in the last word
    const SweepShape sh = sweep_shape(I, a.L, a.Wn, PT, pad);
    a.G = sh.G;
    a.rows_per_thread = sh.rows_per_thread;
    a.Lmagic = (uint32_t)((0x100000000ull + (uint64_t)a.L - 1) / (uint64_t)a.L);
    a.segw = (a.L / 2) * a.Wn;
    const bool f = unit_j ? launch_variant<PT, true>(sh, a, pad, xch, st)
                          : launch_variant<PT, false>(sh, a, pad, xch, st);
    if (fused) *fused = f;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("sweep launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace

bool rows_kernel_supports(int Wn)
{
    const int WG = (Wn % 4 == 0) ? 4 : (Wn % 2 == 0) ? 2 : 1;
    const int CH = (WG == 4 && (Wn / 4) % 2 == 0 && max_chunks() == 2) ? 2 : 1;
    return Wn / (WG * CH) <= 256;
}

int32_t launch_sweep_rows_sa(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_row, bool unit_j, int I, int L, int Wn, int R,
                             uint32_t sweep, int colour, cudaStream_t st, const uint32_t* sweep_base,
                             int* status)
{
    SweepArgs a{};
    a.spins = reinterpret_cast<uint32_t*>(spins);
    a.j6_ptrs = j6_ptrs;
    a.j1_ptrs = j1_ptrs;
    a.keys = keys;
    a.thr = thr_row;
    a.L = L;
    a.Wn = Wn;
    a.Rvalid = R;
    a.sweep = sweep;
    a.colour = colour;
    a.sweep_base = sweep_base;
    a.status = status;
    return launch_rows<false>(a, I, unit_j, false, nullptr, st);
}

int32_t launch_sweep_rows_pt(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_rungs, const uint8_t* rung_of_slot, int32_t* E,
                             bool unit_j, int I, int L, int Wn, int K, uint32_t sweep, int colour,
                             const ExchangeArgs* xch, unsigned* done, bool* fused, cudaStream_t st,
                             const uint32_t* sweep_base, int* status)
{
    SweepArgs a{};
    a.spins = reinterpret_cast<uint32_t*>(spins);
    a.j6_ptrs = j6_ptrs;
    a.j1_ptrs = j1_ptrs;
    a.keys = keys;
    a.thr = thr_rungs;
    a.rung_of_slot = rung_of_slot;
    a.E = E;
    a.L = L;
    a.Wn = Wn;
    a.Rvalid = K;
    a.sweep = sweep;
    a.colour = colour;
    if (xch) a.x = *xch;
    a.done = done;
    a.sweep_base = sweep_base;
    a.status = status;
    return launch_rows<true>(a, I, unit_j, xch != nullptr, fused, st);
}

}  // namespace sg
