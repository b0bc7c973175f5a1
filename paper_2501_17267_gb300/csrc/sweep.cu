// sweep.cu -- one Metropolis half sweep (one checkerboard colour) of every replica of a
// group of instances, spins bit-packed 32 replicas to a word (App. D.1 / D.2).
//
// Work layout:
//   blockIdx.y         instance
//   blockIdx.x, ty     lattice rows (y, z), dealt out grid-stride: thread (bx, ty) takes
//                      rows (c * gridDim.x + bx) * blockDim.y + ty, c < rows_per_thread, so
//                      the blocks of an instance move through the lattice together and the
//                      +-z neighbour rows they read are still in L2
//   tx = j * G + g     site j of the row's colour (colour-split storage: the sites of one
//                      colour in a row are contiguous) and its words g, g + G, ...
// Each (site, word) item loads its own word and the six neighbour words, counts the
// satisfied bonds of all 32 replicas with a bit-sliced adder, compares the leading draw
// bytes with the threshold bytes plane by plane (metropolis.cuh), and stores the word
// back when a replica flipped.  Draws whose leading byte ties with the threshold's are
// queued per warp and decided later, together: sites of one colour never read one
// another within a half sweep, so a late flip changes nothing else.
//
// Parallel tempering: the colour-1 launch also sums every slot's energy afresh: each bond
// joins a colour-0 and a colour-1 site, so E = sum over colour-1 sites of
// s_i sum_q J_q s_q, which for |J| = 1 is 6 - 2c with c the satisfied count after the
// update (kept in bit-sliced vertical counters, reduced through a warp bit transpose).
// The colour-0 launch clears E; the block that finishes the colour-1 launch last for an
// instance performs that instance's replica exchange (exchange.cuh).
//
// Consecutive launches overlap through programmatic dependent launch: every launch waits
// for its predecessor to complete (griddepcontrol.wait) before it reads spins, energies or
// the slot permutation, and only then lets its successor launch.  The successor's blocks
// take the SMs its predecessor's blocks leave during their tail, so the launch gap and,
// in a colour-1 launch, the threshold-table setup are hidden: that setup reads only the
// slot permutation, last written by the exchange two launches back, which has completed
// when the successor's launch is allowed.
#include <stdint.h>
#include <stdlib.h>

#include "exchange.cuh"
#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

// Resident 256-thread blocks per SM the register allocation is sized for.  Two (up to
// 128 registers) measured faster than three (80 registers) for the PT colour-0 launch,
// where three fit without spills: the extra warps do not make up for the lost overlap.
#ifndef SG_SWEEP_MINB
#define SG_SWEEP_MINB 2
#endif
#ifndef SG_SWEEP_MINB_E
#define SG_SWEEP_MINB_E 2
#endif
constexpr int kThrStride = 17;  // per-slot threshold row stride in shared memory (bank spread)
constexpr int kTieCap = 64;     // queued tie entries per warp
// A warp with one item per thread and row adds at most 32 entries a row (about 1.6 on
// average), so it decides its queue only once it is nearly full: at 60 entries, 2.7 %
// faster on the 16 x L=64 x 32-temperature workload than at 32 (a full queue decides
// the overflowing ties on the spot, which is slower again).  Other loops decide it half full.
constexpr int kTieResolvePipe = kTieCap - 4;
constexpr int kVBits = 10;      // planes of the per-thread energy counters
constexpr int kPlanes = 28;     // threshold planes kept per word
constexpr int kVItems = ((1 << kVBits) - 1) / 6;  // items a counter holds before a fold

struct SweepArgs {
    uint32_t* spins;                 // [I][N][Wn] words, storage order
    const uint2* const* j6_ptrs;     // per instance: [N] records of the six int8 couplings
    const uint8_t* const* j1_ptrs;   // per instance: [N] sign bits (used when all |J| = 1)
    const RunKeys* keys;
    const uint32_t* thr;          // SA: one row of kThrRow ([S][kThrRow] with sweep_base); PT: [K][kThrRow]
    const uint8_t* rung_of_slot;  // PT: [I][Rp]
    int32_t* E;                   // PT: [I][Rp] energies, recomputed by colour 1
    int L, Wn, Rvalid, G, rows_per_thread;
    uint32_t Lmagic;              // ceil(2^32 / L): row / L by multiply-high
    uint32_t sweep;
    int colour;
    ExchangeArgs x;               // PT exchange performed by the last block of each instance
    unsigned* done;               // [I] blocks finished in this launch (reset by the last one)
    const uint32_t* sweep_base;   // if set, the sweep index is *sweep_base + sweep
};

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later).  Both are no-ops
// in a launch made without the programmatic-serialization attribute.
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_successor() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t valid_bits(int Rvalid, int w)
{
    const int left = Rvalid - 32 * w;
    return left >= 32 ? 0xFFFFFFFFu : left <= 0 ? 0u : (1u << left) - 1u;
}

// ENERGY: a PT colour-1 launch (sums the energies); XCH: it also performs the exchange.
// PIPE: unit couplings with one (site, word) item per thread and row; the next row's
// words are loaded while the current row is updated.  That is safe: a half sweep reads
// only words of the other colour, which no thread writes during the launch, and its own
// word, which only this thread writes.
template <bool PT, bool UNITJ, bool ENERGY, bool XCH, bool PIPE>
__global__ void __launch_bounds__(256, PT && !ENERGY ? SG_SWEEP_MINB : SG_SWEEP_MINB_E) sweep_bits_kernel(const SweepArgs a)
{
    __shared__ uint32_t s_thr[PT ? 256 * kThrStride : kThrRow];
    // per word: 24 threshold-byte planes, 3 planes "threshold has low bits" (k = 2, 4, 6), 1 spare
    __shared__ __align__(16) uint32_t s_tp[(PT ? 8 : 1) * kPlanes];
    __shared__ int s_E[PT ? 256 : 1];
    __shared__ uint4 s_ties[8 * kTieCap * 2];      // per warp: {site, storage, word index, tie}, {c0, c1, stored word, -}
    __shared__ int s_tie_n[8];

    const int inst = blockIdx.y;
    const int L = a.L, Wn = a.Wn, G = a.G;
    const int Rp = 32 * Wn;
    const int H = L >> 1;
    const int LL = L * L;
    const RunKeys key = a.keys[inst];
    // a colour-1 PT launch sets up its tables first (see the file comment); every other
    // launch reads its predecessor's results from the start
    if constexpr (!ENERGY) {
        wait_for_predecessor();
        allow_successor();
    }
    // the device sweep index is advanced between graph chunks, never between the two
    // colours of a sweep, so a colour-1 launch may read it before its wait too
    const uint32_t sweep = a.sweep + (a.sweep_base ? *a.sweep_base : 0u);
    uint32_t* __restrict__ s = a.spins + (size_t)inst * (size_t)LL * L * Wn;
    const uint8_t* __restrict__ j1 = UNITJ ? a.j1_ptrs[inst] : nullptr;
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    constexpr bool energy = ENERGY;

    if (PT) {
        for (int q = tid; q < Rp * kThrRow; q += nthreads) {
            const int slot = q / kThrRow, k = q % kThrRow;
            s_thr[slot * kThrStride + k] = a.thr[a.rung_of_slot[(size_t)inst * Rp + slot] * kThrRow + k];
        }
        for (int q = tid; q < Rp; q += nthreads) s_E[q] = 0;
        // colour 1 of this sweep sums the energies afresh
        if (a.colour == 0 && blockIdx.x == 0)
            for (int q = tid; q < Rp; q += nthreads) a.E[(size_t)inst * Rp + q] = 0;
    } else {
        // with a device sweep index, thr is the run's [S][kThrRow] schedule table
        const uint32_t* row = a.sweep_base ? a.thr + (size_t)sweep * kThrRow : a.thr;
        for (int q = tid; q < kThrRow; q += nthreads) s_thr[q] = row[q];
    }
    if (tid < 8) s_tie_n[tid] = 0;
    __syncthreads();
    if (UNITJ) {
        const int nw = PT ? Wn : 1;
        for (int q = tid; q < nw * kPlanes; q += nthreads) {
            const int w = q / kPlanes, p = q % kPlanes;
            uint32_t plane = 0;
            if (p < 27) {
                const int m = p < 24 ? p / 8 : p - 24, k = 2 + 2 * m;
                for (int b = 0; b < 32; ++b) {
                    const uint32_t th = PT ? s_thr[(32 * w + b) * kThrStride + k] : s_thr[k];
                    const uint32_t bit = p < 24 ? mp::threshold_plane_bit(th, p % 8) : (uint32_t)((th & 0xFFFFFFu) != 0u);
                    plane |= bit << b;
                }
            }
            s_tp[q] = plane;
        }
        __syncthreads();
    }
    if constexpr (ENERGY) {
        wait_for_predecessor();
        allow_successor();
    }

    const int g = threadIdx.x % G;
    const int j0 = threadIdx.x / G;
    const int JX = blockDim.x / G;
    // the 24 threshold planes of word w, read from shared memory where they are used
    auto load_tp = [&](int w, uint32_t (&tp)[24]) {
        const uint4* v = reinterpret_cast<const uint4*>(s_tp + (PT ? w : 0) * kPlanes);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const uint4 x = v[q];
            tp[4 * q] = x.x, tp[4 * q + 1] = x.y, tp[4 * q + 2] = x.z, tp[4 * q + 3] = x.w;
        }
    };
    // replicas of word w whose threshold for their satisfied count (c0, c1 of c = 4, 5, 6)
    // has nonzero low 24 bits: only those can accept on a tie of the leading bytes
    auto tie_can_accept = [&](int w, uint32_t c0, uint32_t c1) -> uint32_t {
        const uint4 z = reinterpret_cast<const uint4*>(s_tp + (PT ? w : 0) * kPlanes)[6];
        return (c1 & z.z) | (~c1 & ((c0 & z.y) | (~c0 & z.x)));
    };

    // ---- deferred ties of this thread's warp ----
    const int warp = tid >> 5, lane = tid & 31;
    const int warp_lanes = min(32, nthreads - 32 * warp);  // the block's last warp may be partial
    const unsigned wm = warp_lanes == 32 ? 0xFFFFFFFFu : (1u << warp_lanes) - 1u;
    uint4* ties = s_ties + warp * kTieCap * 2;
    auto thr_row = [&](uint32_t w) -> const uint32_t* { return PT ? s_thr + 32 * w * kThrStride : s_thr; };
    // applies the decided ties of one word (and, in a colour-1 PT launch, their energy
    // change 2k to the slots' sums).  `word` is the value the word's owner stored after
    // its other flips; a word has at most one entry and nobody else writes it, so the
    // result is stored without reading the word back.
    auto apply_ties = [&](uint32_t is, uint32_t w, uint32_t acc, uint32_t c0, uint32_t c1, uint32_t word) {
        if (!acc) return;
        s[(size_t)is * Wn + w] = word ^ acc;
        if (energy)
            for (uint32_t m = acc; m; m &= m - 1u) {
                const int b = __ffs(m) - 1;
                const int c = 4 + (int)((c0 >> b) & 1u) + 2 * (int)((c1 >> b) & 1u);
                atomicAdd(&s_E[32 * w + b], 2 * (2 * c - 6));
            }
    };
    auto resolve_list = [&]() {
        __syncwarp(wm);
        const int n = min(s_tie_n[warp], kTieCap);
        const int rank = __popc(wm & ((1u << lane) - 1u));
        for (int e = rank; e < n; e += warp_lanes) {
            const uint4 t = ties[2 * e], u = ties[2 * e + 1];
            const uint32_t acc = mp::resolve_tie_bits(t.w, u.x, u.y, thr_row(t.z), PT ? kThrStride : 0, t.x, sweep,
                                                      t.z, key.k0, key.k1);
            apply_ties(t.y, t.z, acc, u.x, u.y, u.z);
        }
        __syncwarp(wm);
        if (rank == 0) s_tie_n[warp] = 0;
        __syncwarp(wm);
    };
    // a warp stays converged through a row when it lies in one row of threads, every
    // thread of it has the same number of sites in the row, and of words per site
    const bool uniform_rows = blockDim.x % 32 == 0 && H % JX == 0 && Wn % G == 0;
    // queues the ties of one word whose owner stores `word`; when the list is full they
    // are decided here instead and the accepted ones returned, to join the word's flips
    auto queue_tie = [&](uint32_t i, uint32_t is, uint32_t w, uint32_t tie, uint32_t c0, uint32_t c1,
                         uint32_t word) -> uint32_t {
        const int pos = atomicAdd(&s_tie_n[warp], 1);
        if (pos < kTieCap) {
            ties[2 * pos] = make_uint4(i, is, w, tie);
            ties[2 * pos + 1] = make_uint4(c0, c1, word, 0u);
            return 0u;
        }
        return mp::resolve_tie_bits(tie, c0, c1, thr_row(w), PT ? kThrStride : 0, i, sweep, w, key.k0, key.k1);
    };

    // ---- energy counters (colour-1 PT launches) ----
    uint32_t V[kVBits];
#pragma unroll
    for (int j = 0; j < kVBits; ++j) V[j] = 0;
    int nitems = 0;
    auto fold_thread = [&]() {  // this thread's counters into the block sums (any time)
        for (int b = 0; b < 32; ++b) {
            const int e = 6 * nitems - 2 * mp::vcount(V, b);
            if (e) atomicAdd(&s_E[32 * g + b], e);
        }
#pragma unroll
        for (int j = 0; j < kVBits; ++j) V[j] = 0;
        nitems = 0;
    };

    // one word of one site with unit couplings: update, store, queue ties, count energy
    // A: the word's eight leading-byte draw planes
    // wp: the word's address
    auto update_unit = [&](int i, int is, int w, uint32_t* wp, uint32_t self, const uint32_t (&n)[6], uint32_t sbits,
                           const uint32_t (&A)[8]) {
        uint32_t S[6];
        mp::unit_signs(sbits, S);
        const uint32_t valid = valid_bits(a.Rvalid, w);
        uint32_t tp[24];
        load_tp(w, tp);
        uint32_t flip, tie, c0, c1, c2;
        mp::update_word_unit(self, n, S, valid, tp, A, &flip, &tie, &c0, &c1, &c2);
        tie &= tie_can_accept(w, c0, c1);  // the others reject whatever the low bits
        if (tie) flip |= queue_tie((uint32_t)i, (uint32_t)is, (uint32_t)w, tie, c0, c1, self ^ flip);
        if (energy) {
            mp::count_after_flip(flip, c0, c1, c2);
            mp::vadd3(V, c0, c1, c2);
            if (++nitems == kVItems) fold_thread();
        }
        if (flip) *wp = self ^ flip;
    };

    if constexpr (PIPE) {
        // one item per row: site j0 (JX == H) and word g (G == Wn) of rows c = 0, 1, ...
        // The next row's words are loaded and its draw planes computed while the current
        // row is updated: the Philox chains do not depend on spins, so they interleave
        // with the current update's adder and compare.
        const int j = j0, w = g;
        // every word index here is below 2^31 (L/2 * Wn <= 256 and L <= 256), so offsets
        // are 32-bit
        uint32_t* __restrict__ sw = s + w;
        struct Item {
            int i, is;
            uint32_t self, n[6], sbits, A[8];
        };
        auto fetch = [&](int row, Item& it) {
            const int z = (int)__umulhi((uint32_t)row, a.Lmagic);
            const int y = row - z * L;
            const int par = (y + z + a.colour) & 1;
            const int dyp = (y + 1 == L ? 1 - L : 1) * L, dym = (y == 0 ? L - 1 : -1) * L;
            const int dzp = (z + 1 == L ? 1 - L : 1) * LL, dzm = (z == 0 ? L - 1 : -1) * LL;
            const int rowoff = row * L;
            it.i = rowoff + 2 * j + par;
            it.is = rowoff + par * H + j;
            const int ho = rowoff + (1 - par) * H;
            const int jp = j + par == H ? 0 : j + par, jm = j + par == 0 ? H - 1 : j + par - 1;
            const int nb[6] = {ho + jp, ho + jm, it.is + dyp, it.is + dym, it.is + dzp, it.is + dzm};
            it.sbits = j1[it.i];
            it.self = sw[(uint32_t)(it.is * Wn)];
#pragma unroll
            for (int q = 0; q < 6; ++q) it.n[q] = sw[(uint32_t)(nb[q] * Wn)];
            mp::lead_planes((uint32_t)it.i, sweep, (uint32_t)w, key, it.A);
        };
        const int rstride = gridDim.x * blockDim.y;
        int row = blockIdx.x * blockDim.y + threadIdx.y;
        // rows c and c + 1 alternate between two buffers (unrolled by two: no copies)
        Item b0, b1;
        // updates the row in `cur` while fetching the next one into `nxt`; false when
        // there is no next row
        auto step = [&](int c, Item& cur, Item& nxt) -> bool {
            const int nrow = row + rstride;
            const bool more = c + 1 < a.rows_per_thread && nrow < LL;
            if (more) fetch(nrow, nxt);
            update_unit(cur.i, cur.is, w, sw + (uint32_t)(cur.is * Wn), cur.self, cur.n, cur.sbits, cur.A);
            if (uniform_rows) {
                __syncwarp(wm);
                if (s_tie_n[warp] >= kTieResolvePipe) resolve_list();
            }
            row = nrow;
            return more;
        };
        if (a.rows_per_thread > 0 && row < LL) {
            fetch(row, b0);
            for (int c = 0;; c += 2) {
                if (!step(c, b0, b1)) break;
                if (!step(c + 1, b1, b0)) break;
            }
        }
    } else {
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
                const int i = rowoff + 2 * j + par;   // logical site (counters, couplings)
                const int is = rowoff + par * H + j;  // storage position
                const int ho = rowoff + (1 - par) * H;
                const int jp = j + par == H ? 0 : j + par, jm = j + par == 0 ? H - 1 : j + par - 1;
                const int nb[6] = {ho + jp, ho + jm, is + dyp, is + dym, is + dzp, is + dzm};
                uint32_t sbits = 0;
                int J[6];
                if (UNITJ) {
                    sbits = j1[i];
                } else {
                    const uint2 r = a.j6_ptrs[inst][i];
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        J[q] = (int)(int8_t)(((q < 4 ? r.x : r.y) >> (8 * (q & 3))) & 0xFFu);
                }
                for (int w = g; w < Wn; w += G) {
                    const uint32_t self = s[(size_t)is * Wn + w];
                    uint32_t n[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) n[q] = s[(size_t)nb[q] * Wn + w];
                    uint32_t A[8];
                    mp::lead_planes((uint32_t)i, sweep, (uint32_t)w, key, A);
                    if (UNITJ) {
                        update_unit(i, is, w, s + (size_t)is * Wn + w, self, n, sbits, A);
                        continue;
                    }
                    const uint32_t valid = valid_bits(a.Rvalid, w);
                    const uint32_t flip = mp::update_word_general(self, n, J, valid, thr_row((uint32_t)w),
                                                                  PT ? kThrStride : 0, A, (uint32_t)i, sweep,
                                                                  (uint32_t)w, key);
                    if (energy) {  // slow path: each replica's s_i sum_q J_q s_q after the update
                        const uint32_t after = self ^ flip;
                        for (int b = 0; b < 32; ++b) {
                            int h = 0;
#pragma unroll
                            for (int q = 0; q < 6; ++q) h += J[q] * (((n[q] >> b) & 1u) ? -1 : 1);
                            const int e = ((after >> b) & 1u) ? -h : h;
                            if (e) atomicAdd(&s_E[32 * w + b], e);
                        }
                    }
                    if (flip) s[(size_t)is * Wn + w] = self ^ flip;
                }
            }
            if (uniform_rows) {
                __syncwarp(wm);
                if (s_tie_n[warp] >= kTieCap / 2) resolve_list();
            }
        }
    }
    resolve_list();

    if (energy) {
        if (UNITJ) {
            if (warp_lanes == 32) {
                // lane r collects replica r of every lane through a bit transpose per plane
                uint32_t T[kVBits];
#pragma unroll
                for (int jb = 0; jb < kVBits; ++jb) T[jb] = mp::warp_transpose(V[jb], lane);
                for (int w = 0; w < Wn; ++w) {
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, g == w);
                    if (!m) continue;
                    const int items = __reduce_add_sync(0xFFFFFFFFu, g == w ? nitems : 0);
                    int cnt = 0;
#pragma unroll
                    for (int jb = 0; jb < kVBits; ++jb) cnt += __popc(T[jb] & m) << jb;
                    const int e = 6 * items - 2 * cnt;
                    if (e) atomicAdd(&s_E[32 * w + lane], e);
                }
            } else {
                fold_thread();
            }
        }
        __syncthreads();
        int32_t* Ei = a.E + (size_t)inst * Rp;
        for (int q = tid; q < Rp; q += nthreads)
            if (s_E[q]) atomicAdd(&Ei[q], s_E[q]);
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

struct SweepShape {
    dim3 block, grid;
    int G, rows_per_thread;
};

// sms_hint > 0: the launch shares the GPU and gets about that many SMs
SweepShape sweep_shape(int I, int L, int Wn, int bps, int sms_hint)
{
    SweepShape sh;
    sh.G = Wn < 256 ? Wn : 256;
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
    if (sms_hint > 0 && sms_hint < sms) sms = sms_hint;
    // rows per thread: about bps blocks per SM (as many as are resident), so that each
    // block fills its threshold tables and reduces its energies once for many rows
    long long rpt = ((long long)LL * I + (long long)TY * bps * sms - 1) / ((long long)TY * (long long)bps * sms);
    if (rpt < 1) rpt = 1;
    const char* e = getenv("SG_ROWS_RPT");  // tuning knob: rows per thread
    if (e && atoi(e) >= 1) rpt = atoi(e);
    sh.rows_per_thread = (int)rpt;
    sh.block = dim3(TX, TY, 1);
    sh.grid = dim3((LL + TY * (int)rpt - 1) / (TY * (int)rpt), I, 1);
    return sh;
}

template <bool PT>
int32_t launch_rows(SweepArgs a, int I, bool unit_j, bool xch, bool* fused, cudaStream_t st, int sms_hint = 0)
{
    const bool energy = PT && a.colour == 1;
    const SweepShape sh = sweep_shape(I, a.L, a.Wn, PT && !energy ? SG_SWEEP_MINB : SG_SWEEP_MINB_E, sms_hint);
    a.G = sh.G;
    a.rows_per_thread = sh.rows_per_thread;
    a.Lmagic = (uint32_t)((0x100000000ull + (uint64_t)a.L - 1) / (uint64_t)a.L);
    // one (site, word) item per thread and row: the whole colour half row of all words
    const bool pipe = unit_j && sh.G == a.Wn && (int)sh.block.x == sh.G * (a.L / 2);
    // programmatic dependent launch (knob SG_PDL = 0 launches plainly)
    static const bool pdl = [] {
        const char* k = getenv("SG_PDL");
        return !(k && atoi(k) == 0);
    }();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = sh.grid;
    cfg.blockDim = sh.block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e;
    if (!unit_j) {
        if (!energy) e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, false, false, false, false>, a);
        else if (xch) e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, false, PT, PT, false>, a);
        else e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, false, PT, false, false>, a);
    } else if (pipe) {
        if (!energy) e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, true, false, false, true>, a);
        else if (xch) e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, true, PT, PT, true>, a);
        else e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, true, PT, false, true>, a);
    } else {
        if (!energy) e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, true, false, false, false>, a);
        else if (xch) e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, true, PT, PT, false>, a);
        else e = cudaLaunchKernelEx(&cfg, sweep_bits_kernel<PT, true, PT, false, false>, a);
    }
    if (fused) *fused = energy && xch;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("sweep launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace

int32_t launch_sweep_rows_sa(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_row, bool unit_j, int I, int L, int Wn, int R,
                             uint32_t sweep, int colour, cudaStream_t st, const uint32_t* sweep_base,
                             int* /*status*/)
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
    return launch_rows<false>(a, I, unit_j, false, nullptr, st);
}

int32_t launch_sweep_rows_pt(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_rungs, const uint8_t* rung_of_slot, int32_t* E,
                             bool unit_j, int I, int L, int Wn, int K, uint32_t sweep, int colour,
                             const ExchangeArgs* xch, unsigned* done, bool* fused, cudaStream_t st,
                             const uint32_t* sweep_base, int* /*status*/, int sms)
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
    return launch_rows<true>(a, I, unit_j, xch != nullptr && colour == 1, fused, st, sms);
}

}  // namespace sg
