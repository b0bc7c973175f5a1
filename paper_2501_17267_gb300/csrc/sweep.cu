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
#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kThrStride = 17;   // per-slot threshold row stride in shared memory (bank spread)

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
};

template <bool PT, bool UNITJ, int WG, int CH, bool PAD, int MINB = 2, bool DRAW = false,
          bool XCH = false>
__global__ void __launch_bounds__(256, MINB) sweep_rows_kernel(const SweepArgs a)
{
    __shared__ uint32_t s_thr[PT ? 256 * kThrStride : kThrRow];
    __shared__ int s_dE[PT ? 256 : 1];

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
    __syncthreads();

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
                if (mp::update_words<PT, WG, kThrStride, DRAW>(self, P, vmask[ch], cp.msum, (uint32_t)i,
                                                         sweep, (uint32_t)w0, key, thr, acc[ch]))
                    mp::store_words<WG>(s + (size_t)is * Wn + w0, self);
            }
            if (PT && ++items == mp::kLaneCapacity<KMAX>) {
                flush();
                items = 0;
            }
        }
    }

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

struct SweepShape {
    dim3 block, grid;
    int G, CH, WG, rows_per_thread;
};

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

SweepShape sweep_shape(int I, int L, int Wn)
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
    // rows per thread: enough blocks for about two per SM, so that each block fills
    // its threshold table and reduces its energies once for many rows
    const long long bps = rows_min_blocks();
    long long rpt = ((long long)LL * I + (long long)TY * bps * sms - 1) / ((long long)TY * bps * sms);
    if (rpt < 1) rpt = 1;
    const char* e = getenv("SG_ROWS_RPT");  // tuning knob: rows per thread
    if (e && atoi(e) >= 1) rpt = atoi(e);
    sh.rows_per_thread = (int)rpt;
    sh.block = dim3(TX, TY, 1);
    sh.grid = dim3((LL + TY * (int)rpt - 1) / (TY * (int)rpt), I, 1);
    return sh;
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

template <bool PT, bool UNITJ, int CH>
void launch_nopad(const SweepShape& sh, const SweepArgs& a, bool xch, cudaStream_t st)
{
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
    const SweepShape sh = sweep_shape(I, a.L, a.Wn);
    a.G = sh.G;
    a.rows_per_thread = sh.rows_per_thread;
    a.Lmagic = (uint32_t)((0x100000000ull + (uint64_t)a.L - 1) / (uint64_t)a.L);
    const bool pad = a.Rvalid != 4 * a.Wn;  // padding replicas in the last word
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
                             uint32_t sweep, int colour, cudaStream_t st, const uint32_t* sweep_base)
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
                             const uint32_t* sweep_base)
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
    return launch_rows<true>(a, I, unit_j, xch != nullptr, fused, st);
}

}  // namespace sg
