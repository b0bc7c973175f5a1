// ptcluster.cu -- parallel tempering (App. D.2) with every sweep of a chunk in one
// launch: one thread-block cluster per instance, its lattice resident in the blocks'
// shared memory for the whole chunk.
//
// Cluster `inst` of C blocks splits the L^3 lattice of its instance into C z-slabs of
// L / C planes; block r keeps slab r (one 32-bit word of 32 slots per site, storage
// order) and the slab's coupling sign bytes in shared memory.  Both are brought in at
// the start of the launch by bulk asynchronous copies (cp.async.bulk, completion on an
// mbarrier whose wait is bounded) and the spins are written back at the end; in
// between, nothing but the exchange tables is read from global memory.  A half sweep
// reads only sites of the other colour: x and y neighbours lie in the block's own slab,
// z neighbours across a slab boundary in the next block's slab (distributed shared
// memory).  A cluster barrier separates the two half sweeps of a sweep and the sweeps.
//
// Energies and the exchange.  Each bond joins a colour-0 and a colour-1 site, so the
// colour-1 half sweep sums every slot's energy afresh (6 - 2c per site for unit
// couplings, c the satisfied count after the update), in bit-sliced counters per
// thread reduced through a warp bit transpose.  Every block adds its sums into block 0's
// shared memory (distributed atomics, one buffer per sweep parity); after the barrier
// that ends the sweep every block reads the totals and decides the exchange itself --
// the same integer decisions from the same draws -- so its slot-to-rung map and its
// threshold planes are ready for the next sweep without another barrier.  Block 0
// clears a parity's buffer one sweep later, when every block has read it.
//
// Every attempt draws the same counters as the row kernel (site, sweep, word) and the
// exchange the same counters as the stand-alone exchange (pair, sweep), so results are
// bit-identical to the row kernel and to the oracle.
#include <cooperative_groups.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>

#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace cg = cooperative_groups;

namespace sg {
namespace {

// 512 threads (128 registers, no spills): 768 or 1024 threads, and fetching the next item
// before updating the current one, measured slower (spills)
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kTieCap = 48;      // queued tie entries per warp
constexpr int kTieResolve = 16;  // a warp decides its queue from this many (a row of a warp adds <= 32)
constexpr int kThrStride = 17;   // per-slot threshold row stride in shared memory (bank spread)
constexpr int kVBits = 8;        // per-thread energy counters: up to 42 items of at most 6
constexpr int kFoldItems = 42;
// bounded waits: iterations of mbarrier.try_wait (each may suspend the thread briefly)
constexpr int kWaitSpins = 1 << 22;

struct PtcArgs {
    uint32_t* spins;                // [I][N] words (slots 0..31 of a site), storage order
    const uint8_t* const* j1_ptrs;  // per instance: [N] coupling sign bits (all |J| = 1)
    const RunKeys* keys;            // [I]
    const uint32_t* thr;            // [K][kThrRow] thresholds by rung
    uint8_t* rung_of_slot;          // [I][32]
    uint8_t* slot_of_rung;          // [I][K]
    int32_t* E;                     // [I][32] out: slot energies after the last sweep
    unsigned long long* accepts;    // [I][K-1]
    int32_t* minE;                  // [I]
    const uint32_t* xtab;           // exchange thresholds (exchange.cuh)
    const uint32_t* xoff;
    const uint32_t* xlen;
    const uint32_t* xtail;
    int* status;                    // SG_ETIMEOUT when a bounded wait gave up
    int L, K, C, s_begin, s_end;
    uint32_t Hmagic, Lmagic;        // ceil(2^32 / (L / 2)), ceil(2^32 / L)
    int bulk;                       // slabs staged by bulk copies (else by plain loads)
    int bulk_signs;                 // the sign slab is 16-byte aligned: bulk copy (else plain loads)
};

// ---- mbarrier and bulk-copy primitives (PTX, sm_90 and later) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// global -> this block's shared memory, completion counted on `bar` (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar`, giving up after kWaitSpins tries.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    for (int it = 0; it < kWaitSpins; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ uint32_t valid_bits(int K)
{
    return K >= 32 ? 0xFFFFFFFFu : (1u << K) - 1u;
}

__global__ void __launch_bounds__(kThreads, 1) pt_cluster_kernel(const PtcArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_thr[32 * kThrStride];  // per slot: thresholds of its rung, k = 0 .. 15
    __shared__ uint4 s_tp4[8];  // threshold-byte plane j of k = 2, 4, 6 (bit b: slot b)
    __shared__ uint4 s_lz;       // slots whose threshold of k = 2, 4, 6 has nonzero low 24 bits
    __shared__ uint32_t s_rthr[32 * kThrRow];     // per rung (K <= 32): the threshold rows
    __shared__ int s_E[32];                       // this block's energy sums of a colour-1 half sweep
    __shared__ int s_Etot[2][32];                 // block 0: the cluster's sums, by sweep parity
    __shared__ uint32_t s_acc[32];                // block 0: accepted swaps of rung pairs in this launch
    __shared__ uint8_t s_rung[32], s_slot[32];
    __shared__ int s_tie_n[kWarps];
    __shared__ int s_min, s_fail;
    __shared__ __align__(8) uint64_t s_bar;

    cg::cluster_group cluster = cg::this_cluster();
    const int C = a.C;
    const int r = (int)cluster.block_rank();
    const int inst = blockIdx.x / C;
    const int L = a.L, H = L >> 1, LL = L * L, K = a.K;
    const int zc = L / C, z0 = r * zc;
    const int slab_words = zc * LL;
    const int items = zc * L * H;  // sites of one colour in the slab
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const RunKeys key = a.keys[inst];
    const uint32_t valid = valid_bits(K);

    uint32_t* slab = reinterpret_cast<uint32_t*>(smem);
    uint8_t* sgn = smem + (size_t)slab_words * 4;                 // [zc][L][L] sign bytes, logical order
    uint4* s_ties = reinterpret_cast<uint4*>(smem + (((size_t)slab_words * 5 + 15) & ~(size_t)15));
    uint4* ties = s_ties + warp * kTieCap * 2;                     // per warp: {i, is, -, tie}, {c0, c1, word, -}
    uint32_t* g = a.spins + (size_t)inst * LL * L + (size_t)z0 * LL;
    const uint8_t* j1 = a.j1_ptrs[inst] + (size_t)z0 * LL;

    // ---- stage the slab and its coupling signs in shared memory ----
    if (tid == 0) {
        s_fail = 0;
        if (a.bulk) {
            mbar_init(&s_bar, 1);
            const uint32_t sp_bytes = (uint32_t)slab_words * 4u;
            const uint32_t sg_bytes = a.bulk_signs ? (uint32_t)slab_words : 0u;
            mbar_expect_tx(&s_bar, sp_bytes + sg_bytes);
            bulk_load(slab, g, sp_bytes, &s_bar);
            if (sg_bytes) bulk_load(sgn, j1, sg_bytes, &s_bar);
        }
    }
    if (!a.bulk)
        for (int q = tid; q < slab_words; q += kThreads) slab[q] = g[q];
    if (!a.bulk || !a.bulk_signs)
        for (int q = tid; q < slab_words; q += kThreads) sgn[q] = j1[q];
    if (tid < 32) {
        s_rung[tid] = a.rung_of_slot[(size_t)inst * 32 + tid];
        if (tid < K) s_slot[tid] = a.slot_of_rung[(size_t)inst * K + tid];
        s_E[tid] = 0;
        s_Etot[0][tid] = 0;
        s_Etot[1][tid] = 0;
        s_acc[tid] = 0;
    }
    for (int q = tid; q < K * kThrRow; q += kThreads) s_rthr[q] = a.thr[q];
    if (tid < kWarps) s_tie_n[tid] = 0;
    if (tid == 0) s_min = a.minE[inst];
    __syncthreads();  // mbarrier initialised before any thread waits on it
    if (a.bulk && !mbar_wait_bounded(&s_bar, 0)) s_fail = 1;
    // The slot-to-rung map gives every slot its thresholds: per slot rows for ties, and
    // the 24 + 3 bit planes of the word (bit b = slot b) the bit-sliced compare reads.
    auto build_thresholds = [&]() {
        if (warp == 0) {
            const uint32_t* row = s_rthr + (int)s_rung[lane] * kThrRow;
#pragma unroll
            for (int k = 0; k < kThrRow; ++k) s_thr[lane * kThrStride + k] = row[k];
            const uint32_t t2 = row[2], t4 = row[4], t6 = row[6];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t p2 = __ballot_sync(0xFFFFFFFFu, mp::threshold_plane_bit(t2, j) != 0u);
                const uint32_t p4 = __ballot_sync(0xFFFFFFFFu, mp::threshold_plane_bit(t4, j) != 0u);
                const uint32_t p6 = __ballot_sync(0xFFFFFFFFu, mp::threshold_plane_bit(t6, j) != 0u);
                if (lane == 0) s_tp4[j] = make_uint4(p2, p4, p6, 0u);
            }
            const uint32_t l2 = __ballot_sync(0xFFFFFFFFu, (t2 & 0xFFFFFFu) != 0u);
            const uint32_t l4 = __ballot_sync(0xFFFFFFFFu, (t4 & 0xFFFFFFu) != 0u);
            const uint32_t l6 = __ballot_sync(0xFFFFFFFFu, (t6 & 0xFFFFFFu) != 0u);
            if (lane == 0) s_lz = make_uint4(l2, l4, l6, 0u);
        }
    };
    build_thresholds();
    // Every block's slab is in place (and every block's failure flag set) before any block
    // reads a neighbour's slab.
    cluster.sync();
    int fail = 0;
    for (int q = 0; q < C; ++q) fail |= *cluster.map_shared_rank(&s_fail, q);
    if (fail && tid == 0) atomicExch(a.status, SG_ETIMEOUT);

    // slabs of the blocks above (z0 + zc) and below (z0 - 1), periodic in z
    const uint32_t* up = cluster.map_shared_rank(slab, (r + 1) % C);
    const uint32_t* dn = cluster.map_shared_rank(slab, (r + C - 1) % C);
    int* Etot0 = cluster.map_shared_rank(&s_Etot[0][0], 0);

    // ---- the sweeps ----
    const bool uniform = items % kThreads == 0;  // every lane of a warp has the same item count
    uint32_t V[kVBits];
    int nitems = 0;
    uint32_t sweep = (uint32_t)a.s_begin;

    // item q of a colour: its logical site i, slab position is, the words of the site and
    // of its six neighbours (z neighbours in another block's slab at the slab's faces),
    // its coupling sign bits and its eight leading-byte draw planes
    struct Work {
        uint32_t i;
        int is;
        uint32_t self, n[6], sbits, A[8];
    };
    auto fetch = [&](int q, int colour, Work& w) {
        const int rl = H == 1 ? q : (int)__umulhi((uint32_t)q, a.Hmagic);  // slab row
        const int j = q - rl * H;
        const int zl = (int)__umulhi((uint32_t)rl, a.Lmagic), y = rl - zl * L;
        const int par = (y + z0 + zl + colour) & 1;
        const int rowoff = rl * L;
        const int pos = par * H + j;
        const int is = rowoff + pos;
        const int ho = rowoff + (1 - par) * H;
        w.is = is;
        w.i = (uint32_t)(z0 * LL + rowoff + 2 * j + par);
        w.self = slab[is];
        w.n[0] = slab[ho + (j + par == H ? 0 : j + par)];
        w.n[1] = slab[ho + (j + par == 0 ? H - 1 : j + par - 1)];
        w.n[2] = slab[is + (y + 1 == L ? -(L - 1) * L : L)];
        w.n[3] = slab[is + (y == 0 ? (L - 1) * L : -L)];
        w.n[4] = zl + 1 == zc ? up[y * L + pos] : slab[is + LL];
        w.n[5] = zl == 0 ? dn[(zc - 1) * LL + y * L + pos] : slab[is - LL];
        w.sbits = sgn[rowoff + 2 * j + par];
        mp::lead_planes(w.i, sweep, 0u, key, w.A);
    };
    auto fold_thread = [&]() {  // this thread's counters into the block sums (rare)
        for (int b = 0; b < 32; ++b) {
            const int e = 6 * nitems - 2 * mp::vcount(V, b);
            if (e) atomicAdd(&s_E[b], e);
        }
#pragma unroll
        for (int j = 0; j < kVBits; ++j) V[j] = 0;
        nitems = 0;
    };
    // decides the queued ties of this warp (a blind store of the word its owner stored;
    // in a colour-1 half sweep a decided flip adds 2k to the slot's energy)
    auto resolve_list = [&](bool energy) {
        __syncwarp();
        const int n = min(s_tie_n[warp], kTieCap);
        for (int e = lane; e < n; e += 32) {
            const uint4 t = ties[2 * e], u = ties[2 * e + 1];
            const uint32_t acc =
                mp::resolve_tie_bits(t.w, u.x, u.y, s_thr, kThrStride, t.x, sweep, 0u, key.k0, key.k1);
            if (acc) {
                slab[t.y] = u.z ^ acc;
                if (energy)
                    for (uint32_t m = acc; m; m &= m - 1u) {
                        const int b = __ffs(m) - 1;
                        const int c = 4 + (int)((u.x >> b) & 1u) + 2 * (int)((u.y >> b) & 1u);
                        atomicAdd(&s_E[b], 2 * (2 * c - 6));
                    }
            }
        }
        __syncwarp();
        if (lane == 0) s_tie_n[warp] = 0;
        __syncwarp();
    };
    auto update = [&](Work& w, bool energy) {
        uint32_t flip, tie, c0, c1, c2;
        mp::update_word_unit_smem(w.self, w.n, w.sbits, valid, s_tp4, w.A, &flip, &tie, &c0, &c1, &c2);
        {
            const uint4 z = s_lz;
            tie &= (c1 & z.z) | (~c1 & ((c0 & z.y) | (~c0 & z.x)));  // the others reject
        }
        if (tie) {
            const int p = atomicAdd(&s_tie_n[warp], 1);
            if (p < kTieCap) {
                ties[2 * p] = make_uint4(w.i, (uint32_t)w.is, 0u, tie);
                ties[2 * p + 1] = make_uint4(c0, c1, w.self ^ flip, 0u);
            } else {  // queue full: decide here
                const uint32_t acc =
                    mp::resolve_tie_bits(tie, c0, c1, s_thr, kThrStride, w.i, sweep, 0u, key.k0, key.k1);
                flip |= acc;
            }
        }
        if (energy) {
            mp::count_after_flip(flip, c0, c1, c2);
            mp::vadd3(V, c0, c1, c2);
            if (++nitems == kFoldItems) fold_thread();
        }
        if (flip) slab[w.is] = w.self ^ flip;
    };
    // one half sweep of `colour` over this block's slab: items q = tid, tid + kThreads, ...
    auto half = [&](const int colour) {
        const bool energy = colour == 1;
        if (energy) {
#pragma unroll
            for (int j = 0; j < kVBits; ++j) V[j] = 0;
            nitems = 0;
        }
        for (int q = tid; q < items; q += kThreads) {
            Work w;
            fetch(q, colour, w);
            update(w, energy);
            if (uniform) {
                __syncwarp();
                if (s_tie_n[warp] >= kTieResolve) resolve_list(energy);
            }
        }
        resolve_list(energy);
        if (energy) {
            // lane b collects slot b of every lane through a bit transpose per plane
            uint32_t T[kVBits];
#pragma unroll
            for (int jb = 0; jb < kVBits; ++jb) T[jb] = mp::warp_transpose(V[jb], lane);
            const int n = __reduce_add_sync(0xFFFFFFFFu, nitems);
            int cnt = 0;
#pragma unroll
            for (int jb = 0; jb < kVBits; ++jb) cnt += __popc(T[jb]) << jb;
            const int e = 6 * n - 2 * cnt;
            if (e) atomicAdd(&s_E[lane], e);
            __syncthreads();
            if (tid < 32) {  // the block's sums into block 0's buffer of this sweep's parity
                atomicAdd(&Etot0[(sweep & 1u) * 32 + tid], s_E[tid]);
                s_E[tid] = 0;
            }
        }
    };

    if (!fail) {
        for (; (int)sweep < a.s_end; ++sweep) {
            half(0);
            cluster.sync();  // colour 0 complete in every slab
            // block 0 clears the other parity's buffer: every block read it after the
            // previous sweep, before the barrier above
            if (r == 0 && tid < 32) s_Etot[(sweep + 1u) & 1u][tid] = 0;
            half(1);
            cluster.sync();  // colour 1 and the energy sums complete
            // the exchange, decided by every block from the cluster's sums (App. D.2)
            if (warp == 0) {
                const int Eq = Etot0[(sweep & 1u) * 32 + lane];
                const int k = 2 * lane + (int)(sweep & 1u);
                const bool pair = k + 1 < K;
                const int sa = pair ? s_slot[k] : 0, sb = pair ? s_slot[k + 1] : 0;
                const int Ea = __shfl_sync(0xFFFFFFFFu, Eq, sa), Eb = __shfl_sync(0xFFFFFFFFu, Eq, sb);
                if (pair) {
                    const int64_t d = (int64_t)Ea - (int64_t)Eb;
                    bool accept = d <= 0;
                    if (!accept) {
                        const uint32_t u =
                            philox4x32_10((uint32_t)k, sweep, 0u, kDomainExchange, key.k0, key.k1).v[0];
                        const uint32_t T =
                            d <= (int64_t)a.xlen[k] ? a.xtab[a.xoff[k] + (uint32_t)(d - 1)] : a.xtail[k];
                        accept = u < T;
                    }
                    if (accept) {
                        s_rung[sa] = (uint8_t)(k + 1);
                        s_rung[sb] = (uint8_t)k;
                        s_slot[k] = (uint8_t)sb;
                        s_slot[k + 1] = (uint8_t)sa;
                        if (r == 0) s_acc[k] += 1u;
                    }
                }
                int m = lane < K ? Eq : 0x7FFFFFFF;
                m = __reduce_min_sync(0xFFFFFFFFu, m);
                if (lane == 0 && m < s_min) s_min = m;
                if (r == 0 && (int)sweep + 1 == a.s_end) a.E[(size_t)inst * 32 + lane] = Eq;
                __syncwarp();
            }
            build_thresholds();
            __syncthreads();
        }
    }

    // ---- write back ----
    if (!fail)
        for (int q = tid; q < slab_words; q += kThreads) g[q] = slab[q];
    if (r == 0 && !fail && tid < 32) {
        a.rung_of_slot[(size_t)inst * 32 + tid] = s_rung[tid];
        if (tid < K) a.slot_of_rung[(size_t)inst * K + tid] = s_slot[tid];
        if (tid + 1 < K) a.accepts[(size_t)inst * (K - 1) + tid] += (unsigned long long)s_acc[tid];
        if (tid == 0) a.minE[inst] = s_min;
    }
    // after a wait that gave up, copies may still be in flight into this block's shared
    // memory: wait once more (bounded) before the block leaves
    if (fail && a.bulk) mbar_wait_bounded(&s_bar, 0);
    cluster.sync();  // no block leaves while another may still read its shared memory
}

size_t dyn_smem(int L, int C)
{
    const size_t slab_words = (size_t)(L / C) * L * L;
    return ((slab_words * 5 + 15) & ~(size_t)15) + (size_t)kWarps * kTieCap * 2 * sizeof(uint4);
}

cudaLaunchConfig_t cluster_config(int L, int C, int I, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C * I, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = dyn_smem(L, C);
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

// Blocks per cluster for a PT run of I instances of side L with K <= 32 temperatures and
// unit couplings, or 0 when the row kernels should run it.  C is the largest divisor
// C <= 8 of L whose slab fits shared memory and for which all I clusters are resident at
// once (one wave).  The cluster form is taken when its estimated time per sweep is below
// the row kernels', from rates measured on a GB300 (K = 32, L = 8 ... 64, I = 1 ... 15):
// a cluster sweeps about 7.9 attempts per SM clock with about 4 us of fixed cost per sweep
// (barriers, exchange); the row kernels about 6.2 attempts per SM clock over the whole GPU
// with about 10 us per sweep of launch cost.  So it wins for small lattices (L <= 24
// always, L = 32 from a few instances) and, at L = 64, for 15 instances.  Knob
// SG_PT_CLUSTER = 0 turns the form off, = 1 takes it whenever a slab fits.
int pt_cluster_blocks(int I, int L, int K)
{
    const char* e = getenv("SG_PT_CLUSTER");
    const int knob = e ? atoi(e) : -1;
    if (knob == 0 || K > 32 || K < 1 || L < 2 || (L & 1) || I < 1) return 0;
    int dev = 0, smem = 0, sms = 1, clock_khz = 2070000;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
    const double hz = 1e3 * (double)clock_khz;
    for (int C = 8; C >= 1; --C) {
        if (L % C) continue;
        const size_t bytes = dyn_smem(L, C);
        if (bytes + 16 * 1024 > (size_t)smem) continue;
        if (cudaFuncSetAttribute(pt_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (knob == 1) return C;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(L, C, 1, attr);
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, pt_cluster_kernel, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (active < I) continue;
        const double work = (double)L * L * L * K;  // attempts per sweep of one instance
        const double t_cluster = 4e-6 + work / (C * 7.9 * hz);
        const double t_rows = 10e-6 + I * work / (sms * 6.2 * hz);
        return t_cluster < 0.95 * t_rows ? C : 0;
    }
    return 0;
}

int32_t launch_pt_cluster(int8_t* spins, const uint8_t* const* j1_ptrs, const RunKeys* keys, const uint32_t* thr,
                          uint8_t* rung_of_slot, uint8_t* slot_of_rung, int32_t* E, unsigned long long* accepts,
                          int32_t* minE, const ExchangeTablesDev& xt, int* status, int I, int L, int K, int C,
                          int s_begin, int s_end, bool bulk_signs, cudaStream_t st)
{
    PtcArgs a{};
    a.spins = reinterpret_cast<uint32_t*>(spins);
    a.j1_ptrs = j1_ptrs;
    a.keys = keys;
    a.thr = thr;
    a.rung_of_slot = rung_of_slot;
    a.slot_of_rung = slot_of_rung;
    a.E = E;
    a.accepts = accepts;
    a.minE = minE;
    a.xtab = xt.tab;
    a.xoff = xt.off;
    a.xlen = xt.len;
    a.xtail = xt.tail;
    a.status = status;
    a.L = L;
    a.K = K;
    a.C = C;
    a.s_begin = s_begin;
    a.s_end = s_end;
    const int H = L / 2;
    a.Hmagic = H == 1 ? 0u : (uint32_t)((0x100000000ull + (uint64_t)H - 1) / (uint64_t)H);
    a.Lmagic = (uint32_t)((0x100000000ull + (uint64_t)L - 1) / (uint64_t)L);
    // the sign bytes of a slab start at z0 * L^2 bytes into the instance's array: a bulk
    // copy needs its address and size to be multiples of 16
    a.bulk_signs = bulk_signs && ((size_t)(L / C) * L * L) % 16 == 0;
    // knob SG_PT_BULK = 0: plain loads instead of bulk copies (for comparison)
    static const bool bulk = [] {
        const char* k = getenv("SG_PT_BULK");
        return !(k && atoi(k) == 0);
    }();
    a.bulk = bulk ? 1 : 0;
    const size_t smem = dyn_smem(L, C);
    if (cudaFuncSetAttribute(pt_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        set_error("pt_cluster_kernel: cannot use %zu bytes of shared memory", smem);
        return SG_ECUDA;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(L, C, I, attr);
    cfg.stream = st;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, pt_cluster_kernel, a);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("pt_cluster_kernel launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace sg
