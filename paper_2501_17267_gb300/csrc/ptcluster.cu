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
#include "ptslab.cuh"
#include "sg_internal.h"

namespace cg = cooperative_groups;

namespace sg {
namespace {

using pts::kThreads;
using pts::kWarps;
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
    const uint32_t* sweep_base;     // if set, sweeps run from *sweep_base + s_begin to *sweep_base + s_end
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

__global__ void __launch_bounds__(kThreads, 1) pt_cluster_kernel(const PtcArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ pts::Shared sh;
    __shared__ int s_Etot[2][32];  // block 0: the cluster's sums, by sweep parity
    __shared__ int s_fail;
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
    const uint32_t valid = pts::valid_bits(K);

    uint32_t* slab = reinterpret_cast<uint32_t*>(smem);
    uint8_t* sgn = smem + (size_t)slab_words * 4;  // [zc][L][L] sign bytes, logical order
    uint4* s_ties = reinterpret_cast<uint4*>(smem + (((size_t)slab_words * 5 + 15) & ~(size_t)15));
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
    pts::load_state(sh, a.rung_of_slot + (size_t)inst * 32, a.slot_of_rung + (size_t)inst * K, a.thr, K,
                    a.minE[inst], tid);
    if (tid < 32) {
        s_Etot[0][tid] = 0;
        s_Etot[1][tid] = 0;
    }
    __syncthreads();  // mbarrier initialised before any thread waits on it
    if (a.bulk && !mbar_wait_bounded(&s_bar, 0)) s_fail = 1;
    pts::build_thresholds(sh, warp, lane);
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
    const bool uniform = items % kThreads == 0;  // every lane of a warp has the same item count

    // item q of a colour: its site, its words (z neighbours in another block's slab at the
    // slab's faces) and its draws
    auto fetch = [&](int q, int colour, pts::Work& w, const pts::Updater& u) {
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
        u.draws(w);
    };
    // one half sweep of `colour` over this block's slab: items q = tid, tid + kThreads, ...
    auto half = [&](const int colour, uint32_t sweep) {
        pts::Updater u(sh, slab, s_ties, key, valid, sweep, tid, colour == 1);
        int m = 0;
        for (int q = tid; q < items; q += kThreads) {
            pts::Work w;
            fetch(q, colour, w, u);
            u.update(w);
            if (uniform && ++m == pts::kCheckEvery) {
                m = 0;
                u.maybe_resolve();
            }
        }
        u.resolve();
        if (colour == 1) {
            u.energy_to_block();
            __syncthreads();
            if (tid < 32) {  // the block's sums into block 0's buffer of this sweep's parity
                atomicAdd(&Etot0[(sweep & 1u) * 32 + tid], sh.E[tid]);
                sh.E[tid] = 0;
            }
        }
    };

    // a sweep base in device memory lets a captured graph replay the launch for later sweeps
    const uint32_t sb = a.sweep_base ? *a.sweep_base : 0u;
    const uint32_t s_end = sb + (uint32_t)a.s_end;
    if (!fail) {
        for (uint32_t sweep = sb + (uint32_t)a.s_begin; sweep < s_end; ++sweep) {
            half(0, sweep);
            cluster.sync();  // colour 0 complete in every slab
            // block 0 clears the other parity's buffer: every block read it after the
            // previous sweep, before the barrier above
            if (r == 0 && tid < 32) s_Etot[(sweep + 1u) & 1u][tid] = 0;
            half(1, sweep);
            cluster.sync();  // colour 1 and the energy sums complete
            // the exchange, decided by every block from the cluster's sums (App. D.2)
            if (warp == 0) {
                const int Eq = Etot0[(sweep & 1u) * 32 + lane];
                pts::exchange(sh, Eq, sweep, K, key, a.xtab, a.xoff, a.xlen, a.xtail, r == 0, lane);
                if (r == 0 && sweep + 1 == s_end) a.E[(size_t)inst * 32 + lane] = Eq;
            }
            pts::build_thresholds(sh, warp, lane);
            __syncthreads();
        }
    }

    // ---- write back ----
    if (!fail)
        for (int q = tid; q < slab_words; q += kThreads) g[q] = slab[q];
    if (r == 0 && !fail && warp == 0)
        pts::store_state(sh, a.rung_of_slot + (size_t)inst * 32, a.slot_of_rung + (size_t)inst * K,
                         a.accepts + (size_t)inst * (K - 1), a.minE + inst, K, lane);
    // after a wait that gave up, copies may still be in flight into this block's shared
    // memory: wait once more (bounded) before the block leaves
    if (fail && a.bulk) mbar_wait_bounded(&s_bar, 0);
    cluster.sync();  // no block leaves while another may still read its shared memory
}

size_t dyn_smem(int L, int C)
{
    const size_t slab_words = (size_t)(L / C) * L * L;
    return ((slab_words * 5 + 15) & ~(size_t)15) + pts::kTieBytes;
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
    const char* fc = getenv("SG_PT_CLUSTER_C");  // tuning knob: force C (when it divides L and fits)
    const int forced = fc ? atoi(fc) : 0;
    for (int C = 8; C >= 1; --C) {
        if (L % C || (forced > 0 && C != forced)) continue;
        const size_t bytes = dyn_smem(L, C);
        if (bytes + 16 * 1024 > (size_t)smem) continue;
        if (cudaFuncSetAttribute(pt_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (knob == 1 || forced > 0) return C;
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

// A batch with more instances than clusters fit at once: the first M instances on clusters
// (one wave), the other I - M through the row kernels on the SMs the clusters leave, both
// at the same time.  With the rates above, M minimises the longer of the two parts' times
// per sweep, and the split is taken when that beats the row kernels on the whole GPU.  At
// L = 64 with 16 instances of 32 temperatures: 15 clusters of 8 blocks on 120 SMs, one
// instance on the other 32.  Knob SG_PT_HYBRID = 0 turns the split off; SG_PT_CLUSTER = 0
// turns off every cluster form.
int pt_cluster_split(int I, int L, int K, int* M, int* side_sms)
{
    *M = 0;
    *side_sms = 0;
    const char* e = getenv("SG_PT_HYBRID");
    if (e && atoi(e) == 0) return 0;
    const char* c = getenv("SG_PT_CLUSTER");
    if ((c && atoi(c) == 0) || K > 32 || K < 1 || L < 2 || (L & 1) || I < 2) return 0;
    int dev = 0, smem = 0, sms = 1, clock_khz = 2070000;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
    const double hz = 1e3 * (double)clock_khz;
    const double work = (double)L * L * L * K;
    const double t_rows = 10e-6 + I * work / (sms * 6.2 * hz);
    double best = 0.95 * t_rows;
    int bestC = 0;
    for (int C = 8; C >= 1; --C) {
        if (L % C) continue;
        const size_t bytes = dyn_smem(L, C);
        if (bytes + 16 * 1024 > (size_t)smem) continue;
        if (cudaFuncSetAttribute(pt_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(L, C, 1, attr);
        int active = 0, per_sm = 0;
        if (cudaOccupancyMaxActiveClusters(&active, pt_cluster_kernel, &cfg) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pt_cluster_kernel, kThreads, bytes) !=
                cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (active >= I || active < 1 || per_sm < 1) continue;  // one wave: pt_cluster_blocks decides
        const double t_cluster = 4e-6 + work / (C * 7.9 * hz);
        for (int m = active; m >= 1; --m) {
            const int left = sms - (m * C + per_sm - 1) / per_sm;
            if (left < 1) continue;
            const double t_side = 10e-6 + (I - m) * work / (left * 6.2 * hz);
            const double t = t_cluster > t_side ? t_cluster : t_side;
            if (t < best) {
                best = t;
                bestC = C;
                *M = m;
                *side_sms = left;
            }
        }
    }
    return bestC;
}

int32_t launch_pt_cluster(int8_t* spins, const uint8_t* const* j1_ptrs, const RunKeys* keys, const uint32_t* thr,
                          uint8_t* rung_of_slot, uint8_t* slot_of_rung, int32_t* E, unsigned long long* accepts,
                          int32_t* minE, const ExchangeTablesDev& xt, int* status, int I, int L, int K, int C,
                          int s_begin, int s_end, bool bulk_signs, cudaStream_t st, const uint32_t* sweep_base)
{
    PtcArgs a{};
    a.sweep_base = sweep_base;
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
