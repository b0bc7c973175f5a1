// ptcoop.cu -- parallel tempering (App. D.2) with every sweep of a chunk in one
// cooperative launch that holds the whole batch in the GPU's shared memory.
//
// One block per SM.  The L^2 rows (y, z) of each instance are split into contiguous
// row blocks, one per thread block (9 or 10 per instance for 16 instances on 152 SMs);
// a block keeps its rows, the L rows before them and the L rows after them (its halos:
// every neighbour of its rows lies in one of the three), and its rows' coupling sign
// bytes in shared memory for the whole chunk.  After each half sweep a block publishes the
// words it just updated in its first and last L rows to a buffer in device memory and
// raises its flag (the count of half sweeps it has completed); before the next half sweep
// it waits for the flags of the blocks before and after it (a ring within the instance)
// and copies their published rows into its halos.  After the colour-1 half sweep each
// block adds its slot energy sums (6 - 2c per site, c the satisfied count after the
// update) into the instance's sums and every block waits for all blocks of its instance:
// then each decides the exchange from those sums itself (the same draws and integer
// decisions in every block) and goes on.  Every wait polls a bounded number of times;
// when one gives up, the block sets the run's status to SG_ETIMEOUT, raises an abort word
// that every other wait also watches, and all blocks stop.  All blocks are resident at
// once (cooperative launch), so no block waits for one that cannot run.
//
// Every attempt draws the same counters as the row kernel (site, sweep, word) and the
// exchange the same counters as the stand-alone exchange (pair, sweep), so results are
// bit-identical to the row kernels and to the oracle.
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "metropolis.cuh"
#include "philox.cuh"
#include "ptslab.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

using pts::kThreads;
using pts::kWarps;

struct CoopArgs {
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
    int* status;                    // SG_ETIMEOUT when a wait gave up
    // zeroed before every launch:
    int* flags;                     // [blocks] half sweeps each block has completed in this launch
    int* sums;                      // [I][3][32] slot energy sums, by sweep mod 3
    int* abort;                     // raised when a wait gave up
    int* arrived;                   // [I] colour-1 arrivals of each instance's blocks
    uint32_t* pub;                  // [blocks][2 parity][2 side][L][L/2] published halo rows
    const int* plan;                // per block: instance, rank, first row, rows; per instance: first block, blocks
    int L, K, I, s_begin, s_end;
    long long wait_limit;           // polls before a wait gives up
    uint32_t Lmagic, Hmagic;        // ceil(2^32 / L), ceil(2^32 / (L / 2))
};

// 16 bytes global -> shared without registers (both addresses 16-byte aligned), cached in
// L2 only; cp_async_wait waits for this thread's copies
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *p >= target, polling at most wait_limit times (and stopping when the abort
// word is up).  False when it gave up.
__device__ bool wait_at_least(const CoopArgs& a, const int* p, int target)
{
    long long polls = 0;
    while (ld_acquire(p) < target) {
        if (ld_acquire(a.abort) != 0) return false;
        if (++polls > a.wait_limit) {
            atomicExch(a.abort, 1);
            atomicExch(a.status, SG_ETIMEOUT);
            return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 1) pt_coop_kernel(const CoopArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ pts::Shared sh;
    __shared__ int s_ok;

    const int b = blockIdx.x;
    const int inst = a.plan[4 * b], rank = a.plan[4 * b + 1], r0 = a.plan[4 * b + 2], nrows = a.plan[4 * b + 3];
    const int* iplan = a.plan + 4 * gridDim.x;
    const int first = iplan[2 * inst], nblk = iplan[2 * inst + 1];
    const int lower = first + (rank + nblk - 1) % nblk, upper = first + (rank + 1) % nblk;
    const int L = a.L, H = L >> 1, LL = L * L, R = LL, K = a.K;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const RunKeys key = a.keys[inst];
    const uint32_t valid = pts::valid_bits(K);

    // word array: local row lr in [-L, nrows + L) at (lr + L) * L; then the sign bytes of
    // the block's rows (logical order); then the tie queues
    uint32_t* words = reinterpret_cast<uint32_t*>(smem);
    const int max_rows = a.plan[4 * gridDim.x + 2 * a.I];
    uint8_t* sgn = smem + (size_t)(max_rows + 2 * L) * L * 4;
    uint4* s_ties = reinterpret_cast<uint4*>(smem + (((size_t)(max_rows + 2 * L) * L * 4 + (size_t)max_rows * L + 15) &
                                                     ~(size_t)15));
    uint32_t* g = a.spins + (size_t)inst * LL * L;
    const uint8_t* j1 = a.j1_ptrs[inst];

    // ---- stage the rows, the halos and the sign bytes ----
    for (int q = tid; q < (nrows + 2 * L) * L; q += kThreads) {
        const int lr = q / L - L;
        const int r = (r0 + lr + R) % R;
        words[q] = g[(size_t)r * L + (q % L)];
    }
    for (int q = tid; q < nrows * L; q += kThreads) sgn[q] = j1[(size_t)r0 * L + q];
    pts::load_state(sh, a.rung_of_slot + (size_t)inst * 32, a.slot_of_rung + (size_t)inst * K, a.thr, K,
                    a.minE[inst], tid);
    __syncthreads();
    pts::build_thresholds(sh, warp, lane);
    __syncthreads();

    // site j of local row lr in a half sweep of `colour`: its site, its words and its draws
    auto fetch = [&](int lr, int j, int colour, pts::Work& w, const pts::Updater& u) {
        const int r = r0 + lr;
        const int z = (int)__umulhi((uint32_t)r, a.Lmagic), y = r - z * L;
        const int par = (y + z + colour) & 1;
        const int rb = (lr + L) * L;
        const int is = rb + par * H + j;
        const int ho = rb + (1 - par) * H;
        w.is = is;
        w.i = (uint32_t)(r * L + 2 * j + par);
        w.self = words[is];
        w.n[0] = words[ho + (j + par == H ? 0 : j + par)];
        w.n[1] = words[ho + (j + par == 0 ? H - 1 : j + par - 1)];
        w.n[2] = words[is + (y + 1 == L ? -(L - 1) * L : L)];
        w.n[3] = words[is + (y == 0 ? (L - 1) * L : -L)];
        w.n[4] = words[is + LL];
        w.n[5] = words[is - LL];
        w.sbits = sgn[lr * L + 2 * j + par];
        u.draws(w);
    };
    // The rows within L of either end of the block (the only ones that read halo rows, and
    // the ones the neighbours' halos copy) are updated after the interior, so that the halo
    // copies run while the interior is updated.
    const int nbound = min(nrows, 2 * L);
    auto boundary_row = [&](int k) { return k < L || nrows <= 2 * L ? k : nrows - 2 * L + k; };
    // the colour-`colour` half of local row lr (global row r0 + lr, periodic)
    auto half_of = [&](int lr, int colour) {
        const int r = (r0 + lr + R) % R;
        const int z = r / L, y = r - z * L;
        return (y + z + colour) & 1;
    };
    // publishes the first and last L rows' words of `colour` (just updated)
    auto publish = [&](int h, int colour) {
        uint32_t* out = a.pub + ((size_t)b * 4 + (size_t)(h & 1) * 2) * L * H;
        for (int q = tid; q < 2 * L * H; q += kThreads) {
            const int side = q / (L * H), k = q - side * L * H;
            const int row = k / H, j = k - row * H;
            const int lr = side ? nrows - L + row : row;
            out[q] = words[(lr + L) * L + half_of(lr, colour) * H + j];
        }
    };
    // starts copying the neighbours' published rows of `colour` (half sweep h) into the
    // halos: 16-byte asynchronous copies, completed by cp_async_wait before the halos are read
    auto copy_halos_async = [&](int h, int colour) {
        const uint32_t* lo = a.pub + ((size_t)lower * 4 + (size_t)(h & 1) * 2 + 1) * L * H;  // its last L rows
        const uint32_t* hi = a.pub + ((size_t)upper * 4 + (size_t)(h & 1) * 2) * L * H;      // its first L rows
        const int C4 = H / 4;  // 16-byte chunks of a half row
        for (int q = tid; q < 2 * L * C4; q += kThreads) {
            const int side = q / (L * C4), k = q - side * L * C4;
            const int row = k / C4, c = k - row * C4;
            const int lr = side ? nrows + row : row - L;
            cp_async16(words + (lr + L) * L + half_of(lr, colour) * H + 4 * c, (side ? hi : lo) + row * H + 4 * c);
        }
        cp_async_commit();
    };
    // raises this block's flag: its boundary rows of half sweep h are published
    auto raise_flag = [&](int h) {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release(a.flags + b, h + 1);
        }
    };
    // waits (two lanes side by side) until both neighbours have published half sweep h - 1;
    // true when the wait completed
    auto wait_neighbours = [&](int h) -> bool {
        if (warp == 0) {
            bool done = true;
            if (lane < 2) done = wait_at_least(a, a.flags + (lane ? upper : lower), h);
            done = __all_sync(0xFFFFFFFFu, done);
            if (lane == 0) {
                s_ok = done ? 1 : 0;
                __threadfence();
            }
        }
        __syncthreads();
        return s_ok != 0;
    };
    // arrives at the instance's barrier (its energy sums are in) and waits for every block
    // of the instance through the arrival counter; true when the wait completed
    int barriers = 0;
    auto instance_barrier = [&]() -> bool {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.arrived + inst, 1);
            s_ok = wait_at_least(a, a.arrived + inst, nblk * (barriers + 1)) ? 1 : 0;
            __threadfence();
        }
        __syncthreads();
        ++barriers;
        return s_ok != 0;
    };
    // one phase of a half sweep: `nrow` rows, row k at local row row_of(k)
    auto phase = [&](pts::Updater& u, int colour, int nrow, auto row_of) {
        const int n = nrow * H;  // a multiple of 32
        for (int it = warp; 32 * it < n; it += kWarps) {
            const int q = 32 * it + lane;
            const int k = H == 1 ? q : (int)__umulhi((uint32_t)q, a.Hmagic);
            pts::Work w;
            fetch(row_of(k), q - k * H, colour, w, u);
            u.update(w);
            u.maybe_resolve();
        }
        u.resolve();
    };

    bool ok = true;
    int h = 0;  // half sweeps begun in this launch
    for (uint32_t sweep = (uint32_t)a.s_begin; ok && (int)sweep < a.s_end; ++sweep) {
        for (int colour = 0; colour < 2; ++colour, ++h) {
            pts::Updater u(sh, words, s_ties, key, valid, sweep, tid, colour == 1);
            if (h > 0) {  // the neighbours' rows of the previous half sweep into the halos
                ok = wait_neighbours(h);
                if (!ok) break;
                copy_halos_async(h - 1, colour ^ 1);
            }
            phase(u, colour, nrows - nbound, [&](int k) { return L + k; });
            cp_async_wait();
            __syncthreads();
            phase(u, colour, nbound, boundary_row);
            __syncthreads();
            publish(h, colour);
            raise_flag(h);
            if (colour == 1) {
                u.energy_to_block();
                __syncthreads();
                if (tid < 32) {
                    atomicAdd(a.sums + ((size_t)inst * 3 + sweep % 3) * 32 + tid, sh.E[tid]);
                    sh.E[tid] = 0;
                }
                ok = instance_barrier();
                if (!ok) break;
                // the exchange, decided by every block from its instance's sums (App. D.2)
                if (warp == 0) {
                    const int Eq = __ldcg(a.sums + ((size_t)inst * 3 + sweep % 3) * 32 + lane);
                    pts::exchange(sh, Eq, sweep, K, key, a.xtab, a.xoff, a.xlen, a.xtail, rank == 0, lane);
                    if (rank == 0) {
                        // every block read the sums of sweep - 1 before it arrived at this
                        // sweep's barrier: clear that buffer for sweep + 2
                        a.sums[((size_t)inst * 3 + (sweep + 2) % 3) * 32 + lane] = 0;
                        if ((int)sweep + 1 == a.s_end) a.E[(size_t)inst * 32 + lane] = Eq;
                    }
                }
                pts::build_thresholds(sh, warp, lane);
            }
            __syncthreads();
        }
    }

    if (!ok) {
        // release every block that may wait on this one; results are not written
        if (tid == 0) st_release(a.flags + b, 0x3FFFFFFF);
        return;
    }
    for (int q = tid; q < nrows * L; q += kThreads) g[(size_t)r0 * L + q] = words[(size_t)L * L + q];
    if (rank == 0 && warp == 0)
        pts::store_state(sh, a.rung_of_slot + (size_t)inst * 32, a.slot_of_rung + (size_t)inst * K,
                         a.accepts + (size_t)inst * (K - 1), a.minE + inst, K, lane);
}

size_t coop_smem(int L, int max_rows)
{
    return (((size_t)(max_rows + 2 * L) * L * 4 + (size_t)max_rows * L + 15) & ~(size_t)15) + pts::kTieBytes;
}

}  // namespace

// The block plan of a cooperative PT run of I instances of side L (K <= 32, unit
// couplings, L a multiple of 8): blocks per instance (as even as the SM count allows, at
// most L each, so that every block holds at least L rows) and their row ranges (multiples
// of 32 / gcd(L/2, 32) rows, so a block's sites of one colour fill whole warps).  Empty when the form does
// not apply or its shared memory does not fit.
std::vector<int> pt_coop_plan(int I, int L, int K, int* blocks, size_t* smem_bytes)
{
    std::vector<int> plan;
    *blocks = 0;
    // L a multiple of 8: a block's first and last L rows then hold a multiple of 32 sites of
    // a colour, so both phases of a half sweep fill whole warps
    if (K < 1 || K > 32 || L < 8 || (L % 8) || I < 1) return plan;
    int dev = 0, sms = 0, smem = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int H = L / 2, R = L * L;
    const int m = 32 / std::gcd(H, 32);  // rows per unit
    const int units = R / m;
    if (R % m) return plan;
    const int per_inst_max = std::min(L, units);
    if (sms < I) return plan;
    std::vector<int> nb(I);
    int G = 0;
    for (int i = 0; i < I; ++i) {
        nb[i] = std::min(per_inst_max, sms / I + (i < sms % I ? 1 : 0));
        G += nb[i];
    }
    int max_rows = 0;
    std::vector<int> blk;
    for (int i = 0; i < I; ++i)
        for (int k = 0; k < nb[i]; ++k) {
            const int u0 = (int)((long long)k * units / nb[i]), u1 = (int)((long long)(k + 1) * units / nb[i]);
            const int rows = (u1 - u0) * m;
            if (rows < L) return plan;
            max_rows = std::max(max_rows, rows);
            blk.insert(blk.end(), {i, k, u0 * m, rows});
        }
    const size_t bytes = coop_smem(L, max_rows);
    if (bytes + 8 * 1024 > (size_t)smem) return plan;
    if (cudaFuncSetAttribute(pt_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pt_coop_kernel, kThreads, bytes) != cudaSuccess) {
        cudaGetLastError();
        return plan;
    }
    if (per_sm < 1 || G > per_sm * sms) return plan;
    plan = blk;
    int f = 0;
    for (int i = 0; i < I; ++i) {
        plan.push_back(f);
        plan.push_back(nb[i]);
        f += nb[i];
    }
    plan.push_back(max_rows);
    *blocks = G;
    *smem_bytes = bytes;
    return plan;
}

int32_t launch_pt_coop(int8_t* spins, const uint8_t* const* j1_ptrs, const RunKeys* keys, const uint32_t* thr,
                       uint8_t* rung_of_slot, uint8_t* slot_of_rung, int32_t* E, unsigned long long* accepts,
                       int32_t* minE, const ExchangeTablesDev& xt, int* status, const CoopScratch& cs, int I,
                       int L, int K, int blocks, size_t smem_bytes, int s_begin, int s_end, long long wait_limit,
                       cudaStream_t st)
{
    CoopArgs a{};
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
    a.flags = cs.flags;
    a.sums = cs.sums;
    a.abort = cs.abort;
    a.arrived = cs.arrived;
    a.pub = cs.pub;
    a.plan = cs.plan;
    a.L = L;
    a.K = K;
    a.I = I;
    a.s_begin = s_begin;
    a.s_end = s_end;
    a.wait_limit = wait_limit;
    const int H = L / 2;
    a.Hmagic = H == 1 ? 0u : (uint32_t)((0x100000000ull + (uint64_t)H - 1) / (uint64_t)H);
    a.Lmagic = (uint32_t)((0x100000000ull + (uint64_t)L - 1) / (uint64_t)L);
    // the waits count half sweeps of this launch: flags, sums and the abort word start at 0
    SG_TRY_CUDA(cudaMemsetAsync(cs.flags, 0, sizeof(int) * (size_t)blocks, st));
    SG_TRY_CUDA(cudaMemsetAsync(cs.sums, 0, sizeof(int) * (size_t)I * 3 * 32, st));
    SG_TRY_CUDA(cudaMemsetAsync(cs.abort, 0, sizeof(int), st));
    SG_TRY_CUDA(cudaMemsetAsync(cs.arrived, 0, sizeof(int) * (size_t)I, st));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, pt_coop_kernel, a);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("pt_coop_kernel launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace sg
