// cluster.cu -- simulated annealing (App. D.1) of small lattices with many replicas:
// one launch runs every sweep, each word of 32 replicas on its own thread-block cluster.
//
// A half sweep of a small lattice is too little work to pay for a launch, and a whole
// lattice per block (batch.cu) leaves most SMs idle when an instance has few words.
// Here cluster (word w, instance) of C blocks splits the lattice into C slabs of L / C
// z-planes; block r keeps slab r of word w in its shared memory for the whole run.  The
// sites of one colour read only sites of the other colour: x and y neighbours lie in
// the block's own slab, z neighbours across a slab boundary in the next block's slab,
// read through distributed shared memory.  A cluster barrier separates half sweeps.
// Every attempt draws the same counters as the row kernel (site, sweep, word), so the
// results are bit-identical to it and to the oracle.
#include <cooperative_groups.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <cstdint>

#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace cg = cooperative_groups;

namespace sg {
namespace {

// Single runs: 256 or 512 threads a block, chosen with the cluster size (sa_cluster_blocks).
// Batches (planes of up to L = 48 per cluster, tens of words per thread per half sweep):
// 768 threads per block measured fastest on the 512-instance uneven batch -- 1.95 s per
// step against 2.10 at 512, 1.97 at 1024 and 2.89 at 256 -- although at 85 registers a
// thread spills about 100 bytes: more warps hide the update's dependencies better.
constexpr int kListBlock = 768;
constexpr int kTieCap = 32;  // queued tie entries per warp

struct ClusterArgs {
    uint32_t* spins;                // [I][N][Wn] words, storage order
    const uint8_t* const* j1_ptrs;  // per instance: [N] coupling sign bits (all |J| = 1)
    const RunKeys* keys;            // [I]
    const uint32_t* thr;            // [S][kThrRow]
    int L, Wn, R, S, C;             // side, words, replicas, sweeps, blocks per cluster
    uint32_t Hmagic;                // ceil(2^32 / (L / 2))
};

__device__ __forceinline__ uint32_t word_valid_bits(int R, int w)
{
    const int left = R - 32 * w;
    return left >= 32 ? 0xFFFFFFFFu : left <= 0 ? 0u : (1u << left) - 1u;
}

// One word of one lattice, annealed by a cluster of C blocks (block r: z-slab r): the
// plane's word of site s is g[s * stride]; the draws use word index w of the instance.
struct PlaneRun {
    uint32_t* g;
    int stride;
    const uint8_t* j1;    // [N] coupling sign bits (all |J| = 1)
    const uint32_t* thr;  // [S][kThrRow]
    RunKeys key;
    int L, w, R, s_begin, s_end;  // side, word, replicas of the instance, sweeps [s_begin, s_end)
    uint32_t Hmagic;              // ceil(2^32 / (L / 2))
};

// Called by every thread of every block of the cluster; slab: dynamic shared memory of
// at least (L / C) * L * L words.  Ends with the plane written back and a cluster barrier.
template <int NT>
__device__ __forceinline__ void anneal_plane(const PlaneRun& p, const int C, uint32_t* slab, uint4* s_ties,
                                             int* s_tie_n)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int w = p.w;
    const int L = p.L, H = L >> 1, LL = L * L;
    const int zc = L / C;              // z-planes per slab
    const int slab_words = zc * LL;
    const int z0 = r * zc;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const RunKeys key = p.key;
    const uint8_t* __restrict__ j1 = p.j1;
    uint32_t* __restrict__ g = p.g;
    // slabs of the blocks above (z0 + zc) and below (z0 - 1), periodic in z
    const uint32_t* up = cluster.map_shared_rank(slab, (r + 1) % C);
    const uint32_t* dn = cluster.map_shared_rank(slab, (r + C - 1) % C);
    const uint32_t valid = word_valid_bits(p.R, w);
    uint4* ties = s_ties + warp * kTieCap * 2;
    const int items = zc * L * H;  // sites of one colour in the slab

    // geometry of slab item q (site j of slab row rl) in a half sweep of colour `colour`:
    // its slab position, its six neighbours' (z neighbours in another block's slab when
    // `zup` / `zdn`), its logical index and its coupling sign bits
    struct Site {
        int is, nb[6];
        bool zup, zdn;
        uint32_t i, sbits;
    };
    auto site_of = [&](int q, int colour) {
        Site t;
        const int rl = H == 1 ? q : (int)__umulhi((uint32_t)q, p.Hmagic);
        const int j = q - rl * H;
        const int zl = rl / L, y = rl - zl * L;
        const int z = z0 + zl;
        const int par = (y + z + colour) & 1;
        const int rowoff = rl * L;
        const int pos = par * H + j;
        t.is = rowoff + pos;
        const int ho = rowoff + (1 - par) * H;
        t.nb[0] = ho + (j + par == H ? 0 : j + par);
        t.nb[1] = ho + (j + par == 0 ? H - 1 : j + par - 1);
        t.nb[2] = t.is + (y + 1 == L ? -(L - 1) * L : L);
        t.nb[3] = t.is + (y == 0 ? (L - 1) * L : -L);
        t.zup = zl + 1 >= zc;
        t.zdn = zl == 0;
        t.nb[4] = t.zup ? y * L + pos : t.is + LL;
        t.nb[5] = t.zdn ? (zc - 1) * LL + y * L + pos : t.is - LL;
        t.i = (uint32_t)((z * L + y) * L + 2 * j + par);
        t.sbits = j1[t.i];
        return t;
    };
    // this thread's first item of each colour, fixed for the run
    Site first0, first1;
    if (tid < items) {
        first0 = site_of(tid, 0);
        first1 = site_of(tid, 1);
    }
    // The draws of this thread's first item of a half sweep depend only on its site and
    // the sweep, so they are computed while the cluster barrier before it completes.
    uint32_t A0[8];
    auto draws_ahead = [&](int sw, int colour) {
        if (sw < p.s_end && tid < items) mp::lead_planes((colour ? first1 : first0).i, (uint32_t)sw, (uint32_t)w, key, A0);
    };

    for (int q = tid; q < slab_words; q += NT) slab[q] = g[(size_t)(z0 * LL + q) * p.stride];
    if (tid < NT / 32) s_tie_n[tid] = 0;
    cluster.barrier_arrive();
    draws_ahead(p.s_begin, 0);
    cluster.barrier_wait();  // every slab loaded before any block reads its neighbours'

    for (int sw = p.s_begin; sw < p.s_end; ++sw) {
        const uint32_t* thr = p.thr + (size_t)sw * kThrRow;  // the sweep's thresholds, k = 0 .. 15
        uint32_t tp[24], lz[3];  // its threshold planes: the same for every replica
        {
            const uint32_t t2 = thr[2], t4 = thr[4], t6 = thr[6];
#pragma unroll
            for (int m = 0; m < 24; ++m)
                tp[m] = mp::threshold_plane_bit(m < 8 ? t2 : m < 16 ? t4 : t6, m % 8) ? ~0u : 0u;
            lz[0] = (t2 & 0xFFFFFFu) ? ~0u : 0u;
            lz[1] = (t4 & 0xFFFFFFu) ? ~0u : 0u;
            lz[2] = (t6 & 0xFFFFFFu) ? ~0u : 0u;
        }
        // one half sweep of colour `colour`; `fst`: this thread's first item of that colour
        auto half = [&](const int colour, const Site& fst) {
            for (int q = tid; q < items; q += NT) {
                const Site t = q == tid ? fst : site_of(q, colour);
                const uint32_t self = slab[t.is];
                uint32_t n[6];
#pragma unroll
                for (int k = 0; k < 4; ++k) n[k] = slab[t.nb[k]];
                n[4] = t.zup ? up[t.nb[4]] : slab[t.nb[4]];
                n[5] = t.zdn ? dn[t.nb[5]] : slab[t.nb[5]];
                uint32_t S[6];
                mp::unit_signs(t.sbits, S);
                uint32_t A[8];
                if (q == tid) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) A[m] = A0[m];
                } else {
                    mp::lead_planes(t.i, (uint32_t)sw, (uint32_t)w, key, A);
                }
                uint32_t flip, tie, c0, c1, c2;
                mp::update_word_unit(self, n, S, valid, tp, A, &flip, &tie, &c0, &c1, &c2);
                tie &= (c1 & lz[2]) | (~c1 & ((c0 & lz[1]) | (~c0 & lz[0])));  // the others reject
                if (tie) {
                    const int p = atomicAdd(&s_tie_n[warp], 1);
                    if (p < kTieCap) {
                        ties[2 * p] = make_uint4(t.i, (uint32_t)t.is, 0u, tie);
                        ties[2 * p + 1] = make_uint4(c0, c1, self ^ flip, 0u);
                    } else {  // list full: decide here
                        flip |= mp::resolve_tie_bits(tie, c0, c1, thr, 0, t.i, (uint32_t)sw, (uint32_t)w, key.k0,
                                                     key.k1);
                    }
                }
                if (flip) slab[t.is] = self ^ flip;
            }
            // this warp's ties, decided by its lanes together (a word has at most one
            // entry, and its owner stored the entry's word: a blind store)
            __syncwarp();
            const int nt = min(s_tie_n[warp], kTieCap);
            for (int e = lane; e < nt; e += 32) {
                const uint4 t = ties[2 * e], u = ties[2 * e + 1];
                const uint32_t acc =
                    mp::resolve_tie_bits(t.w, u.x, u.y, thr, 0, t.x, (uint32_t)sw, (uint32_t)w, key.k0, key.k1);
                if (acc) slab[t.y] = u.z ^ acc;
            }
            __syncwarp();
            if (lane == 0) s_tie_n[warp] = 0;
            // the half sweep is complete in every slab once all blocks have arrived
            cluster.barrier_arrive();
            if (colour == 0) draws_ahead(sw, 1);
            else draws_ahead(sw + 1, 0);
            cluster.barrier_wait();
        };
        half(0, first0);
        half(1, first1);
    }
    for (int q = tid; q < slab_words; q += NT) g[(size_t)(z0 * LL + q) * p.stride] = slab[q];
    cluster.sync();  // no block goes on (or leaves) while another may still read its slab
}

template <int NT>
__global__ void __launch_bounds__(NT) sa_cluster_kernel(const ClusterArgs a)
{
    extern __shared__ uint32_t slab[];  // [L / C][L][L] words of this block's slab, storage order
    __shared__ uint4 s_ties[(NT / 32) * kTieCap * 2];  // per warp: {site, local, -, tie}, {c0, c1, word, -}
    __shared__ int s_tie_n[NT / 32];
    const int w = blockIdx.y, inst = blockIdx.z;
    PlaneRun p;
    p.g = a.spins + (size_t)inst * a.L * a.L * a.L * a.Wn + w;
    p.stride = a.Wn;
    p.j1 = a.j1_ptrs[inst];
    p.thr = a.thr;
    p.key = a.keys[inst];
    p.L = a.L;
    p.w = w;
    p.R = a.R;
    p.s_begin = 0;
    p.s_end = a.S;
    p.Hmagic = a.Hmagic;
    anneal_plane<NT>(p, a.C, slab, s_ties, s_tie_n);
}

// Persistent form for batches (batch.cu's planes of one word, [N][1]): clusters take
// planes from `order` (longest first) through the counter `next` until none is left;
// every plane's side is a multiple of C.
// (Registers are not capped: one block per SM without spills measured 8 % faster on the
// uneven-batch workload than two per SM with a 128-register cap.)
__global__ void __launch_bounds__(kListBlock, 1) sa_cluster_list_kernel(const Plane* __restrict__ planes,
                                                                 const int* __restrict__ order, int n,
                                                                 unsigned* __restrict__ next, int C)
{
    extern __shared__ uint32_t slab[];
    __shared__ uint4 s_ties[(kListBlock / 32) * kTieCap * 2];
    __shared__ int s_tie_n[kListBlock / 32];
    __shared__ int s_item;
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    for (;;) {
        if (r == 0 && threadIdx.x == 0) {  // claim the next plane for the whole cluster
            const int it = (int)atomicAdd(next, 1u);
            for (int k = 0; k < C; ++k) *cluster.map_shared_rank(&s_item, k) = it;
        }
        cluster.sync();
        const int it = s_item;
        if (it >= n) break;
        const Plane& q = planes[order[it]];
        PlaneRun p;
        p.g = q.spins;
        p.stride = 1;
        p.j1 = q.j1;
        p.thr = q.thr;
        p.key = RunKeys{q.k0, q.k1};
        p.L = q.L;
        p.w = q.w0;
        p.R = q.R;
        p.s_begin = q.s_begin;
        p.s_end = q.s_end;
        p.Hmagic = q.Hmagic;
        anneal_plane<kListBlock>(p, C, slab, s_ties, s_tie_n);  // ends with a cluster barrier
    }
}

}  // namespace

// Blocks per cluster for an SA run of I instances of side L with Wn words, or 0 when the
// run is better served by the row kernel: a divisor C <= 8 of L whose slab fits shared
// memory, the largest for which all I * Wn clusters are resident at once (as the driver
// reports for this kernel, so that the run is one wave).  Knob SG_SA_CLUSTER_C forces C.
const void* sa_cluster_fn(int threads)
{
    return threads == 512 ? (const void*)sa_cluster_kernel<512> : (const void*)sa_cluster_kernel<256>;
}

int sa_cluster_blocks(int I, int L, int Wn, int64_t half_sweep_attempts, int* threads)
{
    *threads = 256;
    if (half_sweep_attempts > ((int64_t)1 << 24)) return 0;  // long half sweeps: the row kernel
    int dev = 0, smem = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t clusters = (int64_t)I * Wn;
    const char* e = getenv("SG_SA_CLUSTER_C");
    const int forced = e ? atoi(e) : 0;
    const char* et = getenv("SG_SA_CLUSTER_THREADS");
    const int forced_t = et ? atoi(et) : 0;
    // For each block size, the largest C whose clusters are all resident at once (one wave);
    // of the two, the one with fewer rounds of items a thread times blocks an SM runs (a
    // half sweep's length), ties to 256 threads.  Measured at L = 16 with 1024 replicas:
    // 512 threads at C = 4 (one block an SM) 3.80 ms a run against 3.93 for 256 threads at
    // C = 8 (two blocks on most SMs); one cluster at L = 4: 1.98 ms with 256, 2.03 with 512.
    int bestC = 0, bestT = 256;
    int64_t best_cost = INT64_MAX;
    for (const int t : {256, 512}) {
        if (forced_t && t != forced_t) continue;
        for (int C = 8; C >= 1; --C) {
            if (L % C || (forced && C != forced)) continue;
            const size_t bytes = (size_t)(L / C) * L * L * 4;
            // static shared memory: t / 32 warps' tie queues (32 entries of 32 bytes) and more
            if (bytes + (size_t)t * 32 + 4096 > (size_t)smem) continue;
            if (!forced) {
                if (bytes > 48 * 1024 && cudaFuncSetAttribute(sa_cluster_fn(t), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              (int)bytes) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                cudaLaunchConfig_t cfg{};
                cfg.gridDim = dim3(C, (unsigned)std::min<int64_t>(clusters, 65535), 1);
                cfg.blockDim = dim3(t, 1, 1);
                cfg.dynamicSmemBytes = bytes;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = C;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int active = 0;
                if (cudaOccupancyMaxActiveClusters(&active, sa_cluster_fn(t), &cfg) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                if (active < clusters) continue;
            }
            const int64_t items = (int64_t)(L / C) * L * (L / 2);  // sites of one colour a block
            const int64_t rounds = (items + t - 1) / t;
            const int64_t per_sm = (clusters * C + sms - 1) / sms;
            const int64_t cost = rounds * per_sm;
            if (cost < best_cost) {
                best_cost = cost;
                bestC = C;
                bestT = t;
            }
            break;
        }
    }
    *threads = bestT;
    return bestC;
}

namespace {
// Resident clusters of C blocks with `smem` bytes each for `fn`, or 0.
int active_clusters(const void* fn, int C, size_t smem, int threads)
{
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return active;
}
}  // namespace

int sa_cluster_list_blocks(const int* Ls, int n, int max_L)
{
    int dev = 0, smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int C = 8; C >= 2; --C) {
        bool ok = true;
        for (int k = 0; k < n && ok; ++k) ok = Ls[k] % C == 0;
        if (!ok) continue;
        const size_t bytes = (size_t)(max_L / C) * max_L * max_L * 4;
        if (bytes + 12 * 1024 > (size_t)smem) continue;
        if (active_clusters((const void*)sa_cluster_list_kernel, C, bytes, kListBlock) > 0) return C;
    }
    return 0;
}

int32_t launch_sa_cluster_planes(const Plane* d_planes, const int* d_order, int n, unsigned* d_next, int C,
                                 int max_L, cudaStream_t st)
{
    const size_t smem = (size_t)(max_L / C) * max_L * max_L * 4;
    const int clusters = active_clusters((const void*)sa_cluster_list_kernel, C, smem, kListBlock);
    if (clusters < 1) {
        set_error("sa_cluster_list_kernel: no cluster of %d blocks with %zu bytes fits", C, smem);
        return SG_ECUDA;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C * std::min(clusters, n), 1, 1);
    cfg.blockDim = dim3(kListBlock, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, sa_cluster_list_kernel, d_planes, d_order, n, d_next, C);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("sa_cluster_list_kernel launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

int32_t launch_sa_cluster(int8_t* spins, const uint8_t* const* j1_ptrs, const RunKeys* keys, const uint32_t* thr,
                          int I, int L, int Wn, int R, int S, int C, int threads, cudaStream_t st)
{
    if (threads != 256 && threads != 512) {
        set_error("sa_cluster_kernel: %d threads a block (256 or 512)", threads);
        return SG_EINVAL;
    }
    ClusterArgs a{};
    a.spins = reinterpret_cast<uint32_t*>(spins);
    a.j1_ptrs = j1_ptrs;
    a.keys = keys;
    a.thr = thr;
    a.L = L;
    a.Wn = Wn;
    a.R = R;
    a.S = S;
    a.C = C;
    const int H = L / 2;
    a.Hmagic = H == 1 ? 0u : (uint32_t)((0x100000000ull + (uint64_t)H - 1) / (uint64_t)H);
    const size_t smem = (size_t)(L / C) * L * L * 4;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(sa_cluster_fn(threads), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        cudaGetLastError();
        set_error("sa_cluster_kernel: cannot use %zu bytes of shared memory", smem);
        return SG_ECUDA;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C, Wn, I);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = threads == 512 ? cudaLaunchKernelEx(&cfg, sa_cluster_kernel<512>, a)
                                         : cudaLaunchKernelEx(&cfg, sa_cluster_kernel<256>, a);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("sa_cluster_kernel launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace sg
