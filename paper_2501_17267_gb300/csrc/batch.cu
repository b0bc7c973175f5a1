// batch.cu -- simulated annealing of many instances of uneven size in one persistent
// launch (App. D.1 run on a batch).
//
// Annealing chains are independent: replicas never interact.  A batch is cut into
// "planes", one per (instance, group of WG consecutive replica words); a plane holds
// its chain's spins for every site, [N][WG] words (32 replicas a word) in storage order,
// so the threads of a block read consecutive 4*WG-byte records.  One persistent kernel runs every plane
// from the first sweep to the last: each block takes the next plane from an atomic
// counter (planes are ordered by decreasing work, largest first), sweeps it colour
// by colour with only block barriers in between -- no other block touches its
// replicas -- and takes another.  No block ever waits on another.
//
// Results are byte-identical to separate runs: every draw is named by (site, sweep,
// word of the instance), independent of how the batch is cut.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <filesystem>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "metropolis.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

__device__ __forceinline__ int div_magic(int v, uint32_t m) { return (int)__umulhi((uint32_t)v, m); }

template <int WG>
__device__ __forceinline__ void load_plane_words(const uint32_t* p, uint32_t (&w)[WG])
{
    if constexpr (WG == 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
    } else if constexpr (WG == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        w[0] = v.x, w[1] = v.y;
    } else {
        w[0] = *p;
    }
}

template <int WG>
__device__ __forceinline__ void store_plane_words(uint32_t* p, const uint32_t (&w)[WG])
{
    if constexpr (WG == 4) *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    else if constexpr (WG == 2) *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    else *p = w[0];
}

// Replicas of word w (of the instance) that exist.
__device__ __forceinline__ uint32_t plane_valid_bits(int R, int w)
{
    const int left = R - 32 * w;
    return left >= 32 ? 0xFFFFFFFFu : left <= 0 ? 0u : (1u << left) - 1u;
}

// Persistent sweep kernel.  `order` lists plane indices by decreasing work.  SMEM: the
// block copies its plane into shared memory (dynamic, [N][WG] words), runs all of the
// plane's sweeps there, and writes it back -- no global traffic and no launches between
// sweeps, for planes that fit.  Every word update is the bit-sliced one of metropolis.cuh.
template <int WG, bool UNITJ, bool SMEM = false>
__global__ void __launch_bounds__(256) sa_planes_kernel(const Plane* __restrict__ planes,
                                                        const int* __restrict__ order, int n_planes,
                                                        unsigned* __restrict__ next)
{
    constexpr int U = 4 / WG;
    constexpr int kTieCap = 32;  // queued tie entries per warp (decided once half full)
    extern __shared__ __align__(16) uint32_t s_plane[];
    __shared__ int s_item;
    __shared__ uint32_t s_thr[kThrRow];
    __shared__ uint4 s_ties[8 * kTieCap * 2];  // per warp: {site, storage, word index, tie}, {c0, c1, stored word, -}
    __shared__ int s_tie_n[8];
    const int tid = threadIdx.x, nthreads = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    uint4* ties = s_ties + warp * kTieCap * 2;
    if (tid < 8) s_tie_n[tid] = 0;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_planes) break;
        const Plane p = planes[order[it]];
        const int L = p.L, H = L >> 1, LL = L * L, N = LL * L;
        const int half = LL * H;  // sites of one colour
        const RunKeys key{p.k0, p.k1};
        uint32_t vmask[WG];
#pragma unroll
        for (int wi = 0; wi < WG; ++wi) vmask[wi] = plane_valid_bits(p.R, p.w0 + wi);
        uint32_t* __restrict__ sp = p.spins;
        if constexpr (SMEM) {
            for (int q = tid; q < N; q += nthreads) {
                uint32_t w[WG];
                load_plane_words<WG>(p.spins + (size_t)q * WG, w);
                store_plane_words<WG>(s_plane + (size_t)q * WG, w);
            }
            __syncthreads();
            sp = s_plane;
        }
        for (int sw = p.s_begin; sw < p.s_end; ++sw) {
            if (tid < kThrRow) s_thr[tid] = p.thr[(size_t)sw * kThrRow + tid];
            __syncthreads();
            uint32_t tp[24];  // threshold planes of the sweep (the same for every replica)
            uint32_t lz[3];   // thresholds k = 2, 4, 6 with nonzero low bits: ties there can accept
            if (UNITJ) {
#pragma unroll
                for (int m = 0; m < 24; ++m) tp[m] = mp::threshold_plane_bit(s_thr[2 + 2 * (m / 8)], m % 8) ? ~0u : 0u;
#pragma unroll
                for (int m = 0; m < 3; ++m) lz[m] = (s_thr[2 + 2 * m] & 0xFFFFFFu) ? ~0u : 0u;
            }
            // Deferred ties of this warp, decided by all its lanes together (every lane
            // runs the same iterations of the site loop below).
            auto resolve_list = [&]() {
                __syncwarp();
                const int n = min(s_tie_n[warp], kTieCap);
                for (int e = lane; e < n; e += 32) {
                    const uint4 t = ties[2 * e], u = ties[2 * e + 1];
                    const uint32_t acc =
                        mp::resolve_tie_bits(t.w, u.x, u.y, s_thr, 0, t.x, (uint32_t)sw, t.z, key.k0, key.k1);
                    // the word's owner stored u.z; nobody else writes it: no read back
                    if (acc) sp[(size_t)t.y * WG + (t.z - (uint32_t)p.w0)] = u.z ^ acc;
                }
                __syncwarp();
                if (lane == 0) s_tie_n[warp] = 0;
                __syncwarp();
            };
            for (int colour = 0; colour < 2; ++colour) {
                // U = 4 / WG sites per thread at a time: all their loads, then all their
                // updates and stores (sites of one colour never read one another), so the
                // U Philox chains and load streams overlap.  The loop bound depends only on
                // the warp, so the warp stays converged; slots past the end are idle.
                for (int qb = tid - lane; qb < half; qb += U * nthreads) {
                    const int q0 = qb + lane;
                    int is_[U], i_[U];
                    bool live[U];
                    uint32_t S[U][6];
                    int J[U][6];
                    uint32_t self[U][WG], n[U][6][WG];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        live[u] = q0 + u * nthreads < half;
                        const int q = live[u] ? q0 + u * nthreads : 0;  // an idle slot reads site 0, unstored
                        const int row = H == 1 ? q : div_magic(q, p.Hmagic);  // ceil(2^32 / 1) does not fit
                        const int j = q - row * H;
                        const int z = div_magic(row, p.Lmagic);
                        const int y = row - z * L;
                        const int par = (y + z + colour) & 1;
                        const int rowoff = row * L;
                        i_[u] = rowoff + 2 * j + par;  // logical site
                        is_[u] = rowoff + par * H + j;  // storage position
                        const int ho = rowoff + (1 - par) * H;
                        const int jp = j + par == H ? 0 : j + par, jm = j + par == 0 ? H - 1 : j + par - 1;
                        const int dyp = (y + 1 == L ? 1 - L : 1) * L, dym = (y == 0 ? L - 1 : -1) * L;
                        const int dzp = (z + 1 == L ? 1 - L : 1) * LL, dzm = (z == 0 ? L - 1 : -1) * LL;
                        const int nb[6] = {ho + jp, ho + jm, is_[u] + dyp, is_[u] + dym, is_[u] + dzp, is_[u] + dzm};
                        if (UNITJ) {
                            mp::unit_signs(p.j1[i_[u]], S[u]);
                        } else {
                            const uint2 r = p.j6[i_[u]];
#pragma unroll
                            for (int qq = 0; qq < 6; ++qq)
                                J[u][qq] = (int)(int8_t)(((qq < 4 ? r.x : r.y) >> (8 * (qq & 3))) & 0xFFu);
                        }
                        load_plane_words<WG>(sp + (size_t)is_[u] * WG, self[u]);
#pragma unroll
                        for (int qq = 0; qq < 6; ++qq) load_plane_words<WG>(sp + (size_t)nb[qq] * WG, n[u][qq]);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        uint32_t out[WG];
                        bool any = false;
#pragma unroll
                        for (int wi = 0; wi < WG; ++wi) {
                            const uint32_t w = (uint32_t)(p.w0 + wi);
                            const uint32_t valid = live[u] ? vmask[wi] : 0u;  // an idle slot flips nothing
                            uint32_t nw[6];
#pragma unroll
                            for (int qq = 0; qq < 6; ++qq) nw[qq] = n[u][qq][wi];
                            uint32_t A[8];
                            mp::lead_planes((uint32_t)i_[u], (uint32_t)sw, w, key, A);
                            uint32_t flip;
                            if (UNITJ) {
                                uint32_t tie, c0, c1, c2;
                                mp::update_word_unit(self[u][wi], nw, S[u], valid, tp, A, &flip, &tie, &c0, &c1, &c2);
                                tie &= (c1 & lz[2]) | (~c1 & ((c0 & lz[1]) | (~c0 & lz[0])));  // others reject
                                if (tie) {
                                    const int pos = atomicAdd(&s_tie_n[warp], 1);
                                    if (pos < kTieCap) {
                                        ties[2 * pos] = make_uint4((uint32_t)i_[u], (uint32_t)is_[u], w, tie);
                                        ties[2 * pos + 1] = make_uint4(c0, c1, self[u][wi] ^ flip, 0u);
                                    } else {  // list full: decide here
                                        flip |= mp::resolve_tie_bits(tie, c0, c1, s_thr, 0, (uint32_t)i_[u],
                                                                     (uint32_t)sw, w, key.k0, key.k1);
                                    }
                                }
                            } else {
                                flip = mp::update_word_general(self[u][wi], nw, J[u], valid, s_thr, 0, A,
                                                               (uint32_t)i_[u], (uint32_t)sw, w, key);
                            }
                            out[wi] = self[u][wi] ^ flip;
                            any |= flip != 0u;
                        }
                        if (any) store_plane_words<WG>(sp + (size_t)is_[u] * WG, out);
                    }
                    __syncwarp();
                    if (s_tie_n[warp] >= kTieCap / 2) resolve_list();
                }
                resolve_list();  // the next colour reads these sites
                __syncthreads();
            }
        }
        if constexpr (SMEM) {
            __syncthreads();
            for (int q = tid; q < N; q += nthreads) {
                uint32_t w[WG];
                load_plane_words<WG>(s_plane + (size_t)q * WG, w);
                store_plane_words<WG>(p.spins + (size_t)q * WG, w);
            }
        }
    }
}

// Initial spins of every plane (grid.y = plane): replica r of site i starts at -1 when
// bit 31 of word r % 4 of Philox(i, kSweepInit, r / 4, 0) is set.
template <int WG>
__global__ void planes_init_kernel(const Plane* __restrict__ planes)
{
    const Plane p = planes[blockIdx.y];
    const int N = p.L * p.L * p.L;
    for (int is = blockIdx.x * blockDim.x + threadIdx.x; is < N; is += gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)logical_of(p.L, is);
        uint32_t words[WG];
#pragma unroll
        for (int wi = 0; wi < WG; ++wi) {
            const int w = p.w0 + wi;
            uint32_t word = 0;
            for (int q = 0; q < 8; ++q) {
                if (32 * w + 4 * q >= p.R) break;
                const Philox4 r = philox4x32_10(i, kSweepInit, (uint32_t)(8 * w + q), kDomainMetropolis, p.k0, p.k1);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (32 * w + 4 * q + m < p.R && (r.v[m] >> 31)) word |= 1u << (4 * q + m);
            }
            words[wi] = word;
        }
        store_plane_words<WG>(p.spins + (size_t)is * WG, words);
    }
}

// Energies (Eq. 1) of every replica of every plane: E_out[plane][32*WG] (grid.y = plane).
// One warp per (row, word) item; lane b sums replica bit b along the row (forward bonds).
template <int WG>
__global__ void planes_energy_kernel(const Plane* __restrict__ planes, unsigned long long* __restrict__ E_out)
{
    const Plane p = planes[blockIdx.y];
    const int L = p.L, LL = L * L, H = L >> 1;
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int t = blockIdx.x * warps + (threadIdx.x >> 5); t < LL * WG; t += gridDim.x * warps) {
        const int r = t / WG, wi = t % WG;
        const int z = r / L, y = r - z * L;
        const int ryp = z * L + (y + 1 == L ? 0 : y + 1);
        const int rzp = (z + 1 == L ? 0 : z + 1) * L + y;
        const uint32_t* __restrict__ row = p.spins + (size_t)r * L * WG + wi;
        const uint32_t* __restrict__ rowy = p.spins + (size_t)ryp * L * WG + wi;
        const uint32_t* __restrict__ rowz = p.spins + (size_t)rzp * L * WG + wi;
        long long e = 0;
        for (int x = 0; x < L; ++x) {
            const int pos = (x & 1) * H + (x >> 1);
            const int xp = x + 1 == L ? 0 : x + 1;
            const int posx = (xp & 1) * H + (xp >> 1);
            const uint2 rec = p.j6[r * L + x];
            const int J[3] = {(int)(int8_t)(rec.x & 0xFFu), (int)(int8_t)((rec.x >> 16) & 0xFFu),
                              (int)(int8_t)(rec.y & 0xFFu)};
            const uint32_t me = row[pos * WG];
            const uint32_t nb[3] = {row[posx * WG], rowy[pos * WG], rowz[pos * WG]};
#pragma unroll
            for (int d = 0; d < 3; ++d) e += J[d] * (1 - 2 * (int)(((me ^ nb[d]) >> lane) & 1u));
        }
        if (e) atomicAdd(&E_out[(size_t)blockIdx.y * 32 * WG + 32 * wi + lane], (unsigned long long)e);
    }
}

// Spins of one plane into the instance's [R][N] output (grid.y = plane).
template <int WG>
__global__ void planes_unpack_kernel(const Plane* __restrict__ planes, int8_t* const* __restrict__ outs)
{
    const Plane p = planes[blockIdx.y];
    int8_t* out = outs[p.out];
    if (!out) return;
    const int L = p.L;
    const int64_t N = (int64_t)L * L * L;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * 32 * WG;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int rb = (int)(q / N);            // replica within the plane
        const int64_t i = q - (int64_t)rb * N;  // logical site
        const int r = 32 * p.w0 + rb;
        if (r < p.R) {
            const uint32_t word = p.spins[storage_of(L, i) * WG + (rb >> 5)];
            out[(int64_t)r * N + i] = ((word >> (rb & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
        }
    }
}

int check(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

// The instantiation for (WG, unit couplings, plane in shared memory).
template <int WG>
const void* planes_kernel_fn(bool unit, bool smem)
{
    if (smem)
        return unit ? (const void*)sa_planes_kernel<WG, true, true> : (const void*)sa_planes_kernel<WG, false, true>;
    return unit ? (const void*)sa_planes_kernel<WG, true, false> : (const void*)sa_planes_kernel<WG, false, false>;
}

const void* planes_kernel_fn(int WG, bool unit, bool smem)
{
    return WG == 4 ? planes_kernel_fn<4>(unit, smem) : WG == 2 ? planes_kernel_fn<2>(unit, smem)
                                                              : planes_kernel_fn<1>(unit, smem);
}

// Tuning knob SG_PLANES_SMEM_KB: largest plane kept in shared memory (default 110 KB, so
// that two blocks fit per SM; 0 keeps every plane in global memory).
size_t planes_smem_limit()
{
    const char* e = getenv("SG_PLANES_SMEM_KB");
    const long kb = e ? atol(e) : 110;
    return kb > 0 ? (size_t)kb * 1024 : 0;
}

}  // namespace

size_t planes_smem_bytes(int WG, int max_L)
{
    const size_t bytes = (size_t)max_L * max_L * max_L * WG * 4;
    int dev = 0, per_block = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return bytes <= planes_smem_limit() && bytes + 1024 <= (size_t)per_block ? bytes : 0;
}

int32_t launch_sa_planes(int WG, const Plane* d_planes, const int* d_order, int n, unsigned* d_next,
                         bool unit, int blocks, cudaStream_t st, size_t smem)
{
    const void* fn = planes_kernel_fn(WG, unit, smem > 0);
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    void* args[] = {(void*)&d_planes, (void*)&d_order, (void*)&n, (void*)&d_next};
    cudaError_t e = cudaLaunchKernel(fn, dim3(blocks), dim3(256), args, smem, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("sa_planes_kernel: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return check("sa_planes_kernel");
}

int planes_blocks(int WG, bool unit, size_t smem)
{
    int dev = 0, sms = 148, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* fn = planes_kernel_fn(WG, unit, smem > 0);
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return sms * per_sm;
}

int32_t launch_planes_init(int WG, const Plane* d_planes, int n, cudaStream_t st)
{
    dim3 grid(64, n);
    if (WG == 4) planes_init_kernel<4><<<grid, 256, 0, st>>>(d_planes);
    else if (WG == 2) planes_init_kernel<2><<<grid, 256, 0, st>>>(d_planes);
    else planes_init_kernel<1><<<grid, 256, 0, st>>>(d_planes);
    return check("planes_init_kernel");
}

int32_t launch_planes_energy(int WG, const Plane* d_planes, int n, unsigned long long* E_out, cudaStream_t st)
{
    dim3 grid(64, n);
    if (WG == 4) planes_energy_kernel<4><<<grid, 256, 0, st>>>(d_planes, E_out);
    else if (WG == 2) planes_energy_kernel<2><<<grid, 256, 0, st>>>(d_planes, E_out);
    else planes_energy_kernel<1><<<grid, 256, 0, st>>>(d_planes, E_out);
    return check("planes_energy_kernel");
}

int32_t launch_planes_unpack(int WG, const Plane* d_planes, int n, int8_t* const* outs, cudaStream_t st)
{
    dim3 grid(64, n);
    if (WG == 4) planes_unpack_kernel<4><<<grid, 256, 0, st>>>(d_planes, outs);
    else if (WG == 2) planes_unpack_kernel<2><<<grid, 256, 0, st>>>(d_planes, outs);
    else planes_unpack_kernel<1><<<grid, 256, 0, st>>>(d_planes, outs);
    return check("planes_unpack_kernel");
}

// ------------------------------------------------------------------ host side

namespace {

uint32_t magic(int d) { return (uint32_t)((0x100000000ull + (uint64_t)d - 1) / (uint64_t)d); }

// Stream-ordered device buffer (freed at scope exit).
struct Buf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    ~Buf()
    {
        if (p) cudaFreeAsync(p, st);
    }
    int32_t alloc(size_t bytes, cudaStream_t s)
    {
        st = s;
        if (cudaMallocAsync(&p, bytes ? bytes : 16, s) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            set_error("device allocation of %zu bytes failed", bytes);
            return SG_ENOMEM;
        }
        return SG_OK;
    }
};

#define SG_B(expr)                      \
    do {                                \
        int32_t _rc = (expr);           \
        if (_rc != SG_OK) return _rc;   \
    } while (0)

// ---- autotuner cache: key -> words per plane, kept in a small JSON object file ----
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_mem;
bool g_tune_loaded = false;

std::string tune_path()
{
    const char* e = getenv("SG_AUTOTUNE_CACHE");
    if (e && *e) return e;
    const char* home = getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/sg_autotune.json";
}

void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    std::ifstream f(tune_path());
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    // flat object {"key": value, ...} written by tune_store
    size_t pos = 0;
    while ((pos = t.find('"', pos)) != std::string::npos) {
        const size_t end = t.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = t.substr(pos + 1, end - pos - 1);
        const size_t colon = t.find(':', end);
        if (colon == std::string::npos) break;
        g_tune_mem[key] = atoi(t.c_str() + colon + 1);
        pos = t.find_first_of(",}", colon);
        if (pos == std::string::npos) break;
    }
}

void tune_store()
{
    const std::string path = tune_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos && slash > 0) {
        std::error_code ec;  // the cache is an optimisation: a directory that cannot be made is skipped
        std::filesystem::create_directories(path.substr(0, slash), ec);
        if (ec) return;
    }
    std::ofstream f(path);
    if (!f) return;
    f << "{";
    bool first = true;
    for (auto& kv : g_tune_mem) {
        f << (first ? "" : ",") << "\n \"" << kv.first << "\": " << kv.second;
        first = false;
    }
    f << "\n}\n";
}

}  // namespace

// Runs the members of a batch (any sizes) through the persistent plane kernel.
int32_t run_sa_planes(const std::vector<int>& members, const sg_instance* const* insts,
                      const sg_sa_params* ps, sg_sa_result* outs, cudaStream_t st, bool* used_graph,
                      int* chosen_wg)
{
    const int I = (int)members.size();
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // words per plane: a common divisor of every instance's word count
    int wg_max = 4;
    for (int a = 0; a < I; ++a) {
        const int Wn = words_for(ps[members[a]].replicas);
        while (Wn % wg_max) wg_max >>= 1;
    }

    // schedules (one threshold table per distinct schedule)
    std::map<std::tuple<int, double, double, int>, size_t> sched_off;
    std::vector<uint32_t> thr;
    std::vector<size_t> inst_thr(I);
    for (int a = 0; a < I; ++a) {
        const sg_sa_params& p = ps[members[a]];
        auto key = std::make_tuple(p.sweeps, p.beta0, p.beta1, p.schedule);
        auto it = sched_off.find(key);
        if (it == sched_off.end()) {
            const size_t off = thr.size();
            std::vector<double> beta((size_t)std::max(p.sweeps, 1));
            beta_schedule(p.sweeps, p.beta0, p.beta1, p.schedule == SG_SCHEDULE_GEOMETRIC, beta.data());
            thr.resize(off + (size_t)std::max(p.sweeps, 1) * kThrRow);
            for (int sw = 0; sw < p.sweeps; ++sw) metropolis_row(beta[sw], &thr[off + (size_t)sw * kThrRow]);
            it = sched_off.emplace(key, off).first;
        }
        inst_thr[a] = it->second;
    }
    bool unit = true;
    for (int a = 0; a < I; ++a) unit &= insts[members[a]]->unit_couplings;

    std::vector<const uint2*> j6(I);
    std::vector<const uint8_t*> j1(I);
    for (int a = 0; a < I; ++a)
        SG_B(instance_device_j6(const_cast<sg_instance*>(insts[members[a]]), st, &j6[a], &j1[a]));

    Buf d_thr;
    SG_B(d_thr.alloc(sizeof(uint32_t) * std::max<size_t>(thr.size(), 1), st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_thr.p, thr.data(), sizeof(uint32_t) * thr.size(), cudaMemcpyHostToDevice, st));

    // planes for a given words-per-plane choice; spins laid out plane after plane
    auto make_planes = [&](int WG, uint32_t* spins_base, std::vector<Plane>* planes,
                           std::vector<double>* work, size_t* words_total) {
        planes->clear();
        work->clear();
        size_t wo = 0;
        for (int a = 0; a < I; ++a) {
            const sg_instance* in = insts[members[a]];
            const sg_sa_params& p = ps[members[a]];
            const int Wn = words_for(p.replicas);
            for (int w0 = 0; w0 < Wn; w0 += WG) {
                Plane pl{};
                pl.spins = spins_base ? spins_base + wo : nullptr;
                pl.j1 = j1[a];
                pl.j6 = j6[a];
                pl.thr = static_cast<const uint32_t*>(d_thr.p) + inst_thr[a];
                const RunKeys k{(uint32_t)p.seed, (uint32_t)(p.seed >> 32) ^ p.instance_id};
                pl.k0 = k.k0;
                pl.k1 = k.k1;
                pl.L = in->L;
                pl.S = p.sweeps;
                pl.s_begin = 0;
                pl.s_end = p.sweeps;
                pl.w0 = w0;
                pl.R = p.replicas;
                pl.Lmagic = magic(in->L);
                pl.Hmagic = magic(in->L / 2);
                pl.out = a;
                planes->push_back(pl);
                work->push_back((double)in->N * 32 * WG * std::max(p.sweeps, 1));
                wo += (size_t)in->N * WG;
            }
        }
        *words_total = wo;
    };
    auto lpt_order = [](const std::vector<double>& work) {
        std::vector<int> order(work.size());
        for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
        return order;
    };
    // planes of a launch sit in shared memory when the largest of them fits
    int max_L = 0;
    for (int a = 0; a < I; ++a) max_L = std::max(max_L, insts[members[a]]->L);
    auto smem_for = [&](int WG) { return planes_smem_bytes(WG, max_L); };
    auto blocks_for = [&](int WG) { return planes_blocks(WG, unit, smem_for(WG)); };
    // Candidate 0: planes of one word, each annealed by a thread-block cluster of Ccl blocks
    // (cluster.cu), so that a large plane is not one block's work alone.
    int Ccl = 0;
    if (unit) {
        std::vector<int> Ls(I);
        for (int a = 0; a < I; ++a) Ls[a] = insts[members[a]]->L;
        Ccl = sa_cluster_list_blocks(Ls.data(), I, max_L);
    }
    auto width = [](int wg) { return wg == 0 ? 1 : wg; };  // words per plane in memory
    // planes running at once: blocks, or clusters (one block per SM)
    auto concurrency = [&](int wg) { return wg == 0 ? std::max(1, sms / Ccl) : blocks_for(wg); };
    auto sweep_launch = [&](int wg, const Plane* d_pl, const int* d_ord, int n, unsigned* d_next,
                            cudaStream_t s) -> int32_t {
        if (wg == 0) return launch_sa_cluster_planes(d_pl, d_ord, n, d_next, Ccl, max_L, s);
        return launch_sa_planes(wg, d_pl, d_ord, n, d_next, unit, blocks_for(wg), s, smem_for(wg));
    };

    // ---- autotune the words per plane (or clusters): measured throughput on the batch
    // itself, then the makespan bound max(total / rate, largest plane / per-plane rate) ----
    std::vector<int> cands;
    for (int wg = wg_max; wg >= 1; wg >>= 1) cands.push_back(wg);
    if (Ccl > 0) cands.push_back(0);
    std::string key;
    {
        std::map<std::tuple<int, int, int>, int> mix;
        for (int a = 0; a < I; ++a)
            mix[std::make_tuple(insts[members[a]]->L, ps[members[a]].replicas, ps[members[a]].sweeps)]++;
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, dev);
        std::ostringstream ks;
        ks << prop.name << "/" << sms << "/" << (unit ? "u" : "g") << "/smem" << smem_for(1) / 1024 << "/c" << Ccl
           << "/t4";
        for (auto& m : mix)
            ks << "/" << std::get<0>(m.first) << "x" << std::get<1>(m.first) << "x" << std::get<2>(m.first) << "x" << m.second;
        key = ks.str();
        for (auto& c : key)
            if (c == '"' || c == '\\') c = '_';
    }
    int WG = cands.front();
    const char* force = getenv("SG_BATCH_WG");
    if (force && atoi(force) >= 1 && wg_max % atoi(force) == 0) {
        WG = atoi(force);
    } else if (force && force[0] == '0' && Ccl > 0) {
        WG = 0;
    } else if (cands.size() > 1) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_load();
        auto hit = g_tune_mem.find(key);
        if (hit != g_tune_mem.end() && (hit->second == 0 ? Ccl > 0 : wg_max % hit->second == 0)) {
            WG = hit->second;
        } else {
            double best = 1e300;
            for (int wg : cands) {
                std::vector<Plane> planes;
                std::vector<double> work;
                size_t words = 0;
                make_planes(width(wg), nullptr, &planes, &work, &words);
                Buf d_sp, d_pl, d_ord, d_next;
                SG_B(d_sp.alloc(words * 4, st));
                make_planes(width(wg), static_cast<uint32_t*>(d_sp.p), &planes, &work, &words);
                // trial: a few sweeps of every plane, enough (up to 64) for about 1e9
                // attempts, so that launch and copy costs do not decide small batches
                double per_sweep = 0;
                int s_min = 1 << 30;
                for (auto& pl : planes) {
                    per_sweep += (double)pl.L * pl.L * pl.L * 32 * width(wg);
                    s_min = std::min(s_min, std::max(pl.S, 1));
                }
                const int trial_sweeps =
                    std::max(2, std::min({64, s_min, (int)std::min(1e9 / std::max(per_sweep, 1.0), 1e6)}));
                double trial_work = 0;
                for (auto& pl : planes) {
                    pl.s_end = std::min(pl.S, trial_sweeps);
                    trial_work += (double)pl.L * pl.L * pl.L * 32 * width(wg) * pl.s_end;
                }
                const std::vector<int> order = lpt_order(work);
                SG_B(d_pl.alloc(sizeof(Plane) * planes.size(), st));
                SG_B(d_ord.alloc(sizeof(int) * order.size(), st));
                SG_B(d_next.alloc(sizeof(unsigned), st));
                SG_TRY_CUDA(cudaMemcpyAsync(d_pl.p, planes.data(), sizeof(Plane) * planes.size(), cudaMemcpyHostToDevice, st));
                SG_TRY_CUDA(cudaMemcpyAsync(d_ord.p, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, st));
                SG_B(launch_planes_init(width(wg), static_cast<Plane*>(d_pl.p), (int)planes.size(), st));
                const int conc = concurrency(wg);
                double t_best = 1e300;
                for (int rep = 0; rep < 2; ++rep) {
                    SG_TRY_CUDA(cudaMemsetAsync(d_next.p, 0, sizeof(unsigned), st));
                    SG_TRY_CUDA(cudaStreamSynchronize(st));
                    const auto t0 = std::chrono::steady_clock::now();
                    SG_B(sweep_launch(wg, static_cast<Plane*>(d_pl.p), static_cast<int*>(d_ord.p),
                                      (int)planes.size(), static_cast<unsigned*>(d_next.p), st));
                    SG_TRY_CUDA(cudaStreamSynchronize(st));
                    t_best = std::min(t_best, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
                }
                const double rate = trial_work / t_best;  // attempts per second, whole GPU
                double total = 0, biggest = 0;
                for (double w : work) {
                    total += w;
                    biggest = std::max(biggest, w);
                }
                const double est = std::max(total / rate, biggest / (rate / std::min<double>(conc, work.size())));
                if (est < best) {
                    best = est;
                    WG = wg;
                }
            }
            g_tune_mem[key] = WG;
            tune_store();
        }
    }
    if (chosen_wg) *chosen_wg = WG;

    // ---- the run ----
    std::vector<Plane> planes;
    std::vector<double> work;
    size_t words = 0;
    const int WGm = width(WG);  // words per plane in memory
    make_planes(WGm, nullptr, &planes, &work, &words);
    Buf d_sp, d_pl, d_ord, d_next, d_E, d_outs, d_stage;
    SG_B(d_sp.alloc(words * 4, st));
    make_planes(WGm, static_cast<uint32_t*>(d_sp.p), &planes, &work, &words);
    const std::vector<int> order = lpt_order(work);
    const int n = (int)planes.size();
    SG_B(d_pl.alloc(sizeof(Plane) * n, st));
    SG_B(d_ord.alloc(sizeof(int) * n, st));
    SG_B(d_next.alloc(sizeof(unsigned), st));
    SG_B(d_E.alloc(sizeof(unsigned long long) * (size_t)n * 32 * WGm, st));
    // spin outputs: device targets directly, host targets through one staging area
    std::vector<int8_t*> outp(I, nullptr);
    size_t stage_bytes = 0;
    std::vector<size_t> stage_off(I, 0);
    for (int a = 0; a < I; ++a) {
        const sg_sa_result& o = outs[members[a]];
        if (o.spins && o.spins_mem == SG_MEM_HOST) {
            stage_off[a] = stage_bytes;
            stage_bytes += (size_t)ps[members[a]].replicas * insts[members[a]]->N;
        }
    }
    if (stage_bytes) SG_B(d_stage.alloc(stage_bytes, st));
    for (int a = 0; a < I; ++a) {
        const sg_sa_result& o = outs[members[a]];
        if (!o.spins) continue;
        outp[a] = o.spins_mem == SG_MEM_DEVICE ? o.spins : static_cast<int8_t*>(d_stage.p) + stage_off[a];
    }
    SG_B(d_outs.alloc(sizeof(int8_t*) * I, st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_pl.p, planes.data(), sizeof(Plane) * n, cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_ord.p, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_outs.p, outp.data(), sizeof(int8_t*) * I, cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaStreamSynchronize(st));  // host arrays above are stack/heap temporaries

    // launch statistics: with timing on, the run launches directly and brackets the
    // persistent sweep launch with events
    const bool timed = stats_timing();
    struct EventPair {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~EventPair()
        {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evp;
    cudaEvent_t* ev = evp.e;
    if (timed && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)) {
        cudaGetLastError();
        set_error("cudaEventCreate failed");
        return SG_ECUDA;
    }
    auto device_work = [&](cudaStream_t s) -> int32_t {
        SG_TRY_CUDA(cudaMemsetAsync(d_next.p, 0, sizeof(unsigned), s));
        SG_TRY_CUDA(cudaMemsetAsync(d_E.p, 0, sizeof(unsigned long long) * (size_t)n * 32 * WGm, s));
        SG_B(launch_planes_init(WGm, static_cast<Plane*>(d_pl.p), n, s));
        if (timed) SG_TRY_CUDA(cudaEventRecord(ev[0], s));
        SG_B(sweep_launch(WG, static_cast<Plane*>(d_pl.p), static_cast<int*>(d_ord.p), n,
                          static_cast<unsigned*>(d_next.p), s));
        if (timed) SG_TRY_CUDA(cudaEventRecord(ev[1], s));
        SG_B(launch_planes_energy(WGm, static_cast<Plane*>(d_pl.p), n, static_cast<unsigned long long*>(d_E.p), s));
        SG_B(launch_planes_unpack(WGm, static_cast<Plane*>(d_pl.p), n, static_cast<int8_t* const*>(d_outs.p), s));
        return SG_OK;
    };
    // the device part of the run is one CUDA graph (knob SG_BATCH_GRAPH=0 launches directly)
    const char* g = getenv("SG_BATCH_GRAPH");
    const bool graph = !(g && atoi(g) == 0) && !timed;
    if (used_graph) *used_graph = graph;
    if (graph) {
        cudaStream_t cs = nullptr;
        SG_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr = nullptr;
        cudaGraphExec_t ge = nullptr;
        int32_t rc = SG_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = SG_ECUDA;
        if (rc == SG_OK) rc = device_work(cs);
        cudaError_t e = cudaStreamEndCapture(cs, &gr);
        if (rc == SG_OK && e != cudaSuccess) rc = SG_ECUDA;
        if (rc == SG_OK && cudaGraphInstantiate(&ge, gr, 0) != cudaSuccess) rc = SG_ECUDA;
        if (rc == SG_OK && cudaGraphLaunch(ge, st) != cudaSuccess) rc = SG_ECUDA;
        if (ge) cudaGraphExecDestroy(ge);
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cs);
        if (rc != SG_OK) {
            cudaGetLastError();
            if (!*sg_last_error_string()) set_error("graph capture of the batch failed");
            return rc;
        }
    } else {
        SG_B(device_work(st));
    }

    std::vector<unsigned long long> E((size_t)n * 32 * WGm);
    SG_TRY_CUDA(cudaMemcpyAsync(E.data(), d_E.p, sizeof(unsigned long long) * E.size(), cudaMemcpyDeviceToHost, st));
    for (int a = 0; a < I; ++a) {
        const sg_sa_result& o = outs[members[a]];
        if (o.spins && o.spins_mem == SG_MEM_HOST)
            SG_TRY_CUDA(cudaMemcpyAsync(o.spins, static_cast<int8_t*>(d_stage.p) + stage_off[a],
                                        (size_t)ps[members[a]].replicas * insts[members[a]]->N,
                                        cudaMemcpyDeviceToHost, st));
    }
    SG_TRY_CUDA(cudaStreamSynchronize(st));
    {
        int64_t attempts = 0, cells = 0;
        for (int a = 0; a < I; ++a) {
            const int64_t N = insts[members[a]]->N, R = ps[members[a]].replicas;
            attempts += N * R * ps[members[a]].sweeps;
            cells += N * R;
        }
        float ms = 0.f;
        if (timed) cudaEventElapsedTime(&ms, ev[0], ev[1]);
        stats_add(SG_KERNEL_INIT, 1, cells, 0.0);
        stats_add(SG_KERNEL_SWEEP_CHUNK, 1, attempts, (double)ms);
        stats_add(SG_KERNEL_ENERGY, 1, cells, 0.0);
        stats_add(SG_KERNEL_OTHER, 1, cells, 0.0);
    }
    for (int q = 0; q < n; ++q) {
        const Plane& pl = planes[q];
        const int a = pl.out;
        const sg_sa_result& o = outs[members[a]];
        const int64_t egs = insts[members[a]]->e_gs;
        for (int rb = 0; rb < 32 * WGm; ++rb) {
            const int r = 32 * pl.w0 + rb;
            if (r >= pl.R) continue;
            o.E[r] = (int64_t)(long long)E[(size_t)q * 32 * WGm + rb];
            if (o.eps) o.eps[r] = (double)(o.E[r] - egs) / (double)(-egs);
        }
    }
    return SG_OK;
}

}  // namespace sg
