// fragment.cu -- the paper's linear-time meta-heuristic (Sec. II; App. A, Fig. 5) with
// simulated-annealing fragment optimisations, wave by wave on the GPU.
//
// Wave w = a + l*(b + l*c) fixes every spin whose coordinates are congruent to (a, b, c)
// mod l.  The fragment of such a spin is the cube of side l centred on it; with L a
// multiple of l the fragments of one wave are disjoint, so one launch anneals all of
// them.  A warp owns one fragment: its 32 reads are the 32 bits of one word per cube
// site, kept in shared memory for the whole anneal, beside the site's couplings (those
// of bonds leaving the cube cleared) and a list of the free sites of each colour.  Sites
// fixed by earlier waves hold all-equal words and are never updated.  Bonds may have
// |J| = 2 or 0: a site's positive bond terms are counted for all 32 reads at once in bit
// planes weighted by |J|, which gives x = s_i h_i of every read; only the reads with
// x < 0 take their draw and threshold one by one.  The read of lowest cube energy fixes
// the centre spin in global memory.
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kWarps = 4;  // fragments per block
constexpr int kLMax = 7;   // largest fragment side
constexpr int kVMax = kLMax * kLMax * kLMax;

struct FragArgs {
    int8_t* spins;                 // [I][N] logical order; 0 = not fixed yet
    const uint2* const* j6_ptrs;   // per instance: [N] six-coupling records (+x, -x, +y, -y, +z, -z)
    const RunKeys* keys;           // [I]
    const uint32_t* thr;           // [S][kThrRow]
    int L, l, S;
};

__device__ __forceinline__ int coupling(uint2 r, int q)
{
    return (int)(int8_t)(((q < 4 ? r.x : r.y) >> (8 * (q & 3))) & 0xFFu);
}

__global__ void __launch_bounds__(kWarps * 32) fragment_wave_kernel(const FragArgs a, int wave)
{
    __shared__ uint32_t s_words[kWarps][kVMax];  // bit r: read r's spin is -1
    __shared__ uint2 s_rec[kWarps][kVMax];       // couplings of the bonds inside the cube (others 0)
    __shared__ uint16_t s_free[kWarps][2][(kVMax + 1) / 2];  // free sites of each colour
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int inst = blockIdx.y;
    const int L = a.L, l = a.l, h = (l - 1) / 2, V = l * l * l;
    const int per = L / l;
    const int frag = blockIdx.x * kWarps + warp;
    if (frag >= per * per * per) return;  // the whole warp
    const int ca = wave % l, cb = (wave / l) % l, cc = wave / (l * l);
    const int cx = ca + l * (frag % per), cy = cb + l * ((frag / per) % per), cz = cc + l * (frag / (per * per));
    const uint32_t centre = (uint32_t)(cx + L * (cy + L * cz));
    const RunKeys key = a.keys[inst];
    const uint2* __restrict__ j6 = a.j6_ptrs[inst];
    int8_t* __restrict__ sp = a.spins + (size_t)inst * L * L * L;
    uint32_t* words = s_words[warp];
    uint2* recs = s_rec[warp];

    auto site_of = [&](int q, int* x, int* y, int* z) {
        const int dx = q % l, dy = (q / l) % l, dz = q / (l * l);
        *x = (cx + dx - h + L) % L;
        *y = (cy + dy - h + L) % L;
        *z = (cz + dz - h + L) % L;
    };
    // fixed by an earlier wave: its residue class precedes this wave's
    auto fixed = [&](int x, int y, int z) { return (x % l) + l * ((y % l) + l * (z % l)) < wave; };

    // cube sites: couplings of the bonds inside the cube, initial words, and the list of
    // the free sites of each colour (compacted by ballot, warp-uniform counts)
    int nfree[2] = {0, 0};
    for (int base = 0; base < V; base += 32) {
        const int q = base + lane;
        bool free_site = false;
        int colour = 0;
        if (q < V) {
            int x, y, z;
            site_of(q, &x, &y, &z);
            const int i = x + L * (y + L * z);
            const int dd[3] = {q % l, (q / l) % l, q / (l * l)};
            uint2 r = j6[i];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int up = 2 * d, dn = 2 * d + 1;  // record bytes of the +d and -d bonds
                if (dd[d] + 1 >= l) (up < 4 ? r.x : r.y) &= ~(0xFFu << (8 * (up & 3)));
                if (dd[d] == 0) (dn < 4 ? r.x : r.y) &= ~(0xFFu << (8 * (dn & 3)));
            }
            recs[q] = r;
            uint32_t word = 0;
            if (fixed(x, y, z)) {
                word = sp[i] < 0 ? 0xFFFFFFFFu : 0u;
            } else {
                free_site = true;
                colour = (x + y + z) & 1;
                for (int g = 0; g < 8; ++g) {
                    const Philox4 u = philox4x32_10(centre, kSweepInit, (uint32_t)(8 * q + g), kDomainFragment,
                                                    key.k0, key.k1);
#pragma unroll
                    for (int m = 0; m < 4; ++m) word |= (u.v[m] >> 31) << (4 * g + m);
                }
            }
            words[q] = word;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const bool mine = free_site && colour == c;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, mine);
            if (mine) s_free[warp][c][nfree[c] + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)q;
            nfree[c] += __popc(bal);
        }
    }
    __syncwarp();

    // One site, all 32 reads: with p_k the reads whose bond term J_k s_i s_k is positive,
    // x = s_i h_i = 2P - M for P = sum |J_k| p_k (kept as bit planes P0..P3) and
    // M = sum |J_k|.  x >= 0 accepts; the others compare their draw with thr[-x].
    for (int sw = 0; sw < a.S; ++sw) {
        const uint32_t* thr = a.thr + (size_t)sw * kThrRow;
        for (int colour = 0; colour < 2; ++colour) {
            for (int e = lane; e < nfree[colour]; e += 32) {
                const int q = s_free[warp][colour][e];
                const uint2 rec = recs[q];
                const uint32_t self = words[q];
                uint32_t P0 = 0, P1 = 0, P2 = 0, P3 = 0;
                int M = 0;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const int J = coupling(rec, k);
                    if (J == 0) continue;  // no bond (or one leaving the cube)
                    const int step = k < 2 ? 1 : k < 4 ? l : l * l;
                    const uint32_t eq = ~(self ^ words[(k & 1) ? q - step : q + step]);
                    const uint32_t p = J > 0 ? eq : ~eq;
                    if (J == 1 || J == -1) {  // add p at weight 1
                        const uint32_t c1 = P0 & p;
                        P0 ^= p;
                        const uint32_t c2 = P1 & c1;
                        P1 ^= c1;
                        P3 ^= P2 & c2;
                        P2 ^= c2;
                        M += 1;
                    } else {  // |J| = 2: add p at weight 2
                        const uint32_t c2 = P1 & p;
                        P1 ^= p;
                        P3 ^= P2 & c2;
                        P2 ^= c2;
                        M += 2;
                    }
                }
                // need: x < 0, i.e. P < T = ceil(M / 2) (borrow of P - T, LSB first)
                const int T = (M + 1) >> 1;
                uint32_t need = 0;
                {
                    const uint32_t Pj[4] = {P0, P1, P2, P3};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t tm = ((T >> j) & 1) ? 0xFFFFFFFFu : 0u;
                        need = (~Pj[j] & tm) | (~(Pj[j] ^ tm) & need);
                    }
                }
                uint32_t flip = ~need;
                for (int g = 0; g < 8; ++g) {  // reads 4g .. 4g + 3
                    const uint32_t nm = (need >> (4 * g)) & 0xFu;
                    if (!nm) continue;
                    const Philox4 u =
                        philox4x32_10(centre, (uint32_t)sw, (uint32_t)(8 * q + g), kDomainFragment, key.k0, key.k1);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (!((nm >> m) & 1u)) continue;
                        const int b = 4 * g + m;
                        const int Pb = (int)(((P0 >> b) & 1u) | (((P1 >> b) & 1u) << 1) | (((P2 >> b) & 1u) << 2) |
                                             (((P3 >> b) & 1u) << 3));
                        if (u.v[m] < thr[M - 2 * Pb]) flip |= 1u << b;
                    }
                }
                words[q] = self ^ flip;
            }
            __syncwarp();
        }
    }

    // lane r: the cube energy of read r (bonds inside the cube, each once)
    long long e = 0;
    for (int q = 0; q < V; ++q) {
        int x, y, z;
        site_of(q, &x, &y, &z);
        const uint2 rec = recs[q];
        const int dd[3] = {q % l, (q / l) % l, q / (l * l)};
        const int sq = ((words[q] >> lane) & 1u) ? -1 : 1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int step = d == 0 ? 1 : d == 1 ? l : l * l;
            if (dd[d] + 1 < l) e += (long long)coupling(rec, 2 * d) * sq * (((words[q + step] >> lane) & 1u) ? -1 : 1);
        }
    }
    // the first read of lowest energy
    long long be = e;
    int br = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long oe = __shfl_xor_sync(0xFFFFFFFFu, be, o);
        const int orr = __shfl_xor_sync(0xFFFFFFFFu, br, o);
        if (oe < be || (oe == be && orr < br)) {
            be = oe;
            br = orr;
        }
    }
    if (lane == 0) sp[centre] = ((words[h + l * (h + l * h)] >> br) & 1u) ? (int8_t)-1 : (int8_t)1;
}

// Exact zero-temperature fragment marginals (l <= 3): the centre spin of each fragment
// is set by comparing the lowest cube energy over the cube's free spins with s_c = +1 and
// with s_c = -1 (+1 on a tie).  One block per fragment; its threads split the 2^F states
// of the F free spins into contiguous stretches of the Gray-code order (state g(n) =
// n ^ (n >> 1)), each energy obtained from the previous one by the flipped spin's change.
constexpr int kTropBlock = 256;

__global__ void __launch_bounds__(kTropBlock) fragment_tropical_kernel(int8_t* spins, const uint2* const* j6_ptrs,
                                                                       int L, int l, int wave)
{
    __shared__ int s_F, s_cf;
    __shared__ int s_h[27], s_nn[27];
    __shared__ int s_nj[27][6], s_nJ[27][6];
    __shared__ int s_mp[kTropBlock / 32], s_mm[kTropBlock / 32];
    const int inst = blockIdx.y, tid = threadIdx.x;
    const int h = (l - 1) / 2, V = l * l * l, per = L / l;
    const int frag = blockIdx.x;
    const int ca = wave % l, cb = (wave / l) % l, cc = wave / (l * l);
    const int cx = ca + l * (frag % per), cy = cb + l * ((frag / per) % per), cz = cc + l * (frag / (per * per));
    int8_t* __restrict__ sp = spins + (size_t)inst * L * L * L;
    const uint2* __restrict__ j6 = j6_ptrs[inst];
    auto site_of = [&](int q) {
        const int dx = q % l, dy = (q / l) % l, dz = q / (l * l);
        return ((cx + dx - h + L) % L) + L * (((cy + dy - h + L) % L) + L * ((cz + dz - h + L) % L));
    };
    if (tid == 0) {
        int idx[27];
        int F = 0;
        for (int q = 0; q < V; ++q) idx[q] = sp[site_of(q)] != 0 ? -1 : F++;
        for (int k = 0; k < F; ++k) s_h[k] = 0, s_nn[k] = 0;
        for (int q = 0; q < V; ++q) {  // bonds inside the cube, each once (+x, +y, +z)
            const int dd[3] = {q % l, (q / l) % l, q / (l * l)};
            const uint2 rec = j6[site_of(q)];
            for (int d = 0; d < 3; ++d) {
                const int step = d == 0 ? 1 : d == 1 ? l : l * l;
                if (dd[d] + 1 >= l) continue;
                const int r = q + step;
                const int J = coupling(rec, 2 * d);
                if (idx[q] >= 0 && idx[r] >= 0) {
                    const int a = idx[q], b = idx[r];
                    s_nj[a][s_nn[a]] = b, s_nJ[a][s_nn[a]++] = J;
                    s_nj[b][s_nn[b]] = a, s_nJ[b][s_nn[b]++] = J;
                } else if (idx[q] >= 0) {
                    s_h[idx[q]] += J * sp[site_of(r)];
                } else if (idx[r] >= 0) {
                    s_h[idx[r]] += J * sp[site_of(q)];
                }
            }
        }
        s_F = F;
        s_cf = idx[h + l * (h + l * h)];
    }
    __syncthreads();
    const int F = s_F, cf = s_cf;
    const uint32_t total = 1u << F;
    const uint32_t seg = (total + kTropBlock - 1) / kTropBlock;
    const uint32_t n0 = tid * seg, n1 = min(n0 + seg, total);
    int mp = 0x7FFFFFFF, mm = 0x7FFFFFFF;
    if (n0 < total) {
        uint32_t st = n0 ^ (n0 >> 1);  // bit k set: free spin k is -1
        auto sv = [&](int k) { return ((st >> k) & 1u) ? -1 : 1; };
        int E = 0;
        for (int k = 0; k < F; ++k) {
            E += s_h[k] * sv(k);
            for (int t = 0; t < s_nn[k]; ++t)
                if (s_nj[k][t] > k) E += s_nJ[k][t] * sv(k) * sv(s_nj[k][t]);
        }
        if (sv(cf) > 0) mp = E; else mm = E;
        for (uint32_t n = n0 + 1; n < n1; ++n) {
            const int k = __ffs(n) - 1;  // the spin that flips from g(n - 1) to g(n)
            int field = s_h[k];
            for (int t = 0; t < s_nn[k]; ++t) field += s_nJ[k][t] * sv(s_nj[k][t]);
            E -= 2 * sv(k) * field;
            st ^= 1u << k;
            if (sv(cf) > 0) mp = min(mp, E); else mm = min(mm, E);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mp = min(mp, __shfl_xor_sync(0xFFFFFFFFu, mp, o));
        mm = min(mm, __shfl_xor_sync(0xFFFFFFFFu, mm, o));
    }
    if ((tid & 31) == 0) s_mp[tid >> 5] = mp, s_mm[tid >> 5] = mm;
    __syncthreads();
    if (tid == 0) {
        for (int k = 1; k < kTropBlock / 32; ++k) mp = min(mp, s_mp[k]), mm = min(mm, s_mm[k]);
        sp[cx + L * (cy + L * cz)] = mp <= mm ? (int8_t)1 : (int8_t)-1;
    }
}

int32_t check(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace

int32_t launch_fragment_waves(int8_t* spins, const uint2* const* j6_ptrs, const RunKeys* keys, const uint32_t* thr,
                              int I, int L, int l, int S, cudaStream_t st)
{
    FragArgs a{};
    a.spins = spins;
    a.j6_ptrs = j6_ptrs;
    a.keys = keys;
    a.thr = thr;
    a.L = L;
    a.l = l;
    a.S = S;
    const int per = L / l;
    const int frags = per * per * per;
    const dim3 grid((frags + kWarps - 1) / kWarps, I);
    for (int w = 0; w < l * l * l; ++w) {
        fragment_wave_kernel<<<grid, kWarps * 32, 0, st>>>(a, w);
        const int32_t rc = check("fragment_wave_kernel");
        if (rc != SG_OK) return rc;
    }
    return SG_OK;
}

int32_t launch_fragment_tropical_waves(int8_t* spins, const uint2* const* j6_ptrs, int I, int L, int l,
                                       cudaStream_t st)
{
    const int per = L / l;
    const dim3 grid(per * per * per, I);
    for (int w = 0; w < l * l * l; ++w) {
        fragment_tropical_kernel<<<grid, kTropBlock, 0, st>>>(spins, j6_ptrs, L, l, w);
        const int32_t rc = check("fragment_tropical_kernel");
        if (rc != SG_OK) return rc;
    }
    return SG_OK;
}

}  // namespace sg
