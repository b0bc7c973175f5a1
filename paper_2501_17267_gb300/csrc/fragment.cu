// fragment.cu -- the paper's linear-time meta-heuristic (Sec. II; App. A, Fig. 5) with
// simulated-annealing fragment optimisations, wave by wave on the GPU.
//
// Wave w = a + l*(b + l*c) fixes every spin whose coordinates are congruent to (a, b, c)
// mod l.  The fragment of such a spin is the cube of side l centred on it; with L a
// multiple of l the fragments of one wave are disjoint, so one launch anneals all of
// them.  A warp owns one fragment: its 32 reads are the 32 bits of one word per cube
// site, kept in shared memory for the whole anneal.  Sites fixed by earlier waves hold
// all-equal words and are never updated; only bonds inside the cube count.  Bonds may
// have |J| = 2 or 0, so each read is updated on its own (a fragment is at most 343
// sites).  The read of lowest cube energy fixes the centre spin in global memory.
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

    auto site_of = [&](int q, int* x, int* y, int* z) {
        const int dx = q % l, dy = (q / l) % l, dz = q / (l * l);
        *x = (cx + dx - h + L) % L;
        *y = (cy + dy - h + L) % L;
        *z = (cz + dz - h + L) % L;
    };
    // fixed by an earlier wave: its residue class precedes this wave's
    auto fixed = [&](int x, int y, int z) { return (x % l) + l * ((y % l) + l * (z % l)) < wave; };

    for (int q = lane; q < V; q += 32) {
        int x, y, z;
        site_of(q, &x, &y, &z);
        const int i = x + L * (y + L * z);
        uint32_t word = 0;
        if (fixed(x, y, z)) {
            word = sp[i] < 0 ? 0xFFFFFFFFu : 0u;
        } else {
            for (int g = 0; g < 8; ++g) {
                const Philox4 r = philox4x32_10(centre, kSweepInit, (uint32_t)(8 * q + g), kDomainFragment, key.k0,
                                                key.k1);
#pragma unroll
                for (int m = 0; m < 4; ++m) word |= (r.v[m] >> 31) << (4 * g + m);
            }
        }
        words[q] = word;
    }
    __syncwarp();

    for (int sw = 0; sw < a.S; ++sw) {
        const uint32_t* thr = a.thr + (size_t)sw * kThrRow;
        for (int colour = 0; colour < 2; ++colour) {
            for (int q = lane; q < V; q += 32) {
                int x, y, z;
                site_of(q, &x, &y, &z);
                if (((x + y + z) & 1) != colour || fixed(x, y, z)) continue;
                const uint2 rec = j6[x + L * (y + L * z)];
                const int dd[3] = {q % l, (q / l) % l, q / (l * l)};
                uint32_t nw[6];
                int J[6];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const int step = d == 0 ? 1 : d == 1 ? l : l * l;
                    const bool up = dd[d] + 1 < l, dn = dd[d] > 0;  // bond inside the cube
                    J[2 * d] = up ? coupling(rec, 2 * d) : 0;
                    J[2 * d + 1] = dn ? coupling(rec, 2 * d + 1) : 0;
                    nw[2 * d] = up ? words[q + step] : 0u;
                    nw[2 * d + 1] = dn ? words[q - step] : 0u;
                }
                const uint32_t self = words[q];
                uint32_t flip = 0;
                for (int g = 0; g < 8; ++g) {  // reads 4g .. 4g + 3
                    int xs[4];
                    bool need = false;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int b = 4 * g + m;
                        int hf = 0;
#pragma unroll
                        for (int k = 0; k < 6; ++k) hf += J[k] * (((nw[k] >> b) & 1u) ? -1 : 1);
                        xs[m] = (((self >> b) & 1u) ? -1 : 1) * hf;
                        need |= xs[m] < 0;
                    }
                    Philox4 u{};
                    if (need)
                        u = philox4x32_10(centre, (uint32_t)sw, (uint32_t)(8 * q + g), kDomainFragment, key.k0, key.k1);
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (xs[m] >= 0 || u.v[m] < thr[-xs[m]]) flip |= 1u << (4 * g + m);
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
        const uint2 rec = j6[x + L * (y + L * z)];
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

}  // namespace sg
