// metropolis.cuh -- the per-site Metropolis arithmetic shared by the sweep kernels
// (App. D.1 / D.2: flip when x = s_i * sum_j J_ij s_j >= 0, else when the draw
// u < thr[k], k = -x, thr[k] = floor(2^32 exp(-beta * 2k))).
//
// Spins are bit-packed: bit b of a 32-bit word is replica 32w + b of a site, 1 meaning
// spin -1.  With all |J| = 1 one word update is bit-sliced: for neighbour q with sign
// mask S_q (all ones when J_q < 0) the bond term J_q s_i s_q is negative -- the bond is
// satisfied -- exactly where self ^ n_q ^ S_q has a 1; six such indicator words go through
// a carry-save adder into three bit planes of the satisfied count c (0..6) of all 32
// replicas at once.  The flip costs dE = 2k with k = 2c - 6: free for c <= 3, else a draw
// decides with k = 2, 4, 6 for c = 4, 5, 6.
//
// Draws (our counter contract): the uniform U of replica 32w + b is A * 2^24 + B.  Bit j
// of its leading byte A is bit b of word j % 4 of Philox(site, sweep, 2w + j / 4, 0) --
// two blocks give the eight bit planes of all 32 leading bytes -- and B is the top 24 bits
// of word (32w + b) % 4 of Philox(site, sweep, (32w + b) / 4, 4).  U < thr[k] is decided
// by comparing A with the leading byte of thr[k] through a bit-sliced borrow chain, for
// all 32 replicas at once; only when the two bytes are equal (probability 1/256) is B
// drawn.
#pragma once
#include <stdint.h>

#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace mp {

constexpr int kRep = 32;  // replicas per spin word

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a | b)); }

// Sign masks of the six couplings of a site with all |J| = 1, from its byte of sign bits
// (bit q set when J_q < 0; q = +x, -x, +y, -y, +z, -z).
__device__ __forceinline__ void unit_signs(uint32_t bits, uint32_t (&S)[6])
{
#pragma unroll
    for (int q = 0; q < 6; ++q) S[q] = 0u - ((bits >> q) & 1u);
}

// Bit planes (c0, c1, c2) of the number of satisfied bonds of every replica.
__device__ __forceinline__ void satisfied_count(uint32_t self, const uint32_t (&n)[6], const uint32_t (&S)[6],
                                                uint32_t& c0, uint32_t& c1, uint32_t& c2)
{
    uint32_t a[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) a[q] = self ^ n[q] ^ S[q];
    const uint32_t s1 = a[0] ^ a[1] ^ a[2], k1 = maj3(a[0], a[1], a[2]);
    const uint32_t s2 = a[3] ^ a[4] ^ a[5], k2 = maj3(a[3], a[4], a[5]);
    c0 = s1 ^ s2;
    const uint32_t t = s1 & s2;
    c1 = k1 ^ k2 ^ t;
    c2 = maj3(k1, k2, t);
}

// The eight bit planes of the leading draw bytes of word w at (site, sweep).
__device__ __forceinline__ void lead_planes(uint32_t site, uint32_t sweep, uint32_t w, const RunKeys& key,
                                            uint32_t (&A)[8])
{
    const Philox4 p0 = philox4x32_10(site, sweep, 2u * w, kDomainMetropolis, key.k0, key.k1);
    const Philox4 p1 = philox4x32_10(site, sweep, 2u * w + 1u, kDomainMetropolis, key.k0, key.k1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        A[j] = p0.v[j];
        A[4 + j] = p1.v[j];
    }
}

// Threshold planes of a word: tp[8 * m + j], m = 0, 1, 2 for k = 2, 4, 6, has bit b equal to
// bit 24 + j of the threshold of slot 32w + b (of the sweep's row for SA).
__device__ __forceinline__ uint32_t threshold_plane_bit(uint32_t thr, int j) { return (thr >> (24 + j)) & 1u; }

// One word of unit-coupling updates.  valid: replicas that exist.  tp: the word's 24
// threshold planes.  Returns the replicas that flip now in *flip and those whose leading
// bytes tied in *tie (decided later by resolve_tie_bits); c0..c2 are the satisfied-count
// planes before the flip.
__device__ __forceinline__ void update_word_unit(uint32_t self, const uint32_t (&n)[6], const uint32_t (&S)[6],
                                                 uint32_t valid, const uint32_t (&tp)[24], const uint32_t (&A)[8],
                                                 uint32_t* flip, uint32_t* tie, uint32_t* c0, uint32_t* c1,
                                                 uint32_t* c2)
{
    satisfied_count(self, n, S, *c0, *c1, *c2);
    const uint32_t need = *c2 & valid;   // c >= 4: the flip raises the energy
    const uint32_t free = ~*c2 & valid;  // c <= 3: it does not
    // A < T through the borrow of A - T, least significant plane first: the borrow out
    // of a plane is the majority of (~A_j, T_j, borrow in), one three-input operation
    uint32_t lt = 0, eq = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        // threshold plane of each replica's k: c = 4 -> k = 2, c = 5 -> 4, c = 6 -> 6
        const uint32_t T = (*c1 & tp[16 + j]) | (~*c1 & ((*c0 & tp[8 + j]) | (~*c0 & tp[j])));
        lt = maj3(~A[j], T, lt);
        eq &= ~(A[j] ^ T);
    }
    *flip = free | (need & lt);
    *tie = need & eq;
}

// Satisfied-count planes after flipping `flip` (a flip turns c into 6 - c).
__device__ __forceinline__ void count_after_flip(uint32_t flip, uint32_t c0, uint32_t& c1, uint32_t& c2)
{
    const uint32_t n1 = c1 ^ (flip & ~c0);
    const uint32_t n2 = c2 ^ (flip & ~(c0 & c1));
    c1 = n1;
    c2 = n2;
}

// Adds the 3-bit value (a0, a1, a2) of every replica to the vertical counter V.
template <int NB>
__device__ __forceinline__ void vadd3(uint32_t (&V)[NB], uint32_t a0, uint32_t a1, uint32_t a2)
{
    uint32_t c = V[0] & a0;
    V[0] ^= a0;
    {
        const uint32_t t = V[1] ^ a1 ^ c;
        c = maj3(V[1], a1, c);
        V[1] = t;
    }
    {
        const uint32_t t = V[2] ^ a2 ^ c;
        c = maj3(V[2], a2, c);
        V[2] = t;
    }
#pragma unroll
    for (int j = 3; j < NB; ++j) {
        const uint32_t t = V[j] & c;
        V[j] ^= c;
        c = t;
    }
}

// Value of replica b in the vertical counter V.
template <int NB>
__device__ __forceinline__ int vcount(const uint32_t (&V)[NB], int b)
{
    int v = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) v |= (int)((V[j] >> b) & 1u) << j;
    return v;
}

// 32 x 32 bit transpose across a full warp: on return lane r holds the word whose bit l
// is bit r of lane l's x.
__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane)
{
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int s = 16 >> st;
        const uint32_t m = masks[st];
        const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, x, s);
        x = (lane & s) ? (((other >> s) & m) | (x & ~m)) : ((x & m) | ((other & m) << s));
    }
    return x;
}

// Decides tied draws: for each replica b of `tie`, k from its satisfied count (c0, c1 of
// c = 4, 5, 6), accepted when the threshold has low bits and the draw's low 24 bits are
// below them (a threshold of exactly A * 2^24 rejects).  thr(b, k) = row[b * stride + k].
// Out of line: it runs rarely, and one copy keeps the sweep loops small.
static __device__ __noinline__ uint32_t resolve_tie_bits(uint32_t tie, uint32_t c0, uint32_t c1,
                                                         const uint32_t* __restrict__ row, int stride, uint32_t site,
                                                         uint32_t sweep, uint32_t w, uint32_t k0, uint32_t k1)
{
    uint32_t acc = 0;
    while (tie) {
        const int b = __ffs(tie) - 1;
        tie &= tie - 1u;
        const int c = 4 + (int)((c0 >> b) & 1u) + 2 * (int)((c1 >> b) & 1u);
        const int k = 2 * c - 6;
        const uint32_t low = row[b * stride + k] & 0xFFFFFFu;
        if (!low) continue;
        const uint32_t slot = 32u * w + (uint32_t)b;
        const Philox4 t = philox4x32_10(site, sweep, slot >> 2, kDomainTail, k0, k1);
        const uint32_t m = slot & 3u;
        const uint32_t word = m == 0 ? t.v[0] : m == 1 ? t.v[1] : m == 2 ? t.v[2] : t.v[3];
        if ((word >> 8) < low) acc |= 1u << b;
    }
    return acc;
}

// General couplings (any |J| <= 2, zeros allowed): one word, replica by replica.  J[q] are
// the six couplings, row[b * stride + k] the threshold of replica b.  Returns the flips.
// Slow; used only for instances that are not all |J| = 1.
__device__ __forceinline__ uint32_t update_word_general(uint32_t self, const uint32_t (&n)[6], const int (&J)[6],
                                                        uint32_t valid, const uint32_t* __restrict__ row, int stride,
                                                        const uint32_t (&A)[8], uint32_t site, uint32_t sweep,
                                                        uint32_t w, const RunKeys& key)
{
    uint32_t flip = 0;
    for (int b = 0; b < 32; ++b) {
        if (!((valid >> b) & 1u)) continue;
        const int si = ((self >> b) & 1u) ? -1 : 1;
        int h = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) h += J[q] * (((n[q] >> b) & 1u) ? -1 : 1);
        const int k = -si * h;
        bool accept = k <= 0;
        if (!accept) {
            uint32_t a = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) a |= ((A[j] >> b) & 1u) << j;
            const uint32_t th = row[b * stride + k];
            const uint32_t t8 = th >> 24;
            accept = a < t8;
            if (a == t8 && (th & 0xFFFFFFu)) {
                const uint32_t slot = 32u * w + (uint32_t)b;
                const Philox4 t = philox4x32_10(site, sweep, slot >> 2, kDomainTail, key.k0, key.k1);
                const uint32_t m = slot & 3u;
                const uint32_t word = m == 0 ? t.v[0] : m == 1 ? t.v[1] : m == 2 ? t.v[2] : t.v[3];
                accept = (word >> 8) < (th & 0xFFFFFFu);
            }
        }
        if (accept) flip |= 1u << b;
    }
    return flip;
}

}  // namespace mp
}  // namespace sg
