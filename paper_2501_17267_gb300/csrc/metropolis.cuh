// metropolis.cuh -- the per-site Metropolis arithmetic shared by the sweep kernels
// (App. D.1 / D.2: accept a flip with x = s_i * sum_j J_ij s_j when x >= 0, else when
// the draw u < thr[k], k = -x, thr[k] = floor(2^32 exp(-beta * 2k))).
//
// Four replicas of a site share one 32-bit word, one byte each: 0x01 is +1, 0xFF is -1,
// so bits 1..7 of a byte say "spin is -1".  For neighbour direction q let S_q be the
// all-ones word when J_q < 0 and M_q the byte pattern 2|J_q| (bit 1 or bit 2).  Then
// (n_q ^ S_q) & M_q is, per byte, 2|J_q| when J_q s_q < 0 and 0 otherwise; their sum
// P counts the negative bond terms seen from a +1 centre (2 sum|J| - P from a -1
// centre).  With W that count, x = sum|J| - W per byte and the energy rises by 2k,
// k = W - sum|J|.
#pragma once
#include <stdint.h>

#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace mp {

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// WG consecutive words (shared or global memory; WG = 4 and 2 need 16- and 8-byte
// alignment).
template <int WG>
__device__ __forceinline__ void load_words(const uint32_t* __restrict__ p, uint32_t (&w)[WG])
{
    if constexpr (WG == 4) {
        const uint4 t = *reinterpret_cast<const uint4*>(p);
        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
    } else if constexpr (WG == 2) {
        const uint2 t = *reinterpret_cast<const uint2*>(p);
        w[0] = t.x; w[1] = t.y;
    } else {
        w[0] = *p;
    }
}

template <int WG>
__device__ __forceinline__ void store_words(uint32_t* __restrict__ p, const uint32_t (&w)[WG])
{
    if constexpr (WG == 4) {
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (WG == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    } else {
        *p = w[0];
    }
}

// Couplings of one site: sign masks S_q, magnitude masks M_q and sum |J|.
struct Couplings {
    uint32_t S[6];
    uint32_t M[6];
    int msum;
};

// All couplings +-1: one byte of sign bits (bit q set when J_q < 0).
__device__ __forceinline__ Couplings decode_unit(uint32_t bits)
{
    Couplings c;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        c.S[q] = 0u - ((bits >> q) & 1u);
        c.M[q] = 0x02020202u;
    }
    c.msum = 6;
    return c;
}

// General couplings |J| <= 2: the eight-byte record, byte q = J_q (q = +x,-x,+y,-y,+z,-z).
__device__ __forceinline__ Couplings decode_general(uint2 r)
{
    Couplings c;
#pragma unroll
    for (int q = 0; q < 6; ++q) c.S[q] = prmt(r.x, r.y, (8u | q) * 0x1111u);
    const uint32_t sl = prmt(r.x, 0u, 0xBA98u), sh = prmt(r.y, 0u, 0xBA98u);
    const uint32_t al = (r.x ^ sl) + (sl & 0x01010101u);  // |J| per byte, no carries (|J| <= 2)
    const uint32_t ah = (r.y ^ sh) + (sh & 0x01010101u);
    const uint32_t ml = al << 1, mh = ah << 1;
#pragma unroll
    for (int q = 0; q < 6; ++q) c.M[q] = prmt(ml, mh, (uint32_t)q * 0x1111u);
    c.msum = (int)__dp4a(al, 0x01010101u, __dp4a(ah, 0x01010101u, 0u));
    return c;
}

// Adds neighbour word n seen along direction q to the negative-term count P.
__device__ __forceinline__ uint32_t bond_term(uint32_t n, const Couplings& c, int q)
{
    return (n ^ c.S[q]) & c.M[q];
}

// Energy lanes.  For parallel tempering each thread sums, per replica byte, the k of
// every flip it makes (the energy rises by 2k).  The four sums share one word: bytes are
// added modulo 256 without carries between them, which is exact while |sum| <= 127,
// i.e. for kLaneCapacity<KMAX> flips of |k| <= KMAX between folds.
template <int KMAX>
constexpr int kLaneCapacity = 127 / KMAX;

// Byte-wise a + b modulo 256 (no carry from one byte into the next).
__device__ __forceinline__ uint32_t add_bytes(uint32_t a, uint32_t b)
{
    return ((a & 0x7F7F7F7Fu) + (b & 0x7F7F7F7Fu)) ^ ((a ^ b) & 0x80808080u);
}

// Sum of byte b of a lane word, as a signed value.
__device__ __forceinline__ int lane_sum(uint32_t acc, int b)
{
    return (int)(int8_t)((acc >> (8 * b)) & 0xFFu);
}

// Metropolis step for WG words (4*WG replicas) of one site.
//   self     spins of the site, updated in place
//   P        negative-term counts from the six neighbours
//   vmask    bit 7 of every byte that is a real replica
//   thr      PT: row of slot 4*w0 (rows THR_STRIDE apart); SA: the sweep's row
//   acc      PT energy lanes (see add_bytes)
// Returns true when some byte flipped.
// DRAW_ALWAYS: compute the draws whether or not a byte needs one.  They depend only on
// (site, sweep, word), so the compiler can then overlap them with the loads of the
// neighbour words; otherwise they sit behind a warp-uniform "any draw needed" branch.
template <bool PT, int WG, int THR_STRIDE, bool DRAW_ALWAYS = false>
__device__ __forceinline__ bool update_words(uint32_t (&self)[WG], const uint32_t (&P)[WG],
                                             const uint32_t (&vmask)[WG], int msum, uint32_t site,
                                             uint32_t sweep, uint32_t w0, const RunKeys& key,
                                             const uint32_t* __restrict__ thr, uint32_t (&acc)[WG])
{
    const uint32_t ones = 0x01010101u;
    const uint32_t C2 = (uint32_t)(2 * msum) * ones;
    const uint32_t T1 = (uint32_t)(msum + 1) * ones;
    const uint32_t Km = (uint32_t)msum * ones;
    uint32_t W[WG], Kg[WG], need[WG], ff[WG];
    uint32_t anyneed = 0;
#pragma unroll
    for (int wi = 0; wi < WG; ++wi) {
        W[wi] = (P[wi] & ~self[wi]) | ((C2 - P[wi]) & self[wi]);
        const uint32_t Wg = W[wi] | 0x80808080u;  // guard bits: byte-wise subtraction, no borrows
        Kg[wi] = Wg - Km;                           // per byte 128 + k
        need[wi] = (Wg - T1) & vmask[wi];           // bit 7: k > 0, needs a draw
        ff[wi] = prmt(vmask[wi] & ~need[wi], 0u, 0xBA98u);  // 0xFF: flips for free
        anyneed |= need[wi];
    }
    if (DRAW_ALWAYS || __any_sync(__activemask(), anyneed != 0)) {
#pragma unroll
        for (int wi = 0; wi < WG; ++wi) {
            const Philox4 u = philox4x32_10(site, sweep, w0 + (uint32_t)wi, kDomainMetropolis,
                                            key.k0, key.k1);
            const uint32_t nf = prmt(need[wi], 0u, 0xBA98u);    // 0xFF: needs a draw
            const uint32_t kidx = Kg[wi] & 0x7F7F7F7Fu & nf;     // k, or 0
            const uint32_t* row = PT ? thr + 4 * wi * THR_STRIDE : thr;
            uint32_t ok = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t kb = prmt(kidx, 0u, 0x4440u + b);
                const uint32_t th = PT ? row[b * THR_STRIDE + kb] : row[kb];
                ok |= (u.v[b] < th) ? (0xFFu << (8 * b)) : 0u;
            }
            ff[wi] |= ok & nf;
        }
    }
    bool any = false;
#pragma unroll
    for (int wi = 0; wi < WG; ++wi) {
        self[wi] ^= ff[wi] & 0xFEFEFEFEu;
        any |= ff[wi] != 0;
        if (PT) acc[wi] = add_bytes(acc[wi], (Kg[wi] ^ 0x80808080u) & ff[wi]);  // k mod 256
    }
    return any;
}

}  // namespace mp
}  // namespace sg
