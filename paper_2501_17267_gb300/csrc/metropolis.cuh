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

// Bit 7 of each byte: byte of a < byte of b (unsigned).  The guarded subtraction gives, per
// byte, whether the low seven bits of a reach those of b; the top bits decide otherwise.
__device__ __forceinline__ uint32_t bytes_lt(uint32_t a, uint32_t b)
{
    const uint32_t d = (a | 0x80808080u) - (b & 0x7F7F7F7Fu);
    return ((~a & b) | (~(a ^ b) & ~d)) & 0x80808080u;
}

// Bit 7 of each byte: byte of a == byte of b.
__device__ __forceinline__ uint32_t bytes_eq(uint32_t a, uint32_t b)
{
    const uint32_t z = a ^ b;
    return ~(((z & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | z) & 0x80808080u;
}

// Leading-byte record of one word's four slots for unit couplings: byte b of x / y / z is
// the leading byte (thr >> 24) of slot b's threshold for k = 2 / 4 / 6.
__device__ __forceinline__ uint4 lead_record(const uint32_t* thr0, const uint32_t* thr1, const uint32_t* thr2,
                                             const uint32_t* thr3)
{
    const uint32_t* t[4] = {thr0, thr1, thr2, thr3};
    uint4 r = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        r.x |= (t[b][2] >> 24) << (8 * b);
        r.y |= (t[b][4] >> 24) << (8 * b);
        r.z |= (t[b][6] >> 24) << (8 * b);
    }
    return r;
}

// The draws.  Replica r = 4w + b compares U = A * 2^24 + B with thr[k], where the leading
// byte A is byte b of word w mod 4 of Philox(site, sweep, w / 4, 0) -- one block serves
// four words -- and B is word b of Philox(site, sweep, w, 4) >> 8.  A < thr >> 24 accepts,
// A > thr >> 24 rejects; only when they are equal (probability 1/256) is B drawn.
template <int WG>
__device__ __forceinline__ void lead_bytes(uint32_t site, uint32_t sweep, uint32_t w0, const RunKeys& key,
                                           uint32_t (&A)[WG])
{
    const Philox4 u = philox4x32_10(site, sweep, w0 >> 2, kDomainMetropolis, key.k0, key.k1);
    if constexpr (WG == 4) {
        A[0] = u.v[0]; A[1] = u.v[1]; A[2] = u.v[2]; A[3] = u.v[3];
    } else if constexpr (WG == 2) {
        const bool hi = (w0 & 2u) != 0;
        A[0] = hi ? u.v[2] : u.v[0];
        A[1] = hi ? u.v[3] : u.v[1];
    } else {
        const uint32_t m = w0 & 3u;
        A[0] = m == 0 ? u.v[0] : m == 1 ? u.v[1] : m == 2 ? u.v[2] : u.v[3];
    }
}

// Decides tied draws (leading byte equal to the threshold's): for each byte of `tie`
// (bit 7 set), accepted when the threshold has low bits and the draw's low 24 bits are
// below them.  thr_k(b) is the full threshold of byte b.  Kept out of line: it runs
// rarely, and one copy keeps the sweep loops small.
static __device__ __noinline__ uint32_t resolve_ties(uint32_t tie, uint32_t kidx, const uint32_t* __restrict__ row,
                                              int stride, uint32_t site, uint32_t sweep, uint32_t w, uint32_t k0,
                                              uint32_t k1)
{
    uint32_t low[4], any = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t kb = (kidx >> (8 * b)) & 0xFFu;
        low[b] = ((tie >> (8 * b + 7)) & 1u) ? row[b * stride + kb] & 0xFFFFFFu : 0u;
        any |= low[b];
    }
    if (!any) return 0;  // a threshold of exactly A * 2^24 rejects its tie
    const Philox4 t = philox4x32_10(site, sweep, w, kDomainTail, k0, k1);
    uint32_t acc = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if ((t.v[b] >> 8) < low[b]) acc |= 0x80u << (8 * b);
    return acc;
}

// Deferred ties of one warp: entries {logical site, storage index, word | tie bits << 16,
// k bytes}, decided later by the whole warp (sites of one colour never read one another,
// so a tie's flip may land after its neighbours' updates within the half sweep).
struct TieList {
    uint4* entries;
    int* count;
    int cap;
};

// Metropolis step for WG words (4*WG replicas) of one site; w0 % WG == 0.
//   self     spins of the site, updated in place
//   P        negative-term counts from the six neighbours
//   vmask    bit 7 of every byte that is a real replica
//   thr      PT: row of slot 4*w0 (rows THR_STRIDE apart); SA: the sweep's row
//   lead     UNITJ: leading-byte records (lead_record) -- PT: of words w0.., SA: one record
//   acc      PT energy lanes (see add_bytes)
//   ties     DEFER: where tied draws are queued (with the site's storage index `is`) for
//            the warp to decide later; a full list, or !DEFER, decides them here
// Returns true when some byte flipped.  The leading bytes depend only on (site, sweep,
// word), so their Philox block overlaps the neighbour loads.
template <bool PT, bool UNITJ, int WG, int THR_STRIDE, bool DEFER = false>
__device__ __forceinline__ bool update_words(uint32_t (&self)[WG], const uint32_t (&P)[WG],
                                             const uint32_t (&vmask)[WG], int msum, uint32_t site,
                                             uint32_t sweep, uint32_t w0, const RunKeys& key,
                                             const uint32_t* __restrict__ thr, const uint4* __restrict__ lead,
                                             uint32_t (&acc)[WG], const TieList* ties = nullptr,
                                             uint32_t is = 0)
{
    const uint32_t ones = 0x01010101u;
    const uint32_t C2 = (uint32_t)(2 * msum) * ones;
    const uint32_t T1 = (uint32_t)(msum + 1) * ones;
    const uint32_t Km = (uint32_t)msum * ones;
    uint32_t A[WG];
    lead_bytes<WG>(site, sweep, w0, key, A);
    bool any = false;
#pragma unroll
    for (int wi = 0; wi < WG; ++wi) {
        const uint32_t W = (P[wi] & ~self[wi]) | ((C2 - P[wi]) & self[wi]);
        const uint32_t Wg = W | 0x80808080u;              // guard bits: byte-wise subtraction, no borrows
        const uint32_t Kg = Wg - Km;                       // per byte 128 + k
        const uint32_t need = (Wg - T1) & vmask[wi];       // bit 7: k > 0, needs a draw
        uint32_t ff = prmt(vmask[wi] & ~need, 0u, 0xBA98u);  // 0xFF: flips for free
        const uint32_t nf = prmt(need, 0u, 0xBA98u);       // 0xFF: needs a draw
        const uint32_t kidx = Kg & 0x7F7F7F7Fu & nf;       // k, or 0
        const uint32_t* row = PT ? thr + 4 * wi * THR_STRIDE : thr;
        uint32_t lt, tie;
        if constexpr (UNITJ) {
            // k in {2, 4, 6}: pick each byte's leading threshold byte with two selects
            const uint4 r = PT ? lead[wi] : lead[0];
            const uint32_t s2 = ((kidx >> 1) & ones) * 0xFFu;  // k in {2, 6}
            const uint32_t s4 = ((kidx >> 2) & ones) * 0xFFu;  // k in {4, 6}
            const uint32_t t8 = (((r.z & s2) | (r.y & ~s2)) & s4) | (r.x & ~s4);
            lt = bytes_lt(A[wi], t8) & need;
            tie = bytes_eq(A[wi], t8) & need;
        } else {
            lt = 0;
            tie = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t kb = prmt(kidx, 0u, 0x4440u + b);
                const uint32_t t8 = (PT ? row[b * THR_STRIDE + kb] : row[kb]) >> 24;
                const uint32_t a = (A[wi] >> (8 * b)) & 0xFFu;
                lt |= (a < t8 ? 0x80u : 0u) << (8 * b);
                tie |= (a == t8 ? 0x80u : 0u) << (8 * b);
            }
            lt &= need;
            tie &= need;
        }
        if (tie) {
            int pos = ties ? ties->cap : 0;
            if (DEFER) pos = atomicAdd(ties->count, 1);
            if (DEFER && pos < ties->cap) {
                const uint32_t nib = (tie >> 7 & 1u) | (tie >> 14 & 2u) | (tie >> 21 & 4u) | (tie >> 28 & 8u);
                ties->entries[pos] = make_uint4(site, is, (w0 + (uint32_t)wi) | (nib << 16), kidx);
            } else {
                lt |= resolve_ties(tie, kidx, row, PT ? THR_STRIDE : 0, site, sweep, w0 + (uint32_t)wi, key.k0,
                                   key.k1);
            }
        }
        ff |= prmt(lt, 0u, 0xBA98u);
        self[wi] ^= ff & 0xFEFEFEFEu;
        any |= ff != 0;
        if (PT) acc[wi] = add_bytes(acc[wi], (Kg ^ 0x80808080u) & ff);  // k mod 256
    }
    return any;
}

}  // namespace mp
}  // namespace sg
