// exchange.cuh -- parallel-tempering label exchange for one instance (App. D.2),
// shared by the stand-alone exchange kernel and the sweep kernel that performs it in
// its last block.
//
// After sweep s, rung pairs (k, k+1) with k = s mod 2, s mod 2 + 2, ... try to swap the
// rungs their slots hold: with slot a at rung k and slot b at rung k+1 and d = E_a - E_b,
// the swap is accepted when d <= 0 or when the exchange draw u < T_k(d),
// T_k(d) = floor(2^32 exp(-(beta_{k+1} - beta_k) d)).  The pairs of one sweep are
// disjoint, so each is decided by its own thread.  The running minimum energy over all
// slots is updated afterwards.
#pragma once
#include <stdint.h>

#include "philox.cuh"
#include "sg_internal.h"

namespace sg {

struct ExchangeArgs {
    const RunKeys* keys;
    int32_t* E;                  // [I][Rp] slot energies
    uint8_t* rung_of_slot;       // [I][Rp]
    uint8_t* slot_of_rung;       // [I][K]
    unsigned long long* accepts; // [I][K-1]
    int32_t* minE;               // [I]
    const uint32_t* xtab;        // exchange thresholds, pair k: xtab[xoff[k] + d - 1], d <= xlen[k]
    const uint32_t* xoff;
    const uint32_t* xlen;
    const uint32_t* xtail;       // threshold for d > xlen[k]
    int Rp, K;
    const uint32_t* sweep_base;  // stand-alone kernel: if set, the sweep is *sweep_base + sweep
};

// Called by every thread of one block (tid in [0, nthreads)); s_min is shared scratch.
// E is read through L2 (ld.cg) because other blocks wrote it with atomics in this launch.
__device__ __forceinline__ void pt_exchange_block(const ExchangeArgs& x, int inst, uint32_t sweep,
                                                  int tid, int nthreads, int32_t* s_min)
{
    const RunKeys key = x.keys[inst];
    const int32_t* Ei = x.E + (size_t)inst * x.Rp;
    uint8_t* perm = x.rung_of_slot + (size_t)inst * x.Rp;
    uint8_t* inv = x.slot_of_rung + (size_t)inst * x.K;
    if (tid == 0) *s_min = 0x7FFFFFFF;
    __syncthreads();
    for (int j = tid;; j += nthreads) {
        const int k = 2 * j + (int)(sweep & 1u);
        if (k + 1 >= x.K) break;
        const int a = inv[k], b = inv[k + 1];
        const int64_t d = (int64_t)__ldcg(&Ei[a]) - (int64_t)__ldcg(&Ei[b]);
        bool accept = d <= 0;
        if (!accept) {
            const uint32_t u =
                philox4x32_10((uint32_t)k, sweep, 0u, kDomainExchange, key.k0, key.k1).v[0];
            const uint32_t T = d <= (int64_t)x.xlen[k] ? x.xtab[x.xoff[k] + (uint32_t)(d - 1)] : x.xtail[k];
            accept = u < T;
        }
        if (accept) {
            perm[a] = (uint8_t)(k + 1);
            perm[b] = (uint8_t)k;
            inv[k] = (uint8_t)b;
            inv[k + 1] = (uint8_t)a;
            x.accepts[(size_t)inst * (x.K - 1) + k] += 1ull;
        }
    }
    for (int r = tid; r < x.K; r += nthreads) atomicMin(s_min, __ldcg(&Ei[r]));
    __syncthreads();
    if (tid == 0 && *s_min < x.minE[inst]) x.minE[inst] = *s_min;
}

}  // namespace sg
