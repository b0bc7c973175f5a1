// kernels.cu -- device kernels of the Metropolis path (sm_103a).
//
// Device layout.  Spins of a run live as int8 [I][N][Rp]: instance, site in storage
// order (see storage_of: colour-split rows), replica (fastest), Rp = R rounded up to 4 so
// that one 32-bit word holds four replicas of one site (padding replicas stay +1 and
// never flip).  A thread owns one such word and updates its four replicas with
// SIMD-within-a-register arithmetic; one Philox4x32-10 call supplies the four
// draws, because the counter (site, sweep, word, 0) names exactly those four
// replicas.  Couplings of a site are one 8-byte record: byte q holds the int8
// coupling to the neighbour in direction q (+x, -x, +y, -y, +z, -z).
//
// Metropolis attempt (App. D.1 / D.2): with x = s_i * sum_q J_q s_q, flip when
// x >= 0, else when the draw u < thr[k], k = -x, thr[k] = floor(2^32 exp(-beta 2k)).
//
// SWAR form of x for four replicas at once.  A spin byte is 0x01 (+1) or 0xFF (-1),
// so bits 1..7 hold "s = -1".  For direction q let S_q be 0xFFFFFFFF when J_q < 0
// and M_q the byte pattern 2|J_q| (bit 1 or bit 2).  Then (n_q ^ S_q) & M_q is,
// per byte, 2|J_q| when J_q s_q < 0 and 0 otherwise.  Their sum P counts the
// negative bond terms seen from a +1 centre; for a -1 centre the count is
// 2 sum|J| - P.  With W the selected count, x = sum|J| - W per byte.
#include <stdio.h>

#include "exchange.cuh"
#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

struct SiteCouplings {
    uint32_t S[6];  // sign masks, 0 or 0xFFFFFFFF
    uint32_t M[6];  // 2|J| broadcast to every byte
    uint32_t C2;    // 2 * sum|J| broadcast to every byte
    int msum;       // sum|J|
};

__device__ __forceinline__ SiteCouplings decode_site(uint2 r)
{
    SiteCouplings c;
    const uint32_t sl = prmt(r.x, 0u, 0xBA98u), sh = prmt(r.y, 0u, 0xBA98u);
    const uint32_t al = (r.x ^ sl) + (sl & 0x01010101u);  // |J| per byte (no carries: |J| <= 2)
    const uint32_t ah = (r.y ^ sh) + (sh & 0x01010101u);
    const uint32_t ml = al << 1, mh = ah << 1;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        c.S[q] = prmt(r.x, r.y, (8u | q) * 0x1111u);
        c.M[q] = prmt(ml, mh, (uint32_t)q * 0x1111u);
    }
    c.msum = (int)__dp4a(al, 0x01010101u, __dp4a(ah, 0x01010101u, 0u));
    c.C2 = (uint32_t)(2 * c.msum) * 0x01010101u;
    return c;
}

struct SiteGeom {
    int64_t i;
    int64_t nb[6];  // +x, -x, +y, -y, +z, -z
};

// Site of colour `colour` with colour-index h in [0, N/2), and its six neighbours.
__device__ __forceinline__ SiteGeom colour_site(int64_t h, int L, int colour)
{
    const int half = L >> 1;
    const int hx = (int)(h % half);
    const int64_t row = h / half;
    const int y = (int)(row % L);
    const int z = (int)(row / L);
    const int x = 2 * hx + ((y + z + colour) & 1);
    const int xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
    const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    const int zp = z + 1 == L ? 0 : z + 1, zm = z == 0 ? L - 1 : z - 1;
    const int64_t LL = (int64_t)L * L;
    const int64_t base = (int64_t)L * y + LL * z;
    SiteGeom g;
    g.i = x + base;
    g.nb[0] = xp + base;
    g.nb[1] = xm + base;
    g.nb[2] = x + (int64_t)L * yp + LL * z;
    g.nb[3] = x + (int64_t)L * ym + LL * z;
    g.nb[4] = x + (int64_t)L * y + LL * zp;
    g.nb[5] = x + (int64_t)L * y + LL * zm;
    return g;
}

// ---------------------------------------------------------------- couplings

__global__ void prepare_j6_kernel(const int8_t* __restrict__ J3, uint2* __restrict__ j6,
                                  uint8_t* __restrict__ j1, int L)
{
    const int64_t N = (int64_t)L * L * L;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((int64_t)L * L));
        const int64_t LL = (int64_t)L * L;
        const int64_t bx = (x == 0 ? L - 1 : x - 1) + (int64_t)L * y + LL * z;
        const int64_t by = x + (int64_t)L * (y == 0 ? L - 1 : y - 1) + LL * z;
        const int64_t bz = x + (int64_t)L * y + LL * (z == 0 ? L - 1 : z - 1);
        const uint32_t b0 = (uint8_t)J3[3 * i + 0], b1 = (uint8_t)J3[3 * bx + 0];
        const uint32_t b2 = (uint8_t)J3[3 * i + 1], b3 = (uint8_t)J3[3 * by + 1];
        const uint32_t b4 = (uint8_t)J3[3 * i + 2], b5 = (uint8_t)J3[3 * bz + 2];
        j6[i] = make_uint2(b0 | (b1 << 8) | (b2 << 16) | (b3 << 24), b4 | (b5 << 8));
        // bit q: coupling q is negative (used only when every coupling is +-1)
        j1[i] = (uint8_t)((b0 >> 7) | ((b1 >> 7) << 1) | ((b2 >> 7) << 2) | ((b3 >> 7) << 3) |
                          ((b4 >> 7) << 4) | ((b5 >> 7) << 5));
    }
}

// ---------------------------------------------------------------- initial state

__global__ void init_spins_kernel(uint32_t* __restrict__ spins, const RunKeys* __restrict__ keys,
                                  int L, int Wn, int R)
{
    const int inst = blockIdx.y;
    const RunKeys key = keys[inst];
    const int64_t N = (int64_t)L * L * L;
    const int64_t items = N * Wn;
    uint32_t* s = spins + (int64_t)inst * items;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(t % Wn);
        const int64_t i = logical_of(L, t / Wn);
        const Philox4 r = philox4x32_10((uint32_t)i, kSweepInit, (uint32_t)w, kDomainMetropolis,
                                        key.k0, key.k1);
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const bool down = (4 * w + b < R) && (r.v[b] >> 31);
            word |= (down ? 0xFFu : 0x01u) << (8 * b);
        }
        s[t] = word;
    }
}

// ---------------------------------------------------------------- Metropolis half sweep

// One colour of one sweep.  Block y = instance.  Each thread keeps a fixed word w
// (the grid stride is a multiple of Wn) and walks colour sites.  MODE_PT selects a
// per-slot threshold row (slot -> rung through rung_of_slot); otherwise one row.
template <bool MODE_PT>
__global__ void __launch_bounds__(kBlock)
half_sweep_kernel(uint32_t* __restrict__ spins, const uint2* const* __restrict__ j6_ptrs,
                  const RunKeys* __restrict__ keys, const uint32_t* __restrict__ thr,
                  const uint8_t* __restrict__ rung_of_slot, int32_t* __restrict__ E, int L,
                  int Wn, int Rvalid, uint32_t sweep, int colour)
{
    __shared__ uint32_t s_thr[MODE_PT ? 256 * kThrRow : kThrRow];
    __shared__ int s_dE[4 * kBlock];

    const int inst = blockIdx.y;
    const int Rp = 4 * Wn;
    const int64_t N = (int64_t)L * L * L;
    const RunKeys key = keys[inst];
    const uint2* __restrict__ j6 = j6_ptrs[inst];
    uint32_t* __restrict__ s = spins + (int64_t)inst * N * Wn;

    if (MODE_PT) {
        for (int q = threadIdx.x; q < Rp * kThrRow; q += blockDim.x) {
            const int slot = q / kThrRow, k = q % kThrRow;
            const int rung = rung_of_slot[(int64_t)inst * Rp + slot];
            s_thr[q] = thr[rung * kThrRow + k];
        }
    } else {
        for (int q = threadIdx.x; q < kThrRow; q += blockDim.x) s_thr[q] = thr[q];
    }
    const bool small_w = Wn <= kBlock;
    if (small_w)
        for (int q = threadIdx.x; q < 4 * Wn; q += blockDim.x) s_dE[q] = 0;
    __syncthreads();

    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int w = (int)(t0 % Wn);
    int valid = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (4 * w + b < Rvalid) valid |= 1 << b;
    int dE[4] = {0, 0, 0, 0};

    const int64_t items = (N / 2) * Wn;
    for (int64_t t = t0; t < items; t += stride) {
        const int64_t h = t / Wn;
        const SiteGeom g = colour_site(h, L, colour);
        const SiteCouplings c = decode_site(j6[g.i]);
        const int64_t is = storage_of(L, g.i);
        const uint32_t self = s[is * Wn + w];
        uint32_t P = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) P += (s[storage_of(L, g.nb[q]) * Wn + w] ^ c.S[q]) & c.M[q];
        const uint32_t W = (P & ~self) | ((c.C2 - P) & self);

        uint32_t flip = 0;
        int kb[4];
        bool need = false;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            kb[b] = (int)((W >> (8 * b)) & 0xFFu) - c.msum;  // k = -x
            if (!((valid >> b) & 1)) continue;
            if (kb[b] <= 0) {
                flip |= 0xFEu << (8 * b);
                dE[b] += 2 * kb[b];
            } else {
                need = true;
            }
        }
        if (need) {
            // the draw of replica 4w + b: leading byte b of word w mod 4 of the block at
            // (site, sweep, w / 4, 0); its low 24 bits (word b of the block at
            // (site, sweep, w, 4), top 24 bits) only when the leading bytes tie
            const Philox4 u = philox4x32_10((uint32_t)g.i, sweep, (uint32_t)w >> 2, kDomainMetropolis,
                                            key.k0, key.k1);
            const int wm = w & 3;
            const uint32_t lead = wm == 0 ? u.v[0] : wm == 1 ? u.v[1] : wm == 2 ? u.v[2] : u.v[3];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (!((valid >> b) & 1) || kb[b] <= 0) continue;
                const uint32_t th = MODE_PT ? s_thr[(4 * w + b) * kThrRow + kb[b]] : s_thr[kb[b]];
                const uint32_t a8 = (lead >> (8 * b)) & 0xFFu, t8 = th >> 24;
                bool accept = a8 < t8;
                if (a8 == t8 && (th & 0xFFFFFFu)) {
                    const Philox4 t = philox4x32_10((uint32_t)g.i, sweep, (uint32_t)w, kDomainTail, key.k0, key.k1);
                    accept = (t.v[b] >> 8) < (th & 0xFFFFFFu);
                }
                if (accept) {
                    flip |= 0xFEu << (8 * b);
                    dE[b] += 2 * kb[b];
                }
            }
        }
        if (flip) s[is * Wn + w] = self ^ flip;
    }

    int32_t* Ei = E + (int64_t)inst * Rp;
    if (small_w) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (dE[b]) atomicAdd(&s_dE[4 * w + b], dE[b]);
        __syncthreads();
        for (int q = threadIdx.x; q < 4 * Wn; q += blockDim.x)
            if (s_dE[q]) atomicAdd(&Ei[q], s_dE[q]);
    } else {
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (dE[b]) atomicAdd(&Ei[4 * w + b], dE[b]);
    }
}

// ---------------------------------------------------------------- energy (Eq. 1)

__global__ void __launch_bounds__(kBlock)
energy_kernel(const uint32_t* __restrict__ spins, const uint2* const* __restrict__ j6_ptrs, int L,
              int Wn, unsigned long long* __restrict__ E_out)
{
    __shared__ long long s_E[4 * kBlock];
    const int inst = blockIdx.y;
    const int64_t N = (int64_t)L * L * L;
    const uint2* __restrict__ j6 = j6_ptrs[inst];
    const uint32_t* __restrict__ s = spins + (int64_t)inst * N * Wn;
    const bool small_w = Wn <= kBlock;
    if (small_w)
        for (int q = threadIdx.x; q < 4 * Wn; q += blockDim.x) s_E[q] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int w = (int)(t0 % Wn);
    long long acc[4] = {0, 0, 0, 0};
    const int64_t items = N * Wn;
    for (int64_t t = t0; t < items; t += stride) {
        const int64_t is = t / Wn;                // storage position
        const int64_t i = logical_of(L, is);      // logical site
        const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((int64_t)L * L));
        const int64_t LL = (int64_t)L * L;
        const int64_t fx = storage_of(L, (x + 1 == L ? 0 : x + 1) + (int64_t)L * y + LL * z);
        const int64_t fy = storage_of(L, x + (int64_t)L * (y + 1 == L ? 0 : y + 1) + LL * z);
        const int64_t fz = storage_of(L, x + (int64_t)L * y + LL * (z + 1 == L ? 0 : z + 1));
        const uint2 r = j6[i];
        const int J[3] = {(int)(int8_t)(r.x & 0xFF), (int)(int8_t)((r.x >> 16) & 0xFF),
                          (int)(int8_t)(r.y & 0xFF)};
        const uint32_t me = s[is * Wn + w];
        const uint32_t nb[3] = {s[fx * Wn + w], s[fy * Wn + w], s[fz * Wn + w]};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int si = (int)(int8_t)((me >> (8 * b)) & 0xFF);
#pragma unroll
            for (int d = 0; d < 3; ++d) acc[b] += J[d] * si * (int)(int8_t)((nb[d] >> (8 * b)) & 0xFF);
        }
    }
    unsigned long long* Ei = E_out + (int64_t)inst * 4 * Wn;
    if (small_w) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (acc[b]) atomicAdd((unsigned long long*)&s_E[4 * w + b], (unsigned long long)acc[b]);
        __syncthreads();
        for (int q = threadIdx.x; q < 4 * Wn; q += blockDim.x)
            if (s_E[q]) atomicAdd(&Ei[q], (unsigned long long)s_E[q]);
    } else {
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (acc[b]) atomicAdd(&Ei[4 * w + b], (unsigned long long)acc[b]);
    }
}

// Energy by rows (used when Wn divides the block size): every edge counted once, as a
// forward bond (+x, +y, +z) of its lower site, with 32-bit indexing.  Thread t owns word
// w = t % Wn of every (kBlock / Wn)-th site of a row, so its four byte sums belong to
// fixed slots.  Per site and byte, sum_d J_d s_i s_{i+e_d} = m3 - W3, where m3 = sum_d |J_d|
// and W3 adds 2|J_d| for every bond whose term J_d s_i s_j is negative; W3 <= 12 per byte,
// so 21 sites add up in the four bytes of one word without carries before a fold.
__global__ void __launch_bounds__(kBlock)
energy_rows_kernel(const uint32_t* __restrict__ spins, const uint2* const* __restrict__ j6_ptrs, int L,
                   int Wn, int rows_per_block, unsigned long long* __restrict__ E_out)
{
    __shared__ unsigned long long s_E[4 * kBlock];
    const int inst = blockIdx.y;
    const int LL = L * L, H = L >> 1;
    const uint2* __restrict__ j6 = j6_ptrs[inst];
    const uint32_t* __restrict__ s = spins + (size_t)inst * (size_t)LL * L * Wn;
    for (int q = threadIdx.x; q < 4 * Wn; q += blockDim.x) s_E[q] = 0;
    __syncthreads();
    const int w = threadIdx.x % Wn, s0 = threadIdx.x / Wn, ds = kBlock / Wn;
    long long m3sum = 0;
    long long acc[4] = {0, 0, 0, 0};
    uint32_t lanes = 0;
    int nl = 0;
    auto fold = [&]() {
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[b] += (lanes >> (8 * b)) & 0xFFu;
        lanes = 0;
        nl = 0;
    };
    const int r0 = blockIdx.x * rows_per_block;
    const int r1 = min(LL, r0 + rows_per_block);
    for (int r = r0; r < r1; ++r) {
        const int z = r / L, y = r - z * L;
        const int ryp = z * L + (y + 1 == L ? 0 : y + 1);
        const int rzp = (z + 1 == L ? 0 : z + 1) * L + y;
        const uint32_t* __restrict__ row = s + (size_t)r * L * Wn;
        const uint32_t* __restrict__ rowy = s + (size_t)ryp * L * Wn;
        const uint32_t* __restrict__ rowz = s + (size_t)rzp * L * Wn;
        for (int pos = s0; pos < L; pos += ds) {
            // colour-split storage: position pos holds x = 2j + par
            const int par = pos >= H ? 1 : 0;
            const int j = pos - par * H;
            const int x = 2 * j + par;
            const int posx = par ? (j + 1 == H ? 0 : j + 1) : H + j;  // site x + 1
            const uint2 rec = j6[r * L + x];
            const int Jd[3] = {(int)(int8_t)(rec.x & 0xFFu), (int)(int8_t)((rec.x >> 16) & 0xFFu),
                               (int)(int8_t)(rec.y & 0xFFu)};
            const uint32_t me = row[pos * Wn + w];
            const uint32_t nb[3] = {row[posx * Wn + w], rowy[pos * Wn + w], rowz[pos * Wn + w]};
            uint32_t W3 = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const uint32_t differ = (me ^ nb[d]) & 0x02020202u;  // 0x02 where the spins differ
                // negative term: J > 0 with different spins, J < 0 with equal spins
                const uint32_t neg = Jd[d] > 0 ? differ : Jd[d] < 0 ? differ ^ 0x02020202u : 0u;
                W3 += neg * (uint32_t)abs(Jd[d]);
                m3sum += abs(Jd[d]);
            }
            lanes += W3;
            if (++nl == 21) fold();
        }
    }
    fold();
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (m3sum - acc[b]) atomicAdd(&s_E[4 * w + b], (unsigned long long)(m3sum - acc[b]));
    __syncthreads();
    unsigned long long* Ei = E_out + (size_t)inst * 4 * Wn;
    for (int q = threadIdx.x; q < 4 * Wn; q += blockDim.x)
        if (s_E[q]) atomicAdd(&Ei[q], s_E[q]);
}

// ---------------------------------------------------------------- parallel tempering

__global__ void pt_setup_kernel(const unsigned long long* __restrict__ E64, int32_t* __restrict__ E,
                                uint8_t* __restrict__ rung_of_slot, uint8_t* __restrict__ slot_of_rung,
                                unsigned long long* __restrict__ accepts, int32_t* __restrict__ minE,
                                int Rp, int K)
{
    const int inst = blockIdx.x;
    __shared__ int32_t s_min;
    if (threadIdx.x == 0) s_min = 0x7FFFFFFF;
    __syncthreads();
    for (int r = threadIdx.x; r < Rp; r += blockDim.x) {
        const int32_t e = (int32_t)(long long)E64[(int64_t)inst * Rp + r];
        E[(int64_t)inst * Rp + r] = e;
        rung_of_slot[(int64_t)inst * Rp + r] = (uint8_t)(r < K ? r : 0);
        if (r < K) {
            slot_of_rung[(int64_t)inst * K + r] = (uint8_t)r;
            atomicMin(&s_min, e);
        }
        if (r + 1 < K) accepts[(int64_t)inst * (K - 1) + r] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) minE[inst] = s_min;
}

// Exchange attempts after sweep `sweep` (see exchange.cuh), one block per instance.
__global__ void pt_exchange_kernel(const ExchangeArgs x, uint32_t sweep)
{
    __shared__ int32_t s_min;
    const uint32_t s = sweep + (x.sweep_base ? *x.sweep_base : 0u);
    pt_exchange_block(x, blockIdx.x, s, threadIdx.x, blockDim.x, &s_min);
}

// ---------------------------------------------------------------- checks and layout

__global__ void narrow_energy_kernel(const unsigned long long* __restrict__ E64,
                                     int32_t* __restrict__ E, int64_t n)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        E[q] = (int32_t)(long long)E64[q];
}

__global__ void check_energy_kernel(const unsigned long long* __restrict__ E64,
                                    const int32_t* __restrict__ E, int Rp, int R, int I,
                                    int* __restrict__ mismatch)
{
    const int64_t n = (int64_t)I * Rp;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q % Rp);
        if (r < R && (long long)E64[q] != (long long)E[q]) atomicAdd(mismatch, 1);
    }
}

__global__ void unpack_spins_kernel(const int8_t* __restrict__ spins, int8_t* __restrict__ out,
                                    int L, int Rp, int R)
{
    const int64_t N = (int64_t)L * L * L;
    const int64_t n = (int64_t)R * N;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / N);
        const int64_t i = q % N;
        out[q] = spins[storage_of(L, i) * Rp + r];
    }
}

__global__ void pack_spins_kernel(const int8_t* __restrict__ in, int8_t* __restrict__ spins,
                                  int L, int Rp, int R, int* __restrict__ bad)
{
    const int64_t N = (int64_t)L * L * L;
    const int64_t n = (int64_t)Rp * N;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = logical_of(L, q / Rp);
        const int r = (int)(q % Rp);
        int8_t v = 1;
        if (r < R) {
            v = in[(int64_t)r * N + i];
            if (v != 1 && v != -1) {
                atomicAdd(bad, 1);
                v = 1;
            }
        }
        spins[q] = v;
    }
}

int grid_for(int64_t items, int multiple_of = 1, int cap = 1 << 20)
{
    int64_t b = (items + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    b = (b + multiple_of - 1) / multiple_of * multiple_of;
    return (int)b;
}

int gcd(int a, int b)
{
    while (b) {
        int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

int32_t check_launch(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s launch failed: %s", what, cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

// Blocks along x so that blocks*kBlock is a multiple of Wn (fixed word per thread).
int sweep_grid_x(int64_t items, int Wn)
{
    const int m = Wn / gcd(Wn, kBlock);
    return grid_for(items, m, 1 << 16);
}

}  // namespace

int32_t launch_prepare_j6(const int8_t* J3_dev, uint2* j6_dev, uint8_t* j1_dev, int L,
                          cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    prepare_j6_kernel<<<grid_for(N, 1, 4096), kBlock, 0, st>>>(J3_dev, j6_dev, j1_dev, L);
    return check_launch("prepare_j6");
}

int32_t launch_init_spins(int8_t* spins, const RunKeys* keys_dev, int I, int L, int Wn, int R,
                          cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    dim3 grid(grid_for(N * Wn, 1, 8192), I);
    init_spins_kernel<<<grid, kBlock, 0, st>>>((uint32_t*)spins, keys_dev, L, Wn, R);
    return check_launch("init_spins");
}

int32_t launch_energy(const int8_t* spins, const uint2* const* j6_ptrs, int I, int L, int Wn,
                      unsigned long long* E_out, cudaStream_t st)
{
    if (kBlock % Wn == 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int LL = L * L;
        int gx = (8 * sms + I - 1) / I;  // about eight blocks per SM over all instances
        if (gx > LL) gx = LL;
        if (gx < 1) gx = 1;
        const int rpb = (LL + gx - 1) / gx;
        dim3 grid((LL + rpb - 1) / rpb, I);
        energy_rows_kernel<<<grid, kBlock, 0, st>>>((const uint32_t*)spins, j6_ptrs, L, Wn, rpb, E_out);
        return check_launch("energy_rows");
    }
    const int64_t N = (int64_t)L * L * L;
    dim3 grid(sweep_grid_x(N * Wn, Wn), I);
    energy_kernel<<<grid, kBlock, 0, st>>>((const uint32_t*)spins, j6_ptrs, L, Wn, E_out);
    return check_launch("energy");
}

int32_t launch_half_sweep_sa(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_row, int32_t* E, int* status, bool unit_j, int I,
                             int L, int Wn, int R, uint32_t sweep, int colour, cudaStream_t st)
{
    if (tile_kernel_supports(I, L, Wn))
        return launch_sweep_tile(spins, j6_ptrs, j1_ptrs, keys, thr_row, nullptr, E, status, false,
                                 unit_j, I, L, Wn, R, sweep, colour, st);
    if (rows_kernel_supports(Wn))
        return launch_sweep_rows_sa(spins, j6_ptrs, j1_ptrs, keys, thr_row, unit_j, I, L, Wn, R, sweep,
                                    colour, st, nullptr, status);
    const int64_t N = (int64_t)L * L * L;
    dim3 grid(sweep_grid_x((N / 2) * Wn, Wn), I);
    half_sweep_kernel<false><<<grid, kBlock, 0, st>>>((uint32_t*)spins, j6_ptrs, keys, thr_row,
                                                     nullptr, E, L, Wn, R, sweep, colour);
    return check_launch("half_sweep_sa");
}

int32_t launch_half_sweep_pt(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_rungs, const uint8_t* rung_of_slot, int32_t* E,
                             int* status, bool unit_j, int I, int L, int Wn, int K, uint32_t sweep,
                             int colour, const ExchangeArgs* xch, unsigned* done, bool* fused,
                             cudaStream_t st)
{
    if (fused) *fused = false;
    if (tile_kernel_supports(I, L, Wn))
        return launch_sweep_tile(spins, j6_ptrs, j1_ptrs, keys, thr_rungs, rung_of_slot, E, status,
                                 true, unit_j, I, L, Wn, K, sweep, colour, st);
    if (rows_kernel_supports(Wn))
        return launch_sweep_rows_pt(spins, j6_ptrs, j1_ptrs, keys, thr_rungs, rung_of_slot, E, unit_j,
                                    I, L, Wn, K, sweep, colour, xch, done, fused, st, nullptr, status);
    const int64_t N = (int64_t)L * L * L;
    dim3 grid(sweep_grid_x((N / 2) * Wn, Wn), I);
    half_sweep_kernel<true><<<grid, kBlock, 0, st>>>((uint32_t*)spins, j6_ptrs, keys, thr_rungs,
                                                    rung_of_slot, E, L, Wn, K, sweep, colour);
    return check_launch("half_sweep_pt");
}

int32_t launch_pt_setup(const unsigned long long* E64, int32_t* E, uint8_t* rung_of_slot,
                        uint8_t* slot_of_rung, unsigned long long* accepts, int32_t* minE, int I,
                        int Rp, int K, cudaStream_t st)
{
    pt_setup_kernel<<<I, kBlock, 0, st>>>(E64, E, rung_of_slot, slot_of_rung, accepts, minE, Rp, K);
    return check_launch("pt_setup");
}

int32_t launch_pt_exchange(const ExchangeArgs& x, int I, uint32_t sweep, cudaStream_t st)
{
    pt_exchange_kernel<<<I, 128, 0, st>>>(x, sweep);
    return check_launch("pt_exchange");
}

int32_t launch_check_energy(const unsigned long long* E64, const int32_t* E, int I, int Rp, int R,
                            int* mismatch, cudaStream_t st)
{
    check_energy_kernel<<<grid_for((int64_t)I * Rp, 1, 1024), kBlock, 0, st>>>(E64, E, Rp, R, I,
                                                                                mismatch);
    return check_launch("check_energy");
}

namespace {
__global__ void copy_energies_kernel(const unsigned long long* __restrict__ E64,
                                     int64_t* __restrict__ E, int n)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        E[q] = (int64_t)(long long)E64[q];
}
}  // namespace

int32_t launch_copy_energies(const unsigned long long* E64, int64_t* E, int n, cudaStream_t st)
{
    copy_energies_kernel<<<grid_for(n, 1, 1024), kBlock, 0, st>>>(E64, E, n);
    return check_launch("copy_energies");
}

int32_t launch_narrow_energy(const unsigned long long* E64, int32_t* E, int64_t n, cudaStream_t st)
{
    narrow_energy_kernel<<<grid_for(n, 1, 1024), kBlock, 0, st>>>(E64, E, n);
    return check_launch("narrow_energy");
}

int32_t launch_unpack_spins(const int8_t* spins, int8_t* out, int L, int Rp, int R, int I_index,
                            cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    unpack_spins_kernel<<<grid_for((int64_t)R * N, 1, 8192), kBlock, 0, st>>>(
        spins + (int64_t)I_index * N * Rp, out, L, Rp, R);
    return check_launch("unpack_spins");
}

int32_t launch_pack_spins(const int8_t* in, int8_t* spins, int L, int Rp, int R, int* bad,
                          cudaStream_t st)
{
    const int64_t N = (int64_t)L * L * L;
    pack_spins_kernel<<<grid_for((int64_t)Rp * N, 1, 8192), kBlock, 0, st>>>(in, spins, L, Rp, R, bad);
    return check_launch("pack_spins");
}

}  // namespace sg
