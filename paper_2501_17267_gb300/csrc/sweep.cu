// sweep.cu -- the Metropolis half-sweep kernel: the hot path (App. D.1, App. D.2).
//
// One launch updates every site of one checkerboard colour, for every replica of a
// group of instances.  Thread mapping (no division except one multiply-high per row):
//   blockIdx.y        instance
//   blockIdx.x, ty    rows (y, z) of the lattice; each thread walks `rows_per_thread` rows
//   tx = j * G + g    site j of the colour inside the row, word group g
// A word holds four replicas (one byte each).  Thread g of a site owns CH chunks of
// WG consecutive words, so it updates 4*WG*CH replicas with one decode of the site's
// couplings, and one Philox4x32-10 call per word (the counter (site, sweep, word, 0)
// names exactly that word's four replicas).
//
// Per word (bit layout in kernels.cu):
//   P  = sum_q ((n_q ^ S_q) & M_q)                 2|J| for each negative bond term
//   W  = s_i == +1 ? P : 2*sum|J| - P                2 * (weight of unsatisfied bonds)
//   k  = W - sum|J|  (= -x; flipping raises E by 2k)
// Bytes with k <= 0 flip unconditionally; the others flip when their Philox word is
// below thr[k].  "k > 0" is found for four bytes by one borrow-free subtraction; the
// draws are taken only when some lane of the warp needs one (a warp-uniform branch,
// so the WG Philox chains of a chunk interleave), and the byte decisions are
// branch-free.  For parallel tempering the energy change of every slot is summed in
// 8-bit lanes (at most 10 updates per thread, each adding <= 24) and reduced once per
// thread with warp reductions.
#include <stdlib.h>

#include "philox.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kThrStride = 17;   // per-slot threshold row stride in shared memory (bank spread)
constexpr int kMaxItems = 10;    // site updates per thread that fit the 8-bit energy lanes

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

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

struct SweepArgs {
    uint32_t* spins;
    const uint2* const* j6_ptrs;
    const RunKeys* keys;
    const uint32_t* thr;          // SA: one row of kThrRow; PT: [K][kThrRow]
    const uint8_t* rung_of_slot;  // PT: [I][Rp]
    int32_t* E;                   // PT: [I][Rp] energies, updated
    int L, Wn, Rvalid, G, rows_per_thread;
    uint32_t Lmagic;              // ceil(2^32 / L): row / L by multiply-high
    uint32_t sweep;
    int colour;
};

template <bool PT, bool UNITJ, int WG, int CH>
__global__ void __launch_bounds__(256) sweep_rows_kernel(const SweepArgs a)
{
    __shared__ uint32_t s_thr[PT ? 256 * kThrStride : kThrRow];
    __shared__ int s_dE[PT ? 256 : 1];

    const int inst = blockIdx.y;
    const int L = a.L, Wn = a.Wn, G = a.G;
    const int Rp = 4 * Wn;
    const int H = L >> 1;
    const int LL = L * L;
    const RunKeys key = a.keys[inst];
    const uint2* __restrict__ j6 = a.j6_ptrs[inst];
    uint32_t* __restrict__ s = a.spins + (size_t)inst * (size_t)LL * L * Wn;
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;

    if (PT) {
        for (int q = tid; q < Rp * kThrRow; q += nthreads) {
            const int slot = q / kThrRow, k = q % kThrRow;
            s_thr[slot * kThrStride + k] = a.thr[a.rung_of_slot[(size_t)inst * Rp + slot] * kThrRow + k];
        }
        for (int q = tid; q < Rp; q += nthreads) s_dE[q] = 0;
    } else {
        for (int q = tid; q < kThrRow; q += nthreads) s_thr[q] = a.thr[q];
    }
    __syncthreads();

    const int g = threadIdx.x % G;
    const int j0 = threadIdx.x / G;
    const int JX = blockDim.x / G;
    const int wbase = g * CH * WG;  // first word owned by this thread

    uint32_t vmask[CH][WG];  // bit 7 of each byte that is a real replica (not padding)
    uint32_t acc[CH][WG], cnt[CH][WG];
#pragma unroll
    for (int ch = 0; ch < CH; ++ch)
#pragma unroll
        for (int wi = 0; wi < WG; ++wi) {
            uint32_t m = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (4 * (wbase + ch * WG + wi) + b < a.Rvalid) m |= 0x80u << (8 * b);
            vmask[ch][wi] = m;
            acc[ch][wi] = 0;
            cnt[ch][wi] = 0;
        }

    const int row_base = blockIdx.x * blockDim.y * a.rows_per_thread + threadIdx.y;
    for (int c = 0; c < a.rows_per_thread; ++c) {
        const int row = row_base + c * blockDim.y;
        if (row >= LL) break;
        const int z = (int)__umulhi((uint32_t)row, a.Lmagic);
        const int y = row - z * L;
        const int par = (y + z + a.colour) & 1;
        const int dyp = (y + 1 == L ? 1 - L : 1) * L, dym = (y == 0 ? L - 1 : -1) * L;
        const int dzp = (z + 1 == L ? 1 - L : 1) * LL, dzm = (z == 0 ? L - 1 : -1) * LL;
        const int rowoff = row * L;
        for (int j = j0; j < H; j += JX) {
            const int x = 2 * j + par;
            const int i = rowoff + x;
            const int nb[6] = {x + 1 == L ? i + 1 - L : i + 1, x == 0 ? i + L - 1 : i - 1,
                               i + dyp, i + dym, i + dzp, i + dzm};

            // couplings of the site: sign masks S_q, magnitude masks M_q, sum |J|
            const uint2 r = j6[i];
            uint32_t S[6], M[6];
            int msum;
#pragma unroll
            for (int q = 0; q < 6; ++q) S[q] = prmt(r.x, r.y, (8u | q) * 0x1111u);
            if (UNITJ) {
#pragma unroll
                for (int q = 0; q < 6; ++q) M[q] = 0x02020202u;
                msum = 6;
            } else {
                const uint32_t sl = prmt(r.x, 0u, 0xBA98u), sh = prmt(r.y, 0u, 0xBA98u);
                const uint32_t al = (r.x ^ sl) + (sl & 0x01010101u);
                const uint32_t ah = (r.y ^ sh) + (sh & 0x01010101u);
                const uint32_t ml = al << 1, mh = ah << 1;
#pragma unroll
                for (int q = 0; q < 6; ++q) M[q] = prmt(ml, mh, (uint32_t)q * 0x1111u);
                msum = (int)__dp4a(al, 0x01010101u, __dp4a(ah, 0x01010101u, 0u));
            }
            const uint32_t ones = 0x01010101u;
            const uint32_t C2 = (uint32_t)(2 * msum) * ones;
            const uint32_t T1 = (uint32_t)(msum + 1) * ones;
            const uint32_t Km = (uint32_t)msum * ones;
            const uint32_t Bias = (uint32_t)(12 - msum) * ones;

#pragma unroll
            for (int ch = 0; ch < CH; ++ch) {
                const int w0 = wbase + ch * WG;
                uint32_t self[WG], P[WG];
                load_words<WG>(s + (size_t)i * Wn + w0, self);
#pragma unroll
                for (int wi = 0; wi < WG; ++wi) P[wi] = 0;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    uint32_t n[WG];
                    load_words<WG>(s + (size_t)nb[q] * Wn + w0, n);
#pragma unroll
                    for (int wi = 0; wi < WG; ++wi) P[wi] += (n[wi] ^ S[q]) & M[q];
                }
                uint32_t W[WG], need[WG], ff[WG];
                uint32_t anyneed = 0;
#pragma unroll
                for (int wi = 0; wi < WG; ++wi) {
                    W[wi] = (P[wi] & ~self[wi]) | ((C2 - P[wi]) & self[wi]);
                    need[wi] = ((W[wi] | 0x80808080u) - T1) & vmask[ch][wi];
                    ff[wi] = prmt(vmask[ch][wi] & ~need[wi], 0u, 0xBA98u);  // 0xFF: free flip
                    anyneed |= need[wi];
                }
                if (__any_sync(__activemask(), anyneed != 0)) {
#pragma unroll
                    for (int wi = 0; wi < WG; ++wi) {
                        const Philox4 u = philox4x32_10((uint32_t)i, a.sweep, (uint32_t)(w0 + wi),
                                                        kDomainMetropolis, key.k0, key.k1);
                        const uint32_t nf = prmt(need[wi], 0u, 0xBA98u);  // 0xFF: needs a draw
                        // k per byte, 0 where no draw is needed; the 0x80 guard bits keep
                        // the subtraction from borrowing across bytes
                        const uint32_t kidx = (((W[wi] | 0x80808080u) - Km) & 0x7F7F7F7Fu) & nf;
                        uint32_t ok = 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const uint32_t kb = prmt(kidx, 0u, 0x4440u + b);
                            const uint32_t th =
                                PT ? s_thr[(4 * (w0 + wi) + b) * kThrStride + kb] : s_thr[kb];
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
                    if (PT) {
                        acc[ch][wi] += (W[wi] + Bias) & ff[wi];  // k + 12 on flipped bytes
                        cnt[ch][wi] += ff[wi] & ones;
                    }
                }
                if (any) store_words<WG>(s + (size_t)i * Wn + w0, self);
            }
        }
    }

    if (PT) {
        // energy change per slot: 2 * (sum (k + 12) - 12 * flips), reduced over the
        // threads of a warp that own the same words.  Lanes are numbered by the linear
        // thread index; the last warp of a block may be partial and then adds directly.
        const int lane = tid & 31;
        const bool full = nthreads - (tid & ~31) >= 32;
        const bool full_warp_same = full && (G == 1);
        const bool shuffle_same = full && G < 32 && (32 % G) == 0;
#pragma unroll
        for (int ch = 0; ch < CH; ++ch)
#pragma unroll
            for (int wi = 0; wi < WG; ++wi)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int slot = 4 * (wbase + ch * WG + wi) + b;
                    int d = 2 * ((int)((acc[ch][wi] >> (8 * b)) & 0xFFu) -
                                 12 * (int)((cnt[ch][wi] >> (8 * b)) & 0xFFu));
                    if (full_warp_same) {
                        d = __reduce_add_sync(0xFFFFFFFFu, d);
                        if (lane == 0 && d) atomicAdd(&s_dE[slot], d);
                    } else if (shuffle_same) {
                        for (int off = G; off < 32; off <<= 1) d += __shfl_xor_sync(0xFFFFFFFFu, d, off);
                        if (lane < G && d) atomicAdd(&s_dE[slot], d);
                    } else if (d) {
                        atomicAdd(&s_dE[slot], d);
                    }
                }
        __syncthreads();
        int32_t* Ei = a.E + (size_t)inst * Rp;
        for (int q = tid; q < Rp; q += nthreads)
            if (s_dE[q]) atomicAdd(&Ei[q], s_dE[q]);
    }
}

struct SweepShape {
    dim3 block, grid;
    int G, CH, WG, rows_per_thread;
};

// Tuning knob: largest number of 4-word chunks per thread (1 or 2), from the
// environment variable SG_SWEEP_MAX_CH (default 2).
int max_chunks()
{
    static const int v = [] {
        const char* e = getenv("SG_SWEEP_MAX_CH");
        return (e && atoi(e) == 1) ? 1 : 2;
    }();
    return v;
}

SweepShape sweep_shape(int I, int L, int Wn)
{
    SweepShape sh;
    sh.WG = (Wn % 4 == 0) ? 4 : (Wn % 2 == 0) ? 2 : 1;
    sh.CH = (sh.WG == 4 && (Wn / 4) % 2 == 0 && max_chunks() == 2) ? 2 : 1;
    sh.G = Wn / (sh.WG * sh.CH);
    const int H = L / 2;
    int JX = 256 / sh.G;
    if (JX < 1) JX = 1;
    if (JX > H) JX = H;
    const int TX = sh.G * JX;
    int TY = 256 / TX;
    if (TY < 1) TY = 1;
    const int LL = L * L;
    if (TY > LL) TY = LL;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_row = (H + JX - 1) / JX;  // site updates per row per thread
    long long rpt = (long long)LL * I / ((long long)TY * 4 * sms);
    if (rpt < 1) rpt = 1;
    if (rpt > 8) rpt = 8;
    if (rpt * per_row > kMaxItems) rpt = kMaxItems / per_row;
    if (rpt < 1) rpt = 1;
    sh.rows_per_thread = (int)rpt;
    sh.block = dim3(TX, TY, 1);
    sh.grid = dim3((LL + TY * (int)rpt - 1) / (TY * (int)rpt), I, 1);
    return sh;
}

template <bool PT, bool UNITJ>
void launch_variant(const SweepShape& sh, const SweepArgs& a, int I, cudaStream_t st)
{
    (void)I;
    if (sh.WG == 4 && sh.CH == 2)
        sweep_rows_kernel<PT, UNITJ, 4, 2><<<sh.grid, sh.block, 0, st>>>(a);
    else if (sh.WG == 4)
        sweep_rows_kernel<PT, UNITJ, 4, 1><<<sh.grid, sh.block, 0, st>>>(a);
    else if (sh.WG == 2)
        sweep_rows_kernel<PT, UNITJ, 2, 1><<<sh.grid, sh.block, 0, st>>>(a);
    else
        sweep_rows_kernel<PT, UNITJ, 1, 1><<<sh.grid, sh.block, 0, st>>>(a);
}

template <bool PT>
int32_t launch_rows(SweepArgs a, int I, bool unit_j, cudaStream_t st)
{
    const SweepShape sh = sweep_shape(I, a.L, a.Wn);
    a.G = sh.G;
    a.rows_per_thread = sh.rows_per_thread;
    a.Lmagic = (uint32_t)((0x100000000ull + (uint64_t)a.L - 1) / (uint64_t)a.L);
    if (unit_j)
        launch_variant<PT, true>(sh, a, I, st);
    else
        launch_variant<PT, false>(sh, a, I, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("sweep launch failed: %s", cudaGetErrorString(e));
        return SG_ECUDA;
    }
    return SG_OK;
}

}  // namespace

bool rows_kernel_supports(int Wn)
{
    const int WG = (Wn % 4 == 0) ? 4 : (Wn % 2 == 0) ? 2 : 1;
    const int CH = (WG == 4 && (Wn / 4) % 2 == 0 && max_chunks() == 2) ? 2 : 1;
    return Wn / (WG * CH) <= 256;
}

int32_t launch_sweep_rows_sa(int8_t* spins, const uint2* const* j6_ptrs, const RunKeys* keys,
                             const uint32_t* thr_row, bool unit_j, int I, int L, int Wn, int R,
                             uint32_t sweep, int colour, cudaStream_t st)
{
    SweepArgs a{};
    a.spins = reinterpret_cast<uint32_t*>(spins);
    a.j6_ptrs = j6_ptrs;
    a.keys = keys;
    a.thr = thr_row;
    a.L = L;
    a.Wn = Wn;
    a.Rvalid = R;
    a.sweep = sweep;
    a.colour = colour;
    return launch_rows<false>(a, I, unit_j, st);
}

int32_t launch_sweep_rows_pt(int8_t* spins, const uint2* const* j6_ptrs, const RunKeys* keys,
                             const uint32_t* thr_rungs, const uint8_t* rung_of_slot, int32_t* E,
                             bool unit_j, int I, int L, int Wn, int K, uint32_t sweep, int colour,
                             cudaStream_t st)
{
    SweepArgs a{};
    a.spins = reinterpret_cast<uint32_t*>(spins);
    a.j6_ptrs = j6_ptrs;
    a.keys = keys;
    a.thr = thr_rungs;
    a.rung_of_slot = rung_of_slot;
    a.E = E;
    a.L = L;
    a.Wn = Wn;
    a.Rvalid = K;
    a.sweep = sweep;
    a.colour = colour;
    return launch_rows<true>(a, I, unit_j, st);
}

}  // namespace sg
