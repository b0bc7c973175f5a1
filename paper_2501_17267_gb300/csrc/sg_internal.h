// sg_internal.h -- internal declarations shared by the libsg translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/sg.h"

namespace sg {

// ---- error reporting (thread-local message behind sg_last_error_string) ----
void set_error(const char* fmt, ...);
void clear_error();

struct Status {
    int32_t code = SG_OK;
    bool ok() const { return code == SG_OK; }
};

#define SG_TRY_CUDA(expr)                                                          \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            ::sg::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                            __FILE__, __LINE__);                                   \
            return SG_ECUDA;                                                       \
        }                                                                          \
    } while (0)

// ---- instances ----
struct DeviceCopy {
    int device = -1;
    uint2* j6 = nullptr;    // [N] per-site record of the six couplings (see kernels.cu)
    uint8_t* j1 = nullptr;  // [N] per-site sign bits of the six couplings (unit couplings)
};

}  // namespace sg

struct sg_instance {
    int32_t L = 0;
    int64_t N = 0;
    int64_t e_gs = 0;
    std::vector<int8_t> J3;      // [N][3]
    std::vector<int8_t> planted; // [N]
    int32_t abs_sum = 0;         // sum over edges of |J| (bounds energy gaps)
    bool unit_couplings = false; // every coupling is +1 or -1
    std::mutex mu;               // guards dev
    std::vector<sg::DeviceCopy> dev;
};

namespace sg {

// Host tile-planting generator (Sec. II).  Returns SG_OK or SG_EINVAL.
int32_t generate_instance(int L, uint64_t seed, const double class_prob[3], int gauge,
                          int8_t* J3, int8_t* planted, int64_t* e_gs);

// ---- schedules and acceptance tables (host) ----
// Metropolis thresholds for one beta: thr[k] = min(floor(2^32 exp(-beta*2k)), 2^32-1),
// k = 0..kMaxK (the accepted energy increase is dE = 2k; entry 0 is unused).
constexpr int kMaxK = 6 * SG_JMAX;  // largest |x| = sum of |J| over six neighbours
constexpr int kThrRow = 16;         // padded row length of a threshold table
void beta_schedule(int S, double b0, double b1, int geometric, double* beta);
void metropolis_row(double beta, uint32_t* row /* kThrRow */);
uint32_t exchange_threshold(double dbeta, int64_t d);

// PT exchange tables: per rung pair k, T_k(d) for d >= 1 is tab[off[k] + d - 1] when
// d <= len[k], else tail[k].
struct ExchangeTables {
    std::vector<uint32_t> tab;
    std::vector<uint32_t> off, len, tail;
};
int32_t build_exchange_tables(const std::vector<double>& ladder, int64_t dmax,
                              ExchangeTables* out);

// Per-instance device copy of the coupling records, uploaded on first use.
int32_t instance_device_j6(sg_instance* inst, cudaStream_t stream, const uint2** j6,
                           const uint8_t** j1);

// ---- spin words ----
// Spins are bit-packed 32 replicas to a 32-bit word (bit b of word w is replica 32w + b,
// set meaning -1); a run of R replicas keeps Wn = words_for(R) words per site and
// Rp = 32 * Wn replica slots.
inline int words_for(int replicas) { return (replicas + 31) / 32; }

// ---- spin storage order ----
// Within every row (y, z) of the lattice the L/2 sites with even x are stored first,
// then the L/2 sites with odd x, so that the sites of one checkerboard colour in a row
// are contiguous.  Logical site i = x + L*(y + L*z) keeps naming a site everywhere else
// (random-number counters, couplings, inputs and outputs).
#if defined(__CUDACC__)
#define SG_HDI __host__ __device__ __forceinline__
#else
#define SG_HDI inline
#endif
SG_HDI int64_t storage_of(int L, int64_t logical)
{
    const int64_t row = logical / L;
    const int x = (int)(logical - row * L);
    return row * L + (x & 1) * (L >> 1) + (x >> 1);
}
SG_HDI int64_t logical_of(int L, int64_t storage)
{
    const int64_t row = storage / L;
    const int pos = (int)(storage - row * L), H = L >> 1;
    return row * L + (pos < H ? 2 * pos : 2 * (pos - H) + 1);
}

// ---- batched annealing of uneven instances (batch.cu) ----
// One annealing chain slice: an instance and a group of WG consecutive replica words,
// spins [N][WG] words in storage order.
struct Plane {
    uint32_t* spins;        // [N][WG] words, storage order
    const uint8_t* j1;      // sign bits (unit couplings) or nullptr
    const uint2* j6;        // six-coupling records
    const uint32_t* thr;    // [S][kThrRow] thresholds of the plane's schedule
    uint32_t k0, k1;        // Philox key of the run
    int L, S, w0, R;        // side, sweeps, first word (of the instance) in the plane, replicas
    int s_begin, s_end;     // sweeps run by this launch: [s_begin, s_end)
    uint32_t Lmagic, Hmagic;  // ceil(2^32 / L), ceil(2^32 / (L/2))
    int out;                // index of the instance in the batch
};
// smem > 0: each block keeps its plane in that many bytes of shared memory
// (planes_smem_bytes gives the size for the largest side of the launch, 0 if it does not fit).
int32_t launch_sa_planes(int WG, const Plane* d_planes, const int* d_order, int n, unsigned* d_next,
                         bool unit, int blocks, cudaStream_t st, size_t smem = 0);
size_t planes_smem_bytes(int WG, int max_L);
int32_t launch_planes_init(int WG, const Plane* d_planes, int n, cudaStream_t st);
int32_t launch_planes_energy(int WG, const Plane* d_planes, int n, unsigned long long* E_out,
                             cudaStream_t st);
int planes_blocks(int WG, bool unit, size_t smem = 0);  // resident blocks of the plane kernel
// Runs members of a batch through one persistent plane kernel (device part captured as
// one CUDA graph unless disabled); reports whether a graph was used and the words per
// plane the autotuner chose.
int32_t run_sa_planes(const std::vector<int>& members, const sg_instance* const* insts,
                      const sg_sa_params* ps, sg_sa_result* outs, cudaStream_t st, bool* used_graph,
                      int* chosen_wg);

// ---- launch statistics shared by all run paths (api.cu) ----
bool stats_timing();
void stats_add(int kind, int64_t launches, int64_t units, double device_ms);

// ---- kernels (kernels.cu) ----
struct RunKeys {
    uint32_t k0, k1;
};
struct ExchangeArgs;  // exchange.cuh

int32_t launch_prepare_j6(const int8_t* J3_dev, uint2* j6_dev, uint8_t* j1_dev, int L,
                          cudaStream_t st);
int32_t launch_init_spins(int8_t* spins, const RunKeys* keys_dev, int I, int L, int Wn, int R,
                          cudaStream_t st);
// j1_ptrs (per instance sign bits) only when every coupling is +-1: the bit-sliced kernel
int32_t launch_energy(const int8_t* spins, const uint2* const* j6_ptrs, int I, int L, int Wn,
                      unsigned long long* E_out /* [I][32*Wn], added to */, cudaStream_t st,
                      const uint8_t* const* j1_ptrs = nullptr);
int32_t launch_half_sweep_sa(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_row /* kThrRow */, int32_t* E, int* status,
                             bool unit_j, int I, int L, int Wn, int R, uint32_t sweep, int colour,
                             cudaStream_t st);
int32_t launch_half_sweep_pt(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_rungs /* [K][kThrRow] */,
                             const uint8_t* rung_of_slot /* [I][32*Wn] */, int32_t* E, int* status,
                             bool unit_j, int I, int L, int Wn, int K, uint32_t sweep, int colour,
                             const ExchangeArgs* xch, unsigned* done, bool* fused,
                             cudaStream_t st);
// sweep.cu: the bit-sliced sweep kernel, one launch per colour (any word count)
// SA variant keeps no energies (the run recomputes them at the end);
// unit_j: every coupling of the group has |J| = 1.  With sweep_base the sweep index is
// *sweep_base + sweep, read on the device, and thr_row is the whole [S][kThrRow] table.
int32_t launch_sweep_rows_sa(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_row, bool unit_j, int I, int L, int Wn, int R,
                             uint32_t sweep, int colour, cudaStream_t st,
                             const uint32_t* sweep_base = nullptr, int* status = nullptr);
// PT: the colour-0 launch clears E [I][32*Wn] and the colour-1 launch sums every slot's
// energy afresh.  xch != nullptr: the colour-1 launch also performs the exchange (last
// block per instance); *fused reports whether it did.  done: [I] zeroed counters.
// status: unused (no launch of this kernel waits).  sms > 0: the launch shares the GPU
// with other work and is shaped for about that many SMs.
int32_t launch_sweep_rows_pt(int8_t* spins, const uint2* const* j6_ptrs,
                             const uint8_t* const* j1_ptrs, const RunKeys* keys,
                             const uint32_t* thr_rungs, const uint8_t* rung_of_slot, int32_t* E,
                             bool unit_j, int I, int L, int Wn, int K, uint32_t sweep, int colour,
                             const ExchangeArgs* xch, unsigned* done, bool* fused, cudaStream_t st,
                             const uint32_t* sweep_base = nullptr, int* status = nullptr, int sms = 0);
// cluster.cu: SA of small lattices, all sweeps in one launch, one thread-block cluster of C
// blocks per (word, instance); sa_cluster_blocks gives C and the threads a block (256 or
// 512), or 0 when the row kernel should run instead (long half sweeps, slabs too large, or
// more clusters than fit at once).
int sa_cluster_blocks(int I, int L, int Wn, int64_t half_sweep_attempts, int* threads);
int32_t launch_sa_cluster(int8_t* spins, const uint8_t* const* j1_ptrs, const RunKeys* keys,
                          const uint32_t* thr /* [S][kThrRow] */, int I, int L, int Wn, int R, int S, int C,
                          int threads, cudaStream_t st);
// The persistent cluster form for batches of one-word planes (batch.cu): C for planes of
// sides Ls (every side a multiple of C, the slab of the largest fitting), or 0.
int sa_cluster_list_blocks(const int* Ls, int n, int max_L);
int32_t launch_sa_cluster_planes(const Plane* d_planes, const int* d_order, int n, unsigned* d_next, int C,
                                 int max_L, cudaStream_t st);
// fragment.cu: the fragment meta-heuristic's waves (one launch per wave) on [I][N] int8 spins
// (0 = not fixed yet; all fixed on return), thr: [S][kThrRow] geometric schedule.
int32_t launch_fragment_waves(int8_t* spins, const uint2* const* j6_ptrs, const RunKeys* keys, const uint32_t* thr,
                              int I, int L, int l, int S, cudaStream_t st);
// the same waves with exact zero-temperature fragment marginals (l <= 3)
int32_t launch_fragment_tropical_waves(int8_t* spins, const uint2* const* j6_ptrs, int I, int L, int l,
                                       cudaStream_t st);
int32_t launch_pt_exchange(const ExchangeArgs& x, int I, uint32_t sweep, cudaStream_t st);
// ptcluster.cu: PT with unit couplings and K <= 32, every sweep of [s_begin, s_end) in one
// launch, one thread-block cluster of C blocks per instance (lattice in shared memory).
// pt_cluster_blocks gives C, or 0 when the row kernels should run the batch.
// bulk_signs: every instance's sign array is 16-byte aligned (slabs then come in by bulk copies).
// sweep_base: if set, the sweeps are *sweep_base + [s_begin, s_end) (graph replays).
struct ExchangeTablesDev {
    const uint32_t *tab, *off, *len, *tail;
};
int pt_cluster_blocks(int I, int L, int K);
// A batch too large for one wave of clusters but faster on them: C for the first *M
// instances on clusters (M < I, all resident at once), the others through the row kernels
// on the side_sms SMs the clusters leave; or 0.
int pt_cluster_split(int I, int L, int K, int* M, int* side_sms);
// ptcoop.cu: the same on one cooperative grid, each instance's rows split into row blocks
// held in shared memory (one block per SM).  pt_coop_plan gives the per-block plan
// (instance, rank, first row, rows; then per instance first block and block count; then
// the largest row count), the block count and the shared memory per block, or an empty plan.
struct CoopScratch {
    int* flags;     // [blocks]
    int* sums;      // [I][3][32]
    int* abort;     // [1]
    int* arrived;   // [I]
    uint32_t* pub;  // [blocks][2][2][L][L/2]
    const int* plan;
};
std::vector<int> pt_coop_plan(int I, int L, int K, int* blocks, size_t* smem_bytes);
int32_t launch_pt_coop(int8_t* spins, const uint8_t* const* j1_ptrs, const RunKeys* keys, const uint32_t* thr,
                       uint8_t* rung_of_slot, uint8_t* slot_of_rung, int32_t* E, unsigned long long* accepts,
                       int32_t* minE, const ExchangeTablesDev& xt, int* status, const CoopScratch& cs, int I,
                       int L, int K, int blocks, size_t smem_bytes, int s_begin, int s_end, long long wait_limit,
                       cudaStream_t st);
int32_t launch_pt_cluster(int8_t* spins, const uint8_t* const* j1_ptrs, const RunKeys* keys, const uint32_t* thr,
                          uint8_t* rung_of_slot, uint8_t* slot_of_rung, int32_t* E, unsigned long long* accepts,
                          int32_t* minE, const ExchangeTablesDev& xt, int* status, int I, int L, int K, int C,
                          int s_begin, int s_end, bool bulk_signs, cudaStream_t st,
                          const uint32_t* sweep_base = nullptr);
int32_t launch_pt_setup(const unsigned long long* E64, int32_t* E, uint8_t* rung_of_slot,
                        uint8_t* slot_of_rung, unsigned long long* accepts, int32_t* minE,
                        int I, int Rp, int K, cudaStream_t st);
int32_t launch_check_energy(const unsigned long long* E64, const int32_t* E, int I, int Rp,
                            int R, int* mismatch, cudaStream_t st);
int32_t launch_copy_energies(const unsigned long long* E64, int64_t* E, int n, cudaStream_t st);
int32_t launch_narrow_energy(const unsigned long long* E64, int32_t* E, int64_t n, cudaStream_t st);
// Rp = 32 * Wn; the int8 side is [R][N] in logical site order
int32_t launch_unpack_spins(const int8_t* spins, int8_t* out, int L, int Rp, int R,
                            int I_index, cudaStream_t st);
int32_t launch_pack_spins(const int8_t* in, int8_t* spins, int L, int Rp, int R, int* bad,
                          cudaStream_t st);

}  // namespace sg
