// api.cu -- the C ABI entry points: validation, device workspace, launch sequence.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <tuple>

#include "exchange.cuh"
#include "sg_internal.h"

namespace sg {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

namespace {

// ---- launch statistics: counts always, CUDA-event durations when enabled ----
struct Stats {
    std::mutex mu;
    bool timing = false;
    sg_kernel_stats totals{};
    std::vector<cudaEvent_t> pool;
};
Stats& stats()
{
    static Stats s;
    return s;
}

}  // namespace

bool stats_timing()
{
    std::lock_guard<std::mutex> g(stats().mu);
    return stats().timing;
}

void stats_add(int kind, int64_t launches, int64_t units, double device_ms)
{
    std::lock_guard<std::mutex> g(stats().mu);
    stats().totals.launches[kind] += launches;
    stats().totals.units[kind] += units;
    stats().totals.device_ms[kind] += device_ms;
}

namespace {

// Per-run recorder.  Each launch is counted; with timing on it is bracketed by two
// events on its stream, resolved by finish() once the run has synchronised.
class LaunchLog {
  public:
    LaunchLog()
    {
        std::lock_guard<std::mutex> g(stats().mu);
        timing_ = stats().timing;
    }
    ~LaunchLog() { release(); }
    // launches: kernels the call enqueues (a graph launch enqueues many)
    template <class F>
    int32_t run(int kind, int64_t units, cudaStream_t st, F&& launch, int64_t launches = 1)
    {
        cudaEvent_t a = nullptr, b = nullptr;
        if (timing_) {
            a = take();
            b = take();
            if (a && b) cudaEventRecord(a, st);
        }
        const int32_t rc = launch();
        if (timing_ && a && b) {
            cudaEventRecord(b, st);
            pending_.push_back({kind, a, b});
        } else {
            give(a);
            give(b);
        }
        {
            std::lock_guard<std::mutex> g(stats().mu);
            stats().totals.launches[kind] += launches;
            stats().totals.units[kind] += units;
        }
        return rc;
    }
    // Call after the stream has been synchronised.
    void finish()
    {
        double ms[SG_KERNEL_KINDS] = {0};
        for (auto& p : pending_) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.kind] += t;
        }
        {
            std::lock_guard<std::mutex> g(stats().mu);
            for (int k = 0; k < SG_KERNEL_KINDS; ++k) stats().totals.device_ms[k] += ms[k];
        }
        release();
    }

  private:
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    cudaEvent_t take()
    {
        {
            std::lock_guard<std::mutex> g(stats().mu);
            if (!stats().pool.empty()) {
                cudaEvent_t e = stats().pool.back();
                stats().pool.pop_back();
                return e;
            }
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    void give(cudaEvent_t e)
    {
        if (!e) return;
        std::lock_guard<std::mutex> g(stats().mu);
        stats().pool.push_back(e);
    }
    void release()
    {
        for (auto& p : pending_) {
            give(p.a);
            give(p.b);
        }
        pending_.clear();
    }
    bool timing_ = false;
    std::vector<Pending> pending_;
};

// Stream-ordered device allocation released when the owner goes out of scope.
class DevBuf {
  public:
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf()
    {
        if (p_) cudaFreeAsync(p_, st_);
    }
    int32_t alloc(size_t bytes, cudaStream_t st)
    {
        st_ = st;
        cudaError_t e = cudaMallocAsync(&p_, bytes ? bytes : 16, st);
        if (e != cudaSuccess) {
            p_ = nullptr;
            cudaGetLastError();
            set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            return SG_ENOMEM;
        }
        return SG_OK;
    }
    template <class T>
    T* as() const
    {
        return reinterpret_cast<T*>(p_);
    }

  private:
    void* p_ = nullptr;
    cudaStream_t st_ = nullptr;
};

#define SG_RET(expr)                    \
    do {                                \
        int32_t _rc = (expr);           \
        if (_rc != SG_OK) return _rc;   \
    } while (0)

__global__ void advance_sweep_base(uint32_t* base, uint32_t by) { *base += by; }

// Runs sweeps 0 .. S-1 as CUDA graphs of up to kGraphSweeps sweeps each, so that the host
// issues one launch per chunk instead of two or three per sweep and a slow host cannot
// leave the GPU idle between sweeps.  enqueue(cs, c) puts sweep c of a chunk on stream cs
// with the sweep index read on the device as *base + c; every chunk ends by advancing
// *base.  per_sweep_launches and units_per_sweep feed the launch statistics.
constexpr int kGraphSweeps = 100;

int32_t run_sweep_graphs(int S, uint32_t* base, cudaStream_t st, LaunchLog& log, int per_sweep_launches,
                         int64_t units_per_sweep, const std::function<int32_t(cudaStream_t, int)>& enqueue)
{
    SG_TRY_CUDA(cudaMemsetAsync(base, 0, sizeof(uint32_t), st));
    struct Graphs {
        cudaStream_t cs = nullptr;
        std::map<int, cudaGraphExec_t> ex;
        ~Graphs()
        {
            for (auto& kv : ex) cudaGraphExecDestroy(kv.second);
            if (cs) cudaStreamDestroy(cs);
        }
    } g;
    SG_TRY_CUDA(cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking));
    auto capture = [&](int n) -> int32_t {
        SG_TRY_CUDA(cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeThreadLocal));
        int32_t rc = SG_OK;
        for (int c = 0; c < n && rc == SG_OK; ++c) rc = enqueue(g.cs, c);
        if (rc == SG_OK) {
            advance_sweep_base<<<1, 1, 0, g.cs>>>(base, (uint32_t)n);
            if (cudaGetLastError() != cudaSuccess) rc = SG_ECUDA;
        }
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g.cs, &gr);
        cudaGraphExec_t ge = nullptr;
        if (rc == SG_OK && (e != cudaSuccess || cudaGraphInstantiate(&ge, gr, 0) != cudaSuccess)) rc = SG_ECUDA;
        if (gr) cudaGraphDestroy(gr);
        if (rc != SG_OK) {
            cudaGetLastError();
            if (!*sg_last_error_string()) set_error("capturing a graph of %d sweeps failed", n);
            return rc;
        }
        g.ex[n] = ge;
        return SG_OK;
    };
    for (int done = 0; done < S;) {
        const int n = std::min(kGraphSweeps, S - done);
        if (!g.ex.count(n)) SG_RET(capture(n));
        cudaGraphExec_t ge = g.ex[n];
        SG_RET(log.run(SG_KERNEL_SWEEP, units_per_sweep * n, st, [&]() -> int32_t {
            const cudaError_t e = cudaGraphLaunch(ge, st);
            if (e != cudaSuccess) {
                set_error("graph launch failed: %s", cudaGetErrorString(e));
                return SG_ECUDA;
            }
            return SG_OK;
        }, (int64_t)per_sweep_launches * n + 1));
        done += n;
    }
    return SG_OK;
}

// Runs of at least this many sweeps go through graphs; shorter ones launch directly.
constexpr int kGraphMinSweeps = 16;

// Sweeps per launch of the thread-block-cluster and cooperative PT kernels (state carried
// in device memory between launches).
constexpr int kClusterChunkSweeps = 2000;

// Polls a bounded wait of the cooperative PT kernel makes before it gives up (each a read
// through L2, well under a microsecond, so several seconds in all); SG_WAIT_LIMIT
// overrides it (a test sets 0 to make a wait give up on purpose).
long long wait_limit()
{
    const char* e = getenv("SG_WAIT_LIMIT");
    if (e && *e) {
        const long long v = atoll(e);
        if (v >= 0) return v;
    }
    return 1ll << 24;
}

// Whether a PT batch goes to the cooperative kernel.  Knob SG_PT_COOP = 0 / 1 turns it
// off / on; otherwise it is off.
bool pt_coop_wanted(int I, int L, int K)
{
    const char* e = getenv("SG_PT_COOP");
    if (e && *e) return atoi(e) != 0;
    (void)I;
    (void)L;
    (void)K;
    return false;
}

// Instances per launch group: the grid's y extent holds one instance per row.
constexpr size_t kMaxGroup = 65535;

RunKeys make_key(uint64_t seed, uint32_t instance_id)
{
    return RunKeys{(uint32_t)seed, (uint32_t)(seed >> 32) ^ instance_id};
}

double eps_of(int64_t E, int64_t egs) { return (double)(E - egs) / (double)(-egs); }

bool beta_ok(double b) { return b > 0 && isfinite(b); }

int32_t check_sa(const sg_instance* inst, const sg_sa_params* p, const sg_sa_result* o)
{
    if (!inst || !p || !o) {
        set_error("NULL argument");
        return SG_EINVAL;
    }
    if (p->replicas < 1 || p->replicas > (1 << 20)) {
        set_error("replicas must be in [1, 2^20] (got %d)", p->replicas);
        return SG_EINVAL;
    }
    if (p->sweeps < 0) {
        set_error("sweeps must be >= 0");
        return SG_EINVAL;
    }
    if (!beta_ok(p->beta0) || !beta_ok(p->beta1)) {
        set_error("beta0 and beta1 must be finite and > 0");
        return SG_EINVAL;
    }
    if (p->schedule != SG_SCHEDULE_LINEAR && p->schedule != SG_SCHEDULE_GEOMETRIC) {
        set_error("unknown schedule %d", p->schedule);
        return SG_EINVAL;
    }
    if (!o->E) {
        set_error("result E must not be NULL");
        return SG_EINVAL;
    }
    if (o->spins && o->spins_mem != SG_MEM_HOST && o->spins_mem != SG_MEM_DEVICE) {
        set_error("bad spins_mem");
        return SG_EINVAL;
    }
    return SG_OK;
}

int32_t check_pt(const sg_instance* inst, const sg_pt_params* p, const sg_pt_result* o)
{
    if (!inst || !p || !o) {
        set_error("NULL argument");
        return SG_EINVAL;
    }
    if (p->temps < 1 || p->temps > 256) {
        set_error("temps must be in [1, 256] (got %d)", p->temps);
        return SG_EINVAL;
    }
    if (p->sweeps < 0) {
        set_error("sweeps must be >= 0");
        return SG_EINVAL;
    }
    if (!beta_ok(p->beta_min) || !beta_ok(p->beta_max)) {
        set_error("beta_min and beta_max must be finite and > 0");
        return SG_EINVAL;
    }
    if (o->spins && o->spins_mem != SG_MEM_HOST && o->spins_mem != SG_MEM_DEVICE) {
        set_error("bad spins_mem");
        return SG_EINVAL;
    }
    return SG_OK;
}

// Shared tail of a run: copy the spins of instance `idx` out of the packed layout.
int32_t emit_spins(const int8_t* packed, int idx, int L, int Rp, int R, int8_t* dst, int mem,
                   cudaStream_t st, DevBuf* staging, LaunchLog* log)
{
    if (!dst) return SG_OK;
    const int64_t N = (int64_t)L * L * L;
    int8_t* target = mem == SG_MEM_DEVICE ? dst : staging->as<int8_t>();
    SG_RET(log->run(SG_KERNEL_OTHER, (int64_t)R * N, st, [&] {
        return launch_unpack_spins(packed, target, L, Rp, R, idx, st);
    }));
    if (mem == SG_MEM_DEVICE) return SG_OK;
    SG_TRY_CUDA(cudaMemcpyAsync(dst, staging->as<int8_t>(), (size_t)R * N, cudaMemcpyDeviceToHost, st));
    return SG_OK;
}

// ------------------------------------------------------------------ SA group

// Instances of one group share L, R, S and schedule; keys differ per instance.
int32_t run_sa_group(const std::vector<int>& members, const sg_instance* const* insts,
                     const sg_sa_params* ps, sg_sa_result* outs, cudaStream_t st)
{
    const int I = (int)members.size();
    const sg_sa_params& p = ps[members[0]];
    sg_instance* first = const_cast<sg_instance*>(insts[members[0]]);
    const int L = first->L;
    const int64_t N = first->N;
    const int R = p.replicas;
    const int Wn = words_for(R), Rp = 32 * Wn;
    const int S = p.sweeps;

    std::vector<double> beta((size_t)std::max(S, 1));
    beta_schedule(S, p.beta0, p.beta1, p.schedule == SG_SCHEDULE_GEOMETRIC, beta.data());
    std::vector<uint32_t> thr((size_t)std::max(S, 1) * kThrRow);
    for (int s = 0; s < S; ++s) metropolis_row(beta[s], &thr[(size_t)s * kThrRow]);

    std::vector<RunKeys> keys(I);
    std::vector<const void*> jp(2 * (size_t)I);  // [I] six-coupling records, then [I] sign bytes
    for (int a = 0; a < I; ++a) {
        const sg_sa_params& q = ps[members[a]];
        keys[a] = make_key(q.seed, q.instance_id);
        const uint2* j6 = nullptr;
        const uint8_t* j1 = nullptr;
        SG_RET(instance_device_j6(const_cast<sg_instance*>(insts[members[a]]), st, &j6, &j1));
        jp[a] = j6;
        jp[I + a] = j1;
    }

    bool unit_j = true;  // every coupling of the group has |J| = 1
    for (int a = 0; a < I; ++a) unit_j &= insts[members[a]]->unit_couplings;
    DevBuf d_spins, d_E, d_E64, d_thr, d_keys, d_j6, d_flag, d_stage, d_base;
    SG_RET(d_spins.alloc((size_t)I * N * Wn * 4, st));
    SG_RET(d_base.alloc(sizeof(uint32_t), st));
    SG_RET(d_E.alloc(sizeof(int32_t) * (size_t)I * Rp, st));
    SG_RET(d_E64.alloc(sizeof(unsigned long long) * (size_t)I * Rp, st));
    SG_RET(d_thr.alloc(sizeof(uint32_t) * thr.size(), st));
    SG_RET(d_keys.alloc(sizeof(RunKeys) * I, st));
    SG_RET(d_j6.alloc(sizeof(void*) * 2 * I, st));
    SG_RET(d_flag.alloc(2 * sizeof(int), st));  // [0] energy mismatches, [1] device status
    bool host_spins = false;
    for (int a = 0; a < I; ++a)
        host_spins |= outs[members[a]].spins && outs[members[a]].spins_mem == SG_MEM_HOST;
    if (host_spins) SG_RET(d_stage.alloc((size_t)R * N, st));

    SG_TRY_CUDA(cudaMemcpyAsync(d_thr.as<void>(), thr.data(), sizeof(uint32_t) * thr.size(),
                                cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_keys.as<void>(), keys.data(), sizeof(RunKeys) * I,
                                cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_j6.as<void>(), jp.data(), sizeof(void*) * 2 * I,
                                cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_E64.as<void>(), 0, sizeof(unsigned long long) * (size_t)I * Rp, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_flag.as<void>(), 0, 2 * sizeof(int), st));

    int8_t* spins = d_spins.as<int8_t>();
    const uint2* const* j6p = d_j6.as<const uint2*>();
    const uint8_t* const* j1p = reinterpret_cast<const uint8_t* const*>(d_j6.as<const void*>() + I);
    const RunKeys* kp = d_keys.as<RunKeys>();
    LaunchLog log;
    const int64_t cells = (int64_t)I * N * Rp;
    unsigned long long* E64d = d_E64.as<unsigned long long>();
    // SA keeps no per-sweep energies: the energy of every replica is computed once,
    // from the final spins.
    SG_RET(log.run(SG_KERNEL_INIT, cells, st, [&] { return launch_init_spins(spins, kp, I, L, Wn, R, st); }));
    // Small lattices with unit couplings: every sweep in one launch, a word per thread-block
    // cluster (cluster.cu).  Knob SG_SA_CLUSTER = 0 / 1 disables or forces it.
    const char* ck = getenv("SG_SA_CLUSTER");
    int threads = 256;
    int C = unit_j && S > 0 && !(ck && atoi(ck) == 0) ? sa_cluster_blocks(I, L, Wn, (int64_t)I * (N / 2) * R, &threads)
                                                      : 0;
    if (ck && atoi(ck) == 1 && unit_j && S > 0 && C == 0) C = sa_cluster_blocks(I, L, Wn, 0, &threads);
    if (C > 0) {
        SG_RET(log.run(SG_KERNEL_SWEEP_CHUNK, (int64_t)I * N * R * S, st, [&] {
            return launch_sa_cluster(spins, j1p, kp, d_thr.as<uint32_t>(), I, L, Wn, R, S, C, threads, st);
        }));
    } else if (S >= kGraphMinSweeps) {
        // the kernel reads row *base + c of the whole [S][kThrRow] table
        SG_RET(run_sweep_graphs(S, d_base.as<uint32_t>(), st, log, 2, (int64_t)I * N * R,
                                [&](cudaStream_t cs, int c) -> int32_t {
                                    for (int colour = 0; colour < 2; ++colour)
                                        SG_RET(launch_sweep_rows_sa(spins, j6p, j1p, kp, d_thr.as<uint32_t>(), unit_j,
                                                                    I, L, Wn, R, (uint32_t)c, colour, cs,
                                                                    d_base.as<uint32_t>(), nullptr));
                                    return SG_OK;
                                }));
    } else {
        for (int s = 0; s < S; ++s)
            for (int c = 0; c < 2; ++c)
                SG_RET(log.run(SG_KERNEL_SWEEP, (int64_t)I * (N / 2) * R, st, [&] {
                    return launch_half_sweep_sa(spins, j6p, j1p, kp, d_thr.as<uint32_t>() + (size_t)s * kThrRow,
                                                d_E.as<int32_t>(), d_flag.as<int>() + 1, unit_j, I, L, Wn, R,
                                                (uint32_t)s, c, st);
                }));
    }
    SG_TRY_CUDA(cudaMemsetAsync(d_E64.as<void>(), 0, sizeof(unsigned long long) * (size_t)I * Rp, st));
    SG_RET(log.run(SG_KERNEL_ENERGY, cells, st, [&] { return launch_energy(spins, j6p, I, L, Wn, E64d, st, unit_j ? j1p : nullptr); }));

    std::vector<long long> E64((size_t)I * Rp);
    int flags[2] = {0, 0};
    int& mismatch = flags[0];
    SG_TRY_CUDA(cudaMemcpyAsync(E64.data(), d_E64.as<void>(), sizeof(long long) * E64.size(),
                                cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaMemcpyAsync(flags, d_flag.as<void>(), 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    for (int a = 0; a < I; ++a) {
        sg_sa_result& o = outs[members[a]];
        SG_RET(emit_spins(spins, a, L, Rp, R, o.spins, o.spins_mem, st, &d_stage, &log));
        if (o.spins && o.spins_mem == SG_MEM_HOST) SG_TRY_CUDA(cudaStreamSynchronize(st));
    }
    SG_TRY_CUDA(cudaStreamSynchronize(st));
    log.finish();
    if (flags[1] != 0) {
        set_error("a bounded device-side wait gave up (status %d)", flags[1]);
        return SG_ETIMEOUT;
    }
    if (mismatch) {
        set_error("incremental energies disagree with the recomputed energies (%d slots)", mismatch);
        return SG_EINTERNAL;
    }
    for (int a = 0; a < I; ++a) {
        const sg_instance* inst = insts[members[a]];
        sg_sa_result& o = outs[members[a]];
        for (int r = 0; r < R; ++r) {
            o.E[r] = E64[(size_t)a * Rp + r];
            if (o.eps) o.eps[r] = eps_of(o.E[r], inst->e_gs);
        }
    }
    return SG_OK;
}

// ------------------------------------------------------------------ PT group

int32_t run_pt_group(const std::vector<int>& members, const sg_instance* const* insts,
                     const sg_pt_params* ps, sg_pt_result* outs, cudaStream_t st)
{
    const int I = (int)members.size();
    const sg_pt_params& p = ps[members[0]];
    const sg_instance* first = insts[members[0]];
    const int L = first->L;
    const int64_t N = first->N;
    const int K = p.temps;
    const int Wn = words_for(K), Rp = 32 * Wn;
    const int S = p.sweeps;

    std::vector<double> ladder(K);
    beta_schedule(K, p.beta_min, p.beta_max, 1, ladder.data());
    std::vector<uint32_t> thr((size_t)K * kThrRow);
    for (int k = 0; k < K; ++k) metropolis_row(ladder[k], &thr[(size_t)k * kThrRow]);
    int64_t dmax = 0;
    for (int a = 0; a < I; ++a) dmax = std::max<int64_t>(dmax, 4 * (int64_t)insts[members[a]]->abs_sum);
    ExchangeTables xt;
    SG_RET(build_exchange_tables(ladder, dmax, &xt));

    std::vector<RunKeys> keys(I);
    std::vector<const void*> jp(2 * (size_t)I);  // [I] six-coupling records, then [I] sign bytes
    for (int a = 0; a < I; ++a) {
        const sg_pt_params& q = ps[members[a]];
        keys[a] = make_key(q.seed, q.instance_id);
        const uint2* j6 = nullptr;
        const uint8_t* j1 = nullptr;
        SG_RET(instance_device_j6(const_cast<sg_instance*>(insts[members[a]]), st, &j6, &j1));
        jp[a] = j6;
        jp[I + a] = j1;
    }
    const int Kp = std::max(K - 1, 1);
    bool unit_j = true;
    for (int a = 0; a < I; ++a) unit_j &= insts[members[a]]->unit_couplings;
    DevBuf d_spins, d_E, d_E64, d_thr, d_keys, d_j6, d_flag, d_stage, d_perm, d_inv, d_acc, d_min,
        d_xtab, d_xoff, d_xlen, d_xtail, d_done, d_base;
    SG_RET(d_spins.alloc((size_t)I * N * Wn * 4, st));
    SG_RET(d_base.alloc(sizeof(uint32_t), st));
    SG_RET(d_E.alloc(sizeof(int32_t) * (size_t)I * Rp, st));
    SG_RET(d_E64.alloc(sizeof(unsigned long long) * (size_t)I * Rp, st));
    SG_RET(d_thr.alloc(sizeof(uint32_t) * thr.size(), st));
    SG_RET(d_keys.alloc(sizeof(RunKeys) * I, st));
    SG_RET(d_j6.alloc(sizeof(void*) * 2 * I, st));
    SG_RET(d_flag.alloc(2 * sizeof(int), st));  // [0] energy mismatches, [1] device status
    SG_RET(d_perm.alloc((size_t)I * Rp, st));
    SG_RET(d_inv.alloc((size_t)I * K, st));
    SG_RET(d_acc.alloc(sizeof(unsigned long long) * (size_t)I * Kp, st));
    SG_RET(d_min.alloc(sizeof(int32_t) * I, st));
    SG_RET(d_done.alloc(sizeof(unsigned) * I, st));
    SG_RET(d_xtab.alloc(sizeof(uint32_t) * xt.tab.size(), st));
    SG_RET(d_xoff.alloc(sizeof(uint32_t) * xt.off.size(), st));
    SG_RET(d_xlen.alloc(sizeof(uint32_t) * xt.len.size(), st));
    SG_RET(d_xtail.alloc(sizeof(uint32_t) * xt.tail.size(), st));
    bool host_spins = false;
    for (int a = 0; a < I; ++a)
        host_spins |= outs[members[a]].spins && outs[members[a]].spins_mem == SG_MEM_HOST;
    if (host_spins) SG_RET(d_stage.alloc((size_t)K * N, st));

    auto h2d = [&](DevBuf& b, const void* src, size_t n) {
        return cudaMemcpyAsync(b.as<void>(), src, n, cudaMemcpyHostToDevice, st);
    };
    SG_TRY_CUDA(h2d(d_thr, thr.data(), sizeof(uint32_t) * thr.size()));
    SG_TRY_CUDA(h2d(d_keys, keys.data(), sizeof(RunKeys) * I));
    SG_TRY_CUDA(h2d(d_j6, jp.data(), sizeof(void*) * 2 * I));
    SG_TRY_CUDA(h2d(d_xtab, xt.tab.data(), sizeof(uint32_t) * xt.tab.size()));
    SG_TRY_CUDA(h2d(d_xoff, xt.off.data(), sizeof(uint32_t) * xt.off.size()));
    SG_TRY_CUDA(h2d(d_xlen, xt.len.data(), sizeof(uint32_t) * xt.len.size()));
    SG_TRY_CUDA(h2d(d_xtail, xt.tail.data(), sizeof(uint32_t) * xt.tail.size()));
    SG_TRY_CUDA(cudaMemsetAsync(d_E64.as<void>(), 0, sizeof(unsigned long long) * (size_t)I * Rp, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_flag.as<void>(), 0, 2 * sizeof(int), st));
    SG_TRY_CUDA(cudaMemsetAsync(d_done.as<void>(), 0, sizeof(unsigned) * I, st));

    int8_t* spins = d_spins.as<int8_t>();
    const uint2* const* j6p = d_j6.as<const uint2*>();
    const uint8_t* const* j1p = reinterpret_cast<const uint8_t* const*>(d_j6.as<const void*>() + I);
    const RunKeys* kp = d_keys.as<RunKeys>();
    int32_t* E = d_E.as<int32_t>();
    uint8_t* perm = d_perm.as<uint8_t>();
    uint8_t* inv = d_inv.as<uint8_t>();
    unsigned long long* acc = d_acc.as<unsigned long long>();
    int32_t* minE = d_min.as<int32_t>();
    LaunchLog log;
    const int64_t cells = (int64_t)I * N * Rp;
    unsigned long long* E64d = d_E64.as<unsigned long long>();
    SG_RET(log.run(SG_KERNEL_INIT, cells, st, [&] { return launch_init_spins(spins, kp, I, L, Wn, K, st); }));
    SG_RET(log.run(SG_KERNEL_ENERGY, cells, st, [&] { return launch_energy(spins, j6p, I, L, Wn, E64d, st, unit_j ? j1p : nullptr); }));
    SG_RET(log.run(SG_KERNEL_OTHER, (int64_t)I * Rp, st, [&] {
        return launch_pt_setup(E64d, E, perm, inv, acc, minE, I, Rp, K, st);
    }));
    ExchangeArgs xa;
    xa.keys = kp;
    xa.E = E;
    xa.rung_of_slot = perm;
    xa.slot_of_rung = inv;
    xa.accepts = acc;
    xa.minE = minE;
    xa.xtab = d_xtab.as<uint32_t>();
    xa.xoff = d_xoff.as<uint32_t>();
    xa.xlen = d_xlen.as<uint32_t>();
    xa.xtail = d_xtail.as<uint32_t>();
    xa.Rp = Rp;
    xa.K = K;
    xa.sweep_base = nullptr;
    unsigned* done = d_done.as<unsigned>();
    // K <= 32 with unit couplings: chunks of sweeps in one cooperative launch holding the
    // batch in shared memory (ptcoop.cu), or on thread-block clusters, one per instance
    // (ptcluster.cu)
    int coop_blocks = 0;
    size_t coop_smem = 0;
    std::vector<int> cplan;
    if (unit_j && Wn == 1 && S > 0 && pt_coop_wanted(I, L, K)) cplan = pt_coop_plan(I, L, K, &coop_blocks, &coop_smem);
    const int Ccl = cplan.empty() && unit_j && Wn == 1 && S > 0 ? pt_cluster_blocks(I, L, K) : 0;
    int Mh = 0, side_sms = 0;
    const int Chy = cplan.empty() && Ccl == 0 && unit_j && Wn == 1 && S >= kGraphMinSweeps
                        ? pt_cluster_split(I, L, K, &Mh, &side_sms)
                        : 0;
    if (!cplan.empty()) {
        DevBuf d_cflags, d_csums, d_cabort, d_carr, d_cpub, d_cplan;
        SG_RET(d_cflags.alloc(sizeof(int) * (size_t)coop_blocks, st));
        SG_RET(d_csums.alloc(sizeof(int) * (size_t)I * 3 * 32, st));
        SG_RET(d_cabort.alloc(sizeof(int), st));
        SG_RET(d_carr.alloc(sizeof(int) * (size_t)I, st));
        SG_RET(d_cpub.alloc(sizeof(uint32_t) * (size_t)coop_blocks * 4 * L * (L / 2), st));
        SG_RET(d_cplan.alloc(sizeof(int) * cplan.size(), st));
        SG_TRY_CUDA(cudaMemcpyAsync(d_cplan.as<void>(), cplan.data(), sizeof(int) * cplan.size(),
                                    cudaMemcpyHostToDevice, st));
        const CoopScratch cs{d_cflags.as<int>(), d_csums.as<int>(), d_cabort.as<int>(), d_carr.as<int>(),
                             d_cpub.as<uint32_t>(), d_cplan.as<int>()};
        const ExchangeTablesDev xd{d_xtab.as<uint32_t>(), d_xoff.as<uint32_t>(), d_xlen.as<uint32_t>(),
                                   d_xtail.as<uint32_t>()};
        const long long limit = wait_limit();
        for (int s0 = 0; s0 < S; s0 += kClusterChunkSweeps) {
            const int s1 = std::min(S, s0 + kClusterChunkSweeps);
            SG_RET(log.run(SG_KERNEL_SWEEP_CHUNK, (int64_t)I * N * K * (s1 - s0), st, [&] {
                return launch_pt_coop(spins, j1p, kp, d_thr.as<uint32_t>(), perm, inv, E, acc, minE, xd,
                                      d_flag.as<int>() + 1, cs, I, L, K, coop_blocks, coop_smem, s0, s1, limit, st);
            }));
        }
    } else if (Ccl > 0) {
        bool aligned = true;
        for (int a = 0; a < I; ++a) aligned &= (reinterpret_cast<uintptr_t>(jp[I + a]) & 15u) == 0;
        const ExchangeTablesDev xd{d_xtab.as<uint32_t>(), d_xoff.as<uint32_t>(), d_xlen.as<uint32_t>(),
                                   d_xtail.as<uint32_t>()};
        for (int s0 = 0; s0 < S; s0 += kClusterChunkSweeps) {
            const int s1 = std::min(S, s0 + kClusterChunkSweeps);
            SG_RET(log.run(SG_KERNEL_SWEEP_CHUNK, (int64_t)I * N * K * (s1 - s0), st, [&] {
                return launch_pt_cluster(spins, j1p, kp, d_thr.as<uint32_t>(), perm, inv, E, acc, minE, xd,
                                         d_flag.as<int>() + 1, I, L, K, Ccl, s0, s1, aligned, st);
            }));
        }
    } else if (Chy > 0) {
        // Instances [0, Mh) on clusters, on a stream of the highest priority so that their
        // blocks are placed first; instances [Mh, I) through the row kernels on the
        // caller's stream, shaped for the SMs the clusters leave.  Every per-instance array
        // of the second part starts Mh instances in.  The guard joins the side stream into
        // the caller's on every way out, so nothing is freed while a cluster launch runs.
        struct Side {
            cudaStream_t own, side = nullptr;
            cudaEvent_t fork = nullptr, join = nullptr;
            ~Side()
            {
                if (side && join && cudaEventRecord(join, side) == cudaSuccess) cudaStreamWaitEvent(own, join, 0);
                if (side) cudaStreamDestroy(side);
                if (fork) cudaEventDestroy(fork);
                if (join) cudaEventDestroy(join);
            }
        } sd{st};
        int prio_lo = 0, prio_hi = 0;
        SG_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        SG_TRY_CUDA(cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming));
        SG_TRY_CUDA(cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming));
        SG_TRY_CUDA(cudaStreamCreateWithPriority(&sd.side, cudaStreamNonBlocking, prio_hi));
        SG_TRY_CUDA(cudaEventRecord(sd.fork, st));
        SG_TRY_CUDA(cudaStreamWaitEvent(sd.side, sd.fork, 0));
        bool aligned = true;
        for (int a = 0; a < Mh; ++a) aligned &= (reinterpret_cast<uintptr_t>(jp[I + a]) & 15u) == 0;
        const ExchangeTablesDev xd{d_xtab.as<uint32_t>(), d_xoff.as<uint32_t>(), d_xlen.as<uint32_t>(),
                                   d_xtail.as<uint32_t>()};
        for (int s0 = 0; s0 < S; s0 += kClusterChunkSweeps) {
            const int s1 = std::min(S, s0 + kClusterChunkSweeps);
            SG_RET(log.run(SG_KERNEL_SWEEP_CHUNK, (int64_t)Mh * N * K * (s1 - s0), sd.side, [&] {
                return launch_pt_cluster(spins, j1p, kp, d_thr.as<uint32_t>(), perm, inv, E, acc, minE, xd,
                                         d_flag.as<int>() + 1, Mh, L, K, Chy, s0, s1, aligned, sd.side);
            }));
        }
        const size_t o = (size_t)Mh;
        const int Ir = I - Mh;
        int8_t* rspins = spins + o * (size_t)N * Wn * 4;
        ExchangeArgs xg = xa;
        xg.keys = kp + o;
        xg.E = E + o * Rp;
        xg.rung_of_slot = perm + o * Rp;
        xg.slot_of_rung = inv + o * K;
        xg.accepts = acc + o * (K - 1);
        xg.minE = minE + o;
        xg.sweep_base = d_base.as<uint32_t>();
        SG_RET(run_sweep_graphs(S, d_base.as<uint32_t>(), st, log, 2, (int64_t)Ir * N * K,
                                [&](cudaStream_t cs, int c) -> int32_t {
                                    bool fused = false;
                                    for (int colour = 0; colour < 2; ++colour)
                                        SG_RET(launch_sweep_rows_pt(rspins, j6p + o, j1p + o, kp + o,
                                                                    d_thr.as<uint32_t>(), perm + o * Rp, E + o * Rp,
                                                                    unit_j, Ir, L, Wn, K, (uint32_t)c, colour,
                                                                    colour == 1 ? &xg : nullptr, done + o,
                                                                    colour == 1 ? &fused : nullptr, cs,
                                                                    d_base.as<uint32_t>(), nullptr, side_sms));
                                    if (!fused) SG_RET(launch_pt_exchange(xg, Ir, (uint32_t)c, cs));
                                    return SG_OK;
                                }));
    } else if (S >= kGraphMinSweeps) {
        ExchangeArgs xg = xa;
        xg.sweep_base = d_base.as<uint32_t>();
        SG_RET(run_sweep_graphs(S, d_base.as<uint32_t>(), st, log, 2, (int64_t)I * N * K,
                                [&](cudaStream_t cs, int c) -> int32_t {
                                    bool fused = false;
                                    for (int colour = 0; colour < 2; ++colour)
                                        SG_RET(launch_sweep_rows_pt(spins, j6p, j1p, kp, d_thr.as<uint32_t>(), perm, E,
                                                                    unit_j, I, L, Wn, K, (uint32_t)c, colour,
                                                                    colour == 1 ? &xg : nullptr, done,
                                                                    colour == 1 ? &fused : nullptr, cs,
                                                                    d_base.as<uint32_t>(), nullptr));
                                    if (!fused) SG_RET(launch_pt_exchange(xg, I, (uint32_t)c, cs));
                                    return SG_OK;
                                }));
    }
    for (int s = 0; s < (S >= kGraphMinSweeps || Ccl > 0 || Chy > 0 || !cplan.empty() ? 0 : S); ++s) {
        bool fused = false;
        for (int c = 0; c < 2; ++c)
            SG_RET(log.run(SG_KERNEL_SWEEP, (int64_t)I * (N / 2) * K, st, [&] {
                // the colour-1 launch may perform the exchange in its last blocks
                return launch_half_sweep_pt(spins, j6p, j1p, kp, d_thr.as<uint32_t>(), perm, E,
                                            d_flag.as<int>() + 1, unit_j, I, L, Wn, K,
                                            (uint32_t)s, c, c == 1 ? &xa : nullptr, done,
                                            c == 1 ? &fused : nullptr, st);
            }));
        if (!fused)
            SG_RET(log.run(SG_KERNEL_EXCHANGE, (int64_t)I * (K / 2), st,
                           [&] { return launch_pt_exchange(xa, I, (uint32_t)s, st); }));
    }
    SG_TRY_CUDA(cudaMemsetAsync(d_E64.as<void>(), 0, sizeof(unsigned long long) * (size_t)I * Rp, st));
    SG_RET(log.run(SG_KERNEL_ENERGY, cells, st, [&] { return launch_energy(spins, j6p, I, L, Wn, E64d, st, unit_j ? j1p : nullptr); }));
    SG_RET(log.run(SG_KERNEL_OTHER, (int64_t)I * Rp, st, [&] {
        return launch_check_energy(E64d, E, I, Rp, K, d_flag.as<int>(), st);
    }));

    std::vector<long long> E64((size_t)I * Rp);
    std::vector<uint8_t> hperm((size_t)I * Rp);
    std::vector<unsigned long long> hacc((size_t)I * Kp);
    std::vector<int32_t> hmin(I);
    int flags[2] = {0, 0};
    int& mismatch = flags[0];
    SG_TRY_CUDA(cudaMemcpyAsync(E64.data(), d_E64.as<void>(), sizeof(long long) * E64.size(),
                                cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaMemcpyAsync(hperm.data(), perm, hperm.size(), cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaMemcpyAsync(hacc.data(), acc, sizeof(unsigned long long) * hacc.size(),
                                cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaMemcpyAsync(hmin.data(), minE, sizeof(int32_t) * I, cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaMemcpyAsync(flags, d_flag.as<void>(), 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    for (int a = 0; a < I; ++a) {
        sg_pt_result& o = outs[members[a]];
        SG_RET(emit_spins(spins, a, L, Rp, K, o.spins, o.spins_mem, st, &d_stage, &log));
        if (o.spins && o.spins_mem == SG_MEM_HOST) SG_TRY_CUDA(cudaStreamSynchronize(st));
    }
    SG_TRY_CUDA(cudaStreamSynchronize(st));
    log.finish();
    if (flags[1] != 0) {
        set_error("a bounded device-side wait gave up (status %d)", flags[1]);
        return SG_ETIMEOUT;
    }
    if (mismatch) {
        set_error("incremental energies disagree with the recomputed energies (%d slots)", mismatch);
        return SG_EINTERNAL;
    }
    for (int a = 0; a < I; ++a) {
        const sg_instance* inst = insts[members[a]];
        sg_pt_result& o = outs[members[a]];
        for (int r = 0; r < K; ++r) {
            if (o.E) o.E[r] = E64[(size_t)a * Rp + r];
            if (o.perm) o.perm[r] = hperm[(size_t)a * Rp + r];
        }
        if (o.accepts)
            for (int k = 0; k + 1 < K; ++k) o.accepts[k] = (int64_t)hacc[(size_t)a * Kp + k];
        o.minE = hmin[a];
        o.min_eps = eps_of(o.minE, inst->e_gs);
    }
    return SG_OK;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" const char* sg_last_error_string(void) { return g_err; }

extern "C" int32_t sg_version(void) { return 100; }

extern "C" int32_t sg_stats_enable(int32_t timing)
{
    clear_error();
    std::lock_guard<std::mutex> g(stats().mu);
    stats().timing = timing != 0;
    return SG_OK;
}

extern "C" int32_t sg_stats_read(sg_kernel_stats* out, int32_t reset)
{
    clear_error();
    if (!out) {
        set_error("NULL argument");
        return SG_EINVAL;
    }
    std::lock_guard<std::mutex> g(stats().mu);
    *out = stats().totals;
    if (reset) stats().totals = sg_kernel_stats{};
    return SG_OK;
}

extern "C" int32_t sg_sa_run_batch(const sg_instance* const* insts, const sg_sa_params* ps, int32_t n,
                                   sg_sa_result* outs, void* stream)
{
    clear_error();
    if (n < 0 || (n > 0 && (!insts || !ps || !outs))) {
        set_error("bad batch arguments");
        return SG_EINVAL;
    }
    for (int a = 0; a < n; ++a) SG_RET(check_sa(insts[a], &ps[a], &outs[a]));
    cudaStream_t st = (cudaStream_t)stream;
    // group instances that can share launches
    std::map<std::tuple<int, int, int, double, double, int>, std::vector<int>> groups;
    for (int a = 0; a < n; ++a) {
        const sg_sa_params& p = ps[a];
        groups[std::make_tuple(insts[a]->L, p.replicas, p.sweeps, p.beta0, p.beta1, p.schedule)]
            .push_back(a);
    }
    // A batch of uneven shapes runs in one persistent launch (batch.cu), and so does a
    // batch of small lattices whose half sweeps are too short to pay for a launch each
    // (every plane then lives in shared memory for the whole run) -- provided it has
    // enough words of 32 replicas to give every SM two planes, since a plane is one
    // block's work.  Other batches of one shape use the sweep kernel that spreads each
    // instance over many blocks.  Knob SG_BATCH_PLANES = 1 / 0 forces one or the other.
    bool small = n > 0;
    int64_t half_sweep = 0;  // attempts per half sweep of the whole batch
    int64_t words = 0;       // planes of one word
    for (int a = 0; a < n; ++a) {
        small &= planes_smem_bytes(1, insts[a]->L) > 0;
        half_sweep += insts[a]->N / 2 * (int64_t)ps[a].replicas;
        words += words_for(ps[a].replicas);
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    small &= half_sweep <= (int64_t)1 << 24 && words >= 2 * (int64_t)sms;
    const char* knob = getenv("SG_BATCH_PLANES");
    const bool planes = knob ? atoi(knob) == 1 : (groups.size() > 1 || small);
    if (planes && n > 0) {
        std::vector<int> all(n);
        for (int a = 0; a < n; ++a) all[a] = a;
        return run_sa_planes(all, insts, ps, outs, st, nullptr, nullptr);  // records its launches
    }
    for (auto& g : groups)
        for (size_t at = 0; at < g.second.size(); at += kMaxGroup) {
            std::vector<int> part(g.second.begin() + at,
                                  g.second.begin() + std::min(g.second.size(), at + kMaxGroup));
            SG_RET(run_sa_group(part, insts, ps, outs, st));
        }
    return SG_OK;
}

extern "C" int32_t sg_sa_run(const sg_instance* inst, const sg_sa_params* p, sg_sa_result* out,
                             void* stream)
{
    return sg_sa_run_batch(&inst, p, 1, out, stream);
}

extern "C" int32_t sg_pt_run_batch(const sg_instance* const* insts, const sg_pt_params* ps, int32_t n,
                                   sg_pt_result* outs, void* stream)
{
    clear_error();
    if (n < 0 || (n > 0 && (!insts || !ps || !outs))) {
        set_error("bad batch arguments");
        return SG_EINVAL;
    }
    for (int a = 0; a < n; ++a) SG_RET(check_pt(insts[a], &ps[a], &outs[a]));
    cudaStream_t st = (cudaStream_t)stream;
    std::map<std::tuple<int, int, int, double, double>, std::vector<int>> groups;
    for (int a = 0; a < n; ++a) {
        const sg_pt_params& p = ps[a];
        groups[std::make_tuple(insts[a]->L, p.temps, p.sweeps, p.beta_min, p.beta_max)].push_back(a);
    }
    for (auto& g : groups)
        for (size_t at = 0; at < g.second.size(); at += kMaxGroup) {
            std::vector<int> part(g.second.begin() + at,
                                  g.second.begin() + std::min(g.second.size(), at + kMaxGroup));
            SG_RET(run_pt_group(part, insts, ps, outs, st));
        }
    return SG_OK;
}

extern "C" int32_t sg_pt_run(const sg_instance* inst, const sg_pt_params* p, sg_pt_result* out,
                             void* stream)
{
    return sg_pt_run_batch(&inst, p, 1, out, stream);
}

namespace {
int32_t fragment_batch(const sg_instance* const* insts, const sg_fragment_params* ps, int32_t n,
                       sg_fragment_result* outs, void* stream, bool tropical)
{
    clear_error();
    if (n < 0 || (n > 0 && (!insts || !ps || !outs))) {
        set_error("bad batch arguments");
        return SG_EINVAL;
    }
    if (n == 0) return SG_OK;
    const sg_fragment_params& p = ps[0];
    for (int a = 0; a < n; ++a) {
        if (!insts[a] || !outs) {
            set_error("NULL instance");
            return SG_EINVAL;
        }
        const sg_fragment_params& q = ps[a];
        if (insts[a]->L != insts[0]->L || q.l != p.l || q.sweeps != p.sweeps || q.beta0 != p.beta0 ||
            q.beta1 != p.beta1) {
            set_error("a fragment batch needs one L and one (l, sweeps, beta0, beta1)");
            return SG_EINVAL;
        }
        if (outs[a].spins && outs[a].spins_mem != SG_MEM_HOST && outs[a].spins_mem != SG_MEM_DEVICE) {
            set_error("bad spins_mem");
            return SG_EINVAL;
        }
    }
    const int L = insts[0]->L, l = p.l, S = tropical ? 0 : p.sweeps;
    if (l < 1 || l > (tropical ? 3 : 7) || (l % 2) == 0 || l >= L || L % l != 0 ||
        (!tropical && (S < 0 || !beta_ok(p.beta0) || !beta_ok(p.beta1)))) {
        set_error("fragment side l must be odd, 1 <= l <= %d, l < L and divide L; sweeps >= 0; betas > 0",
                  tropical ? 3 : 7);
        return SG_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int I = n;
    const int64_t N = insts[0]->N;
    std::vector<double> beta((size_t)std::max(S, 1));
    if (S > 0) beta_schedule(S, p.beta0, p.beta1, 1, beta.data());
    std::vector<uint32_t> thr((size_t)std::max(S, 1) * kThrRow);
    for (int s = 0; s < S; ++s) metropolis_row(beta[s], &thr[(size_t)s * kThrRow]);
    std::vector<RunKeys> keys(I);
    std::vector<const void*> jp((size_t)I);
    for (int a = 0; a < I; ++a) {
        keys[a] = make_key(ps[a].seed, ps[a].instance_id);
        const uint2* j6 = nullptr;
        SG_RET(instance_device_j6(const_cast<sg_instance*>(insts[a]), st, &j6, nullptr));
        jp[a] = j6;
    }
    DevBuf d_spins, d_thr, d_keys, d_j6, d_words, d_E64, d_bad, d_one;
    SG_RET(d_spins.alloc((size_t)I * N, st));
    SG_RET(d_thr.alloc(sizeof(uint32_t) * thr.size(), st));
    SG_RET(d_keys.alloc(sizeof(RunKeys) * I, st));
    SG_RET(d_j6.alloc(sizeof(void*) * I, st));
    SG_RET(d_words.alloc((size_t)N * 4, st));
    SG_RET(d_E64.alloc(sizeof(unsigned long long) * 32 * (size_t)I, st));
    SG_RET(d_bad.alloc(sizeof(int), st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_thr.as<void>(), thr.data(), sizeof(uint32_t) * thr.size(), cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_keys.as<void>(), keys.data(), sizeof(RunKeys) * I, cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_j6.as<void>(), jp.data(), sizeof(void*) * I, cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_spins.as<void>(), 0, (size_t)I * N, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_E64.as<void>(), 0, sizeof(unsigned long long) * 32 * (size_t)I, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_bad.as<void>(), 0, sizeof(int), st));
    LaunchLog log;
    const int64_t V = (int64_t)l * l * l;
    // attempts: wave w anneals V - w free sites of each of N / V fragments, 32 reads, S sweeps;
    // tropical: wave w enumerates 2^(V - w) states of each of N / V fragments
    int64_t units = (int64_t)I * N * 32 * S * (V + 1) / 2;
    if (tropical) {
        units = 0;
        for (int w = 0; w < V; ++w) units += (int64_t)I * (N / V) * ((int64_t)1 << (V - w));
    }
    SG_RET(log.run(SG_KERNEL_SWEEP, units, st, [&] {
        if (tropical) return launch_fragment_tropical_waves(d_spins.as<int8_t>(), d_j6.as<const uint2*>(), I, L, l, st);
        return launch_fragment_waves(d_spins.as<int8_t>(), d_j6.as<const uint2*>(), d_keys.as<RunKeys>(),
                                     d_thr.as<uint32_t>(), I, L, l, S, st);
    }, V));
    // energies (Eq. 1): each configuration packed as one word of a single replica
    for (int a = 0; a < I; ++a) {
        SG_RET(log.run(SG_KERNEL_OTHER, N, st, [&] {
            return launch_pack_spins(d_spins.as<int8_t>() + (size_t)a * N, d_words.as<int8_t>(), L, 32, 1,
                                     d_bad.as<int>(), st);
        }));
        SG_RET(log.run(SG_KERNEL_ENERGY, N, st, [&] {
            return launch_energy(d_words.as<int8_t>(), d_j6.as<const uint2*>() + a, 1, L, 1,
                                 d_E64.as<unsigned long long>() + 32 * (size_t)a, st);
        }));
    }
    std::vector<unsigned long long> E64((size_t)32 * I);
    SG_TRY_CUDA(cudaMemcpyAsync(E64.data(), d_E64.as<void>(), sizeof(unsigned long long) * E64.size(),
                                cudaMemcpyDeviceToHost, st));
    for (int a = 0; a < I; ++a)
        if (outs[a].spins)
            SG_TRY_CUDA(cudaMemcpyAsync(outs[a].spins, d_spins.as<int8_t>() + (size_t)a * N, (size_t)N,
                                        outs[a].spins_mem == SG_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                           : cudaMemcpyDeviceToHost,
                                        st));
    SG_TRY_CUDA(cudaStreamSynchronize(st));
    log.finish();
    for (int a = 0; a < I; ++a) {
        outs[a].E = (int64_t)(long long)E64[(size_t)32 * a];
        outs[a].eps = eps_of(outs[a].E, insts[a]->e_gs);
    }
    return SG_OK;
}
}  // namespace

extern "C" int32_t sg_fragment_run_batch(const sg_instance* const* insts, const sg_fragment_params* ps, int32_t n,
                                         sg_fragment_result* outs, void* stream)
{
    return fragment_batch(insts, ps, n, outs, stream, false);
}

extern "C" int32_t sg_fragment_tropical_run_batch(const sg_instance* const* insts, const sg_fragment_params* ps,
                                                  int32_t n, sg_fragment_result* outs, void* stream)
{
    return fragment_batch(insts, ps, n, outs, stream, true);
}

extern "C" int32_t sg_fragment_run(const sg_instance* inst, const sg_fragment_params* p, sg_fragment_result* out,
                                   void* stream)
{
    return sg_fragment_run_batch(&inst, p, 1, out, stream);
}

extern "C" int32_t sg_energy(const sg_instance* inst_c, const int8_t* spins, int32_t n_configs,
                             int32_t mem_kind, int64_t* E_out, void* stream)
{
    clear_error();
    if (!inst_c || !E_out || n_configs < 0 || (n_configs > 0 && !spins) ||
        (mem_kind != SG_MEM_HOST && mem_kind != SG_MEM_DEVICE)) {
        set_error("bad sg_energy arguments");
        return SG_EINVAL;
    }
    if (n_configs == 0) return SG_OK;
    if (n_configs > (1 << 20)) {
        set_error("n_configs must be <= 2^20");
        return SG_EINVAL;
    }
    sg_instance* inst = const_cast<sg_instance*>(inst_c);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = inst->N;
    const int R = n_configs, Wn = words_for(R), Rp = 32 * Wn;
    const uint2* j6 = nullptr;
    SG_RET(instance_device_j6(inst, st, &j6, nullptr));
    DevBuf d_in, d_packed, d_E64, d_j6, d_bad;
    const int8_t* src = spins;
    if (mem_kind == SG_MEM_HOST) {
        SG_RET(d_in.alloc((size_t)R * N, st));
        SG_TRY_CUDA(cudaMemcpyAsync(d_in.as<void>(), spins, (size_t)R * N, cudaMemcpyHostToDevice, st));
        src = d_in.as<int8_t>();
    }
    SG_RET(d_packed.alloc((size_t)Wn * 4 * N, st));
    SG_RET(d_E64.alloc(sizeof(unsigned long long) * Rp, st));
    SG_RET(d_j6.alloc(sizeof(uint2*), st));
    SG_RET(d_bad.alloc(sizeof(int), st));
    SG_TRY_CUDA(cudaMemcpyAsync(d_j6.as<void>(), &j6, sizeof(uint2*), cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_E64.as<void>(), 0, sizeof(unsigned long long) * Rp, st));
    SG_TRY_CUDA(cudaMemsetAsync(d_bad.as<void>(), 0, sizeof(int), st));
    LaunchLog log;
    SG_RET(log.run(SG_KERNEL_OTHER, (int64_t)Rp * N, st, [&] {
        return launch_pack_spins(src, d_packed.as<int8_t>(), inst->L, Rp, R, d_bad.as<int>(), st);
    }));
    SG_RET(log.run(SG_KERNEL_ENERGY, (int64_t)Rp * N, st, [&] {
        return launch_energy(d_packed.as<int8_t>(), d_j6.as<const uint2*>(), 1, inst->L, Wn,
                             d_E64.as<unsigned long long>(), st);
    }));
    std::vector<long long> E((size_t)Rp);
    int bad = 0;
    SG_TRY_CUDA(cudaMemcpyAsync(E.data(), d_E64.as<void>(), sizeof(long long) * Rp,
                                cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaMemcpyAsync(&bad, d_bad.as<void>(), sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_TRY_CUDA(cudaStreamSynchronize(st));
    log.finish();
    if (bad) {
        set_error("%d spin values are not -1 or +1", bad);
        return SG_EINVAL;
    }
    for (int r = 0; r < R; ++r) E_out[r] = E[r];
    return SG_OK;
}
