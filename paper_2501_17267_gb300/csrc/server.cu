// server.cu -- continuously batched solve server: requests run until their lowest energy
// reaches a target gap (time to target, TT-eps, Eq. 2) or a sweep cap.
//
// One worker thread per server owns the device work.  Requests wait in a FIFO queue;
// the worker admits them while their device memory fits the budget and a slot is free,
// keeps their state resident, and advances every admitted request by one chunk of
// sweeps per round:
//   - all SA requests together in one persistent plane launch (batch.cu), each with its
//     own sweep range inside its current restart;
//   - each PT request by replaying its own CUDA graph (one chunk of sweeps and
//     exchanges, the sweep index read from device memory) on its own stream,
// so requests that arrive while others run join the next round and their kernels
// overlap on the GPU.  Completion is checked between rounds, at sweep counts that do
// not depend on what else runs, so each result is the same alone and in any mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "exchange.cuh"
#include "sg_internal.h"

namespace sg {
namespace {

using Clock = std::chrono::steady_clock;

__global__ void advance_kernel(uint32_t* base, uint32_t by) { *base += by; }

// Device allocation owned by a request (freed synchronously at retirement).
struct DMem {
    void* p = nullptr;
    DMem() = default;
    DMem(const DMem&) = delete;
    DMem& operator=(const DMem&) = delete;
    ~DMem() { reset(); }
    void reset()
    {
        if (p) cudaFree(p);
        p = nullptr;
    }
    bool alloc(size_t bytes)
    {
        reset();
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        return true;
    }
    template <class T>
    T* as() const
    {
        return static_cast<T*>(p);
    }
};

// Device or pinned host buffer that only grows (reused across rounds).
struct GrowBuf {
    void* p = nullptr;
    size_t cap = 0;
    bool host = false;
    GrowBuf() = default;
    GrowBuf(const GrowBuf&) = delete;
    GrowBuf& operator=(const GrowBuf&) = delete;
    ~GrowBuf() { release(); }
    void release()
    {
        if (p) host ? cudaFreeHost(p) : cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    bool ensure(size_t bytes)
    {
        if (bytes <= cap) return true;
        release();
        const size_t n = std::max<size_t>(bytes, 4096);
        if ((host ? cudaMallocHost(&p, n) : cudaMalloc(&p, n)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        cap = n;
        return true;
    }
    template <class T>
    T* as() const
    {
        return static_cast<T*>(p);
    }
};

struct Request {
    uint64_t ticket = 0;
    sg_request req{};
    Clock::time_point t_submit, t_admit, t_done;
    size_t bytes = 0;
    bool admitted = false;
    bool finished = false;  // guarded by the server mutex: the result may be read
    bool cancelled = false; // guarded by the server mutex
    bool done = false;      // worker only: stop after this round
    sg_result result{};
    sg_instance* inst = nullptr;
    int64_t target = 0;       // done when min energy <= target
    int64_t sweeps = 0;       // sweeps run so far (all restarts)
    int64_t minE = INT64_MAX;
    // SA
    int WG = 1, restart = 0, in_restart = 0;
    bool need_init = true;
    const uint32_t* thr = nullptr;  // shared schedule table (owned by the server)
    DMem sa_spins;
    // PT
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    DMem pt_spins, pt_E, pt_E64, pt_thr, pt_keys, pt_jp, pt_perm, pt_inv, pt_acc, pt_min, pt_done,
        pt_base, pt_xtab, pt_xoff, pt_xlen, pt_xtail;
    int32_t* h_min = nullptr;  // pinned
    // Frees every device resource (the result stays).
    void release()
    {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        if (stream) cudaStreamDestroy(stream);
        stream = nullptr;
        if (h_min) cudaFreeHost(h_min);
        h_min = nullptr;
        for (DMem* d : {&sa_spins, &pt_spins, &pt_E, &pt_E64, &pt_thr, &pt_keys, &pt_jp, &pt_perm, &pt_inv,
                        &pt_acc, &pt_min, &pt_done, &pt_base, &pt_xtab, &pt_xoff, &pt_xlen, &pt_xtail})
            d->reset();
        if (inst) sg_instance_destroy(inst);
        inst = nullptr;
    }
    ~Request() { release(); }
};

// Per plane width: a stream and reusable launch buffers for the SA requests of a round.
struct SaGroup {
    int WG = 1;
    cudaStream_t st = nullptr;
    GrowBuf pl, ord, next, E, init, hE;
    std::vector<Request*> reqs;
    std::vector<Plane> planes, init_planes;
    std::vector<int> first, steps;
    int32_t rc = SG_OK;
};

int largest_wg(int Wn)
{
    int wg = 4;
    while (Wn % wg) wg >>= 1;
    return wg;
}

size_t request_bytes(const sg_request& r)
{
    const size_t N = (size_t)r.instance.L * r.instance.L * r.instance.L;
    const size_t Rp = 4 * (size_t)((r.width + 3) / 4);
    size_t b = N * Rp + 9 * N + 4096;  // spins, coupling records, small state
    if (r.kind == SG_REQ_SA)
        b += (size_t)r.sweeps_per_restart * 64;
    else
        b += 16 * Rp * sizeof(uint32_t) + (size_t)r.width * (1u << 14);  // thresholds, exchange tables
    return b;
}

}  // namespace
}  // namespace sg

struct sg_server {
    sg_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<sg::Request*> queue;
    std::map<uint64_t, std::unique_ptr<sg::Request>> all;
    std::vector<sg::Request*> active;
    uint64_t next_ticket = 1;
    size_t in_use = 0;
    bool stop = false;
    std::thread worker;
    // device resources of the worker
    cudaStream_t setup_stream = nullptr;
    sg::SaGroup groups[3];  // plane widths 4, 2, 1
    std::map<std::tuple<int, double, double, int>, sg::DMem*> schedules;
    ~sg_server()
    {
        for (auto& kv : schedules) delete kv.second;
        all.clear();
        for (auto& g : groups) {
            g.pl.release(), g.ord.release(), g.next.release(), g.E.release(), g.init.release(), g.hE.release();
            if (g.st) cudaStreamDestroy(g.st);
        }
        if (setup_stream) cudaStreamDestroy(setup_stream);
    }
};

namespace sg {
namespace {

double secs(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double>(b - a).count();
}

// Device state of an admitted request; false on failure (result.status set).
bool admit_request(sg_server* srv, Request* q)
{
    const sg_request& r = q->req;
    auto fail = [&](int32_t code) {
        q->result.status = code;
        return false;
    };
    if (sg_instance_create(&r.instance, &q->inst) != SG_OK) return fail(SG_EINVAL);
    q->result.e_gs = q->inst->e_gs;
    const int64_t abs_gs = q->inst->e_gs < 0 ? -q->inst->e_gs : q->inst->e_gs;
    q->target = q->inst->e_gs + (int64_t)floor(r.eps_target * (double)abs_gs);
    const uint2* j6 = nullptr;
    const uint8_t* j1 = nullptr;
    if (instance_device_j6(q->inst, srv->setup_stream, &j6, &j1) != SG_OK) return fail(SG_ENOMEM);
    const int L = q->inst->L;
    const size_t N = (size_t)q->inst->N;
    const int Wn = (r.width + 3) / 4, Rp = 4 * Wn;
    if (r.kind == SG_REQ_SA) {
        auto key = std::make_tuple(r.sweeps_per_restart, r.beta0, r.beta1, r.schedule);
        auto it = srv->schedules.find(key);
        if (it == srv->schedules.end()) {
            const int S = r.sweeps_per_restart;
            std::vector<double> beta(S);
            beta_schedule(S, r.beta0, r.beta1, r.schedule == SG_SCHEDULE_GEOMETRIC, beta.data());
            std::vector<uint32_t> t((size_t)S * kThrRow);
            for (int s = 0; s < S; ++s) metropolis_row(beta[s], &t[(size_t)s * kThrRow]);
            DMem* d = new DMem;
            if (!d->alloc(t.size() * 4) ||
                cudaMemcpy(d->p, t.data(), t.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
                delete d;
                return fail(SG_ENOMEM);
            }
            it = srv->schedules.emplace(key, d).first;
        }
        q->thr = it->second->as<uint32_t>();
        q->WG = largest_wg(Wn);
        if (!q->sa_spins.alloc(N * Rp)) return fail(SG_ENOMEM);
        return true;
    }
    // PT: state, thresholds, exchange tables, and the captured chunk graph
    if (!rows_kernel_supports(Wn)) return fail(SG_EINVAL);
    const int K = r.width;
    std::vector<double> ladder(K);
    beta_schedule(K, r.beta0, r.beta1, 1, ladder.data());
    std::vector<uint32_t> thr((size_t)K * kThrRow);
    for (int k = 0; k < K; ++k) metropolis_row(ladder[k], &thr[(size_t)k * kThrRow]);
    ExchangeTables xt;
    if (build_exchange_tables(ladder, 4 * (int64_t)q->inst->abs_sum, &xt) != SG_OK) return fail(SG_EINVAL);
    const int Kp = std::max(K - 1, 1);
    const RunKeys key{(uint32_t)r.seed, (uint32_t)(r.seed >> 32)};
    const void* jp[2] = {j6, j1};
    bool ok = q->pt_spins.alloc(N * Rp) && q->pt_E.alloc(4 * Rp) && q->pt_E64.alloc(8 * Rp) &&
              q->pt_thr.alloc(thr.size() * 4) && q->pt_keys.alloc(sizeof(RunKeys)) &&
              q->pt_jp.alloc(sizeof(jp)) && q->pt_perm.alloc(Rp) && q->pt_inv.alloc(K) &&
              q->pt_acc.alloc(8 * Kp) && q->pt_min.alloc(4) && q->pt_done.alloc(4) &&
              q->pt_base.alloc(4) && q->pt_xtab.alloc(4 * xt.tab.size()) &&
              q->pt_xoff.alloc(4 * xt.off.size()) && q->pt_xlen.alloc(4 * xt.len.size()) &&
              q->pt_xtail.alloc(4 * xt.tail.size());
    if (!ok) return fail(SG_ENOMEM);
    if (cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&q->h_min, sizeof(int32_t)) != cudaSuccess)
        return fail(SG_ECUDA);
    cudaStream_t st = q->stream;
    bool cu = cudaMemcpyAsync(q->pt_thr.p, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(q->pt_keys.p, &key, sizeof(key), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(q->pt_jp.p, jp, sizeof(jp), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(q->pt_xtab.p, xt.tab.data(), 4 * xt.tab.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(q->pt_xoff.p, xt.off.data(), 4 * xt.off.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(q->pt_xlen.p, xt.len.data(), 4 * xt.len.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemcpyAsync(q->pt_xtail.p, xt.tail.data(), 4 * xt.tail.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
              cudaMemsetAsync(q->pt_E64.p, 0, 8 * Rp, st) == cudaSuccess &&
              cudaMemsetAsync(q->pt_done.p, 0, 4, st) == cudaSuccess &&
              cudaMemsetAsync(q->pt_base.p, 0, 4, st) == cudaSuccess;
    if (!cu) return fail(SG_ECUDA);
    int8_t* spins = q->pt_spins.as<int8_t>();
    const uint2* const* j6p = q->pt_jp.as<const uint2*>();
    const uint8_t* const* j1p = reinterpret_cast<const uint8_t* const*>(q->pt_jp.as<const void*>() + 1);
    const RunKeys* kp = q->pt_keys.as<RunKeys>();
    if (launch_init_spins(spins, kp, 1, L, Wn, K, st) != SG_OK ||
        launch_energy(spins, j6p, 1, L, Wn, q->pt_E64.as<unsigned long long>(), st) != SG_OK ||
        launch_pt_setup(q->pt_E64.as<unsigned long long>(), q->pt_E.as<int32_t>(), q->pt_perm.as<uint8_t>(),
                        q->pt_inv.as<uint8_t>(), q->pt_acc.as<unsigned long long>(), q->pt_min.as<int32_t>(), 1,
                        Rp, K, st) != SG_OK)
        return fail(SG_ECUDA);
    // one chunk as a graph: chunk x (colour 0, colour 1 with the exchange), then advance
    ExchangeArgs xa;
    xa.keys = kp;
    xa.E = q->pt_E.as<int32_t>();
    xa.rung_of_slot = q->pt_perm.as<uint8_t>();
    xa.slot_of_rung = q->pt_inv.as<uint8_t>();
    xa.accepts = q->pt_acc.as<unsigned long long>();
    xa.minE = q->pt_min.as<int32_t>();
    xa.xtab = q->pt_xtab.as<uint32_t>();
    xa.xoff = q->pt_xoff.as<uint32_t>();
    xa.xlen = q->pt_xlen.as<uint32_t>();
    xa.xtail = q->pt_xtail.as<uint32_t>();
    xa.Rp = Rp;
    xa.K = K;
    xa.sweep_base = q->pt_base.as<uint32_t>();
    const bool unit = q->inst->unit_couplings;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(SG_ECUDA);
    int32_t rc = SG_OK;
    for (int c = 0; c < srv->cfg.chunk_sweeps && rc == SG_OK; ++c) {
        bool fused = false;
        rc = launch_sweep_rows_pt(spins, j6p, j1p, kp, q->pt_thr.as<uint32_t>(), q->pt_perm.as<uint8_t>(),
                                  q->pt_E.as<int32_t>(), unit, 1, L, Wn, K, (uint32_t)c, 0, nullptr,
                                  q->pt_done.as<unsigned>(), nullptr, st, q->pt_base.as<uint32_t>());
        if (rc == SG_OK)
            rc = launch_sweep_rows_pt(spins, j6p, j1p, kp, q->pt_thr.as<uint32_t>(), q->pt_perm.as<uint8_t>(),
                                      q->pt_E.as<int32_t>(), unit, 1, L, Wn, K, (uint32_t)c, 1, &xa,
                                      q->pt_done.as<unsigned>(), &fused, st, q->pt_base.as<uint32_t>());
        if (rc == SG_OK && !fused) rc = launch_pt_exchange(xa, 1, (uint32_t)c, st);
    }
    if (rc == SG_OK) {
        advance_kernel<<<1, 1, 0, st>>>(q->pt_base.as<uint32_t>(), (uint32_t)srv->cfg.chunk_sweeps);
        if (cudaGetLastError() != cudaSuccess) rc = SG_ECUDA;
    }
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc == SG_OK && (e != cudaSuccess || cudaGraphInstantiate(&q->graph, g, 0) != cudaSuccess)) rc = SG_ECUDA;
    if (g) cudaGraphDestroy(g);
    if (rc != SG_OK) {
        cudaGetLastError();
        return fail(rc);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(SG_ECUDA);
    return true;
}

// SA requests of one plane width: one persistent launch over all their planes, each
// plane running sweeps [in_restart, in_restart + n) of its current restart; energies of
// every replica come back through pinned memory.  Asynchronous on the group's stream.
void launch_sa_group(SaGroup& g, int chunk)
{
    g.rc = SG_OK;
    g.planes.clear();
    g.init_planes.clear();
    g.first.assign(1, 0);
    g.steps.clear();
    if (g.reqs.empty()) return;
    bool unit = true;
    for (Request* q : g.reqs) unit &= q->inst->unit_couplings;
    for (Request* q : g.reqs) {
        const sg_request& r = q->req;
        const int Wn = (r.width + 3) / 4;
        const int n = (int)std::min<int64_t>({(int64_t)chunk, (int64_t)(r.sweeps_per_restart - q->in_restart),
                                              r.sweep_cap - q->sweeps});
        g.steps.push_back(n);
        const uint2* j6 = nullptr;
        const uint8_t* j1 = nullptr;
        if (instance_device_j6(q->inst, g.st, &j6, &j1) != SG_OK) {
            g.rc = SG_ENOMEM;
            return;
        }
        for (int w0 = 0; w0 < Wn; w0 += g.WG) {
            Plane pl{};
            pl.spins = q->sa_spins.as<uint32_t>() + (size_t)q->inst->N * w0;
            pl.j1 = j1;
            pl.j6 = j6;
            pl.thr = q->thr;
            pl.k0 = (uint32_t)r.seed;
            pl.k1 = (uint32_t)(r.seed >> 32) ^ (uint32_t)q->restart;  // restart k runs as instance id k
            pl.L = q->inst->L;
            pl.S = r.sweeps_per_restart;
            pl.w0 = w0;
            pl.R = r.width;
            pl.s_begin = q->in_restart;
            pl.s_end = q->in_restart + n;
            pl.Lmagic = (uint32_t)((0x100000000ull + pl.L - 1) / pl.L);
            pl.Hmagic = (uint32_t)((0x100000000ull + pl.L / 2 - 1) / (pl.L / 2));
            pl.out = (int)(g.first.size() - 1);
            g.planes.push_back(pl);
            if (q->need_init) g.init_planes.push_back(pl);
        }
        g.first.push_back((int)g.planes.size());
    }
    const int np = (int)g.planes.size(), nI = (int)g.init_planes.size();
    // longest planes first (work = sites x sweeps)
    std::vector<int> order(np);
    for (int k = 0; k < np; ++k) order[k] = k;
    auto work = [&](int k) {
        const Plane& p = g.planes[k];
        return (double)p.L * p.L * p.L * (p.s_end - p.s_begin);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    const size_t nE = (size_t)np * 4 * g.WG;
    cudaStream_t st = g.st;
    bool ok = g.pl.ensure(sizeof(Plane) * np) && g.ord.ensure(sizeof(int) * np) && g.next.ensure(4) &&
              g.E.ensure(8 * nE) && g.hE.ensure(8 * nE) && g.init.ensure(sizeof(Plane) * std::max(nI, 1));
    ok = ok && cudaMemcpyAsync(g.pl.p, g.planes.data(), sizeof(Plane) * np, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(g.ord.p, order.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemsetAsync(g.next.p, 0, 4, st) == cudaSuccess && cudaMemsetAsync(g.E.p, 0, 8 * nE, st) == cudaSuccess &&
         (nI == 0 ||
          cudaMemcpyAsync(g.init.p, g.init_planes.data(), sizeof(Plane) * nI, cudaMemcpyHostToDevice, st) == cudaSuccess);
    int32_t rc = ok ? SG_OK : SG_ECUDA;
    if (rc == SG_OK && nI) rc = launch_planes_init(g.WG, g.init.as<Plane>(), nI, st);
    if (rc == SG_OK)
        rc = launch_sa_planes(g.WG, g.pl.as<Plane>(), g.ord.as<int>(), np, g.next.as<unsigned>(), unit,
                              planes_blocks(g.WG, unit), st);
    if (rc == SG_OK) rc = launch_planes_energy(g.WG, g.pl.as<Plane>(), np, g.E.as<unsigned long long>(), st);
    if (rc == SG_OK && cudaMemcpyAsync(g.hE.p, g.E.p, 8 * nE, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = SG_ECUDA;
    for (Request* q : g.reqs) q->need_init = false;
    g.rc = rc;
}

// One round: every admitted request advances by one chunk of sweeps, then the
// completion tests run at sweep counts that do not depend on the other requests.
void run_round(sg_server* srv, const std::vector<Request*>& act)
{
    const int chunk = srv->cfg.chunk_sweeps;
    // PT requests: replay their graphs, then read the running minimum
    for (Request* q : act) {
        if (q->req.kind != SG_REQ_PT || q->done) continue;
        if (cudaGraphLaunch(q->graph, q->stream) != cudaSuccess ||
            cudaMemcpyAsync(q->h_min, q->pt_min.p, sizeof(int32_t), cudaMemcpyDeviceToHost, q->stream) !=
                cudaSuccess) {
            cudaGetLastError();
            q->result.status = SG_ECUDA;
            q->done = true;
        }
    }
    // SA requests: one launch per plane width, each on its own stream
    for (SaGroup& g : srv->groups) {
        g.reqs.clear();
        for (Request* q : act)
            if (q->req.kind == SG_REQ_SA && !q->done && q->WG == g.WG) g.reqs.push_back(q);
        launch_sa_group(g, chunk);
    }
    for (SaGroup& g : srv->groups)
        if (!g.reqs.empty() && cudaStreamSynchronize(g.st) != cudaSuccess) g.rc = SG_ECUDA;
    for (Request* q : act)
        if (q->req.kind == SG_REQ_PT && !q->done && cudaStreamSynchronize(q->stream) != cudaSuccess) {
            q->result.status = SG_ECUDA;
            q->done = true;
        }
    cudaGetLastError();
    for (Request* q : act)
        if (q->req.kind == SG_REQ_PT && !q->done) {
            q->sweeps += chunk;
            q->minE = std::min<int64_t>(q->minE, *q->h_min);
        }
    for (SaGroup& g : srv->groups) {
        for (size_t a = 0; a < g.reqs.size(); ++a) {
            Request* q = g.reqs[a];
            if (g.rc != SG_OK) {
                q->result.status = g.rc;
                q->done = true;
                continue;
            }
            const unsigned long long* E = g.hE.as<unsigned long long>();
            for (int k = g.first[a]; k < g.first[a + 1]; ++k)
                for (int rb = 0; rb < 4 * g.WG; ++rb)
                    if (4 * g.planes[k].w0 + rb < q->req.width)
                        q->minE = std::min<int64_t>(q->minE, (int64_t)(long long)E[(size_t)k * 4 * g.WG + rb]);
            q->sweeps += g.steps[a];
            q->in_restart += g.steps[a];
            if (q->in_restart == q->req.sweeps_per_restart) {  // next round starts restart + 1
                q->restart += 1;
                q->in_restart = 0;
                q->need_init = true;
            }
        }
    }
    for (Request* q : act) {
        if (q->done) continue;
        if (q->minE <= q->target) {
            q->result.reached = 1;
            q->done = true;
        } else if (q->sweeps >= q->req.sweep_cap) {
            q->done = true;
        }
    }
}

void retire(sg_server* srv, Request* q)
{
    q->t_done = Clock::now();
    q->release();
    q->finished = true;
    if (q->admitted) srv->in_use -= q->bytes;
}

void worker_main(sg_server* srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lock(srv->mu);
    for (;;) {
        // admission: FIFO while memory and slots allow
        while (!srv->stop && !srv->queue.empty() && (int)srv->active.size() < srv->cfg.max_active) {
            Request* q = srv->queue.front();
            if (srv->in_use + q->bytes > srv->cfg.hbm_budget_bytes) break;
            srv->queue.pop_front();
            srv->in_use += q->bytes;
            q->admitted = true;
            q->t_admit = Clock::now();
            lock.unlock();
            const bool ok = admit_request(srv, q);
            lock.lock();
            if (!ok) {
                retire(srv, q);
                srv->cv_done.notify_all();
                continue;
            }
            srv->active.push_back(q);
        }
        if (srv->stop && srv->active.empty()) break;
        if (srv->active.empty()) {
            srv->cv_work.wait_for(lock, std::chrono::milliseconds(50));
            continue;
        }
        for (Request* q : srv->active)
            if (q->cancelled || srv->stop) {
                q->result.status = SG_ECANCELED;
                q->done = true;
            }
        const std::vector<Request*> act = srv->active;
        lock.unlock();
        run_round(srv, act);
        lock.lock();
        std::vector<Request*> keep;
        for (Request* q : srv->active) {
            if (!q->done && q->cancelled) {
                q->result.status = SG_ECANCELED;
                q->done = true;
            }
            if (q->done)
                retire(srv, q);
            else
                keep.push_back(q);
        }
        srv->active.swap(keep);
        srv->cv_done.notify_all();
    }
}

void finish_result(Request* q)
{
    sg_result& r = q->result;
    r.sweeps = q->sweeps;
    const bool ran = q->minE != INT64_MAX;
    r.minE = ran ? q->minE : 0;
    r.min_eps = ran && r.e_gs != 0 ? (double)(r.minE - r.e_gs) / (double)(r.e_gs < 0 ? -r.e_gs : r.e_gs) : NAN;
    const Clock::time_point admit = q->admitted ? q->t_admit : q->t_done;
    r.queue_s = secs(q->t_submit, admit);
    r.run_s = secs(admit, q->t_done);
    r.total_s = secs(q->t_submit, q->t_done);
}

bool valid_request(const sg_request& r)
{
    if (r.kind != SG_REQ_SA && r.kind != SG_REQ_PT) return false;
    if (r.instance.L < 2 || r.instance.L > SG_LMAX || (r.instance.L & 1)) return false;
    if (r.width < 1 || (r.kind == SG_REQ_PT && r.width > 256) || r.width > 4096) return false;
    if (!(r.beta0 > 0 && r.beta1 > 0 && isfinite(r.beta0) && isfinite(r.beta1))) return false;
    if (!(r.eps_target >= 0) || r.sweep_cap < 1) return false;
    if (r.kind == SG_REQ_SA && (r.sweeps_per_restart < 1 ||
                                (r.schedule != SG_SCHEDULE_LINEAR && r.schedule != SG_SCHEDULE_GEOMETRIC)))
        return false;
    const double* cp = r.instance.class_prob;
    if (!(cp[0] >= 0 && cp[1] >= 0 && cp[2] >= 0 && cp[0] + cp[1] + cp[2] > 0)) return false;
    return true;
}

}  // namespace
}  // namespace sg

using namespace sg;

extern "C" int32_t sg_server_create(const sg_server_config* cfg, sg_server** out)
{
    clear_error();
    if (!cfg || !out || cfg->max_active < 1 || cfg->chunk_sweeps < 1 || cfg->queue_capacity < 1 ||
        cfg->hbm_budget_bytes == 0) {
        set_error("bad server config (max_active, chunk_sweeps, queue_capacity >= 1; budget > 0)");
        return SG_EINVAL;
    }
    sg_server* srv = new (std::nothrow) sg_server;
    if (!srv) return SG_ENOMEM;
    srv->cfg = *cfg;
    bool ok = cudaGetDevice(&srv->device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&srv->setup_stream, cudaStreamNonBlocking) == cudaSuccess;
    const int widths[3] = {4, 2, 1};
    for (int k = 0; k < 3 && ok; ++k) {
        srv->groups[k].WG = widths[k];
        srv->groups[k].hE.host = true;
        ok = cudaStreamCreateWithFlags(&srv->groups[k].st, cudaStreamNonBlocking) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        delete srv;
        set_error("server: creating streams failed");
        return SG_ECUDA;
    }
    try {
        srv->worker = std::thread(worker_main, srv);
    } catch (...) {
        delete srv;
        set_error("server: starting the worker thread failed");
        return SG_EINTERNAL;
    }
    *out = srv;
    return SG_OK;
}

extern "C" int32_t sg_submit(sg_server* srv, const sg_request* req, uint64_t* ticket)
{
    clear_error();
    if (!srv || !req || !ticket) {
        set_error("NULL argument");
        return SG_EINVAL;
    }
    if (!valid_request(*req)) {
        set_error("bad request (kind, L even in [2, %d], width, betas > 0, eps_target >= 0, "
                  "sweep_cap >= 1, SA sweeps_per_restart >= 1 and schedule, class weights)", SG_LMAX);
        return SG_EINVAL;
    }
    const size_t bytes = request_bytes(*req);
    if (bytes > srv->cfg.hbm_budget_bytes) {
        set_error("request needs %zu bytes of device memory, more than the server budget", bytes);
        return SG_ENOMEM;
    }
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stop) {
        set_error("server is stopping");
        return SG_EINVAL;
    }
    if ((int)srv->queue.size() >= srv->cfg.queue_capacity) {
        set_error("queue full (%d waiting)", (int)srv->queue.size());
        return SG_EBUSY;
    }
    auto q = std::make_unique<Request>();
    q->ticket = srv->next_ticket++;
    q->req = *req;
    q->bytes = bytes;
    q->t_submit = Clock::now();
    q->result.status = SG_OK;
    q->WG = largest_wg((req->width + 3) / 4);
    srv->queue.push_back(q.get());
    *ticket = q->ticket;
    srv->all.emplace(q->ticket, std::move(q));
    srv->cv_work.notify_one();
    return SG_OK;
}

extern "C" int32_t sg_poll(sg_server* srv, uint64_t ticket, int32_t timeout_ms, sg_result* out)
{
    clear_error();
    if (!srv || !out) {
        set_error("NULL argument");
        return SG_EINVAL;
    }
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return SG_EINVAL;
    }
    Request* q = it->second.get();
    auto is_done = [q] { return q->finished; };
    if (timeout_ms < 0)
        srv->cv_done.wait(lock, is_done);
    else if (timeout_ms > 0)
        srv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), is_done);
    if (!q->finished) return SG_PENDING;
    finish_result(q);
    *out = q->result;
    srv->all.erase(it);
    return SG_OK;
}

extern "C" int32_t sg_cancel(sg_server* srv, uint64_t ticket)
{
    clear_error();
    if (!srv) {
        set_error("NULL server");
        return SG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return SG_EINVAL;
    }
    Request* q = it->second.get();
    if (q->finished) return SG_OK;
    auto pos = std::find(srv->queue.begin(), srv->queue.end(), q);
    if (pos != srv->queue.end()) {
        srv->queue.erase(pos);
        q->result.status = SG_ECANCELED;
        retire(srv, q);
        srv->cv_done.notify_all();
    } else {
        q->cancelled = true;  // admitted: the worker stops it at the next round boundary
    }
    return SG_OK;
}

extern "C" int32_t sg_server_destroy(sg_server* srv)
{
    clear_error();
    if (!srv) return SG_OK;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        for (Request* q : srv->queue) {
            q->result.status = SG_ECANCELED;
            retire(srv, q);
        }
        srv->queue.clear();
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    delete srv;
    return SG_OK;
}
