// server.cu -- continuously batched solve server: requests run until their lowest energy
// reaches a target gap (time to target, TT-eps, Eq. 2) or a sweep cap.
//
// sg_submit generates the request's instance and host tables in the caller's thread and
// queues it.  One worker thread per server owns the device work: it admits queued
// requests (FIFO) while their device memory fits the budget and a slot is free, keeps
// their state resident in one stream-ordered allocation each, and keeps every admitted
// request busy, one chunk of sweeps at a time, with no barrier between requests:
//   - PT requests, and SA requests on lattices too large for one thread block, replay
//     their own CUDA graph (a chunk of multi-block sweeps whose sweep index lives in
//     device memory, then the energy check) on their own stream;
//   - small SA requests share a persistent plane launch (batch.cu) per plane width,
//     relaunched with whatever small requests are ready whenever the previous one ends.
// The worker polls events, so a chunk that ends lets its request check for completion
// and start the next chunk at once, and arrivals join as soon as they are admitted.
// Completion is checked only at chunk ends, at sweep counts fixed by the request alone,
// so each result is the same alone and in any mix.
#include <limits.h>
#include <math.h>
#include <stdlib.h>
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

// Start of an SA restart: key (k0, k1) and sweep index 0.
__global__ void restart_kernel(RunKeys* keys, uint32_t k0, uint32_t k1, uint32_t* base)
{
    keys->k0 = k0;
    keys->k1 = k1;
    *base = 0;
}

// out = min over the R valid replicas of the energy sums (two's complement in 64 bits).
__global__ void min_energy_kernel(const unsigned long long* E64, int R, long long* out)
{
    __shared__ long long s[256];
    long long m = LLONG_MAX;
    for (int r = threadIdx.x; r < R; r += blockDim.x) m = min(m, (long long)E64[r]);
    s[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] = min(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// The PT running minimum (int32) as the 64-bit word the host reads.
__global__ void widen_kernel(const int32_t* minE, long long* out) { *out = *minE; }

enum Mode { kPlanes = 0, kRowsSA = 1, kPT = 2 };

// A stream, an event and a little pinned memory, reused by successive requests.
struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    long long* h_out = nullptr;  // pinned: [0] min energy of the last chunk, [1] its status word
};

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Offsets into the request's single device allocation.
struct Layout {
    size_t j6 = 0, j1 = 0, J3 = 0, spins = 0, thr = 0, keys = 0, jp = 0, base = 0, E = 0, E64 = 0,
           perm = 0, inv = 0, acc = 0, minE = 0, done = 0, xtab = 0, xoff = 0, xlen = 0, xtail = 0,
           out = 0, status = 0, total = 0;
};

struct Request {
    uint64_t ticket = 0;
    sg_request req{};
    Clock::time_point t_submit, t_admit, t_done;
    size_t bytes = 0;
    bool admitted = false;
    bool finished = false;   // guarded by the server mutex: the result may be read
    bool cancelled = false;  // guarded by the server mutex
    // worker only
    bool stopping = false;   // cancelled or server stopping: stop when idle
    bool done = false;       // retire
    bool inflight = false;   // a chunk (own stream or plane launch) is running
    sg_result result{};
    std::unique_ptr<sg_instance, int32_t (*)(sg_instance*)> inst{nullptr, sg_instance_destroy};
    int mode = kPlanes;
    int ptc = -1;              // PT: blocks per cluster of the cluster kernel, 0: row kernels (-1: not chosen yet)
    int L = 0, Wn = 0, Rp = 0, WG = 1;
    int64_t N = 0;
    int64_t target = 0;        // done when min energy <= target
    int64_t sweeps = 0;        // sweeps run so far (all restarts)
    int64_t minE = INT64_MAX;
    int step = 0;              // sweeps of the chunk in flight
    // host tables made at submit
    std::shared_ptr<const std::vector<uint32_t>> thr;  // SA: [S][kThrRow]; PT: [K][kThrRow]
    ExchangeTables xt;
    // SA
    int restart = 0, in_restart = 0;
    bool need_init = true;
    // device state
    Layout lay;
    unsigned char* mem = nullptr;
    Slot* slot = nullptr;
    std::map<int, cudaGraphExec_t> graphs;  // chunk length -> graph
    template <class T>
    T* at(size_t off) const
    {
        return reinterpret_cast<T*>(mem + off);
    }
};

Layout layout_of(const Request& q)
{
    Layout y;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + std::max<size_t>(bytes, 1));
        return at;
    };
    const size_t N = (size_t)q.N, Rp = (size_t)q.Rp;
    y.j6 = take(8 * N);
    y.j1 = take(N);
    y.J3 = take(3 * N);
    y.spins = take(N * (Rp / 32) * 4);  // bit-packed words
    if (q.mode == kPlanes) {
        y.thr = take(4 * q.thr->size());
    } else if (q.mode == kRowsSA) {
        y.thr = take(4 * q.thr->size());
        y.keys = take(sizeof(RunKeys));
        y.jp = take(2 * sizeof(void*));
        y.base = take(4);
        y.E64 = take(8 * Rp);
        y.out = take(8);
        y.status = take(4);
    } else {
        const size_t K = (size_t)q.req.width, Kp = std::max<size_t>(K - 1, 1);
        y.thr = take(4 * q.thr->size());
        y.keys = take(sizeof(RunKeys));
        y.jp = take(2 * sizeof(void*));
        y.base = take(4);
        y.E = take(4 * Rp);
        y.E64 = take(8 * Rp);
        y.perm = take(Rp);
        y.inv = take(K);
        y.acc = take(8 * Kp);
        y.minE = take(4);
        y.done = take(4);
        y.xtab = take(4 * q.xt.tab.size());
        y.xoff = take(4 * q.xt.off.size());
        y.xlen = take(4 * q.xt.len.size());
        y.xtail = take(4 * q.xt.tail.size());
        y.out = take(8);
        y.status = take(4);
    }
    y.total = o;
    return y;
}

// Small SA requests of one plane width: one persistent launch over all their planes, each
// plane running sweeps [in_restart, in_restart + step) of its current restart.
struct PlaneGroup {
    int WG = 1;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool inflight = false;
    void *pl = nullptr, *ord = nullptr, *next = nullptr, *E = nullptr, *init = nullptr;
    unsigned long long* hE = nullptr;  // pinned
    size_t cap_planes = 0;
    std::vector<Request*> reqs;
    std::vector<Plane> planes, init_planes;
    std::vector<int> first;
};

// Host schedule tables shared by requests with the same SA schedule.
struct ScheduleCache {
    std::mutex mu;
    std::map<std::tuple<int, double, double, int>, std::shared_ptr<const std::vector<uint32_t>>> tables;
};

int largest_wg(int Wn)
{
    int wg = 4;
    while (Wn % wg) wg >>= 1;
    return wg;
}

// Largest side that runs in the shared plane launch (one thread block per plane); larger
// SA lattices run multi-block sweeps on their own stream.  Knob: SG_SERVER_PLANE_MAX_L.
int plane_max_L()
{
    static const int v = [] {
        const char* e = getenv("SG_SERVER_PLANE_MAX_L");
        const int x = e ? atoi(e) : 16;
        return x < 0 ? 0 : x;
    }();
    return v;
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
    sg::ScheduleCache schedules;  // used by the submitting threads
    // device resources of the worker
    cudaMemPool_t pool = nullptr;
    std::vector<std::unique_ptr<sg::Slot>> slots;  // all slots made
    std::vector<sg::Slot*> free_slots;
    sg::PlaneGroup groups[3];  // plane widths 4, 2, 1
    ~sg_server()
    {
        all.clear();
        for (auto& g : groups) {
            for (void* p : {g.pl, g.ord, g.next, g.E, g.init})
                if (p) cudaFree(p);
            if (g.hE) cudaFreeHost(g.hE);
            if (g.ev) cudaEventDestroy(g.ev);
            if (g.st) cudaStreamDestroy(g.st);
        }
        for (auto& s : slots) {
            if (s->h_out) cudaFreeHost(s->h_out);
            if (s->ev) cudaEventDestroy(s->ev);
            if (s->st) cudaStreamDestroy(s->st);
        }
        if (pool) cudaMemPoolDestroy(pool);
    }
};

namespace sg {
namespace {

double secs(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double>(b - a).count();
}

Slot* take_slot(sg_server* srv)
{
    if (!srv->free_slots.empty()) {
        Slot* s = srv->free_slots.back();
        srv->free_slots.pop_back();
        return s;
    }
    auto s = std::make_unique<Slot>();
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&s->h_out, 64) != cudaSuccess) {
        cudaGetLastError();
        if (s->h_out) cudaFreeHost(s->h_out);
        if (s->ev) cudaEventDestroy(s->ev);
        if (s->st) cudaStreamDestroy(s->st);
        return nullptr;
    }
    srv->slots.push_back(std::move(s));
    return srv->slots.back().get();
}

// Host part of a request, in the submitting thread: the instance, its target and the
// acceptance tables.  SG_OK or SG_EINVAL.
int32_t prepare_request(ScheduleCache& cache, Request* q)
{
    const sg_request& r = q->req;
    sg_instance* inst = nullptr;
    int32_t rc = sg_instance_create(&r.instance, &inst);
    if (rc != SG_OK) return rc;
    q->inst.reset(inst);
    q->L = inst->L;
    q->N = inst->N;
    q->Wn = words_for(r.width);
    q->Rp = 32 * q->Wn;
    q->WG = largest_wg(q->Wn);
    q->result.e_gs = inst->e_gs;
    const int64_t abs_gs = inst->e_gs < 0 ? -inst->e_gs : inst->e_gs;
    q->target = inst->e_gs + (int64_t)floor(r.eps_target * (double)abs_gs);
    if (r.kind == SG_REQ_SA) {
        q->mode = q->L <= plane_max_L() ? kPlanes : kRowsSA;
        const auto key = std::make_tuple(r.sweeps_per_restart, r.beta0, r.beta1, r.schedule);
        std::lock_guard<std::mutex> lock(cache.mu);
        auto it = cache.tables.find(key);
        if (it == cache.tables.end()) {
            const int S = r.sweeps_per_restart;
            std::vector<double> beta(S);
            beta_schedule(S, r.beta0, r.beta1, r.schedule == SG_SCHEDULE_GEOMETRIC, beta.data());
            auto t = std::make_shared<std::vector<uint32_t>>((size_t)S * kThrRow);
            for (int s = 0; s < S; ++s) metropolis_row(beta[s], t->data() + (size_t)s * kThrRow);
            it = cache.tables.emplace(key, std::move(t)).first;
        }
        q->thr = it->second;
    } else {
        q->mode = kPT;
        const int K = r.width;
        std::vector<double> ladder(K);
        beta_schedule(K, r.beta0, r.beta1, 1, ladder.data());
        auto t = std::make_shared<std::vector<uint32_t>>((size_t)K * kThrRow);
        for (int k = 0; k < K; ++k) metropolis_row(ladder[k], t->data() + (size_t)k * kThrRow);
        q->thr = t;
        rc = build_exchange_tables(ladder, 4 * (int64_t)inst->abs_sum, &q->xt);
        if (rc != SG_OK) return rc;
    }
    q->lay = layout_of(*q);
    q->bytes = q->lay.total;
    return SG_OK;
}

// Device part of admission, on the request's own stream: one allocation from the
// server's pool, couplings and tables uploaded, PT state initialised.  Returns a status;
// on failure the caller releases what was taken.
int32_t admit_request(sg_server* srv, Request* q)
{
    q->slot = take_slot(srv);
    if (!q->slot) return SG_ECUDA;
    cudaStream_t st = q->slot->st;
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, q->lay.total, srv->pool, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("device memory for a request of %zu bytes is not available", q->lay.total);
        return SG_ENOMEM;
    }
    q->mem = static_cast<unsigned char*>(p);
    const Layout& y = q->lay;
    const sg_instance* inst = q->inst.get();
    const size_t N = (size_t)q->N;
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.J3), inst->J3.data(), 3 * N, cudaMemcpyHostToDevice, st));
    int32_t rc = launch_prepare_j6(q->at<int8_t>(y.J3), q->at<uint2>(y.j6), q->at<uint8_t>(y.j1), q->L, st);
    if (rc != SG_OK) return rc;
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.thr), q->thr->data(), 4 * q->thr->size(), cudaMemcpyHostToDevice, st));
    if (q->mode == kPlanes) {  // the shared plane launch waits for these uploads
        SG_TRY_CUDA(cudaEventRecord(q->slot->ev, st));
        return SG_OK;
    }
    const void* jp[2] = {q->at<void>(y.j6), q->at<void>(y.j1)};
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.jp), jp, sizeof(jp), cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemsetAsync(q->at<void>(y.base), 0, 4, st));
    SG_TRY_CUDA(cudaMemsetAsync(q->at<void>(y.status), 0, 4, st));
    if (q->mode == kRowsSA) return SG_OK;
    // PT: keys, exchange tables, initial spins and energies, the identity permutation
    const RunKeys key{(uint32_t)q->req.seed, (uint32_t)(q->req.seed >> 32)};
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.keys), &key, sizeof(key), cudaMemcpyHostToDevice, st));
    const ExchangeTables& xt = q->xt;
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.xtab), xt.tab.data(), 4 * xt.tab.size(), cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.xoff), xt.off.data(), 4 * xt.off.size(), cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.xlen), xt.len.data(), 4 * xt.len.size(), cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemcpyAsync(q->at<void>(y.xtail), xt.tail.data(), 4 * xt.tail.size(), cudaMemcpyHostToDevice, st));
    SG_TRY_CUDA(cudaMemsetAsync(q->at<void>(y.E64), 0, 8 * (size_t)q->Rp, st));
    SG_TRY_CUDA(cudaMemsetAsync(q->at<void>(y.done), 0, 4, st));
    const RunKeys* kp = q->at<RunKeys>(y.keys);
    const uint2* const* j6p = q->at<const uint2*>(y.jp);
    const uint8_t* const* j1p = reinterpret_cast<const uint8_t* const*>(q->at<const void*>(y.jp) + 1);
    rc = launch_init_spins(q->at<int8_t>(y.spins), kp, 1, q->L, q->Wn, q->req.width, st);
    if (rc == SG_OK)
        rc = launch_energy(q->at<int8_t>(y.spins), j6p, 1, q->L, q->Wn, q->at<unsigned long long>(y.E64), st,
                           q->inst->unit_couplings ? j1p : nullptr);
    if (rc == SG_OK)
        rc = launch_pt_setup(q->at<unsigned long long>(y.E64), q->at<int32_t>(y.E), q->at<uint8_t>(y.perm),
                             q->at<uint8_t>(y.inv), q->at<unsigned long long>(y.acc), q->at<int32_t>(y.minE), 1,
                             q->Rp, q->req.width, st);
    return rc;
}

// Captures one chunk of n sweeps of a PT or large-SA request as a graph: the sweeps
// (sweep index = device base + c), the base advanced by n, and the chunk's lowest energy
// copied to the slot's pinned word.
int32_t capture_chunk(Request* q, int n, cudaGraphExec_t* out)
{
    const Layout& y = q->lay;
    cudaStream_t st = q->slot->st;
    int8_t* spins = q->at<int8_t>(y.spins);
    const uint2* const* j6p = q->at<const uint2*>(y.jp);
    const uint8_t* const* j1p = reinterpret_cast<const uint8_t* const*>(q->at<const void*>(y.jp) + 1);
    const RunKeys* kp = q->at<RunKeys>(y.keys);
    uint32_t* base = q->at<uint32_t>(y.base);
    const uint32_t* thr = q->at<uint32_t>(y.thr);
    const bool unit = q->inst->unit_couplings;
    int* status = q->at<int>(y.status);
    ExchangeArgs xa{};
    if (q->mode == kPT) {
        xa.keys = kp;
        xa.E = q->at<int32_t>(y.E);
        xa.rung_of_slot = q->at<uint8_t>(y.perm);
        xa.slot_of_rung = q->at<uint8_t>(y.inv);
        xa.accepts = q->at<unsigned long long>(y.acc);
        xa.minE = q->at<int32_t>(y.minE);
        xa.xtab = q->at<uint32_t>(y.xtab);
        xa.xoff = q->at<uint32_t>(y.xoff);
        xa.xlen = q->at<uint32_t>(y.xlen);
        xa.xtail = q->at<uint32_t>(y.xtail);
        xa.Rp = q->Rp;
        xa.K = q->req.width;
        xa.sweep_base = base;
    }
    // PT of a lattice the cluster kernel sweeps faster (its cost model; small L): the
    // chunk is one launch of it instead of two launches per sweep
    if (q->mode == kPT && q->ptc < 0)
        q->ptc = unit && q->Wn == 1 ? pt_cluster_blocks(1, q->L, q->req.width) : 0;
    SG_TRY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int32_t rc = SG_OK;
    if (q->mode == kPT && q->ptc > 0) {
        const ExchangeTablesDev xd{xa.xtab, xa.xoff, xa.xlen, xa.xtail};
        const bool aligned = (reinterpret_cast<uintptr_t>(q->at<uint8_t>(y.j1)) & 15u) == 0;
        rc = launch_pt_cluster(spins, j1p, kp, thr, xa.rung_of_slot, xa.slot_of_rung, xa.E, xa.accepts, xa.minE, xd,
                               status, 1, q->L, q->req.width, q->ptc, 0, n, aligned, st, base);
    }
    for (int c = 0; c < n && rc == SG_OK && !(q->mode == kPT && q->ptc > 0); ++c) {
        if (q->mode == kRowsSA) {
            for (int colour = 0; colour < 2 && rc == SG_OK; ++colour)
                rc = launch_sweep_rows_sa(spins, j6p, j1p, kp, thr, unit, 1, q->L, q->Wn, q->req.width,
                                          (uint32_t)c, colour, st, base, status);
        } else {
            bool fused = false;
            rc = launch_sweep_rows_pt(spins, j6p, j1p, kp, thr, xa.rung_of_slot, xa.E, unit, 1, q->L, q->Wn,
                                      q->req.width, (uint32_t)c, 0, nullptr, q->at<unsigned>(y.done), nullptr,
                                      st, base, status);
            if (rc == SG_OK)
                rc = launch_sweep_rows_pt(spins, j6p, j1p, kp, thr, xa.rung_of_slot, xa.E, unit, 1, q->L,
                                          q->Wn, q->req.width, (uint32_t)c, 1, &xa, q->at<unsigned>(y.done),
                                          &fused, st, base, status);
            if (rc == SG_OK && !fused) rc = launch_pt_exchange(xa, 1, (uint32_t)c, st);
        }
    }
    if (rc == SG_OK) {
        advance_kernel<<<1, 1, 0, st>>>(base, (uint32_t)n);
        if (q->mode == kRowsSA) {
            cudaMemsetAsync(q->at<void>(y.E64), 0, 8 * (size_t)q->Rp, st);
            rc = launch_energy(spins, j6p, 1, q->L, q->Wn, q->at<unsigned long long>(y.E64), st, unit ? j1p : nullptr);
            if (rc == SG_OK)
                min_energy_kernel<<<1, 256, 0, st>>>(q->at<unsigned long long>(y.E64), q->req.width,
                                                     q->at<long long>(y.out));
        } else {
            widen_kernel<<<1, 1, 0, st>>>(q->at<int32_t>(y.minE), q->at<long long>(y.out));
        }
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(q->slot->h_out, q->at<void>(y.out), 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(q->slot->h_out + 1, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = SG_ECUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc == SG_OK && e != cudaSuccess) rc = SG_ECUDA;
    if (rc == SG_OK && cudaGraphInstantiate(out, g, 0) != cudaSuccess) rc = SG_ECUDA;
    if (g) cudaGraphDestroy(g);
    if (rc != SG_OK) {
        cudaGetLastError();
        set_error("capturing a chunk of %d sweeps failed", n);
    }
    return rc;
}

// Sweeps of the next chunk: a whole chunk, cut at the end of an SA restart and at the cap.
int next_step(const Request* q, int chunk)
{
    if (q->mode == kPT) return chunk;
    return (int)std::min<int64_t>({(int64_t)chunk, (int64_t)(q->req.sweeps_per_restart - q->in_restart),
                                   q->req.sweep_cap - q->sweeps});
}

// Folds a finished chunk into the request: lowest energy, sweep counts, restart end,
// and the completion test.
void finish_chunk(Request* q, int64_t chunk_min)
{
    q->minE = std::min(q->minE, chunk_min);
    q->sweeps += q->step;
    if (q->mode != kPT) {
        q->in_restart += q->step;
        if (q->in_restart == q->req.sweeps_per_restart) {  // the next chunk starts restart + 1
            q->restart += 1;
            q->in_restart = 0;
            q->need_init = true;
        }
    }
    q->step = 0;
    q->inflight = false;
    if (q->minE <= q->target) {
        q->result.reached = 1;
        q->done = true;
    } else if (q->sweeps >= q->req.sweep_cap) {
        q->done = true;
    }
}

void fail_request(Request* q, int32_t code)
{
    q->result.status = code;
    q->inflight = false;
    q->done = true;
}

// Launches the next chunk of a PT or large-SA request on its own stream.
void launch_own_chunk(Request* q, int chunk)
{
    cudaStream_t st = q->slot->st;
    const int n = next_step(q, chunk);
    if (q->mode == kRowsSA && q->need_init) {
        const uint32_t k0 = (uint32_t)q->req.seed;
        const uint32_t k1 = (uint32_t)(q->req.seed >> 32) ^ (uint32_t)q->restart;  // restart k = instance id k
        restart_kernel<<<1, 1, 0, st>>>(q->at<RunKeys>(q->lay.keys), k0, k1, q->at<uint32_t>(q->lay.base));
        if (cudaGetLastError() != cudaSuccess ||
            launch_init_spins(q->at<int8_t>(q->lay.spins), q->at<RunKeys>(q->lay.keys), 1, q->L, q->Wn,
                              q->req.width, st) != SG_OK) {
            cudaGetLastError();
            return fail_request(q, SG_ECUDA);
        }
        q->need_init = false;
    }
    auto it = q->graphs.find(n);
    if (it == q->graphs.end()) {
        cudaGraphExec_t g = nullptr;
        if (capture_chunk(q, n, &g) != SG_OK) return fail_request(q, SG_ECUDA);
        it = q->graphs.emplace(n, g).first;
    }
    if (cudaGraphLaunch(it->second, st) != cudaSuccess || cudaEventRecord(q->slot->ev, st) != cudaSuccess) {
        cudaGetLastError();
        return fail_request(q, SG_ECUDA);
    }
    q->step = n;
    q->inflight = true;
}

// True once the request's chunk has ended (and then folds it in).
bool poll_own_chunk(Request* q)
{
    const cudaError_t e = cudaEventQuery(q->slot->ev);
    if (e == cudaErrorNotReady) return false;
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail_request(q, SG_ECUDA);
        return true;
    }
    if (*reinterpret_cast<const int*>(q->slot->h_out + 1) != 0) {  // a bounded device wait gave up
        fail_request(q, SG_ETIMEOUT);
        return true;
    }
    finish_chunk(q, q->slot->h_out[0]);
    return true;
}

bool grow_group(PlaneGroup& g, size_t np)
{
    if (np <= g.cap_planes) return true;
    size_t cap = std::max<size_t>(1024, g.cap_planes);
    while (cap < np) cap *= 2;
    for (void** p : {&g.pl, &g.ord, &g.next, &g.E, &g.init})
        if (*p) cudaFree(*p), *p = nullptr;
    if (g.hE) cudaFreeHost(g.hE), g.hE = nullptr;
    g.cap_planes = 0;
    if (cudaMalloc(&g.pl, sizeof(Plane) * cap) != cudaSuccess || cudaMalloc(&g.ord, sizeof(int) * cap) != cudaSuccess ||
        cudaMalloc(&g.next, 16) != cudaSuccess || cudaMalloc(&g.E, 8 * 128 * cap) != cudaSuccess ||
        cudaMalloc(&g.init, sizeof(Plane) * cap) != cudaSuccess ||
        cudaMallocHost(&g.hE, 8 * 128 * cap) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    g.cap_planes = cap;
    return true;
}

// Launches the ready small SA requests of one plane width together.
void launch_group(PlaneGroup& g, const std::vector<Request*>& act, int chunk)
{
    g.reqs.clear();
    for (Request* q : act)
        if (q->mode == kPlanes && q->WG == g.WG && !q->done && !q->inflight && !q->stopping) g.reqs.push_back(q);
    if (g.reqs.empty()) return;
    g.planes.clear();
    g.init_planes.clear();
    g.first.assign(1, 0);
    bool unit = true;
    for (Request* q : g.reqs) unit &= q->inst->unit_couplings;
    for (Request* q : g.reqs) {
        q->step = next_step(q, chunk);
        for (int w0 = 0; w0 < q->Wn; w0 += g.WG) {
            Plane pl{};
            pl.spins = q->at<uint32_t>(q->lay.spins) + (size_t)q->N * w0;
            pl.j1 = q->at<uint8_t>(q->lay.j1);
            pl.j6 = q->at<uint2>(q->lay.j6);
            pl.thr = q->at<uint32_t>(q->lay.thr);
            pl.k0 = (uint32_t)q->req.seed;
            pl.k1 = (uint32_t)(q->req.seed >> 32) ^ (uint32_t)q->restart;  // restart k = instance id k
            pl.L = q->L;
            pl.S = q->req.sweeps_per_restart;
            pl.w0 = w0;
            pl.R = q->req.width;
            pl.s_begin = q->in_restart;
            pl.s_end = q->in_restart + q->step;
            pl.Lmagic = (uint32_t)((0x100000000ull + pl.L - 1) / pl.L);
            pl.Hmagic = (uint32_t)((0x100000000ull + pl.L / 2 - 1) / (pl.L / 2));
            pl.out = (int)(g.first.size() - 1);
            g.planes.push_back(pl);
            if (q->need_init) g.init_planes.push_back(pl);
        }
        g.first.push_back((int)g.planes.size());
    }
    const int np = (int)g.planes.size(), nI = (int)g.init_planes.size();
    std::vector<int> order(np);
    for (int k = 0; k < np; ++k) order[k] = k;
    auto work = [&](int k) {
        const Plane& p = g.planes[k];
        return (double)p.L * p.L * p.L * (p.s_end - p.s_begin);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });  // longest first
    const size_t nE = (size_t)np * 32 * g.WG;
    cudaStream_t st = g.st;
    int32_t rc = grow_group(g, (size_t)np) ? SG_OK : SG_ENOMEM;
    // uploads of newly admitted requests ran on their own streams
    for (Request* q : g.reqs)
        if (rc == SG_OK && q->need_init && cudaStreamWaitEvent(st, q->slot->ev, 0) != cudaSuccess) rc = SG_ECUDA;
    if (rc == SG_OK &&
        (cudaMemcpyAsync(g.pl, g.planes.data(), sizeof(Plane) * np, cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(g.ord, order.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemsetAsync(g.next, 0, 4, st) != cudaSuccess || cudaMemsetAsync(g.E, 0, 8 * nE, st) != cudaSuccess ||
         (nI && cudaMemcpyAsync(g.init, g.init_planes.data(), sizeof(Plane) * nI, cudaMemcpyHostToDevice, st) !=
                    cudaSuccess)))
        rc = SG_ECUDA;
    if (rc == SG_OK && nI) rc = launch_planes_init(g.WG, static_cast<Plane*>(g.init), nI, st);
    {
        int max_L = 0;
        for (Request* q : g.reqs) max_L = std::max(max_L, q->L);
        const size_t smem = planes_smem_bytes(g.WG, max_L);
        if (rc == SG_OK)
            rc = launch_sa_planes(g.WG, static_cast<Plane*>(g.pl), static_cast<int*>(g.ord), np,
                                  static_cast<unsigned*>(g.next), unit, planes_blocks(g.WG, unit, smem), st, smem);
    }
    if (rc == SG_OK) rc = launch_planes_energy(g.WG, static_cast<Plane*>(g.pl), np, static_cast<unsigned long long*>(g.E), st);
    if (rc == SG_OK && (cudaMemcpyAsync(g.hE, g.E, 8 * nE, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                        cudaEventRecord(g.ev, st) != cudaSuccess))
        rc = SG_ECUDA;
    if (rc != SG_OK) {
        cudaGetLastError();
        for (Request* q : g.reqs) fail_request(q, rc);
        g.reqs.clear();
        return;
    }
    for (Request* q : g.reqs) {
        q->need_init = false;
        q->inflight = true;
    }
    g.inflight = true;
}

// True once the group's launch has ended (and then folds it into its requests).
bool poll_group(PlaneGroup& g)
{
    if (!g.inflight) return false;
    const cudaError_t e = cudaEventQuery(g.ev);
    if (e == cudaErrorNotReady) return false;
    g.inflight = false;
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (Request* q : g.reqs) fail_request(q, SG_ECUDA);
        return true;
    }
    for (size_t a = 0; a < g.reqs.size(); ++a) {
        Request* q = g.reqs[a];
        int64_t m = INT64_MAX;
        for (int k = g.first[a]; k < g.first[a + 1]; ++k)
            for (int rb = 0; rb < 32 * g.WG; ++rb)
                if (32 * g.planes[k].w0 + rb < q->req.width)
                    m = std::min<int64_t>(m, (int64_t)(long long)g.hE[(size_t)k * 32 * g.WG + rb]);
        finish_chunk(q, m);
    }
    return true;
}

// Gives back a request's device state (stream-ordered: no device synchronisation) and
// marks its result readable.  Caller holds the server mutex; the request is idle.
void retire(sg_server* srv, Request* q)
{
    for (auto& kv : q->graphs) cudaGraphExecDestroy(kv.second);
    q->graphs.clear();
    if (q->mem) cudaFreeAsync(q->mem, q->slot->st);
    q->mem = nullptr;
    if (q->slot) srv->free_slots.push_back(q->slot);
    q->slot = nullptr;
    cudaGetLastError();
    q->inst.reset();
    q->thr.reset();
    q->xt = ExchangeTables();
    q->t_done = Clock::now();
    q->finished = true;
    if (q->admitted) srv->in_use -= q->bytes;
}

void worker_main(sg_server* srv)
{
    cudaSetDevice(srv->device);
    const int chunk = srv->cfg.chunk_sweeps;
    std::unique_lock<std::mutex> lock(srv->mu);
    for (;;) {
        bool progress = false;
        // admission: FIFO while memory and slots allow
        while (!srv->stop && !srv->queue.empty() && (int)srv->active.size() < srv->cfg.max_active) {
            Request* q = srv->queue.front();
            if (srv->in_use + q->bytes > srv->cfg.hbm_budget_bytes) break;
            srv->queue.pop_front();
            srv->in_use += q->bytes;
            q->admitted = true;
            q->t_admit = Clock::now();
            lock.unlock();
            const int32_t rc = admit_request(srv, q);
            lock.lock();
            progress = true;
            if (rc != SG_OK) {
                q->result.status = rc;
                retire(srv, q);
                srv->cv_done.notify_all();
                continue;
            }
            srv->active.push_back(q);
        }
        for (Request* q : srv->active)
            if (q->cancelled || srv->stop) q->stopping = true;
        const std::vector<Request*> act = srv->active;
        lock.unlock();

        // chunks that ended
        for (Request* q : act)
            if (q->inflight && q->mode != kPlanes && poll_own_chunk(q)) progress = true;
        for (PlaneGroup& g : srv->groups)
            if (poll_group(g)) progress = true;
        for (Request* q : act)
            if (q->stopping && !q->inflight && !q->done) {
                q->result.status = SG_ECANCELED;
                q->done = true;
            }
        // next chunks
        for (Request* q : act)
            if (!q->done && !q->inflight && q->mode != kPlanes) {
                launch_own_chunk(q, chunk);
                progress = true;
            }
        for (PlaneGroup& g : srv->groups)
            if (!g.inflight) {
                launch_group(g, act, chunk);
                progress |= g.inflight;
            }

        lock.lock();
        std::vector<Request*> keep;
        bool retired = false;
        for (Request* q : srv->active) {
            if (q->done && !q->inflight) {
                retire(srv, q);
                retired = true;
            } else {
                keep.push_back(q);
            }
        }
        srv->active.swap(keep);
        if (retired) srv->cv_done.notify_all();
        if (srv->stop && srv->active.empty()) break;
        if (!progress && !retired) {
            // idle: wake on a submit, cancel or stop; poll the device every 50 us while busy
            if (srv->active.empty())
                srv->cv_work.wait_for(lock, std::chrono::milliseconds(20));
            else
                srv->cv_work.wait_for(lock, std::chrono::microseconds(50));
        }
    }
    lock.unlock();
    for (auto& s : srv->slots) cudaStreamSynchronize(s->st);
    for (PlaneGroup& g : srv->groups) cudaStreamSynchronize(g.st);
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
    if (!cfg || !out || cfg->max_active < 1 || cfg->max_active > 65536 || cfg->chunk_sweeps < 1 ||
        cfg->queue_capacity < 1 || cfg->hbm_budget_bytes == 0) {
        set_error("bad server config (max_active in [1, 65536], chunk_sweeps and queue_capacity >= 1, "
                  "budget > 0)");
        return SG_EINVAL;
    }
    sg_server* srv = new (std::nothrow) sg_server;
    if (!srv) return SG_ENOMEM;
    srv->cfg = *cfg;
    bool ok = cudaGetDevice(&srv->device) == cudaSuccess;
    if (ok) {
        // the requests' device memory: a pool of its own that keeps up to the budget cached
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = srv->device;
        ok = cudaMemPoolCreate(&srv->pool, &props) == cudaSuccess;
        uint64_t keep = cfg->hbm_budget_bytes;
        ok = ok && cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess;
    }
    const int widths[3] = {4, 2, 1};
    for (int k = 0; k < 3 && ok; ++k) {
        srv->groups[k].WG = widths[k];
        ok = cudaStreamCreateWithFlags(&srv->groups[k].st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&srv->groups[k].ev, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        delete srv;
        set_error("server: CUDA set-up failed (device, memory pool or streams)");
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
    auto q = std::make_unique<Request>();
    q->t_submit = Clock::now();
    q->req = *req;
    q->result.status = SG_OK;
    int32_t rc = prepare_request(srv->schedules, q.get());
    if (rc != SG_OK) return rc;
    if (q->bytes > srv->cfg.hbm_budget_bytes) {
        set_error("request needs %zu bytes of device memory, more than the server budget", q->bytes);
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
    q->ticket = srv->next_ticket++;
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
    if (pos != srv->queue.end()) {  // waiting: no device state yet
        srv->queue.erase(pos);
        q->result.status = SG_ECANCELED;
        retire(srv, q);
        srv->cv_done.notify_all();
    } else {
        q->cancelled = true;  // admitted: the worker stops it when its chunk ends
        srv->cv_work.notify_one();
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

extern "C" int32_t sg_request_bytes(const sg_request* req, uint64_t* bytes)
{
    clear_error();
    if (!req || !bytes || !valid_request(*req)) {
        set_error("bad request");
        return SG_EINVAL;
    }
    ScheduleCache cache;
    Request q;
    q.req = *req;
    const int32_t rc = prepare_request(cache, &q);
    if (rc == SG_OK) *bytes = q.bytes;
    return rc;
}
