/*
 * sg.h -- C ABI of libsg, the GB300 (sm_103a) Metropolis simulated-annealing and
 * parallel-tempering library for tile-planted cubic-lattice Ising spin glasses.
 *
 * Problem statement (arXiv:2501.17267):
 *   H = sum over lattice edges <i,j> of J_ij s_i s_j, s_i in {-1,+1}      (Eq. 1)
 *   on the periodic L x L x L simple-cubic lattice (Sec. II, Fig. 4 caption),
 *   scored by the optimality gap eps = (E - E_gs) / |E_gs|                   (Eq. 2)
 *   where E_gs is the planted ground-state energy of a tile-planting instance
 *   (Sec. II).  The solvers are Metropolis single-spin-flip simulated annealing
 *   along a beta schedule (App. D.1) and parallel tempering over a geometric beta
 *   ladder (App. D.2).
 *
 * Conventions shared by every entry point:
 *   - Every call returns int32_t status: SG_OK (0) or a negative SG_E* code.  On
 *     error, sg_last_error_string() gives a message for the calling thread.  No C++
 *     exception crosses the ABI.
 *   - Site index i = x + L*(y + L*z).  Couplings "J3" are int8 [N][3] (N = L^3);
 *     J3[i][d] couples site i to its +1 neighbour along axis d (0=x, 1=y, 2=z),
 *     periodic.  |J| <= SG_JMAX.  Spins are int8 in {-1, +1}.
 *   - Handles (sg_instance) are owned by the library and released with
 *     sg_instance_destroy.  Caller buffers are borrowed for the duration of the
 *     call only: host pointers, or device pointers when the matching *_mem field
 *     is SG_MEM_DEVICE (device memory of the current CUDA device).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; every run call returns after its host outputs are
 *     written (it synchronises the stream before returning).
 *   - Runs are deterministic: the same instance, parameters and seed give the same
 *     bytes on every call, batch composition and GPU.  Every random number is word
 *     w of Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed_lo32, seed_hi32 ^ instance_id) at a counter that names its use:
 *       Metropolis draw of replica r at site i, sweep s: the 32-bit uniform
 *         U = A * 2^24 + B, with g = r / 32, b = r % 32: bit j (j = 0..7) of the
 *         leading byte A is bit b of word j % 4 at counter (i, s, 2g + j/4, 0), and
 *         B is the top 24 bits of word r % 4 at counter (i, s, r/4, 4)
 *       initial spin of replica r at site i:             counter (i, 0xFFFFFFFF, r/4, 0), w = r%4,
 *                                                         spin = -1 iff bit 31 is set
 *       PT exchange of rungs (k, k+1) after sweep s:      counter (k, s, 0, 1), w = 0
 *   - A Metropolis attempt at site i computes x = s_i * sum_j J_ij s_j (flipping
 *     changes E by dE = -2x) and flips when x >= 0, or when the draw U satisfies
 *     U < floor(2^32 * exp(-beta * dE)) (clamped to 2^32 - 1).  Sites are swept in checkerboard order:
 *     all sites with x+y+z even, then all with x+y+z odd.
 */
#ifndef SG_H
#define SG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SG_OK 0
#define SG_EINVAL (-1)    /* invalid argument (odd L, beta <= 0, R = 0, |J| > SG_JMAX, ...) */
#define SG_ENOMEM (-2)    /* host or device allocation failed, or request exceeds a budget */
#define SG_ECUDA (-3)     /* a CUDA runtime call failed */
#define SG_ETIMEOUT (-4)  /* a bounded device-side wait gave up */
#define SG_EBUSY (-5)     /* a queue or slot pool is full */
#define SG_EINTERNAL (-6) /* a self-check failed (e.g. incremental energy != recomputed) */
#define SG_ECANCELED (-7) /* the request was cancelled */
#define SG_PENDING 1      /* sg_poll: the request has not finished */

#define SG_MEM_HOST 0
#define SG_MEM_DEVICE 1

#define SG_SCHEDULE_LINEAR 0    /* beta_s = b0 + (b1 - b0) * s / (S - 1)      */
#define SG_SCHEDULE_GEOMETRIC 1 /* beta_s = b0 * (b1 / b0) ^ (s / (S - 1))    */

#define SG_JMAX 2      /* largest |J| the kernels accept */
#define SG_LMAX 256    /* largest lattice side */

typedef struct sg_instance sg_instance;

/* ------------------------------------------------------------------------ */
/* Instances: tile planting (Sec. II).                                       */
/* ------------------------------------------------------------------------ */

typedef struct sg_instance_desc {
    int32_t L;             /* even, 2 <= L <= SG_LMAX */
    int32_t gauge;         /* 1: scramble the planted state with a random gauge (Sec. II) */
    uint64_t seed;         /* instance seed */
    double class_prob[3];  /* weights of tile classes F22, F42, F6 (>= 0, sum > 0) */
} sg_instance_desc;

/* Generate a tile-planted instance (Sec. II).  The lattice is split into the
 * N/4 unit cubes whose origin has all-even or all-odd coordinates; every edge lies
 * in exactly one.  Each cube draws a class (F22: two adjacent frustrated faces,
 * F42: four frustrated faces with the two others opposite, F6: all six frustrated;
 * |J| = 1) and one of the 48 cube symmetries; E_gs is the sum of the cube minima
 * and the planted state is all +1, then gauged by a random tau when gauge = 1.
 * Counters: class and symmetry from words 0 and 1 of Philox at (tile, 0, 0, 2),
 * gauge from bit 31 of word 0 at (site, 0, 0, 3), key (seed_lo32, seed_hi32).
 * Errors: SG_EINVAL for bad L or weights; SG_ENOMEM. */
int32_t sg_instance_create(const sg_instance_desc* desc, sg_instance** out);

/* Wrap caller couplings J3 [N][3] (host or device per mem_kind) with a known
 * ground-state energy e_gs (used only for eps; pass 0 if unknown, eps is then
 * not finite).  The planted state is reported as all +1.  The couplings are copied.
 * Errors: SG_EINVAL for bad L, a NULL pointer or |J| > SG_JMAX. */
int32_t sg_instance_create_from_couplings(int32_t L, const int8_t* J3, int32_t mem_kind,
                                          int64_t e_gs, sg_instance** out);

/* Read back an instance.  Any output pointer may be NULL.  J3_out: host int8
 * [N][3]; planted_out: host int8 [N]. */
int32_t sg_instance_get(const sg_instance* inst, int32_t* L_out, int8_t* J3_out,
                        int8_t* planted_out, int64_t* e_gs_out);

/* Release an instance (and its cached device copy).  NULL is a no-op. */
int32_t sg_instance_destroy(sg_instance* inst);

/* ------------------------------------------------------------------------ */
/* Simulated annealing (App. D.1).                                           */
/* ------------------------------------------------------------------------ */

typedef struct sg_sa_params {
    int32_t replicas;      /* R >= 1: independent chains (num_reads), run side by side */
    int32_t sweeps;        /* S >= 0: one checkerboard sweep per schedule value */
    double beta0, beta1;   /* schedule end points, > 0 */
    int32_t schedule;      /* SG_SCHEDULE_LINEAR or SG_SCHEDULE_GEOMETRIC */
    uint32_t instance_id;  /* mixed into the RNG key */
    uint64_t seed;         /* run seed */
} sg_sa_params;

typedef struct sg_sa_result {
    int64_t* E;            /* [R] host: final energy of each replica (required) */
    double* eps;           /* [R] host: final optimality gap (Eq. 2), may be NULL */
    int8_t* spins;         /* [R][N]: final spins, may be NULL */
    int32_t spins_mem;     /* SG_MEM_HOST or SG_MEM_DEVICE for `spins` */
} sg_sa_result;

/* Anneal R replicas of one instance for S sweeps.  The energy of each replica is
 * computed (Eq. 1) from its final spins.  Errors: SG_EINVAL, SG_ENOMEM, SG_ECUDA. */
int32_t sg_sa_run(const sg_instance* inst, const sg_sa_params* p, sg_sa_result* out,
                  void* stream);

/* Anneal n instances in one call; instances of equal L and equal (R, S, beta0,
 * beta1, schedule) share launches.  Results are byte-identical to n separate
 * sg_sa_run calls. */
int32_t sg_sa_run_batch(const sg_instance* const* insts, const sg_sa_params* ps, int32_t n,
                        sg_sa_result* outs, void* stream);

/* ------------------------------------------------------------------------ */
/* Fragment meta-heuristic (Sec. II; App. A, Fig. 5) with SA fragment        */
/* anneals.                                                                 */
/* ------------------------------------------------------------------------ */

/* The paper's linear-time meta-heuristic bootstraps local optimisations of small
 * cubic fragments (its own runs contract tensor networks; it notes that SA can take
 * their place).  Our reading: spins are fixed in l^3 waves -- wave a + l*(b + l*c)
 * fixes every spin with coordinates congruent to (a, b, c) mod l -- and spin i is
 * fixed from the cube of side l centred on it: the cube's spins fixed by earlier waves
 * keep their values, the others are annealed (32 independent reads, `sweeps`
 * checkerboard sweeps along the geometric schedule beta0 -> beta1) with only the
 * bonds inside the cube, and spin i takes its value in the read of lowest cube
 * energy (the first such read).  With L a multiple of l the cubes of one wave are
 * disjoint and are annealed in parallel.  Draws: read r at cube site q (q = dx +
 * l*(dy + l*dz), offsets from the cube's corner) uses word r % 4 of the Philox block
 * at counter (i, sweep, 8q + r/4, 5); initial values sweep 0xFFFFFFFF, bit 31. */
typedef struct sg_fragment_params {
    int32_t l;             /* fragment side: odd, 1 <= l < L, L a multiple of l, l <= 7 */
    int32_t sweeps;        /* >= 0 sweeps per fragment anneal */
    double beta0, beta1;   /* geometric schedule end points, > 0 */
    uint32_t instance_id;  /* mixed into the RNG key */
    uint64_t seed;         /* run seed */
} sg_fragment_params;

typedef struct sg_fragment_result {
    int64_t E;             /* energy (Eq. 1) of the configuration reached */
    double eps;            /* its optimality gap (Eq. 2) */
    int8_t* spins;         /* [N] the configuration, may be NULL */
    int32_t spins_mem;     /* SG_MEM_HOST or SG_MEM_DEVICE for `spins` */
} sg_fragment_result;

/* Run the meta-heuristic on n instances of one side L with one set of parameters
 * (wave by wave, all instances' fragments of a wave in one launch).  Errors:
 * SG_EINVAL (unequal L or parameters, l not as stated), SG_ENOMEM, SG_ECUDA. */
int32_t sg_fragment_run_batch(const sg_instance* const* insts, const sg_fragment_params* p, int32_t n,
                              sg_fragment_result* outs, void* stream);
int32_t sg_fragment_run(const sg_instance* inst, const sg_fragment_params* p, sg_fragment_result* out,
                        void* stream);

/* The same waves and cubes with the centre spin set by the exact zero-temperature
 * (tropical) marginal of its cube, the limit beta -> infinity of the paper's
 * tensor-network fragment contraction (App. A; the tropical form is suggested in
 * Sec. III): the lowest cube energy over the cube's free spins with s_c = +1 is compared
 * with that with s_c = -1 (+1 on a tie), by enumerating all states of the free spins.
 * Only p->l is used, l in {1, 3} (at most 27 free spins).  Errors as sg_fragment_run. */
int32_t sg_fragment_tropical_run_batch(const sg_instance* const* insts, const sg_fragment_params* p, int32_t n,
                                       sg_fragment_result* outs, void* stream);

/* ------------------------------------------------------------------------ */
/* Parallel tempering (App. D.2).                                            */
/* ------------------------------------------------------------------------ */

typedef struct sg_pt_params {
    int32_t temps;         /* K >= 1 rungs (one replica slot per rung) */
    int32_t sweeps;        /* S >= 0 */
    double beta_min, beta_max; /* geometric ladder beta_k = bmin (bmax/bmin)^(k/(K-1)), > 0 */
    uint32_t instance_id;
    uint64_t seed;
} sg_pt_params;

typedef struct sg_pt_result {
    int64_t* E;            /* [K] host, by slot: final energies (may be NULL) */
    int32_t* perm;         /* [K] host, by slot: rung held at the end (may be NULL) */
    int64_t* accepts;      /* [K-1] host: accepted swaps of rungs (k, k+1) (may be NULL) */
    int64_t minE;          /* out: lowest energy seen in any slot, after init and every sweep */
    double min_eps;        /* out: eps of minE (Eq. 2) */
    int8_t* spins;         /* [K][N] by slot, may be NULL */
    int32_t spins_mem;
} sg_pt_result;

/* Run PT: slot energies are tracked incrementally on the device (the exchange needs
 * them after every sweep) and checked against a full recompute at the end
 * (mismatch: SG_EINTERNAL).  After every sweep s, rung pairs (k, k+1) with k = s mod 2 attempt a
 * label swap, accepted when d = E_a - E_b <= 0 (slot a at rung k, b at k+1) or
 * when the draw u < floor(2^32 exp(-(beta_{k+1} - beta_k) d)).  Errors: SG_EINVAL
 * (also when the ladder is so fine that an exchange table would exceed 2^22
 * entries), SG_ENOMEM, SG_ECUDA, SG_EINTERNAL. */
int32_t sg_pt_run(const sg_instance* inst, const sg_pt_params* p, sg_pt_result* out,
                  void* stream);

/* n instances in one call; instances of equal L and equal (K, S, beta range)
 * share launches.  Byte-identical to n separate sg_pt_run calls. */
int32_t sg_pt_run_batch(const sg_instance* const* insts, const sg_pt_params* ps, int32_t n,
                        sg_pt_result* outs, void* stream);

/* ------------------------------------------------------------------------ */
/* Energy (Eq. 1).                                                           */
/* ------------------------------------------------------------------------ */

/* E_out[c] = sum_i sum_d J3[i][d] s_c[i] s_c[i + e_d] for n_configs spin
 * configurations s_c laid out [n_configs][N] (host or device per mem_kind);
 * E_out is host.  Errors: SG_EINVAL (also for a spin not in {-1,+1}), SG_ECUDA. */
int32_t sg_energy(const sg_instance* inst, const int8_t* spins, int32_t n_configs,
                  int32_t mem_kind, int64_t* E_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: solve requests to a target gap, continuously batched.            */
/* ------------------------------------------------------------------------ */
/* A server owns one worker thread and the device it was created on.  Requests (a
 * fresh tile-planted instance plus SA or PT parameters, Sec. II and App. D) wait in a
 * FIFO queue and are admitted while their device memory fits the budget and a slot
 * is free; admitted requests stay resident and advance together, chunk_sweeps sweeps
 * per round: all SA requests in one persistent launch, each PT request as a captured
 * CUDA graph on its own stream, so their work overlaps on the GPU.  A request is done
 * at the first round boundary where its lowest energy E satisfies
 * E <= E_gs + floor(eps_target * |E_gs|) (time to target, TT-eps, Eq. 2), or at the
 * first round boundary at or past sweep_cap sweeps (censored; SA rounds also end
 * exactly at the cap and at the end of every restart, PT rounds are whole chunks).
 * "Lowest energy" is the minimum over replicas at round boundaries for SA and the
 * running minimum PT keeps after every exchange (as sg_pt_run reports it).  Results do not depend on what else is running:
 * every draw is named by the request's own seed, sites, sweeps and replicas, and the
 * checks happen at fixed sweep counts.  SA requests anneal in restarts of
 * sweeps_per_restart sweeps; restart k is the run sg_sa_run gives with instance_id = k. */

#define SG_REQ_SA 0
#define SG_REQ_PT 1

typedef struct sg_server sg_server;

typedef struct sg_server_config {
    uint64_t hbm_budget_bytes;  /* device memory the server may hold for admitted requests */
    int32_t max_active;         /* requests resident at once (>= 1) */
    int32_t chunk_sweeps;       /* sweeps per round; completion is checked between rounds */
    int32_t queue_capacity;     /* waiting requests; beyond it sg_submit returns SG_EBUSY */
} sg_server_config;

typedef struct sg_request {
    int32_t kind;               /* SG_REQ_SA or SG_REQ_PT */
    sg_instance_desc instance;  /* the instance the server generates for this request */
    int32_t width;              /* SA: replicas R; PT: temperatures K (1..256) */
    int32_t sweeps_per_restart; /* SA: sweeps of one anneal; ignored for PT */
    double beta0, beta1;        /* SA: schedule ends; PT: geometric ladder ends; > 0 */
    int32_t schedule;           /* SA: SG_SCHEDULE_LINEAR or _GEOMETRIC */
    uint64_t seed;              /* run seed */
    double eps_target;          /* target optimality gap (>= 0) */
    int64_t sweep_cap;          /* stop after this many sweeps (all restarts) */
} sg_request;

typedef struct sg_result {
    int32_t status;             /* SG_OK, SG_ECANCELED, or the error that ended the request */
    int32_t reached;            /* 1: target reached; 0: stopped at the sweep cap */
    int64_t sweeps;             /* sweeps run when it stopped (all restarts) */
    int64_t minE;               /* lowest energy seen */
    int64_t e_gs;               /* planted ground-state energy */
    double min_eps;             /* gap of minE (Eq. 2) */
    double queue_s;             /* submit -> admitted */
    double run_s;               /* admitted -> done */
    double total_s;             /* submit -> done: the time to target */
} sg_result;

/* Start a server on the current CUDA device.  Errors: SG_EINVAL (bad config),
 * SG_ECUDA, SG_ENOMEM. */
int32_t sg_server_create(const sg_server_config* cfg, sg_server** out);

/* Queue a request; *ticket identifies it.  Errors: SG_EINVAL (bad request), SG_ENOMEM
 * (it alone needs more than the budget), SG_EBUSY (queue full). */
int32_t sg_submit(sg_server* srv, const sg_request* req, uint64_t* ticket);

/* Device memory the server would hold for this request while it runs (the amount
 * admission counts against hbm_budget_bytes): spins, couplings, tables and run state.
 * The instance is generated to size its tables.  Errors: SG_EINVAL. */
int32_t sg_request_bytes(const sg_request* req, uint64_t* bytes);

/* Wait up to timeout_ms (0: just look; < 0: wait until done) for a request.  Returns
 * SG_OK with *out filled once it is done (a ticket is reported once, then forgotten),
 * SG_PENDING while it is not, SG_EINVAL for an unknown ticket. */
int32_t sg_poll(sg_server* srv, uint64_t ticket, int32_t timeout_ms, sg_result* out);

/* Cancel a request: a waiting one leaves the queue, a running one stops at the next
 * round boundary; its result has status SG_ECANCELED.  SG_EINVAL for an unknown ticket. */
int32_t sg_cancel(sg_server* srv, uint64_t ticket);

/* Stop the worker (running requests are cancelled) and release everything. */
int32_t sg_server_destroy(sg_server* srv);

/* ------------------------------------------------------------------------ */
/* Energy without device allocation (no counterpart in the paper).           */
/* ------------------------------------------------------------------------ */

/* Size of the fixed device scratch array behind sg_energy_noalloc (16 MiB).  Every
 * GPU that loads the library holds this array until the process exits. */
#define SG_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* The energies sg_energy computes, for callers that must not let a library allocate
 * device memory -- for example a server that owns the device-memory budget through its
 * own pool, or a latency-critical loop where cudaMalloc/cudaFree (which can synchronise
 * the device and can fail under fragmentation) is not allowed.  The paper has no
 * counterpart: this is an interface for such callers only.
 *   L          lattice side (even, 2 <= L <= SG_LMAX)
 *   J3_dev     device int8 [L^3][3] couplings (|J| <= SG_JMAX), read only
 *   spins_dev  device int8 [n_configs][L^3] configurations in {-1, +1}, read only
 *   E_dev      device int64 [n_configs], written
 * All pointers are device memory of the current device.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  All scratch lives in one fixed array of
 * SG_NOALLOC_SCRATCH_BYTES per device; a request that needs more (about
 * 9*L^3 + L^3 * 4*ceil(n_configs/32) bytes) fails with SG_EINVAL and a message.
 * The first call on a device is its set-up: it looks up the array's device address
 * with that device current (loading the library's device code there); make that first
 * call before any stream capture.  Every call repeats the lookup, so a device reset
 * between calls is harmless.  Every call shares the array and it keeps the last call's
 * contents (the call clears what must start at zero): calls that overlap on the GPU --
 * on different streams or from different host threads -- race on it, so serialise
 * them.  The call enqueues on `stream` and returns after it has completed.
 * Errors: SG_EINVAL (bad arguments, too large, a spin not in {-1,+1}), SG_ECUDA. */
int32_t sg_energy_noalloc(int32_t L, const int8_t* J3_dev, const int8_t* spins_dev,
                          int32_t n_configs, int64_t* E_dev, void* stream);

/* ------------------------------------------------------------------------ */
/* Launch statistics (diagnostics; no counterpart in the paper).             */
/* ------------------------------------------------------------------------ */

#define SG_KERNEL_INIT 0         /* initial spins */
#define SG_KERNEL_ENERGY 1       /* full energy recompute */
#define SG_KERNEL_SWEEP 2        /* Metropolis sweep kernels, one or two launches per sweep
                                    (the row kernels; fragment waves) */
#define SG_KERNEL_EXCHANGE 3     /* PT exchange */
#define SG_KERNEL_OTHER 4        /* layout conversion, checks, set-up */
#define SG_KERNEL_SWEEP_CHUNK 5  /* Metropolis sweep kernels that run many sweeps per launch
                                    with the lattice in shared memory (thread-block cluster,
                                    cooperative and persistent batch forms) */
#define SG_KERNEL_KINDS 6

/* A PT batch may run both sweep kinds at once on different streams (some instances on
 * clusters, the others through the row kernels), so device_ms of one kind is the time of
 * that kind's launches alone. */
typedef struct sg_kernel_stats {
    int64_t launches[SG_KERNEL_KINDS];  /* kernels launched by this library, per kind */
    double device_ms[SG_KERNEL_KINDS];  /* summed launch durations (only while timing is on) */
    int64_t units[SG_KERNEL_KINDS];     /* work units processed: spin-flip attempts for the
                                           two sweep kinds, spin sites x replicas otherwise */
} sg_kernel_stats;

/* timing = 1: every later launch is bracketed by CUDA events recorded on the
 * launch's own stream, and its duration is added to device_ms when the run that
 * issued it completes.  Launch counts and units are always kept.  Process-wide. */
int32_t sg_stats_enable(int32_t timing);

/* Copy the process-wide counters into *out; reset = 1 zeroes them afterwards. */
int32_t sg_stats_read(sg_kernel_stats* out, int32_t reset);

/* Generator throughput: the rate, in blocks per second, at which this device
 * produces Philox4x32-10 blocks (Salmon, Moraes, Dror, Shaw, SC'11) when drawing is
 * all it does.  Every thread of 8 x (SM count) blocks of 256 threads draws
 * blocks_per_thread blocks (even, >= 2), two independent ones at a time, as a sweep
 * thread draws its planes.  The Metropolis draws of the SA / PT sweeps (App. D.1,
 * D.2) take two blocks per word of 32 replicas, so 16 x this rate bounds the attempt
 * rate of the sweeps' integer work.  One warm-up and one timed launch on `stream`
 * (a cudaStream_t, NULL for the default stream), timed with CUDA events; returns
 * once the timed launch has completed.  Allocates 4 bytes per thread, stream-ordered,
 * freed before returning.
 * Errors: SG_EINVAL (blocks_per_thread odd or < 2, NULL output), SG_ECUDA. */
int32_t sg_philox_rate(int32_t blocks_per_thread, double* blocks_per_second, void* stream);

/* ------------------------------------------------------------------------ */
/* Misc.                                                                     */
/* ------------------------------------------------------------------------ */

/* Message of the last failed call on this thread ("" if none). */
const char* sg_last_error_string(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t sg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
