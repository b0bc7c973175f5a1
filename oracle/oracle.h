/*
 * oracle.h -- declarations of the CPU oracle (test infrastructure only; see oracle.c).
 * All pointers are host pointers owned by the caller.  Functions returning int
 * give 0 on success, -1 on invalid arguments, -2 on allocation failure, -3 when
 * the tile set fails to partition the edges (never expected).
 */
#ifndef SG_ORACLE_H
#define SG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_CLASS_F22 = 0, OR_CLASS_F42 = 1, OR_CLASS_F6 = 2 };
enum {
    OR_DOMAIN_METROPOLIS = 0, /* init: (site, 0xFFFFFFFF, replica/4, 0); draws: (site, sweep, 2*(replica/32) + j/4, 0) */
    OR_DOMAIN_EXCHANGE = 1,   /* counter (rung pair k, sweep, 0, 1)  */
    OR_DOMAIN_GENERATE = 2,   /* counter (tile, 0, 0, 2)              */
    OR_DOMAIN_GAUGE = 3,      /* counter (site, 0, 0, 3)              */
    OR_DOMAIN_TAIL = 4,       /* counter (site, sweep, replica/4, 4): low 24 bits of a draw */
    OR_DOMAIN_FRAGMENT = 5    /* counter (centre, sweep, 8*q + read/4, 5): fragment anneals */
};
#define OR_FRAGMENT_READS 32
#define OR_SWEEP_INIT 0xFFFFFFFFu

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

int64_t or_site(int L, int x, int y, int z);
int64_t or_energy(int L, const int8_t* J3, const int8_t* s);
int or_local_field(int L, const int8_t* J3, const int8_t* s, int64_t i);
double or_epsilon(int64_t E, int64_t E_gs);

void or_cube_edge(int e, int* u, int* v);
int or_tile_template(int cls, int8_t J12[12]);
int or_tile_energy(const int8_t J12[12], int state);
void or_tile_bruteforce(const int8_t J12[12], int* emin, int* degeneracy);
int or_cube_symmetry(int sym, int corner);

int or_generate(int L, uint64_t seed, const double class_prob[3], int gauge,
                int8_t* J3, int8_t* tau, int64_t* e_gs);

void or_beta_schedule(int S, double b0, double b1, int geometric, double* beta);
void or_pt_ladder(int K, double bmin, double bmax, double* beta);
uint32_t or_metropolis_threshold(double beta, int dE);
uint32_t or_exchange_threshold(double dbeta, int64_t d);

int8_t or_init_spin(uint64_t seed, uint32_t instance_id, int64_t i, int rep);
void or_metropolis_uniform_grid(uint64_t seed, uint32_t instance_id, int64_t i0, int n_i, uint32_t s0,
                                int n_s, const int32_t* reps, int n_reps, uint32_t* out);
int or_sa_run(int L, const int8_t* J3, uint64_t seed, uint32_t instance_id,
              int S, double b0, double b1, int geometric,
              const int32_t* reps, int nreps, int8_t* spins_out, int64_t* E_out);
int or_pt_run(int L, const int8_t* J3, uint64_t seed, uint32_t instance_id,
              int K, int S, double bmin, double bmax,
              int8_t* spins_out, int64_t* E_out, int32_t* perm_out,
              int64_t* minE_out, int64_t* accepts_out);

int or_fragment_run(int L, const int8_t* J3, int l, int S, double b0, double b1, uint64_t seed,
                    uint32_t instance_id, int8_t* spins_out, int64_t* E_out);
int or_fragment_min_energies(int F, const int* h, const int8_t* Jff, int c, int64_t* m_plus, int64_t* m_minus);
int or_fragment_tropical(int L, const int8_t* J3, int l, int8_t* spins_out, int64_t* E_out);

#ifdef __cplusplus
}
#endif
#endif
