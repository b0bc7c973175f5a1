/*
 * oracle.c -- plain, sequential CPU statement of the spin-glass Metropolis path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  The product path (the CUDA library) never
 * links, includes or calls it, and shares no code with it.
 *
 * What it computes, each function citing the passage of arXiv:2501.17267 it follows:
 *   - the zero-field Ising Hamiltonian on the periodic simple-cubic lattice (Eq. 1);
 *   - the optimality gap eps = (E - E_gs)/|E_gs| (Eq. 2);
 *   - cubic tile planting with gauge scrambling (Sec. II, instance paragraph);
 *   - simulated annealing with Metropolis sweeps along a beta schedule (App. D.1);
 *   - parallel tempering over a geometric beta ladder (App. D.2).
 * The RNG is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11), written here from that published description.
 *
 * Everything is deliberately slow: nine Philox blocks per spin-flip attempt (eight
 * for the bit planes of the draw's leading byte, one for its low bits), one site at a
 * time, no blocking or vectorisation.
 *
 * Readings of points the paper leaves open that shape this file: the three tile
 * classes are fixed by their sets of
 * frustrated faces (F22: two adjacent faces, F42: four faces with the two
 * unfrustrated ones opposite, F6: all six); the sum in Eq. 1 runs once over each
 * lattice edge; sites are swept in checkerboard order (colour 0, then colour 1);
 * the Metropolis draw is accepted when u < floor(2^32 exp(-beta dE)), with the
 * 32-bit uniform u of an attempt assembled from Philox words (metropolis_uniform).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11).                                     */
/* ------------------------------------------------------------------------ */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u; /* key increments    */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)mult0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)mult1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One 32-bit word of the Philox block at counter (c0, c1, c2, c3). */
static uint32_t philox_word(uint32_t k0, uint32_t k1,
                            uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {k0, k1};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------------------ */
/* Lattice (Eq. 1 on the periodic L x L x L simple-cubic lattice).           */
/* ------------------------------------------------------------------------ */

int64_t or_site(int L, int x, int y, int z)
{
    x = ((x % L) + L) % L;
    y = ((y % L) + L) % L;
    z = ((z % L) + L) % L;
    return (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * (int64_t)z);
}

static void site_coords(int L, int64_t i, int* x, int* y, int* z)
{
    *x = (int)(i % L);
    *y = (int)((i / L) % L);
    *z = (int)(i / ((int64_t)L * L));
}

/* Neighbour of site i one step along axis d (0=x, 1=y, 2=z) in direction dir (+1/-1). */
static int64_t neighbour(int L, int64_t i, int d, int dir)
{
    int c[3];
    site_coords(L, i, &c[0], &c[1], &c[2]);
    c[d] += dir;
    return or_site(L, c[0], c[1], c[2]);
}

/* Eq. 1, read as one term per lattice edge: E = sum_i sum_d J[i][d] s_i s_{i+e_d}. */
int64_t or_energy(int L, const int8_t* J3, const int8_t* s)
{
    int64_t N = (int64_t)L * L * L;
    int64_t E = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d)
            E += (int64_t)J3[3 * i + d] * s[i] * s[neighbour(L, i, d, +1)];
    return E;
}

/* Local field h_i = sum over the six neighbours j of J_ij s_j. */
int or_local_field(int L, const int8_t* J3, const int8_t* s, int64_t i)
{
    int h = 0;
    for (int d = 0; d < 3; ++d) {
        int64_t fwd = neighbour(L, i, d, +1);
        int64_t bwd = neighbour(L, i, d, -1);
        h += J3[3 * i + d] * s[fwd];     /* edge (i, i+e_d) is stored at i      */
        h += J3[3 * bwd + d] * s[bwd];   /* edge (i-e_d, i) is stored at i-e_d  */
    }
    return h;
}

/* Eq. 2. */
double or_epsilon(int64_t E, int64_t E_gs)
{
    return (double)(E - E_gs) / (double)(-E_gs);
}

/* ------------------------------------------------------------------------ */
/* Cubic tiles (Sec. II: tile planting, classes F22, F42, F6).               */
/* ------------------------------------------------------------------------ */

/* Corner (a, b, c) of the unit cube has index a + 2b + 4c.  Edge e = 4*d + j is
 * the edge along axis d whose other two coordinates, in increasing axis order,
 * form the two bits of j.  Returns the two corner indices of edge e. */
void or_cube_edge(int e, int* u, int* v)
{
    int d = e / 4, j = e % 4;
    int other[2], n = 0;
    for (int a = 0; a < 3; ++a)
        if (a != d) other[n++] = a;
    int coord[3] = {0, 0, 0};
    coord[other[0]] = j & 1;
    coord[other[1]] = (j >> 1) & 1;
    *u = coord[0] + 2 * coord[1] + 4 * coord[2];
    coord[d] = 1;
    *v = coord[0] + 2 * coord[1] + 4 * coord[2];
}

/* Templates: every edge ferromagnetic (J = -1) except the listed ones (J = +1),
 * which are chosen so that the frustrated faces are the ones the class names. */
int or_tile_template(int cls, int8_t J12[12])
{
    for (int e = 0; e < 12; ++e) J12[e] = -1;
    switch (cls) {
    case OR_CLASS_F22: /* x-edge at (y=0,z=0): frustrates faces y=0 and z=0 (adjacent) */
        J12[0] = +1;
        break;
    case OR_CLASS_F42: /* x-edges at (0,0) and (1,1): all faces but x=0 and x=1 */
        J12[0] = +1;
        J12[3] = +1;
        break;
    case OR_CLASS_F6:  /* x(0,0), y(x=0,z=1), z(x=1,y=1): each face once */
        J12[0] = +1;
        J12[4 + 2] = +1;
        J12[8 + 3] = +1;
        break;
    default:
        return -1;
    }
    return 0;
}

/* Energy of one cube for a corner state given as 8 bits (bit v set = spin -1). */
int or_tile_energy(const int8_t J12[12], int state)
{
    int E = 0;
    for (int e = 0; e < 12; ++e) {
        int u, v;
        or_cube_edge(e, &u, &v);
        int su = ((state >> u) & 1) ? -1 : +1;
        int sv = ((state >> v) & 1) ? -1 : +1;
        E += J12[e] * su * sv;
    }
    return E;
}

/* Exhaustive search over the 2^8 corner states. */
void or_tile_bruteforce(const int8_t J12[12], int* emin, int* degeneracy)
{
    int best = 1 << 30, count = 0;
    for (int st = 0; st < 256; ++st) {
        int E = or_tile_energy(J12, st);
        if (E < best) { best = E; count = 1; }
        else if (E == best) ++count;
    }
    *emin = best;
    *degeneracy = count;
}

/* The 48 symmetries of the cube: sym = 8*p + r, p indexing the axis permutations
 * in lexicographic order, r the reflection bits.  New coordinate along axis a is
 * the old coordinate along perm[a], reflected when bit a of r is set. */
int or_cube_symmetry(int sym, int corner)
{
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                    {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int p = sym / 8, r = sym % 8;
    int old[3] = {corner & 1, (corner >> 1) & 1, (corner >> 2) & 1};
    int nw[3];
    for (int a = 0; a < 3; ++a) nw[a] = old[perms[p][a]] ^ ((r >> a) & 1);
    return nw[0] + 2 * nw[1] + 4 * nw[2];
}

/* ------------------------------------------------------------------------ */
/* Instance generator (Sec. II: tile planting + gauge scrambling).           */
/* ------------------------------------------------------------------------ */

int or_generate(int L, uint64_t seed, const double class_prob[3], int gauge,
                int8_t* J3, int8_t* tau, int64_t* e_gs)
{
    if (L < 2 || (L % 2) != 0) return -1;
    double total = class_prob[0] + class_prob[1] + class_prob[2];
    if (!(class_prob[0] >= 0 && class_prob[1] >= 0 && class_prob[2] >= 0 && total > 0))
        return -1;
    /* class = inverse CDF of a uniform 32-bit word against the cumulative
     * probabilities in 2^32 fixed point */
    uint64_t cut0 = (uint64_t)floor(ldexp(class_prob[0] / total, 32));
    uint64_t cut1 = (uint64_t)floor(ldexp((class_prob[0] + class_prob[1]) / total, 32));

    int8_t templ[3][12];
    int tmin[3];
    for (int c = 0; c < 3; ++c) {
        int deg;
        or_tile_template(c, templ[c]);
        or_tile_bruteforce(templ[c], &tmin[c], &deg);
    }

    int64_t N = (int64_t)L * L * L;
    int8_t* covered = (int8_t*)calloc((size_t)(3 * N), 1);
    if (!covered) return -2;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    int H = L / 2;
    int64_t ntiles = 2 * (int64_t)H * H * H;
    int64_t E = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        /* tiles 0 .. H^3-1 sit at all-even origins, the rest at all-odd origins */
        int64_t tt = t % ((int64_t)H * H * H);
        int odd = t >= (int64_t)H * H * H;
        int ox = 2 * (int)(tt % H) + odd;
        int oy = 2 * (int)((tt / H) % H) + odd;
        int oz = 2 * (int)(tt / ((int64_t)H * H)) + odd;
        uint32_t u0 = philox_word(k0, k1, (uint32_t)t, 0, 0, OR_DOMAIN_GENERATE, 0);
        uint32_t u1 = philox_word(k0, k1, (uint32_t)t, 0, 0, OR_DOMAIN_GENERATE, 1);
        int cls = (u0 < cut0) ? 0 : ((u0 < cut1) ? 1 : 2);
        int sym = (int)(((uint64_t)u1 * 48u) >> 32);
        E += tmin[cls];
        for (int e = 0; e < 12; ++e) {
            int u, v;
            or_cube_edge(e, &u, &v);
            int gu = or_cube_symmetry(sym, u), gv = or_cube_symmetry(sym, v);
            /* the image edge joins corners gu and gv; find its axis and base corner */
            int diff = gu ^ gv;
            int d = (diff == 1) ? 0 : (diff == 2) ? 1 : 2;
            int base = gu < gv ? gu : gv;
            int64_t i = or_site(L, ox + (base & 1), oy + ((base >> 1) & 1), oz + ((base >> 2) & 1));
            if (covered[3 * i + d]) { free(covered); return -3; } /* not a partition */
            covered[3 * i + d] = 1;
            J3[3 * i + d] = templ[cls][e];
        }
    }
    for (int64_t q = 0; q < 3 * N; ++q)
        if (!covered[q]) { free(covered); return -3; }
    free(covered);

    for (int64_t i = 0; i < N; ++i) {
        uint32_t w = philox_word(k0, k1, (uint32_t)i, 0, 0, OR_DOMAIN_GAUGE, 0);
        tau[i] = (gauge && (w >> 31)) ? -1 : +1;
    }
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d)
            J3[3 * i + d] = (int8_t)(J3[3 * i + d] * tau[i] * tau[neighbour(L, i, d, +1)]);
    *e_gs = E;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Schedules and acceptance thresholds (App. D.1, App. D.2).                 */
/* ------------------------------------------------------------------------ */

void or_beta_schedule(int S, double b0, double b1, int geometric, double* beta)
{
    for (int s = 0; s < S; ++s) {
        if (s == S - 1 && S > 1)
            beta[s] = b1;
        else if (S == 1)
            beta[s] = b0;
        else if (geometric)
            beta[s] = b0 * pow(b1 / b0, (double)s / (double)(S - 1));
        else
            beta[s] = b0 + (b1 - b0) * (double)s / (double)(S - 1);
    }
}

void or_pt_ladder(int K, double bmin, double bmax, double* beta)
{
    or_beta_schedule(K, bmin, bmax, 1, beta);
}

/* floor(2^32 exp(-beta * dE)), clamped to 2^32 - 1, for an energy increase dE > 0. */
uint32_t or_metropolis_threshold(double beta, int dE)
{
    double v = floor(ldexp(exp(-(beta * (double)dE)), 32));
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)v;
}

/* Same form for a replica exchange between rungs dbeta apart and energy gap d > 0. */
uint32_t or_exchange_threshold(double dbeta, int64_t d)
{
    double v = floor(ldexp(exp(-(dbeta * (double)d)), 32));
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)v;
}

/* ------------------------------------------------------------------------ */
/* Metropolis dynamics.                                                      */
/* ------------------------------------------------------------------------ */

static void run_key(uint64_t seed, uint32_t instance_id, uint32_t* k0, uint32_t* k1)
{
    *k0 = (uint32_t)seed;
    *k1 = (uint32_t)(seed >> 32) ^ instance_id;
}

/* Initial spin of replica rep at site i: uniform random from the init draw. */
int8_t or_init_spin(uint64_t seed, uint32_t instance_id, int64_t i, int rep)
{
    uint32_t k0, k1;
    run_key(seed, instance_id, &k0, &k1);
    uint32_t w = philox_word(k0, k1, (uint32_t)i, OR_SWEEP_INIT, (uint32_t)(rep / 4),
                             OR_DOMAIN_METROPOLIS, rep % 4);
    return (w >> 31) ? -1 : +1;
}

/* The 32-bit uniform of replica rep's attempt at site i in sweep `sweep` (our RNG
 * contract; the paper fixes none).  Replicas come in groups of 32 (g = rep / 32, bit
 * b = rep % 32).  The leading byte A of the draw has, for j = 0..7, bit j equal to bit b
 * of word j % 4 of the block at counter (i, sweep, 2g + j / 4, METROPOLIS): two blocks
 * give the eight bit planes of the leading bytes of all 32 replicas of a group.  Its low
 * 24 bits are the top 24 bits of word rep % 4 of the block at counter
 * (i, sweep, rep / 4, TAIL).  The blocks are independent and uniform, so u is uniform on
 * [0, 2^32).  (A fast implementation needs the tail only when A equals the threshold's
 * leading byte; the result is the same.) */
static uint32_t metropolis_uniform(uint32_t k0, uint32_t k1, int64_t i, uint32_t sweep, int rep)
{
    int g = rep / 32, b = rep % 32;
    uint32_t a = 0;
    for (int j = 0; j < 8; ++j) {
        uint32_t plane = philox_word(k0, k1, (uint32_t)i, sweep, (uint32_t)(2 * g + j / 4),
                                     OR_DOMAIN_METROPOLIS, j % 4);
        a |= ((plane >> b) & 1u) << j;
    }
    uint32_t tail = philox_word(k0, k1, (uint32_t)i, sweep, (uint32_t)(rep / 4),
                                OR_DOMAIN_TAIL, rep % 4);
    return (a << 24) | (tail >> 8);
}

/* The draws of replicas reps[0..n_reps) at sites i0 .. i0+n_i-1 and sweeps
 * s0 .. s0+n_s-1, out[((s - s0) * n_i + (i - i0)) * n_reps + k] = U of replica reps[k]:
 * exposed so that tests can check the law of the draws (uniform, independent across
 * replicas, sites and sweeps) without going through a run. */
void or_metropolis_uniform_grid(uint64_t seed, uint32_t instance_id, int64_t i0, int n_i, uint32_t s0,
                                int n_s, const int32_t* reps, int n_reps, uint32_t* out)
{
    uint32_t k0, k1;
    run_key(seed, instance_id, &k0, &k1);
    for (int s = 0; s < n_s; ++s)
        for (int i = 0; i < n_i; ++i)
            for (int k = 0; k < n_reps; ++k)
                out[((int64_t)s * n_i + i) * n_reps + k] =
                    metropolis_uniform(k0, k1, i0 + i, s0 + (uint32_t)s, reps[k]);
}

/* One Metropolis attempt at site i of replica rep during sweep `sweep`.
 * x = s_i h_i; flipping changes E by -2x.  Accept when x >= 0, else when the
 * draw u is below the threshold for dE = -2x.  Returns the energy change. */
static int metropolis_attempt(int L, const int8_t* J3, int8_t* s, int64_t i,
                              uint32_t k0, uint32_t k1, uint32_t sweep, int rep,
                              double beta)
{
    int x = s[i] * or_local_field(L, J3, s, i);
    int accept;
    if (x >= 0) {
        accept = 1;
    } else {
        uint32_t u = metropolis_uniform(k0, k1, i, sweep, rep);
        accept = u < or_metropolis_threshold(beta, -2 * x);
    }
    if (!accept) return 0;
    s[i] = (int8_t)(-s[i]);
    return -2 * x;
}

/* One checkerboard sweep: all sites with (x+y+z) even, then all with it odd. */
static int64_t sweep_replica(int L, const int8_t* J3, int8_t* s, uint32_t k0, uint32_t k1,
                             uint32_t sweep, int rep, double beta)
{
    int64_t dE = 0;
    for (int colour = 0; colour < 2; ++colour)
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x)
                    if (((x + y + z) & 1) == colour)
                        dE += metropolis_attempt(L, J3, s, or_site(L, x, y, z), k0, k1,
                                                 sweep, rep, beta);
    return dE;
}

int or_sa_run(int L, const int8_t* J3, uint64_t seed, uint32_t instance_id,
              int S, double b0, double b1, int geometric,
              const int32_t* reps, int nreps, int8_t* spins_out, int64_t* E_out)
{
    if (L < 2 || (L % 2) != 0 || S < 0 || nreps < 0) return -1;
    int64_t N = (int64_t)L * L * L;
    double* beta = (double*)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
    if (!beta) return -2;
    or_beta_schedule(S, b0, b1, geometric, beta);
    uint32_t k0, k1;
    run_key(seed, instance_id, &k0, &k1);
    for (int n = 0; n < nreps; ++n) {
        int rep = reps[n];
        int8_t* s = spins_out + (int64_t)n * N;
        for (int64_t i = 0; i < N; ++i) s[i] = or_init_spin(seed, instance_id, i, rep);
        int64_t E = or_energy(L, J3, s);
        for (int sw = 0; sw < S; ++sw)
            E += sweep_replica(L, J3, s, k0, k1, (uint32_t)sw, rep, beta[sw]);
        E_out[n] = E;
    }
    free(beta);
    return 0;
}

int or_pt_run(int L, const int8_t* J3, uint64_t seed, uint32_t instance_id,
              int K, int S, double bmin, double bmax,
              int8_t* spins_out, int64_t* E_out, int32_t* perm_out,
              int64_t* minE_out, int64_t* accepts_out)
{
    if (L < 2 || (L % 2) != 0 || K < 1 || S < 0) return -1;
    int64_t N = (int64_t)L * L * L;
    double* beta = (double*)malloc(sizeof(double) * (size_t)K);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)K); /* slot -> rung */
    int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)K); /* rung -> slot */
    if (!beta || !perm || !slot) { free(beta); free(perm); free(slot); return -2; }
    or_pt_ladder(K, bmin, bmax, beta);
    uint32_t k0, k1;
    run_key(seed, instance_id, &k0, &k1);

    for (int r = 0; r < K; ++r) {
        int8_t* s = spins_out + (int64_t)r * N;
        for (int64_t i = 0; i < N; ++i) s[i] = or_init_spin(seed, instance_id, i, r);
        E_out[r] = or_energy(L, J3, s);
        perm[r] = r;
        slot[r] = r;
    }
    for (int k = 0; k + 1 < K; ++k) accepts_out[k] = 0;
    int64_t minE = E_out[0];
    for (int r = 1; r < K; ++r) if (E_out[r] < minE) minE = E_out[r];

    for (int sw = 0; sw < S; ++sw) {
        /* Metropolis sweep of every slot at the temperature it currently holds */
        for (int r = 0; r < K; ++r)
            E_out[r] += sweep_replica(L, J3, spins_out + (int64_t)r * N, k0, k1,
                                      (uint32_t)sw, r, beta[perm[r]]);
        /* exchange attempts between rungs k and k+1 for k of the sweep's parity */
        for (int k = sw % 2; k + 1 < K; k += 2) {
            int a = slot[k], b = slot[k + 1];
            int64_t d = E_out[a] - E_out[b];
            uint32_t u = philox_word(k0, k1, (uint32_t)k, (uint32_t)sw, 0,
                                     OR_DOMAIN_EXCHANGE, 0);
            int accept = (d <= 0) || (u < or_exchange_threshold(beta[k + 1] - beta[k], d));
            if (accept) {
                perm[a] = k + 1;
                perm[b] = k;
                slot[k] = b;
                slot[k + 1] = a;
                accepts_out[k] += 1;
            }
        }
        for (int r = 0; r < K; ++r) if (E_out[r] < minE) minE = E_out[r];
    }
    for (int r = 0; r < K; ++r) perm_out[r] = perm[r];
    *minE_out = minE;
    free(beta); free(perm); free(slot);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Linear-time fragment meta-heuristic (Sec. II; App. A, Fig. 5), with      */
/* simulated annealing as the subsystem optimizer (the paper's suggestion;  */
/* its own runs contract tensor-network fragments).                          */
/* ------------------------------------------------------------------------ */

/* Our reading of the bootstrapping.  Spins are fixed ("decimated") in l^3 waves; wave
 * w = a + l*(b + l*c) fixes every spin whose coordinates are congruent to (a, b, c)
 * mod l.  The fragment of spin i is the cube of side l centred on it (offsets -h .. h,
 * h = (l - 1) / 2, periodic); with L a multiple of l the fragments of one wave are
 * disjoint.  Inside the fragment the spins fixed by earlier waves keep their values,
 * the others are annealed: OR_FRAGMENT_READS independent reads, S checkerboard sweeps
 * (colour by x + y + z as for the whole lattice) along the geometric schedule
 * b0 -> b1, Metropolis with only the bonds whose two ends lie in the fragment (bonds
 * leaving it are dropped).  Spin i then takes its value in the read of lowest fragment
 * energy (the first such read).  Draws: read r at fragment site q = dx + l*(dy + l*dz)
 * (d = offset + h) uses word r % 4 of the block at counter (i, sweep, 8*q + r/4,
 * FRAGMENT) as its 32-bit uniform; initial values use sweep 0xFFFFFFFF, bit 31. */
int or_fragment_run(int L, const int8_t* J3, int l, int S, double b0, double b1, uint64_t seed,
                    uint32_t instance_id, int8_t* spins_out, int64_t* E_out)
{
    if (L < 2 || (L % 2) != 0 || l < 1 || (l % 2) == 0 || (L % l) != 0 || l >= L || S < 0) return -1;
    const int64_t N = (int64_t)L * L * L;
    const int h = (l - 1) / 2, V = l * l * l, R = OR_FRAGMENT_READS;
    double* beta = (double*)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
    int8_t* f = (int8_t*)malloc((size_t)V * (size_t)R);   /* f[r * V + q] */
    int8_t* fixed = (int8_t*)malloc((size_t)V);
    int64_t* site = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
    if (!beta || !f || !fixed || !site) {
        free(beta); free(f); free(fixed); free(site);
        return -2;
    }
    or_beta_schedule(S, b0, b1, 1, beta);
    uint32_t k0, k1;
    run_key(seed, instance_id, &k0, &k1);
    for (int64_t i = 0; i < N; ++i) spins_out[i] = 0; /* 0: not fixed yet */

    for (int w = 0; w < l * l * l; ++w) {
        const int a = w % l, b = (w / l) % l, c = w / (l * l);
        for (int cz = c; cz < L; cz += l)
            for (int cy = b; cy < L; cy += l)
                for (int cx = a; cx < L; cx += l) {
                    const int64_t centre = or_site(L, cx, cy, cz);
                    /* the fragment's sites, and which of them earlier waves fixed */
                    for (int q = 0; q < V; ++q) {
                        const int dx = q % l, dy = (q / l) % l, dz = q / (l * l);
                        site[q] = or_site(L, cx + dx - h, cy + dy - h, cz + dz - h);
                        fixed[q] = spins_out[site[q]] != 0;
                    }
                    /* anneal every read */
                    for (int r = 0; r < R; ++r) {
                        int8_t* s = f + (int64_t)r * V;
                        for (int q = 0; q < V; ++q) {
                            if (fixed[q]) {
                                s[q] = spins_out[site[q]];
                            } else {
                                uint32_t u = philox_word(k0, k1, (uint32_t)centre, OR_SWEEP_INIT,
                                                         (uint32_t)(8 * q + r / 4), OR_DOMAIN_FRAGMENT, r % 4);
                                s[q] = (u >> 31) ? -1 : +1;
                            }
                        }
                        for (int sw = 0; sw < S; ++sw)
                            for (int colour = 0; colour < 2; ++colour)
                                for (int q = 0; q < V; ++q) {
                                    const int dx = q % l, dy = (q / l) % l, dz = q / (l * l);
                                    if (fixed[q] || ((cx + dx - h + cy + dy - h + cz + dz - h) & 1) != colour)
                                        continue;
                                    /* local field over the bonds inside the fragment */
                                    int hf = 0;
                                    const int dd[3] = {dx, dy, dz};
                                    for (int d = 0; d < 3; ++d) {
                                        const int step = d == 0 ? 1 : d == 1 ? l : l * l;
                                        if (dd[d] + 1 < l) hf += J3[3 * site[q] + d] * s[q + step];
                                        if (dd[d] > 0) hf += J3[3 * site[q - step] + d] * s[q - step];
                                    }
                                    const int x = s[q] * hf;
                                    int accept = x >= 0;
                                    if (!accept) {
                                        const uint32_t u = philox_word(k0, k1, (uint32_t)centre, (uint32_t)sw,
                                                                       (uint32_t)(8 * q + r / 4),
                                                                       OR_DOMAIN_FRAGMENT, r % 4);
                                        accept = u < or_metropolis_threshold(beta[sw], -2 * x);
                                    }
                                    if (accept) s[q] = (int8_t)(-s[q]);
                                }
                    }
                    /* the read of lowest fragment energy sets the centre spin */
                    int best = 0;
                    int64_t best_e = 0;
                    for (int r = 0; r < R; ++r) {
                        const int8_t* s = f + (int64_t)r * V;
                        int64_t e = 0;
                        for (int q = 0; q < V; ++q) {
                            const int dx = q % l, dy = (q / l) % l, dz = q / (l * l);
                            if (dx + 1 < l) e += (int64_t)J3[3 * site[q] + 0] * s[q] * s[q + 1];
                            if (dy + 1 < l) e += (int64_t)J3[3 * site[q] + 1] * s[q] * s[q + l];
                            if (dz + 1 < l) e += (int64_t)J3[3 * site[q] + 2] * s[q] * s[q + l * l];
                        }
                        if (r == 0 || e < best_e) {
                            best = r;
                            best_e = e;
                        }
                    }
                    spins_out[centre] = f[(int64_t)best * V + (h + l * (h + l * h))];
                }
    }
    *E_out = or_energy(L, J3, spins_out);
    free(beta); free(f); free(fixed); free(site);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact fragment decimation in the zero-temperature (tropical) limit:      */
/* the tensor-network step of App. A with the fragment contracted exactly   */
/* by enumeration.                                                          */
/* ------------------------------------------------------------------------ */

/* Free spins k = 0 .. F-1 with fields h[k] and couplings Jff[k*F + j] (symmetric, zero
 * diagonal); energy E(s) = sum_k h_k s_k + sum_{k<j} Jff[k][j] s_k s_j.  m_plus / m_minus:
 * the lowest energy over the states with s_c = +1 / -1.  Enumerates all 2^F states in
 * Gray-code order (state g = n ^ (n >> 1), bit k set: s_k = -1), each energy obtained
 * from the previous one by the change of the one spin that flips. */
int or_fragment_min_energies(int F, const int* h, const int8_t* Jff, int c, int64_t* m_plus, int64_t* m_minus)
{
    if (F < 1 || F > 30 || c < 0 || c >= F) return -1;
    int8_t s[32];
    int nn[32], nj[32][32];  /* the spins coupled to spin k */
    int8_t nJ[32][32];
    int64_t E = 0;
    for (int k = 0; k < F; ++k) {
        s[k] = 1;
        E += h[k];
        nn[k] = 0;
        for (int j = 0; j < F; ++j)
            if (j != k && Jff[k * F + j] != 0) {
                nj[k][nn[k]] = j;
                nJ[k][nn[k]++] = Jff[k * F + j];
            }
    }
    for (int k = 0; k < F; ++k)
        for (int j = k + 1; j < F; ++j) E += Jff[k * F + j];
    int64_t mp = E, mm = INT64_MAX;
    const uint64_t total = (uint64_t)1 << F;
    for (uint64_t n = 1; n < total; ++n) {
        int k = 0;
        while (!((n >> k) & 1u)) ++k;  /* the bit that changes from g(n-1) to g(n) */
        int64_t field = h[k];
        for (int t = 0; t < nn[k]; ++t) field += (int64_t)nJ[k][t] * s[nj[k][t]];
        E -= 2 * (int64_t)s[k] * field;
        s[k] = (int8_t)(-s[k]);
        if (s[c] > 0) {
            if (E < mp) mp = E;
        } else {
            if (E < mm) mm = E;
        }
    }
    *m_plus = mp;
    *m_minus = mm;
    return 0;
}

/* The waves and cubes of or_fragment_run (readings A13, A14), with the centre spin set
 * by the exact zero-temperature marginal: +1 when the lowest cube energy with s_c = +1
 * is at most the lowest with s_c = -1, else -1.  Cube sides l <= 3 (2^27 states). */
int or_fragment_tropical(int L, const int8_t* J3, int l, int8_t* spins_out, int64_t* E_out)
{
    if (L < 2 || (L % 2) != 0 || l < 1 || l > 3 || (l % 2) == 0 || (L % l) != 0 || l >= L) return -1;
    const int64_t N = (int64_t)L * L * L;
    const int h = (l - 1) / 2, V = l * l * l;
    int64_t site[27];
    int idx[27];
    int hf[27];
    int8_t Jff[27 * 27];
    for (int64_t i = 0; i < N; ++i) spins_out[i] = 0;
    for (int w = 0; w < V; ++w) {
        const int a = w % l, b = (w / l) % l, c = w / (l * l);
        for (int cz = c; cz < L; cz += l)
            for (int cy = b; cy < L; cy += l)
                for (int cx = a; cx < L; cx += l) {
                    int F = 0, cf = -1;
                    for (int q = 0; q < V; ++q) {
                        const int dx = q % l, dy = (q / l) % l, dz = q / (l * l);
                        site[q] = or_site(L, cx + dx - h, cy + dy - h, cz + dz - h);
                        idx[q] = spins_out[site[q]] != 0 ? -1 : F++;
                        if (q == h + l * (h + l * h)) cf = idx[q];
                    }
                    for (int k = 0; k < F; ++k) hf[k] = 0;
                    for (int k = 0; k < F * F; ++k) Jff[k] = 0;
                    /* bonds inside the cube: fixed-free ones become fields */
                    for (int q = 0; q < V; ++q) {
                        const int dd[3] = {q % l, (q / l) % l, q / (l * l)};
                        for (int d = 0; d < 3; ++d) {
                            const int step = d == 0 ? 1 : d == 1 ? l : l * l;
                            if (dd[d] + 1 >= l) continue;
                            const int r = q + step, J = J3[3 * site[q] + d];
                            if (idx[q] >= 0 && idx[r] >= 0) {
                                Jff[idx[q] * F + idx[r]] = (int8_t)(Jff[idx[q] * F + idx[r]] + J);
                                Jff[idx[r] * F + idx[q]] = (int8_t)(Jff[idx[r] * F + idx[q]] + J);
                            } else if (idx[q] >= 0) {
                                hf[idx[q]] += J * spins_out[site[r]];
                            } else if (idx[r] >= 0) {
                                hf[idx[r]] += J * spins_out[site[q]];
                            }
                        }
                    }
                    int64_t mp, mm;
                    if (or_fragment_min_energies(F, hf, Jff, cf, &mp, &mm) != 0) return -3;
                    spins_out[site[h + l * (h + l * h)]] = mp <= mm ? 1 : -1;
                }
    }
    *E_out = or_energy(L, J3, spins_out);
    return 0;
}
