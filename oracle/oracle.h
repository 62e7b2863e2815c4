/*
 * oracle.h -- plain, slow FP64 CPU oracle for asynchronous replica-exchange
 * Lennard-Jones molecular dynamics (Bussi, "A simple asynchronous
 * replica-exchange implementation", arXiv:0812.1633).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: it is used by tests/, by the smoke check and by the CPU
 * baseline leg of bench.py.  It shares no code with the CUDA library.
 *
 * Conventions (LJ reduced units, sigma = epsilon = m = k_B = 1; Example section):
 *   positions, velocities, forces: AoS doubles, atom i at [3i, 3i+1, 3i+2].
 *   box: cubic, side L, periodic, positions wrapped into [0, L).
 *
 * Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), used as a
 * counter-based generator.  key = (seed, stream), counter = (index, tag, sub, 0).
 * The CUDA library implements the same generator from the same published
 * definition; the tags below fix which draw feeds which step of the method.
 */
#ifndef RE_ORACLE_H
#define RE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_TAG_VEL = 1,    /* initial Maxwell-Boltzmann velocities; index = atom */
  ORC_TAG_SVR_R1 = 2, /* thermostat Gaussian R1; index = step */
  ORC_TAG_SVR_GAM = 3,/* thermostat chi-square (Gamma trials); index = step, sub = trial */
  ORC_TAG_EXCH = 4,   /* Metropolis uniform of a replica; index = attempt */
  ORC_TAG_PARITY = 5  /* random pairing offset; stream = ~0, index = attempt */
};

/* One replica of the LJ liquid.  Arrays are owned by the caller. */
typedef struct orc_rep {
  int N;            /* atoms */
  int shift;        /* 1: energy shifted to zero at rc; 0: plain truncation */
  double L, rc, skin, dt, tau, T; /* box, cutoff, list skin, time step, SVR tau (<=0: NVE), target T */
  uint64_t seed, stream;          /* Philox key of this replica (stream = replica id) */
  int64_t step;                   /* MD steps done (counter of the thermostat draws) */
  int64_t nrebuild;               /* neighbour-list rebuilds done */
  double U, K, econs;             /* potential, kinetic, thermostat work (H~ = U + K + econs) */
  double *x, *v, *f, *xref;       /* 3N each */
  int *pi, *pj;                   /* half Verlet list (i < j pairs), capacity maxpairs */
  int npairs, maxpairs;
  int list_valid;
  int status;                     /* 0 ok, -1 list overflow */
  double lam;                     /* potential scale: the replica's Hamiltonian is K + lam U_LJ */
} orc_rep;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* Four uniforms in [0, 1) with 53-bit resolution from one Philox block. */
void orc_uniform4(uint64_t seed, uint64_t stream, uint64_t index, uint64_t tag,
                  uint64_t sub, double u[4]);
/* Box-Muller pair from two uniforms: g0 = rho cos(2 pi u1), g1 = rho sin(2 pi u1). */
void orc_box_muller(double u0, double u1, double *g0, double *g1);
/* Gamma(a, 1), a >= 1, by Marsaglia & Tsang (2000); trials drawn from the stream. */
double orc_gamma_mt(double a, uint64_t seed, uint64_t stream, uint64_t index, uint64_t tag,
                    int *ntrials);
/* Stochastic velocity rescaling (Bussi, Donadio, Parrinello 2007): new kinetic
 * energy and the velocity factor alpha for one step of length dt. */
double orc_svr_alpha(double K, double Kbar, int Nf, double c, double R1, double S,
                     double *Knew);

/* LJ pair: for squared distance r2 < rc2 returns the pair energy (shifted by
 * Uc) and sets *fs so that the force on i is -fs * (x_j - x_i). */
double orc_lj_pair(double r2, double Uc, double *fs);
double orc_lj_shift(double rc, int shift);
/* Brute-force O(N^2) minimum-image forces; returns U.  The definition. */
double orc_forces_brute(int N, double L, double rc, int shift, const double *x, double *f);
/* Half Verlet list with cells (cells >= rlist wide; all pairs below 3 cells/side).
 * Returns the number of pairs, or -1 if more than maxpairs. */
int orc_build_list(int N, double L, double rlist, const double *x, int maxpairs, int *pi, int *pj);
double orc_forces_list(int N, double L, double rc, int shift, const double *x, int npairs,
                       const int *pi, const int *pj, double *f);

void orc_fcc_lattice(int N, double L, double *x);
void orc_init_velocities(int N, double T, uint64_t seed, uint64_t stream, double *v);
double orc_kinetic(int N, const double *v);

/* Lattice + velocities + list + forces. Returns 0 or -1 (bad N or list overflow). */
int orc_init_replica(orc_rep *r);
/* Rebuild list, forces, U and K from the current x, v (after an external state change). */
int orc_refresh(orc_rep *r);
/* nsteps of velocity Verlet + SVR with neighbour-list maintenance. */
int orc_md_steps(orc_rep *r, int nsteps);
/* Every replica advances its own number of steps (threads over replicas). */
int orc_advance(orc_rep **reps, int R, const int32_t *steps, int nthreads);

/* One exchange attempt over an ensemble of R replicas indexed by replica id.
 * T (in/out): current temperature of each replica; U: potential energies.
 * Outputs per replica: partner (-1 if unpaired), accepted flag, velocity
 * factor sqrt(T_new / T_old) (1 when not exchanged).  Returns accepted pairs. */
int orc_exchange(int R, double *T, const double *U, uint64_t seed, int64_t attempt,
                 int parity_mode, int32_t *partner, uint8_t *accepted, double *vscale);
/* Apply an exchange to replica states: scale v, update T, K and econs. */
void orc_apply_exchange(orc_rep **reps, int R, const double *Tnew, const double *vscale);

/* Generalised (Hamiltonian) exchange with pairs at ladder distance
 * `distance`: replica k has parameters (T_k, lam_k) and potential energy
 * U_k = lam_k U_LJ(x_k).  Ladder order = ascending T/lam; pairs (q, q + d)
 * for q - o in [0, d) mod 2d, o = p d with p the parity offset;
 * D = (lam_a/T_a - lam_b/T_b)(U_a/lam_a - U_b/lam_b); on acceptance the pair
 * swaps (T, lam), vscale = sqrt(T_new/T_old), uscale = lam_new/lam_old.
 * lam NULL: all 1 (then identical to orc_exchange when distance == 1). */
int orc_exchange_h(int R, double *T, double *lam, const double *U, uint64_t seed,
                   int64_t attempt, int parity_mode, int distance, int32_t *partner,
                   uint8_t *accepted, double *vscale, double *uscale);
/* Applies an exchange to the replicas: v *= vscale (K and econs follow),
 * f *= uscale and U *= uscale (econs absorbs the change of U), new T, lam. */
void orc_apply_exchange_h(orc_rep **reps, int R, const double *Tnew, const double *lamnew,
                          const double *vscale, const double *uscale);

#ifdef __cplusplus
}
#endif
#endif
