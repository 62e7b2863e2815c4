/*
 * oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Every routine below is the textbook form of one step of the method, written
 * for a reader to check by eye.  No blocking, fusion or reordering.  Built with
 * -O2 -ffp-contract=off (no fused multiply-add), IEEE round-to-nearest.
 *
 * Paper: G. Bussi, "A simple asynchronous replica-exchange implementation",
 * arXiv:0812.1633.  Section "Implementation" defines the exchange protocol
 * (temperatures, not coordinates, are exchanged; Metropolis test with the
 * uniform number of the lower-rank node; temperature and velocities scaled on
 * success).  Section "Example" defines the test system (LJ liquid, cutoff 2.5,
 * Verlet list to 3.0 rebuilt when a displacement exceeds half the skin, time
 * step 0.005, stochastic velocity rescaling, geometric temperature ladder).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Philox */
/* Philox4x64-10, Salmon et al., "Parallel random numbers: as easy as 1, 2, 3"
 * (SC'11): ten rounds of two 64x64->128 multiplications, with the key bumped
 * by the Weyl constants between rounds. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, x0, &hi0, &lo0);
    mulhilo64(M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_uniform4(uint64_t seed, uint64_t stream, uint64_t index, uint64_t tag,
                  uint64_t sub, double u[4]) {
  uint64_t c[4] = {index, tag, sub, 0}, k[2] = {seed, stream}, o[4];
  orc_philox4x64_10(c, k, o);
  for (int i = 0; i < 4; ++i) u[i] = (double)(o[i] >> 11) * 0x1.0p-53;
}

/* Box-Muller transform (1958); 1 - u0 lies in (0, 1] so the logarithm is finite. */
void orc_box_muller(double u0, double u1, double *g0, double *g1) {
  const double two_pi = 6.283185307179586476925286766559;
  double rho = sqrt(-2.0 * log(1.0 - u0));
  *g0 = rho * cos(two_pi * u1);
  *g1 = rho * sin(two_pi * u1);
}

/* Marsaglia & Tsang, "A simple method for generating gamma variables",
 * ACM TOMS 26 (2000): d = a - 1/3, c = 1/sqrt(9d); propose v = (1 + c x)^3
 * with x standard normal; accept with the squeeze u < 1 - 0.0331 x^4 or with
 * log u < x^2/2 + d (1 - v + log v).  Trial t uses Philox block (index, tag, t). */
double orc_gamma_mt(double a, uint64_t seed, uint64_t stream, uint64_t index, uint64_t tag,
                    int *ntrials) {
  double d = a - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  for (uint64_t t = 0;; ++t) {
    double u[4], x, unused;
    orc_uniform4(seed, stream, index, tag, t, u);
    orc_box_muller(u[0], u[1], &x, &unused);
    double w = 1.0 + c * x;
    if (w <= 0.0) continue;
    double v = w * w * w;
    double uu = u[2];
    if (ntrials) *ntrials = (int)t + 1;
    if (uu < 1.0 - 0.0331 * (x * x) * (x * x)) return d * v;
    if (log(uu) < 0.5 * x * x + d * (1.0 - v + log(v))) return d * v;
  }
}

/* Stochastic velocity rescaling, Bussi, Donadio & Parrinello, J. Chem. Phys.
 * 126, 014101 (2007) (the thermostat the Example section cites).  Exact
 * propagation of the kinetic energy over one step:
 *   K' = c K + (1-c) Kbar (R1^2 + S)/Nf + 2 R1 sqrt(c (1-c) Kbar K / Nf),
 * c = exp(-dt/tau), Kbar = Nf T / 2, R1 ~ N(0,1), S ~ chi^2 with Nf-1 degrees.
 * alpha = sqrt(K'/K), negative when R1 + sqrt(c Nf K / ((1-c) Kbar)) < 0. */
double orc_svr_alpha(double K, double Kbar, int Nf, double c, double R1, double S,
                     double *Knew) {
  double nf = (double)Nf;
  double Kp = c * K + (1.0 - c) * Kbar * (R1 * R1 + S) / nf +
              2.0 * R1 * sqrt(c * (1.0 - c) * Kbar * K / nf);
  double alpha = sqrt(Kp / K);
  if (R1 + sqrt(c * nf * K / ((1.0 - c) * Kbar)) < 0.0) alpha = -alpha;
  if (Knew) *Knew = Kp;
  return alpha;
}

/* ------------------------------------------------------------ LJ forces */
/* Lennard-Jones pair in reduced units (Example section: cutoff at 2.5).
 * u(r) = 4 (r^-12 - r^-6) - Uc;  force on i = -fs (x_j - x_i) with
 * fs = -(1/r) du/dr = 48 r^-14 - 24 r^-8. */
double orc_lj_pair(double r2, double Uc, double *fs) {
  double s = 1.0 / r2;
  double s3 = s * s * s;
  *fs = 48.0 * s3 * s3 * s - 24.0 * s3 * s;
  return 4.0 * (s3 * s3 - s3) - Uc;
}

double orc_lj_shift(double rc, int shift) {
  if (!shift) return 0.0;
  double s3 = 1.0 / (rc * rc * rc * rc * rc * rc);
  return 4.0 * (s3 * s3 - s3);
}

static double minimg(double d, double L) { return d - L * nearbyint(d / L); }

double orc_forces_brute(int N, double L, double rc, int shift, const double *x, double *f) {
  double rc2 = rc * rc, Uc = orc_lj_shift(rc, shift), U = 0.0;
  memset(f, 0, sizeof(double) * 3 * (size_t)N);
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = minimg(x[3 * j + k] - x[3 * i + k], L);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 < rc2) {
        double fs;
        U += orc_lj_pair(r2, Uc, &fs);
        for (int k = 0; k < 3; ++k) {
          f[3 * i + k] -= fs * d[k];
          f[3 * j + k] += fs * d[k];
        }
      }
    }
  return U;
}

/* Verlet neighbour list (Allen & Tildesley, cited in the Example section):
 * all pairs closer than rlist = rc + skin, found through a linked-cell list
 * with cells at least rlist wide.  With fewer than 3 cells per side the 27
 * neighbour cells would repeat, so every pair is examined instead. */
int orc_build_list(int N, double L, double rlist, const double *x, int maxpairs, int *pi, int *pj) {
  double rl2 = rlist * rlist;
  int n = 0;
  int nc = (int)floor(L / rlist);
  if (nc < 3) {
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j) {
        double r2 = 0.0;
        for (int k = 0; k < 3; ++k) {
          double d = minimg(x[3 * j + k] - x[3 * i + k], L);
          r2 += d * d;
        }
        if (r2 < rl2) {
          if (n >= maxpairs) return -1;
          pi[n] = i; pj[n] = j; ++n;
        }
      }
    return n;
  }
  int ncell = nc * nc * nc;
  int *head = (int *)malloc(sizeof(int) * (size_t)ncell);
  int *next = (int *)malloc(sizeof(int) * (size_t)N);
  for (int c = 0; c < ncell; ++c) head[c] = -1;
  for (int i = N - 1; i >= 0; --i) {
    int c3[3];
    for (int k = 0; k < 3; ++k) {
      int ck = (int)floor(x[3 * i + k] / L * nc);
      if (ck < 0) ck = 0;
      if (ck >= nc) ck = nc - 1;
      c3[k] = ck;
    }
    int c = (c3[0] * nc + c3[1]) * nc + c3[2];
    next[i] = head[c];
    head[c] = i;
  }
  for (int cx = 0; cx < nc; ++cx)
    for (int cy = 0; cy < nc; ++cy)
      for (int cz = 0; cz < nc; ++cz) {
        int c = (cx * nc + cy) * nc + cz;
        for (int i = head[c]; i >= 0; i = next[i])
          for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dz = -1; dz <= 1; ++dz) {
                int ox = (cx + dx + nc) % nc, oy = (cy + dy + nc) % nc, oz = (cz + dz + nc) % nc;
                int c2 = (ox * nc + oy) * nc + oz;
                for (int j = head[c2]; j >= 0; j = next[j]) {
                  if (j <= i) continue;
                  double r2 = 0.0;
                  for (int k = 0; k < 3; ++k) {
                    double d = minimg(x[3 * j + k] - x[3 * i + k], L);
                    r2 += d * d;
                  }
                  if (r2 < rl2) {
                    if (n >= maxpairs) { free(head); free(next); return -1; }
                    pi[n] = i; pj[n] = j; ++n;
                  }
                }
              }
      }
  free(head);
  free(next);
  return n;
}

double orc_forces_list(int N, double L, double rc, int shift, const double *x, int npairs,
                       const int *pi, const int *pj, double *f) {
  double rc2 = rc * rc, Uc = orc_lj_shift(rc, shift), U = 0.0;
  memset(f, 0, sizeof(double) * 3 * (size_t)N);
  for (int p = 0; p < npairs; ++p) {
    int i = pi[p], j = pj[p];
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = minimg(x[3 * j + k] - x[3 * i + k], L);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 < rc2) {
      double fs;
      U += orc_lj_pair(r2, Uc, &fs);
      for (int k = 0; k < 3; ++k) {
        f[3 * i + k] -= fs * d[k];
        f[3 * j + k] += fs * d[k];
      }
    }
  }
  return U;
}

/* ------------------------------------------------------------ set-up */
/* Face-centred cubic start: N = 4 k^3 atoms, k cells of side a = L/k per
 * side, four-atom basis; atom 4*((ix*k + iy)*k + iz) + b.  Offset by a/4 so
 * that no atom sits on the box face. */
void orc_fcc_lattice(int N, double L, double *x) {
  int k = 1;
  while (4 * k * k * k < N) ++k;
  double a = L / k;
  static const double basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
  int n = 0;
  for (int ix = 0; ix < k; ++ix)
    for (int iy = 0; iy < k; ++iy)
      for (int iz = 0; iz < k; ++iz)
        for (int b = 0; b < 4; ++b) {
          if (n >= N) return;
          x[3 * n + 0] = (ix + basis[b][0] + 0.25) * a;
          x[3 * n + 1] = (iy + basis[b][1] + 0.25) * a;
          x[3 * n + 2] = (iz + basis[b][2] + 0.25) * a;
          ++n;
        }
}

double orc_kinetic(int N, const double *v) {
  double K = 0.0;
  for (int i = 0; i < 3 * N; ++i) K += v[i] * v[i];
  return 0.5 * K;
}

/* Maxwell-Boltzmann velocities at T: atom i takes Philox block (i, VEL):
 * Box-Muller on (u0, u1) gives vx, vy; on (u2, u3) gives vz (cosine branch).
 * The centre-of-mass velocity is removed and the result rescaled so that
 * 2K/Nf equals T exactly, Nf = 3N - 3. */
void orc_init_velocities(int N, double T, uint64_t seed, uint64_t stream, double *v) {
  double mean[3] = {0, 0, 0};
  for (int i = 0; i < N; ++i) {
    double u[4], g0, g1, g2, g3;
    orc_uniform4(seed, stream, (uint64_t)i, ORC_TAG_VEL, 0, u);
    orc_box_muller(u[0], u[1], &g0, &g1);
    orc_box_muller(u[2], u[3], &g2, &g3);
    v[3 * i + 0] = g0;
    v[3 * i + 1] = g1;
    v[3 * i + 2] = g2;
  }
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < 3; ++k) mean[k] += v[3 * i + k];
  for (int k = 0; k < 3; ++k) mean[k] /= N;
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < 3; ++k) v[3 * i + k] -= mean[k];
  double K = orc_kinetic(N, v);
  int Nf = 3 * N - 3;
  double Tinst = 2.0 * K / Nf;
  double scale = sqrt(T / Tinst);
  for (int i = 0; i < 3 * N; ++i) v[i] *= scale;
}

static int rebuild(orc_rep *r) {
  int n = orc_build_list(r->N, r->L, r->rc + r->skin, r->x, r->maxpairs, r->pi, r->pj);
  if (n < 0) { r->status = -1; return -1; }
  r->npairs = n;
  memcpy(r->xref, r->x, sizeof(double) * 3 * (size_t)r->N);
  r->list_valid = 1;
  r->nrebuild += 1;
  return 0;
}

/* Forces and potential energy of the replica's Hamiltonian lam U_LJ. */
static double replica_forces(orc_rep *r) {
  double U = orc_forces_list(r->N, r->L, r->rc, r->shift, r->x, r->npairs, r->pi, r->pj, r->f);
  for (int i = 0; i < 3 * r->N; ++i) r->f[i] *= r->lam;
  return r->lam * U;
}

int orc_refresh(orc_rep *r) {
  if (rebuild(r)) return -1;
  r->U = replica_forces(r);
  r->K = orc_kinetic(r->N, r->v);
  return 0;
}

int orc_init_replica(orc_rep *r) {
  int k = 1;
  while (4 * k * k * k < r->N) ++k;
  if (4 * k * k * k != r->N) return -1;
  orc_fcc_lattice(r->N, r->L, r->x);
  orc_init_velocities(r->N, r->T, r->seed, r->stream, r->v);
  r->step = 0;
  r->nrebuild = 0;
  r->econs = 0.0;
  r->status = 0;
  return orc_refresh(r);
}

/* ------------------------------------------------------------ MD step */
/* One velocity-Verlet step (time step 0.005 in the Example section) with the
 * list maintained as the Example section states: after the drift the list is
 * rebuilt when some atom has moved (minimum image) more than half the skin
 * since the last rebuild.  The thermostat acts once per step, after the
 * second half-kick, with the draws of step index r->step. */
static void md_step(orc_rep *r) {
  int N = r->N;
  double hdt = 0.5 * r->dt;
  for (int i = 0; i < 3 * N; ++i) r->v[i] += hdt * r->f[i];
  for (int i = 0; i < 3 * N; ++i) {
    r->x[i] += r->dt * r->v[i];
    r->x[i] -= r->L * floor(r->x[i] / r->L);
  }
  double half = 0.5 * r->skin, maxd2 = 0.0;
  for (int i = 0; i < N; ++i) {
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      double d = minimg(r->x[3 * i + k] - r->xref[3 * i + k], r->L);
      d2 += d * d;
    }
    if (d2 > maxd2) maxd2 = d2;
  }
  if (!r->list_valid || maxd2 > half * half) {
    if (rebuild(r)) return;
  }
  r->U = replica_forces(r);
  for (int i = 0; i < 3 * N; ++i) r->v[i] += hdt * r->f[i];
  double K = orc_kinetic(N, r->v);
  if (r->tau > 0.0) {
    int Nf = 3 * N - 3;
    double c = exp(-r->dt / r->tau);
    double Kbar = 0.5 * Nf * r->T;
    double u[4], R1, unused;
    orc_uniform4(r->seed, r->stream, (uint64_t)r->step, ORC_TAG_SVR_R1, 0, u);
    orc_box_muller(u[0], u[1], &R1, &unused);
    double S = 2.0 * orc_gamma_mt(0.5 * (Nf - 1), r->seed, r->stream, (uint64_t)r->step,
                                  ORC_TAG_SVR_GAM, NULL);
    double Kp;
    double alpha = orc_svr_alpha(K, Kbar, Nf, c, R1, S, &Kp);
    for (int i = 0; i < 3 * N; ++i) r->v[i] *= alpha;
    r->econs += K - Kp;
    r->K = Kp;
  } else {
    r->K = K;
  }
  r->step += 1;
}

int orc_md_steps(orc_rep *r, int nsteps) {
  for (int s = 0; s < nsteps; ++s) {
    md_step(r);
    if (r->status) return r->status;
  }
  return 0;
}

/* Asynchronous stride: replica k performs steps[k] steps before the next
 * attempt (Example section: replicas need not do equal numbers of steps). */
int orc_advance(orc_rep **reps, int R, const int32_t *steps, int nthreads) {
  int err = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
  for (int k = 0; k < R; ++k) err |= orc_md_steps(reps[k], steps[k]) ? 1 : 0;
  (void)nthreads;
  return err ? -1 : 0;
}

/* ------------------------------------------------------------ exchange */
typedef struct { double T; int id; } tk;
static int cmp_tk(const void *a, const void *b) {
  const tk *x = (const tk *)a, *y = (const tk *)b;
  if (x->T < y->T) return -1;
  if (x->T > y->T) return 1;
  return x->id - y->id;
}

/* Exchange attempt as the Implementation section describes it: the
 * temperatures are collected and sorted; neighbours in sorted order form the
 * pairs (the first pair starts at position p, p alternating with the attempt
 * number or drawn at random); each pair takes the uniform number of its
 * lower-rank (lower id) member and applies the Metropolis rule of
 * Sugita & Okamoto, accept iff D >= 0 or r < exp(D) with
 * D = (1/T_a - 1/T_b)(U_a - U_b); on success the temperatures are swapped and
 * the velocities scaled by sqrt(T_new / T_old). */
int orc_exchange(int R, double *T, const double *U, uint64_t seed, int64_t attempt,
                 int parity_mode, int32_t *partner, uint8_t *accepted, double *vscale) {
  tk *order = (tk *)malloc(sizeof(tk) * (size_t)R);
  for (int i = 0; i < R; ++i) { order[i].T = T[i]; order[i].id = i; }
  qsort(order, (size_t)R, sizeof(tk), cmp_tk);
  int p;
  if (parity_mode == 0) {
    p = (int)(attempt & 1);
  } else {
    double u[4];
    orc_uniform4(seed, ~0ULL, (uint64_t)attempt, ORC_TAG_PARITY, 0, u);
    p = u[0] < 0.5 ? 0 : 1;
  }
  for (int i = 0; i < R; ++i) { partner[i] = -1; accepted[i] = 0; vscale[i] = 1.0; }
  int nacc = 0;
  for (int k = p; k + 1 < R; k += 2) {
    int a = order[k].id, b = order[k + 1].id;
    double Ta = T[a], Tb = T[b];
    double delta = (1.0 / Ta - 1.0 / Tb) * (U[a] - U[b]);
    int lo = a < b ? a : b;
    double u[4];
    orc_uniform4(seed, (uint64_t)lo, (uint64_t)attempt, ORC_TAG_EXCH, 0, u);
    int ok = (delta >= 0.0) || (u[0] < exp(delta));
    partner[a] = b;
    partner[b] = a;
    if (ok) {
      accepted[a] = accepted[b] = 1;
      vscale[a] = sqrt(Tb / Ta);
      vscale[b] = sqrt(Ta / Tb);
      T[a] = Tb;
      T[b] = Ta;
      ++nacc;
    }
  }
  free(order);
  return nacc;
}

void orc_apply_exchange(orc_rep **reps, int R, const double *Tnew, const double *vscale) {
  for (int k = 0; k < R; ++k) {
    orc_rep *r = reps[k];
    double s = vscale[k];
    if (s != 1.0) {
      for (int i = 0; i < 3 * r->N; ++i) r->v[i] *= s;
      double Knew = r->K * (s * s);
      r->econs += r->K - Knew;
      r->K = Knew;
    }
    r->T = Tnew[k];
  }
}

/* ------------------------------------------------ generalised exchange */
/* The Implementation section's exchange with two extensions it mentions
 * (non-nearest-neighbour pairs) or allows (parameters other than T): replica
 * k samples exp(-(K + lam_k U_LJ)/T_k); swapping the parameter sets of a and b
 * is accepted with min(1, exp(D)), D = (lam_a/T_a - lam_b/T_b)(u_a - u_b),
 * u = U/lam the unscaled LJ energy (the kinetic part is handled by the
 * velocity rescaling, as for temperatures). */
typedef struct { double key; int id; } kk;
static int cmp_kk(const void *a, const void *b) {
  const kk *x = (const kk *)a, *y = (const kk *)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return x->id - y->id;
}

int orc_exchange_h(int R, double *T, double *lam, const double *U, uint64_t seed,
                   int64_t attempt, int parity_mode, int distance, int32_t *partner,
                   uint8_t *accepted, double *vscale, double *uscale) {
  const int d = distance < 1 ? 1 : distance;
  kk *order = (kk *)malloc(sizeof(kk) * (size_t)R);
  for (int i = 0; i < R; ++i) {
    order[i].key = T[i] / (lam ? lam[i] : 1.0);
    order[i].id = i;
  }
  qsort(order, (size_t)R, sizeof(kk), cmp_kk);
  int p;
  if (parity_mode == 0) {
    p = (int)(attempt & 1);
  } else {
    double u[4];
    orc_uniform4(seed, ~0ULL, (uint64_t)attempt, ORC_TAG_PARITY, 0, u);
    p = u[0] < 0.5 ? 0 : 1;
  }
  for (int i = 0; i < R; ++i) {
    partner[i] = -1;
    accepted[i] = 0;
    vscale[i] = 1.0;
    uscale[i] = 1.0;
  }
  const int o = p * d;
  int nacc = 0;
  for (int q = o; q + d < R; ++q) {
    if ((q - o) % (2 * d) >= d) continue; /* q is the upper member of a pair */
    int a = order[q].id, b = order[q + d].id;
    double Ta = T[a], Tb = T[b];
    double la = lam ? lam[a] : 1.0, lb = lam ? lam[b] : 1.0;
    double delta = (la / Ta - lb / Tb) * (U[a] / la - U[b] / lb);
    int lo = a < b ? a : b;
    double u[4];
    orc_uniform4(seed, (uint64_t)lo, (uint64_t)attempt, ORC_TAG_EXCH, 0, u);
    int ok = (delta >= 0.0) || (u[0] < exp(delta));
    partner[a] = b;
    partner[b] = a;
    if (ok) {
      accepted[a] = accepted[b] = 1;
      vscale[a] = sqrt(Tb / Ta);
      vscale[b] = sqrt(Ta / Tb);
      uscale[a] = lb / la;
      uscale[b] = la / lb;
      T[a] = Tb;
      T[b] = Ta;
      if (lam) {
        lam[a] = lb;
        lam[b] = la;
      }
      ++nacc;
    }
  }
  free(order);
  return nacc;
}

void orc_apply_exchange_h(orc_rep **reps, int R, const double *Tnew, const double *lamnew,
                          const double *vscale, const double *uscale) {
  for (int k = 0; k < R; ++k) {
    orc_rep *r = reps[k];
    double s = vscale[k];
    if (s != 1.0) {
      for (int i = 0; i < 3 * r->N; ++i) r->v[i] *= s;
      double Knew = r->K * (s * s);
      r->econs += r->K - Knew;
      r->K = Knew;
    }
    double us = uscale[k];
    if (us != 1.0) {
      for (int i = 0; i < 3 * r->N; ++i) r->f[i] *= us;
      double Unew = r->U * us;
      r->econs += r->U - Unew;
      r->U = Unew;
    }
    r->T = Tnew[k];
    r->lam = lamnew[k];
  }
}
