// re_internal.h -- data layout shared by the host side (re_capi.cu) and the
// kernels (re_kernels.cu) of the replica-exchange library.  Not installed.
//
// Device memory of a context (all replicas of all ensembles, SoA):
//   qx,qy,qz  uint64 [atoms]   positions, fixed point x/L * 2^64 (wrapping)
//   vx,vy,vz  double [atoms]   velocities
//   fx,fy,fz  double [atoms]   forces at the current positions
//   rx,ry,rz  uint32 [atoms]   top 32 bits of the positions at the last rebuild
//   ncnt      int32  [8 * atoms] neighbour count of each (atom, lane) sub-list
//   nbr       uint16 [sum over replicas of cap * N]  neighbour indices (local
//             atom indices).  With P threads per atom each atom's list is split
//             into P sub-lists of cap/P entries; entry k of sub-list (i, q) at
//             ((k / 4) * N * P + i * P + q) * 4 + k % 4 (P = 1 on the plain path)
//   per replica: T, U, K, econs, vscale (pending velocity factor), step,
//             nreb, status, valid
//   per ensemble: attempt counter; per sorted pair position: attempts, accepts
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace re {

enum StatusBits : int {
  kStOverflow = 1,
  kStNumeric = 2,
  kStRngCap = 4,
  kStStop = 8,     // not an error: free-running stop request seen
  kStTimeout = 16, // free-running exchange: this replica's own bounded wait ran out (or it
                   // was told to stop answering: host-side fault injection)
  kStXchg = 32,    // not an error: an exchange pattern is waiting at this step boundary
  kStAborted = 64  // free-running exchange: left before the last pattern because another
                   // replica of the ensemble gave up (raised the abort flag)
};

// Per-ensemble step constants, formed once on the host (FP64 transcendentals
// and divisions run at 1/64 of the FP32 rate on the GPU).  The fields that
// depend on the thermostat's target T (kbar, af, bf, gf) are filled per
// replica by set_thermo_target.
struct StepConst {
  double lam32, lam64, inv_l, dtq, hdt, inv_hdt, uc, rc2, c_th, kbar;
  double kbar1, af1, bf1, gf1;  // kbar = kbar1 T, af = af1 T, bf = bf1 sqrt(T), gf = gf1 / sqrt(T)
  double lamv;                  // the replica's potential scale (set_potential_scale)
  double rc2x;                  // rc^2 in units (L / 2^42)^2 (exact cutoff test, mixed path)
  float hlf;                    // FP32 half-kick factor per force unit, times lamv
  float rc2u, rl2u, half2u, inv_lam2;
  float rc2u_lo, rc2u_hi;       // rc2u (1 -+ 2e-6): the band decided on 42-bit separations
  // thermostat constants of the mixed path (used in FP32): c - 1,
  // (1 - c) Kbar / Nf, 2 sqrt(c (1 - c) Kbar / Nf), sqrt(c Nf / ((1 - c) Kbar))
  float cm1f, af, bf, gf;
  int nf, pad_;
};

struct EnsHdr {
  int N, R, rep_off, pair_off;  // replicas [rep_off, rep_off + R); stats at pair_off
  int nc, m;                    // list cells per side (0: all pairs), reach in cells
  int cap;                      // neighbour entries per atom: max over P of P * capsub[P]
  int capsub[4];                // sub-list capacity (multiple of 4) for P = 1, 2, 4, 8
  int shift, parity_mode, xdist;  // xdist: exchange pairs at ladder distance xdist (>= 1)
  double L, rc, rlist, skin, dt, tau;
  uint64_t seed;
};

// An ensemble: its parameters and the step constants derived from them (the
// batched kernel keeps the two apart in shared memory, the constants per
// replica).
struct EnsDev : EnsHdr {
  StepConst kc;  // filled by finish_ens (host) once the fields above are set
};

// The constants of StepConst that depend on the replica's potential scale
// (its Hamiltonian is K + lam U_LJ: forces and U scale by lam).
__host__ __device__ inline void set_potential_scale(StepConst& k, double lam) {
  k.lamv = lam;
  k.hlf = (float)(k.hdt * k.lam32 * lam);
}

// The constants of StepConst that depend on the target temperature T.
__host__ __device__ inline void set_thermo_target(StepConst& k, double T) {
  k.kbar = k.kbar1 * T;
  k.af = (float)(k.af1 * T);
  const float ts = sqrtf((float)T);
  k.bf = (float)k.bf1 * ts;
  k.gf = (float)k.gf1 / ts;
}

struct RepDev {
  int ens, id, atom_off;
  int stream;  // Philox stream of the replica's own draws (velocities, thermostat): id_offset + id
  int64_t nbr_off;
};

struct StateDev {
  uint64_t *qx, *qy, *qz;
  double *vx, *vy, *vz, *fx, *fy, *fz;
  uint32_t *rx, *ry, *rz;
  int32_t* ncnt;
  uint16_t* nbr;
  double *T, *U, *K, *econs, *vscale;
  double *lam, *fscale;  // per replica: potential scale; pending force factor (null: 1)
  int64_t *step, *nreb;
  int32_t *status, *valid;
  int64_t* attempt;                  // per ensemble
  int64_t *pair_att, *pair_acc;      // per ensemble pair position
  double* red;                       // plain path: per replica reduction scratch
  uint32_t* dmax;                    // plain path: per replica max displacement^2 (float bits)
  int32_t* stop;                     // per ensemble: free-running mode, the master's "done" flag
  int32_t* perm;                     // per atom: original index (within its replica) of the
                                     // atom held in this slot (atoms are renumbered in space order)
  int32_t* order;                    // per atom: spatial re-sort order (scratch)
  uint64_t* sbuf;                    // 7 words per atom: re-sort staging (scratch)
  // 1: the v and f arrays hold the mixed kernel's own words (v: 64-bit fixed
  // point in units of 2^-48; f: the FP32 half-kick increment dt/2 F in the
  // low 4 bytes), so a launch loads and stores its state without FP64
  // conversions; 0: doubles (FP64 and plain paths)
  int vfix;
};

// Free-running replica exchange inside one persistent launch (Implementation
// section).  Per ensemble e: `issue` counts the exchange patterns issued in
// this launch, `abort_` is raised by a replica that leaves early.  Per replica
// r (global index): the current pattern's partner (ensemble member id, -1 for
// none) and position in the sorted-temperature order, the number of patterns
// it has processed (`done`), and its published (T, U) with the pattern number
// + 1 they belong to (`flag`).  The log holds, per pattern k < log_cap and
// replica, the step count at which the replica took part, its temperature
// afterwards, its partner and the decision.  Zeroed by the host before every
// launch (except the log).
struct FreeDev {
  int nx;            // > 0: free-running mode; the master's own steps between patterns
  int n_att;         // patterns per ensemble in this launch
  int log_cap;       // patterns logged (0: none)
  int rtot;          // replicas in the launch (log row stride)
  uint64_t wait_ns;  // limit of every bounded wait (nanoseconds of the global timer)
  int stall_rep;     // host-side fault injection: this replica (global index; -1: none)
  int stall_from;    // stops answering at its part in pattern stall_from of the launch
  int32_t* issue;    // [E]
  int32_t* abort_;   // [E]
  int32_t* partner;  // [Rtot]
  int32_t* pos;      // [Rtot]
  int32_t* done;     // [Rtot]
  int32_t* flag;     // [Rtot]
  int32_t* order;    // [Rtot] scratch of the master (sorted order, at the ensemble's rep_off)
  double* slot;      // [3 Rtot] published (T, U, lam)
  double* key;       // [Rtot] scratch of the master (ladder keys T/lam)
  int64_t* log_step;    // [log_cap x rtot]
  double* log_T;        // [log_cap x rtot]
  int32_t* log_partner; // [log_cap x rtot]
  int32_t* log_acc;     // [log_cap x rtot]
};

struct LaunchCfg {
  int cluster, threads, cell_div, atom_threads;  // CTAs per replica, threads per CTA,
                                                 // list cells per list radius, threads per atom
  int lists_smem;  // 1: each CTA's sub-lists in shared memory during a launch (when they fit)
  // Budget mode of a one-ensemble context: the wide_n hottest replicas (by
  // current temperature) run in a second, concurrent launch with clusters of
  // wide_cluster CTAs (wide_threads threads each, wide_atom_threads per atom);
  // wide_n = 0: one launch for all.  Hot replicas move faster and rebuild their lists
  // more often (the load imbalance of the paper's Introduction): more SMs
  // for them shorten the slowest replica, and the extra CTAs fill SMs that a
  // uniform launch leaves idle.
  int wide_n, wide_cluster, wide_threads, wide_atom_threads;
};

// Host helpers (re_capi.cu): list cells of an ensemble and neighbour capacities.
void choose_cells(double L, double rlist, int N, int want_m, int* nc_out, int* m_out);
void set_capacity(EnsDev& e, int user_cap);
// e.kc from L, rc, rlist, skin, dt, tau, shift and N (target T = 1)
void finish_ens(EnsDev& e);

// Host-side launchers (re_kernels.cu).  All return the launch status.
cudaError_t launch_init_lattice(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, int max_threads, cudaStream_t st);
size_t batched_smem_bytes(int max_n, int max_ncell, int threads, bool fp64, size_t list_elems);
// Shared memory the batched kernel declares statically (replica constants and
// hand-over words), reserved on top of batched_smem_bytes; launches check it.
constexpr size_t kBatchedStaticSmem = 512;
// list_elems > 0: each CTA keeps its atoms' neighbour sub-lists (list_elems
// uint16 entries) in shared memory during the launch
// async_nx > 0: master-stop mode (budgets ignored): in every ensemble the
// master replica (attempt mod R) does async_nx steps and then raises the
// ensemble's stop flag; the others stop after the step in which they see it.
// fr && fr->nx > 0: free-running mode with exchanges inside the launch (all
// replicas must be resident at once; see FreeDev).  Both modes need
// list_elems == 0 (lists in global memory).
cudaError_t launch_batched(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                           const int* d_work, int n_work, const int32_t* d_budget, bool fp64,
                           const LaunchCfg& cfg, int max_n, int max_ncell, size_t list_elems,
                           int async_nx, cudaStream_t st, const FreeDev* fr = nullptr);
// Clusters of the batched kernel that can be resident at once with this
// launch shape (0 when the query fails).
int batched_max_active_clusters(bool fp64, const LaunchCfg& cfg, int max_n, int max_ncell);

// One instantiation of the batched kernel (precision, threads per atom, list
// placement, mode) and its launch; defined in re_batched.cuh, instantiated in
// the re_batched_*.cu translation units.
#define BATCHED_LAUNCH_ARGS                                                               \
  const StateDev &s, const EnsDev *d_ens, const RepDev *d_rep, const int *d_work,        \
      int n_work, const int32_t *d_budget, const LaunchCfg &cfg, int max_n, int max_ncell, \
      size_t list_elems, int async_nx, cudaStream_t st, const FreeDev *fr
// MAXT: 1024, or kNarrowThreads for launches of at most that many threads
// per CTA (a larger register budget per thread).
constexpr int kNarrowThreads = 896;
template <bool FP64, int P, bool LSM, int MODE, int MAXT>
cudaError_t launch_batched_t(BATCHED_LAUNCH_ARGS);
template <bool FP64, int P, bool LSM, int MAXT>
int max_active_clusters_t(const LaunchCfg& cfg, int max_n, int max_ncell, size_t list_elems);
// Work lists of a split launch: replicas ranked by decreasing temperature T
// (ties by index); the wide_n hottest go to work[R - wide_n .. R), in rank
// order, the others to work[0 .. R - wide_n).  One ensemble of R replicas.
cudaError_t launch_split_work(const double* T, int R, int wide_n, int* work, cudaStream_t st);
// Work list of a budget-mode launch with uneven budgets, longest job first:
// the replicas of [r0, r0 + n) by decreasing budget x atoms, then index,
// written to work[r0 .. r0 + n) (n <= 4096).  A grid of many waves then ends
// with short jobs instead of long ones started late.
cudaError_t launch_order_work(const int32_t* budget, const RepDev* d_rep, const EnsDev* d_ens,
                              int r0, int n, int* work, cudaStream_t st);
// applies externally decided exchange results, d_in = [T_new | lam_new |
// vscale | uscale] (R values each, device)
cudaError_t launch_apply_exchange(const StateDev& s, const double* d_in, int R, cudaStream_t st);
// attempt[e] += n for every ensemble (after a free-running launch)
cudaError_t launch_attempt_add(const StateDev& s, int n_ens, int n, cudaStream_t st);
cudaError_t launch_plain_advance(const StateDev& s, const EnsDev& e, const RepDev& r, int rep,
                                 const EnsDev* d_ens, const RepDev* d_rep, int steps,
                                 int max_ncell, cudaStream_t st, int refresh);
// d_rec (may be null): record row of rtot replicas, see exchange_kernel
cudaError_t launch_exchange(const StateDev& s, const EnsDev* d_ens, int n_ens, int max_r,
                            int32_t* d_partner, uint8_t* d_acc, cudaStream_t st,
                            double* d_rec = nullptr, int rtot = 0);
cudaError_t launch_apply_vscale(const StateDev& s, const RepDev* d_rep, const EnsDev* d_ens,
                                int n_rep, cudaStream_t st);
cudaError_t launch_export_state(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, double* d_x, double* d_v, double* d_f,
                                cudaStream_t st);
cudaError_t launch_import_state(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, const double* d_x, const double* d_v,
                                cudaStream_t st);
// perm = identity for every replica (every context starts in original order)
cudaError_t launch_identity_perm(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                 int n_rep, cudaStream_t st);
// Renumber the atoms of every replica in cell order (state permuted, lists
// invalidated); getters and setters map slots back through perm.
cudaError_t launch_spatial_sort(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, int max_n, int max_ncell, int64_t n_atoms,
                                cudaStream_t st);
cudaError_t launch_exchange_raw(int R, const double* T, const double* lam, const double* U,
                                uint64_t seed, int64_t attempt, int parity_mode, int distance,
                                double* T_out, double* lam_out, int32_t* partner,
                                uint8_t* accepted, double* vscale, double* uscale,
                                cudaStream_t st);

}  // namespace re
