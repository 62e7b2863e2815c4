/*
 * re.h -- C ABI of the GB300 (sm_103a) asynchronous replica-exchange
 * Lennard-Jones molecular-dynamics library.
 *
 * Method: G. Bussi, "A simple asynchronous replica-exchange implementation",
 * arXiv:0812.1633.  Replicas of an LJ liquid run velocity-Verlet MD with the
 * stochastic-velocity-rescaling thermostat (Example section) at different
 * temperatures; exchanges swap temperatures, not coordinates, with a
 * Metropolis test on the lower-rank replica's uniform number, and rescale
 * velocities by sqrt(T_new/T_old) (Implementation section).  Replicas may
 * perform different numbers of steps between attempts (asynchronous stride,
 * Example section).
 *
 * Conventions for every entry point:
 *   - Units: LJ reduced units (sigma = epsilon = m = k_B = 1).
 *   - Host arrays are owned by the caller; inputs are copied during the call,
 *     outputs are written before the call returns.  Array lengths are given
 *     per argument.  Device arrays ("_device" entry points) are owned by the
 *     caller and must stay valid until the work on the given stream is done.
 *   - Replica order: replicas of a context are numbered 0..n_rep-1; in a group
 *     (re_group) the replicas of its members follow one another in member order.
 *   - Positions/velocities/forces: doubles, AoS per replica, [replica][atom][xyz].
 *   - Return value: RE_OK (0) or a negative RE_E* code; re_last_error() gives
 *     a one-line message.  Errors raised by device work of an asynchronous
 *     call (list overflow, non-finite energy) are reported by the next call
 *     that synchronises (getters, re_sync).
 *   - Threads: one host thread per context at a time.  Calls are queued on the
 *     context's CUDA stream (re_set_stream); getters synchronise that stream.
 *   - The library allocates its own device memory with cudaMalloc at creation.
 *
 * Random numbers: Philox4x64-10 (Salmon et al., SC'11) used as a
 * counter-based generator; key = (seed, stream), counter = (index, tag, sub, 0):
 *   tag 1 initial velocities  (stream = id_offset + replica id, index = atom)
 *   tag 2 thermostat Gaussian (stream = id_offset + replica id, index = step)
 *   tag 3 thermostat Gamma trials (stream = id_offset + replica id, index = step,
 *                                  sub = trial)
 *   tag 4 Metropolis uniform  (stream = member id in the ladder, index = attempt)
 *   tag 5 random pair offset  (stream = 2^64-1, index = attempt)
 * A uniform is (word >> 11) * 2^-53.
 */
#ifndef RE_GB300_H
#define RE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RE_OK 0
#define RE_EINVAL (-1)    /* bad argument (see re_last_error)                 */
#define RE_ECUDA (-2)     /* CUDA runtime error                               */
#define RE_ENOMEM (-3)    /* device allocation failed                         */
#define RE_ENUMERIC (-4)  /* non-finite energy in some replica                */
#define RE_EOVERFLOW (-5) /* neighbour list or scratch capacity exceeded      */
#define RE_ETIMEOUT (-6)  /* a bounded device wait gave up                    */

#define RE_PREC_FP64 0    /* FP64 pair forces                                 */
#define RE_PREC_MIXED 1   /* FP32 pair forces on exact fixed-point separations,
                             64-bit fixed-point positions and velocities, exact
                             integer energy sums                               */

#define RE_PATH_BATCHED 0 /* one persistent launch runs every replica's budget */
#define RE_PATH_PLAIN 1   /* per replica and per step a sequence of launches  */

typedef struct re_ctx re_ctx; /* opaque; created by re_create/re_group, freed by re_destroy */

typedef struct re_opts {
  double dt;        /* time step; default 0.005 (Example section)                    */
  double skin;      /* Verlet skin; list radius rc + skin; default 0.5 (list to 3.0) */
  double tau_T;     /* thermostat relaxation time; default 0.5; <= 0: NVE            */
  int shift_energy; /* 1 (default): pair energy shifted to 0 at rc; 0: truncated      */
  int precision;    /* RE_PREC_MIXED (default) or RE_PREC_FP64                        */
  int path;         /* RE_PATH_BATCHED (default) or RE_PATH_PLAIN                     */
  int pair_parity;  /* 0 (default): first pair offset alternates 0,1; 1: random      */
  int nx;           /* steps per replica used by re_advance(c, NULL); default 10      */
  int nbr_capacity; /* neighbours per atom; 0: from the density with a 6-sigma margin */
  int cell_div;     /* list cells per list radius (1..3); 0: automatic               */
  int cluster;      /* CTAs cooperating on one replica (1, 2, 3, 4, 8); 0: automatic  */
  int atom_threads; /* threads sharing one atom's neighbour list (1, 2, 4, 8); 0: auto */
  int sort_interval;/* mixed batched path: renumber each replica's atoms in space order
                       every this many steps (0: every 200; < 0: never).  Results
                       differ only in summation order; atom order in the API is
                       always the original one. */
  int exch_distance;/* exchange pairs at ladder distance d (default 1: nearest
                       neighbours).  Non-nearest exchanges are the extension the
                       Implementation section mentions: positions (q, q + d) in
                       blocks of 2d, offset by d on odd attempts (parity). */
  int id_offset;    /* Philox stream of replica k's own draws (initial velocities,
                       thermostat) is id_offset + k (default 0).  A ladder sharded
                       over several contexts gives each shard the global id of its
                       first member, so every replica keeps its own stream. */
  int lists_smem;   /* neighbour lists of the batched path: 0 (default) global memory
                       (cached in L1/L2); 1: each CTA's sub-lists in shared memory when
                       they fit (copied in and out at every launch, so they pay off only
                       for long launches); -1: global memory, also for re_autotune.
                       re_autotune tries both unless this is 1 or -1. */
  int wide_launch;  /* split launch of a one-ensemble batched context (budget mode):
                       when the uniform launch leaves SMs idle, the hottest replicas
                       (by current temperature; they rebuild their lists most often)
                       run concurrently with one more CTA each, filling those SMs.
                       0 (default): one launch, and re_autotune times the split
                       against it; 1: always where it applies; -1: never.
                       The wide replicas take clusters of twice the CTAs with the
                       same threads per atom (re_config_wide), so the trajectories do
                       not change: the mixed path's sums are exact integers, and the
                       FP64 path differs only in the summation order of its energies. */
  int group_launch; /* a context of several ensembles (re_group), budget mode: 0
                       (default): one launch per ensemble, all concurrent on their own
                       streams, each ensemble in its own launch shape (re_config_class;
                       re_autotune tunes each on its own), so that small replicas do
                       not run in the shape sized for the largest; -1: one launch for
                       all replicas in one shape.  The free-running modes always use
                       one launch (their waits stay inside it). */
} re_opts;

/* Fills *o with the defaults listed above. */
void re_default_opts(re_opts *o);

/* Creates one ensemble of n_rep replicas of N atoms in a cubic periodic box of
 * side L with LJ cutoff rc.  Replica k starts at temperature temps[k] on an
 * FCC lattice (N must be 4 k^3) with Maxwell-Boltzmann velocities drawn from
 * seed, centre-of-mass motion removed and rescaled to exactly temps[k]
 * (3N - 3 degrees of freedom).  temps: n_rep distinct positive values (host).
 * opt: NULL for defaults.  Requires rc + skin < L/2, N <= 65535 for the
 * batched path.  *out receives the new context. */
int re_create(int N, double L, double rc, int n_rep, const double *temps, uint64_t seed,
              const re_opts *opt, re_ctx **out);

/* Generalised (Hamiltonian) replica exchange: as re_create, and replica k
 * also carries a potential scale lams[k] > 0 (host; NULL: all 1), so that its
 * Hamiltonian is K + lams[k] U_LJ (forces and reported U scale by lams[k]).
 * Exchanges then swap the parameter sets (T, lam): the ladder is ordered by
 * T/lam (keys must be distinct), D = (lam_a/T_a - lam_b/T_b)(U_a/lam_a -
 * U_b/lam_b), and on acceptance velocities scale by sqrt(T_new/T_old) and
 * forces and U by lam_new/lam_old (econs absorbs the jump, so H~ stays
 * continuous).  lam = 1 everywhere is the paper's temperature exchange.  The
 * paper implements temperatures only; it states the scheme extends to other
 * exchanges. */
int re_create_h(int N, double L, double rc, int n_rep, const double *temps, const double *lams,
                uint64_t seed, const re_opts *opt, re_ctx **out);

/* Builds one context holding the replicas of n contexts (ensembles of uneven
 * sizes), so that one launch advances all of them.  The members are copied;
 * they stay valid and independent.  All members must share precision and
 * path.  Exchanges never mix ensembles. */
int re_group(re_ctx *const *ctxs, int n, re_ctx **out);

/* Advances replica k by steps[k] MD steps (k over all replicas of the
 * context; host array; NULL: opt.nx for every replica).  Each step: half
 * kick, drift, list rebuild if some atom moved more than skin/2 since the
 * last rebuild, LJ forces, half kick, thermostat.  Asynchronous. */
int re_advance(re_ctx *c, const int32_t *steps);

/* Free-running (asynchronous) advance, the paper's scheme on one GPU
 * (Implementation section): in every ensemble the master replica, which
 * rotates with the attempt counter (replica attempt mod R), performs nx steps
 * and then raises the ensemble's flag; every other replica checks the flag
 * after each of its steps and stops after the step in which it sees it (and
 * after at most 16 nx + 16 steps).  Replicas therefore do different numbers of
 * steps between attempts (re_counters reports them).  Meaningful when all
 * replicas of an ensemble run at once (replicas x cluster CTAs within the
 * GPU's resident capacity); no thread ever waits on the flag.  Batched path
 * only.  Asynchronous. */
int re_advance_async(re_ctx *c, int nx);
/* n_cycles times { re_advance_async(nx); re_exchange }, optionally as one
 * CUDA graph. */
int re_run_async(re_ctx *c, int n_cycles, int nx, int use_graph);

/* The paper's asynchronous replica exchange inside ONE persistent launch
 * (Implementation section): replicas integrate without stopping; in every
 * ensemble the master of attempt a (member a mod R, rotating) waits, after nx
 * of its own steps since it took part in attempt a - 1, until every member has
 * finished attempt a - 1, sorts the ladder and publishes the pattern (the
 * pairs of re_exchange: ladder distance opt.exch_distance, offset by parity).
 * Every replica looks for a new pattern after each of its steps; a paired
 * replica publishes (T, U, lam), waits for its partner's, and both apply the
 * Metropolis rule with the uniform of the lower replica id for attempt a; on
 * acceptance the parameters are swapped and velocities (and forces) rescaled
 * exactly as re_exchange does.  n_att attempts per ensemble, then the launch
 * ends.
 *
 * Requires the batched path and all replicas resident on the GPU at once:
 * when the tuned launch shape cannot hold them all, the call runs in the first
 * shape with fewer CTAs per replica (the same threads per atom first, then
 * fewer) that can, rebuilding the neighbour lists for it and again for the
 * tuned shape afterwards; RE_EINVAL when no shape can.  Every device wait is bounded (1 s by default,
 * re_set_wait_limit); a wait that gives up ends the launch with RE_ETIMEOUT,
 * reported here when logging or by the next getter.  The launch then leaves
 * every replica at a step boundary with a consistent state: an exchange pair
 * has swapped on both sides or on neither, and T stays a permutation of the
 * ladder.  Once reported, the timeout marks are cleared and the context goes
 * on with the next call.  The number of steps each replica makes is decided
 * at run time; re_counters reports them.
 *
 * log_step, log_T (n_att x n_rep, row a = this call's attempt a): the
 * replica's step count when it took part (-1: it did not take part, the
 * launch having ended before), and its temperature afterwards; log_partner:
 * partner member id (-1 unpaired); log_acc: 1 if accepted.  Any non-NULL log
 * pointer makes the call synchronous; with all NULL it is asynchronous.  The
 * log is written also when the call returns RE_ETIMEOUT. */
int re_run_free(re_ctx *c, int n_att, int nx, int64_t *log_step, double *log_T,
                int32_t *log_partner, uint8_t *log_acc);

/* Limit of every bounded device wait of re_run_free (the master's collection
 * of temperatures, a replica's wait for its partner's pair message), in
 * seconds of the GPU's global timer: [1e-4, 10], default 1.  The paper's
 * blocking calls (Implementation section) become these waits. */
int re_set_wait_limit(re_ctx *c, double seconds);

/* Host-side fault injection for failure detection: in the next re_run_free
 * call (one call only), replica `replica` stops answering at its part in
 * attempt from_attempt (counted from that call's first attempt): it publishes
 * no pair message, reports nothing and leaves the launch at that step
 * boundary, as a stalled or lost process would.  Its partner's bounded wait
 * then runs out and the call returns RE_ETIMEOUT.  replica = -1 cancels.
 * Nothing faults on the device: the replica only skips its messages. */
int re_inject_stall(re_ctx *c, int replica, int from_attempt);

/* One exchange attempt in every ensemble: the ladder sorted (by temperature;
 * by T/lam with potential scales), ladder positions (q, q + d) paired for
 * d = opt.exch_distance (1: neighbours) from offset 0 or d, Metropolis with
 * the lower replica id's uniform, accepted pairs swap T (and lam) and rescale
 * velocities (and forces).  Outputs (host, n_rep each, may be NULL): partner
 * id or -1, accepted flag.  Synchronises only when an output is requested. */
int re_exchange(re_ctx *c, int32_t *partner_out, uint8_t *accepted_out);

/* n_cycles times { re_advance(steps + cycle * n_rep); re_exchange }.  steps:
 * host array n_cycles * n_rep, or NULL for opt.nx.  use_graph != 0 captures
 * the launches of all cycles in one CUDA graph and replays it. */
int re_run(re_ctx *c, int n_cycles, const int32_t *steps, int use_graph);

/* re_run with the run's log read back every cycle (the Example section's
 * record of a replica-exchange run: who exchanged, and the energies and
 * temperatures after every attempt).  Cycle k: row k of the budgets is
 * copied host -> device (steps: host, n_cycles x n_rep; NULL: opt.nx), the
 * replicas advance, one exchange attempt runs, and the cycle's record is
 * copied device -> host.  The copies run on two streams of their own and
 * overlap the following cycles; the call returns when the last record has
 * arrived (synchronous).  Outputs (host, n_cycles x n_rep each, row k =
 * cycle k, replica ids as in re_exchange; any may be NULL): partner id (-1:
 * unpaired), accepted flag, temperature after the attempt, U, K and H~ (as
 * re_energies would report after the attempt).  use_graph != 0 captures the
 * cycles, their copies included, in one CUDA graph, kept for the next call
 * with the same n_cycles (the budgets are read from the host array at every
 * call); the batched path only (the plain path runs eagerly).  Errors as
 * re_run; a replica error (status) is reported after the last cycle, the
 * outputs written. */
int re_run_record(re_ctx *c, int n_cycles, const int32_t *steps, int use_graph, int32_t *partner,
                  uint8_t *accepted, double *T, double *U, double *K, double *H);

/* Per replica (host, n_rep each, K and H may be NULL): potential energy U,
 * kinetic energy K and H~ = U + K + (energy removed by the thermostat). */
int re_energies(re_ctx *c, double *U, double *K, double *H);
/* Current temperature of every replica (host, n_rep). */
int re_temps(re_ctx *c, double *T);
/* Potential scale lam of every replica id (host, n_rep values). */
int re_lambdas(re_ctx *c, double *lam);

/* Applies exchange results decided outside the context (a ladder sharded
 * over several contexts or processes, each holding a block of its members):
 * per replica id (host, n_rep values) the new T, the new lam (NULL: kept),
 * the velocity factor sqrt(T_new/T_old) and the force/energy factor
 * lam_new/lam_old (NULL: 1), with the same bookkeeping as re_exchange
 * (K, U and econs).  All values must be positive.  Synchronous. */
int re_apply_exchange(re_ctx *c, const double *T_new, const double *lam_new,
                      const double *vscale, const double *uscale);
/* Positions (wrapped into [0, L)) and velocities, host arrays of
 * 3 * (atoms of all replicas) doubles each; either may be NULL. */
int re_get_state(re_ctx *c, double *x, double *v);
/* Replaces positions and velocities (same layout); lists and forces are
 * recomputed before the next step.  Step counters are unchanged. */
int re_set_state(re_ctx *c, const double *x, const double *v);
/* Checkpoint and resume.  A checkpoint holds everything the next call reads:
 * the fixed-point positions, velocities and forces, the neighbour lists and
 * their reference positions, the atom order, per replica T, lam, U, K, econs,
 * the pending exchange factors, step and rebuild counters, per ensemble the
 * exchange-attempt counter and per ladder pair the statistics, and the
 * launch configuration.  The random numbers are counter-based (Philox keyed
 * by seed and replica, counted by step and attempt), so a context restored
 * from a checkpoint continues bit for bit as the original would have.
 * re_checkpoint_size gives the bytes; re_checkpoint_save writes them into a
 * caller-owned host buffer of at least that size (synchronises the stream);
 * re_checkpoint_load restores them into a context created with the same
 * ensembles, seed and options (RE_EINVAL if the buffer is not a checkpoint of
 * a context of that shape; the context is unchanged then). */
int re_checkpoint_size(const re_ctx *c, size_t *bytes);
int re_checkpoint_save(re_ctx *c, void *buf, size_t bytes);
int re_checkpoint_load(re_ctx *c, const void *buf, size_t bytes);
/* Forces at the current positions (host, 3 * atoms). */
int re_forces(re_ctx *c, double *f);
/* Per replica steps done and list rebuilds done (host, n_rep each; may be NULL). */
int re_counters(re_ctx *c, int64_t *steps, int64_t *rebuilds);
/* Per ensemble and per sorted-temperature pair position k (k = 0..R_e-2), the
 * number of attempts and of accepted exchanges; ensembles concatenated,
 * sum over ensembles of (R_e - 1) entries. */
int re_accept_stats(re_ctx *c, int64_t *attempts, int64_t *accepts);
/* Shape of the context: replicas, atoms of all replicas, ensembles, pair
 * stats entries (any may be NULL). */
int re_info(const re_ctx *c, int *n_rep, int64_t *n_atoms, int *n_ens, int *n_pairs);
/* Launch configuration in use: CTAs per replica, threads per CTA, list cells
 * per list radius, threads per atom (any may be NULL). */
int re_config(const re_ctx *c, int *cluster, int *threads, int *cell_div, int *atom_threads);
/* re_config and whether the neighbour lists are kept in shared memory. */
int re_config_ex(const re_ctx *c, int *cluster, int *threads, int *cell_div, int *atom_threads,
                 int *lists_smem);
/* Launch shape of ensemble e's launch in a context of several ensembles with
 * per-ensemble launches (re_opts.group_launch): CTAs per replica, threads
 * per CTA, list cells per list radius, threads per atom, lists in shared
 * memory (any pointer may be NULL).  RE_EINVAL when e is out of range or the
 * context runs one launch. */
int re_config_class(const re_ctx *c, int e, int *cluster, int *threads, int *cell_div,
                    int *atom_threads, int *lists_smem);
/* The split launch in use (re_opts.wide_launch): replicas in the wide class,
 * CTAs per wide replica, threads per wide CTA, threads per atom in the wide
 * class (all 0: one launch).  Any pointer may be NULL. */
int re_config_wide(const re_ctx *c, int *wide_n, int *wide_cluster, int *wide_threads,
                   int *wide_atom_threads);
/* Times candidate launch configurations (cluster, atom_threads, cell_div,
 * the lists' placement, global or shared memory, and each as one launch or
 * split, see re_opts.wide_launch) over `steps` steps each on a copy of the
 * state and keeps the fastest; the state is restored afterwards.  With
 * per-ensemble launches (re_opts.group_launch) every ensemble's shape is
 * tuned on its own launch. */
int re_autotune(re_ctx *c, int steps);
/* Queues subsequent work on stream (a cudaStream_t; NULL: legacy default). */
int re_set_stream(re_ctx *c, void *stream);
/* Waits for the context's queued work and reports deferred device errors. */
int re_sync(re_ctx *c);
/* Last error message of the context (or of the last failed create when c is NULL). */
const char *re_last_error(const re_ctx *c);
void re_destroy(re_ctx *c);

/* ---------------------------------------------------------------------------
 * Stateless device entry points (device pointers, caller-owned, on `stream`).
 */

/* One exchange attempt over R <= 4096 replicas (Implementation section), as
 * in re_exchange: T, U device arrays (R doubles); outputs T_out (R doubles,
 * new temperatures), partner (R int32, -1 if unpaired), accepted (R uint8),
 * vscale (R doubles, sqrt(T_new/T_old) or 1).  T must hold distinct positive values. */
int re_exchange_device(int R, const double *T, const double *U, uint64_t seed, int64_t attempt,
                       int parity_mode, double *T_out, int32_t *partner, uint8_t *accepted,
                       double *vscale, void *stream);

/* re_exchange_device generalised like re_create_h: lam (device, R values,
 * NULL: all 1) and pairs at ladder distance `distance` (>= 1).  Outputs as
 * re_exchange_device, plus lam_out (NULL allowed) = the swapped scales and
 * uscale (NULL allowed) = lam_new/lam_old per replica.  Keys T/lam must be
 * distinct and positive.  The same decisions as re_exchange for the same
 * state. */
int re_exchange_device_h(int R, const double *T, const double *lam, const double *U,
                         uint64_t seed, int64_t attempt, int parity_mode, int distance,
                         double *T_out, double *lam_out, int32_t *partner, uint8_t *accepted,
                         double *vscale, double *uscale, void *stream);

/* Truncated LJ forces and potential energy of N atoms in a cubic periodic box
 * of side L with cutoff rc (Example section): x device array of 3N doubles
 * (AoS), f device array of 3N doubles, U device pointer to one double.
 * Pairs are found with the same cell binning and neighbour-list kernels as
 * the MD path (list radius rc + skin, skin = 0.5).  precision: RE_PREC_FP64
 * or RE_PREC_MIXED.  Scratch (cells, lists) is allocated with cudaMalloc and
 * freed before return; the call synchronises `stream`.  Requires 2 <= N <=
 * 65535 and rc + 0.5 < L/2. */
int re_lj_forces_device(int N, double L, double rc, int shift, int precision, const double *x,
                        double *f, double *U, void *stream);

/* The computation of re_lj_forces_device (FP64 pair forces) without any
 * allocation, for callers that cannot call cudaMalloc (code running inside
 * another framework's memory pool or under a fixed memory budget, plug-ins
 * that may not touch the allocator).  The paper has no counterpart: this is a
 * deployment variant.  Scratch lives in one fixed device array of about
 * 2.6 MB that every device loading the library keeps until the process exits.
 * Limits: 2 <= N <= 4096 atoms, at most 256 neighbour-list entries per atom
 * (RE_EOVERFLOW beyond), rc + 0.5 < L/2.  Arguments as re_lj_forces_device
 * (device pointers, caller-owned).  The first call on a device looks up the
 * array's device address and caches it: make that first call before any
 * stream capture.  Every call shares the array and leaves its contents
 * behind; calls that overlap on the GPU race.  The call synchronises
 * `stream`.  Errors: return code only (re_last_error is not updated). */
int re_lj_forces_device_noalloc(int N, double L, double rc, int shift, const double *x,
                                double *f, double *U, void *stream);

#ifdef __cplusplus
}
#endif
#endif
