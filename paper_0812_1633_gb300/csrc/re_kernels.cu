// re_kernels.cu -- sm_103a kernels of the asynchronous replica-exchange LJ MD
// library (G. Bussi, arXiv:0812.1633).
//
// Hot path (Example section: LJ liquid, cutoff rc, Verlet list to rc + skin
// rebuilt when a displacement exceeds skin/2, velocity Verlet with time step
// dt, stochastic velocity rescaling), run for every replica at once:
//   md_batched_kernel  one thread-block cluster per replica runs that
//                      replica's whole step budget: kick, drift, displacement
//                      test, [cell binning + counting sort + list build], LJ
//                      forces, kick, thermostat.  Positions of the replica
//                      live in shared memory of every CTA of the cluster
//                      (broadcast through distributed shared memory).
//   plain_*            the same step as a sequence of launches for one
//                      replica at a time, FP64 throughout (comparison path).
//   exchange_kernel    Implementation section: sort temperatures, pair
//                      sorted neighbours, Metropolis with the lower-id
//                      replica's uniform, swap T, rescale velocities.
#include <climits>

#include "re_md.cuh"

namespace re {

namespace {

// ------------------------------------------------------------------ set-up
// FCC lattice (N = 4 k^3, cell a = L/k, four-atom basis, offset a/4) and
// Maxwell-Boltzmann velocities: atom i takes Philox block (i, tag 1) of the
// replica's stream; Box-Muller gives vx, vy from (u0, u1) and vz from (u2, u3);
// centre-of-mass velocity removed; rescaled to exactly T with Nf = 3N - 3.
__global__ void init_lattice_kernel(StateDev S, const EnsDev* __restrict__ ens,
                                    const RepDev* __restrict__ reps) {
  __shared__ double red[kMaxWarps];
  const int r = blockIdx.x;
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const int N = E.N;
  int k = 1;
  while (4 * k * k * k < N) ++k;
  const double a = E.L / k;
  const double inv_l = 1.0 / E.L;
  const double bx[4] = {0.0, 0.5, 0.5, 0.0}, by[4] = {0.0, 0.5, 0.0, 0.5},
               bz[4] = {0.0, 0.0, 0.5, 0.5};
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int b = i & 3, cell = i >> 2;
    const int iz = cell % k, iy = (cell / k) % k, ix = cell / (k * k);
    const double x = (ix + bx[b] + 0.25) * a, y = (iy + by[b] + 0.25) * a,
                 z = (iz + bz[b] + 0.25) * a;
    const int g = rd.atom_off + i;
    S.perm[g] = i;
    S.qx[g] = fix_from_double(x, inv_l);
    S.qy[g] = fix_from_double(y, inv_l);
    S.qz[g] = fix_from_double(z, inv_l);
    const Uni4 u = uniforms(E.seed, (uint64_t)rd.stream, (uint64_t)i, kTagVel, 0ull);
    double g0, g1, g2, g3;
    box_muller(u.u0, u.u1, &g0, &g1);
    box_muller(u.u2, u.u3, &g2, &g3);
    S.vx[g] = g0;
    S.vy[g] = g1;
    S.vz[g] = g2;
    sx += g0;
    sy += g1;
    sz += g2;
  }
  const double mx = block_sum(sx, red) / N, my = block_sum(sy, red) / N,
               mz = block_sum(sz, red) / N;
  double kin = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int g = rd.atom_off + i;
    const double vx = S.vx[g] - mx, vy = S.vy[g] - my, vz = S.vz[g] - mz;
    S.vx[g] = vx;
    S.vy[g] = vy;
    S.vz[g] = vz;
    kin += vx * vx + vy * vy + vz * vz;
  }
  const double K = 0.5 * block_sum(kin, red);
  const int nf = 3 * N - 3;
  const double scale = sqrt(S.T[r] / (2.0 * K / nf));
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int g = rd.atom_off + i;
    const double vx = S.vx[g] * scale, vy = S.vy[g] * scale, vz = S.vz[g] * scale;
    if (S.vfix) {
      vfix_put(S.vx, g, vfix_from_double(vx));
      vfix_put(S.vy, g, vfix_from_double(vy));
      vfix_put(S.vz, g, vfix_from_double(vz));
      hfix_put(S.fx, g, 0.0f);
      hfix_put(S.fy, g, 0.0f);
      hfix_put(S.fz, g, 0.0f);
    } else {
      S.vx[g] = vx;
      S.vy[g] = vy;
      S.vz[g] = vz;
    }
  }
  if (threadIdx.x == 0) {
    S.K[r] = K * scale * scale;
    S.U[r] = 0.0;
    S.econs[r] = 0.0;
    S.vscale[r] = 1.0;
    S.fscale[r] = 1.0;
    S.step[r] = 0;
    S.nreb[r] = 0;
    S.status[r] = 0;
    S.valid[r] = 0;
  }
}

// ------------------------------------------------------------------ plain path
// One replica, one step, a sequence of small FP64 launches (the comparison
// path).  Positions use the same fixed-point words as the batched path.

__device__ __forceinline__ void atomic_max_float_pos(uint32_t* addr, float v) {
  atomicMax(addr, __float_as_uint(v));  // non-negative floats order like their bits
}

__global__ void plain_kick_drift(StateDev S, const EnsDev* __restrict__ ens,
                                 const RepDev* __restrict__ reps, int r) {
  __shared__ float scr[kMaxWarps];
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const StepConst& K = E.kc;
  const double vs = S.vscale[r];
  const double fs = S.fscale ? S.fscale[r] : 1.0;  // pending force factor (exchange of lam)
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float md = 0.0f;
  if (i < E.N) {
    const int g = rd.atom_off + i;
    const double vx = fma(S.vx[g], vs, K.hdt * (S.fx[g] * fs));
    const double vy = fma(S.vy[g], vs, K.hdt * (S.fy[g] * fs));
    const double vz = fma(S.vz[g], vs, K.hdt * (S.fz[g] * fs));
    S.vx[g] = vx;
    S.vy[g] = vy;
    S.vz[g] = vz;
    const uint64_t qx = S.qx[g] + (uint64_t)__double2ll_rn(vx * K.dtq);
    const uint64_t qy = S.qy[g] + (uint64_t)__double2ll_rn(vy * K.dtq);
    const uint64_t qz = S.qz[g] + (uint64_t)__double2ll_rn(vz * K.dtq);
    S.qx[g] = qx;
    S.qy[g] = qy;
    S.qz[g] = qz;
    const Hi3 ref{S.rx[g], S.ry[g], S.rz[g]};
    const Hi3 now{(uint32_t)(qx >> 32), (uint32_t)(qy >> 32), (uint32_t)(qz >> 32)};
    md = sep2_hi(ref, now);
  }
  md = block_max(md, scr);
  if (threadIdx.x == 0) atomic_max_float_pos(S.dmax + r, md);
}

// Whole-replica list rebuild in one CTA when needed (or forced).
__global__ void plain_rebuild(StateDev S, const EnsDev* __restrict__ ens,
                              const RepDev* __restrict__ reps, int r, int max_ncell) {
  extern __shared__ __align__(16) unsigned char sh[];
  __shared__ int scr[64];
  __shared__ int ovf;
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const StepConst& K = E.kc;
  const bool need = !S.valid[r] || __uint_as_float(S.dmax[r]) > K.half2u;
  __syncthreads();
  if (threadIdx.x == 0) {
    S.dmax[r] = 0u;
    ovf = 0;
  }
  if (!need) return;
  const int N = E.N;
  uint4* spos = reinterpret_cast<uint4*>(sh);
  Hi3* hp = reinterpret_cast<Hi3*>(spos + N);
  int* cstart = reinterpret_cast<int*>(hp + N);
  int* ccnt = cstart + (max_ncell + 1);
  uint16_t* acell = reinterpret_cast<uint16_t*>(ccnt + (max_ncell + 1));
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int g = rd.atom_off + i;
    hp[i] = Hi3{(uint32_t)(S.qx[g] >> 32), (uint32_t)(S.qy[g] >> 32), (uint32_t)(S.qz[g] >> 32)};
  }
  __syncthreads();
  auto hi_of = [&](int i) { return hp[i]; };
  if (E.nc > 0) cta_build_cells(hi_of, N, E.nc, cstart, ccnt, spos, acell, scr);
  int overflow = 0;
  uint16_t* nb = S.nbr + rd.nbr_off;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int g = rd.atom_off + i;
    S.ncnt[(size_t)rd.atom_off * 8 + i] =
        build_sublist<1>(i, 0, hi_of, N, E.nc, E.m, cstart, spos, K.rl2u, nb, (uint32_t)i,
                         (uint32_t)N, E.capsub[0], &overflow);
    S.rx[g] = hp[i].x;
    S.ry[g] = hp[i].y;
    S.rz[g] = hp[i].z;
  }
  if (overflow) atomicOr(&ovf, overflow);
  __syncthreads();
  if (threadIdx.x == 0) {
    S.valid[r] = (ovf & kStOverflow) ? 0 : 1;
    S.nreb[r] += 1;
    S.status[r] |= ovf;
  }
}

// FP64 forces of one replica from its list, positions read from global memory;
// per-block energy partials to red[r][block].
__global__ void plain_forces(StateDev S, const EnsDev* __restrict__ ens,
                             const RepDev* __restrict__ reps, int r) {
  __shared__ double scr[kMaxWarps];
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const StepConst& K = E.kc;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < E.N) {
    const int g = rd.atom_off + i;
    const uint64_t xi = S.qx[g], yi = S.qy[g], zi = S.qz[g];
    const int cnt = S.ncnt[(size_t)rd.atom_off * 8 + i];
    const uint16_t* nb = S.nbr + rd.nbr_off;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int k = 0; k < cnt; ++k) {
      const int j = nb[((size_t)(k >> 2) * E.N + i) * 4 + (k & 3)];
      const int gj = rd.atom_off + j;
      const double dx = (double)(long long)(S.qx[gj] - xi) * K.lam64;
      const double dy = (double)(long long)(S.qy[gj] - yi) * K.lam64;
      const double dz = (double)(long long)(S.qz[gj] - zi) * K.lam64;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < K.rc2) {
        const double s = 1.0 / r2;
        const double s3 = s * s * s;
        const double fs = 48.0 * s3 * s3 * s - 24.0 * s3 * s;
        fx -= fs * dx;
        fy -= fs * dy;
        fz -= fs * dz;
        e += 4.0 * (s3 * s3 - s3) - K.uc;
      }
    }
    const double lam = S.lam ? S.lam[r] : 1.0;
    S.fx[g] = lam * fx;
    S.fy[g] = lam * fy;
    S.fz[g] = lam * fz;
    e *= lam;
  }
  e = block_sum(e, scr);
  if (threadIdx.x == 0) S.red[(size_t)r * kPlainRed + blockIdx.x] = e;
  // the forces are new: no pending factor (plain_kick_drift of this step has run)
  if (S.fscale && blockIdx.x == 0 && threadIdx.x == 0) S.fscale[r] = 1.0;
}

// Second half kick (optional) and per-block sums of v^2 to red[r][512 + block].
__global__ void plain_kick(StateDev S, const EnsDev* __restrict__ ens,
                           const RepDev* __restrict__ reps, int r, int kick) {
  __shared__ double scr[kMaxWarps];
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const double hdt = 0.5 * E.dt;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double k2 = 0.0;
  if (i < E.N) {
    const int g = rd.atom_off + i;
    double vx = S.vx[g], vy = S.vy[g], vz = S.vz[g];
    if (kick) {
      vx += hdt * S.fx[g];
      vy += hdt * S.fy[g];
      vz += hdt * S.fz[g];
      S.vx[g] = vx;
      S.vy[g] = vy;
      S.vz[g] = vz;
    }
    k2 = vx * vx + vy * vy + vz * vz;
  }
  k2 = block_sum(k2, scr);
  if (threadIdx.x == 0) S.red[(size_t)r * kPlainRed + kPlainRed / 2 + blockIdx.x] = k2;
}

// Energies of the step (fixed-order sums of the block partials) and the
// thermostat factor, stored as the pending velocity factor of the next kick.
__global__ void plain_thermo(StateDev S, const EnsDev* __restrict__ ens,
                             const RepDev* __restrict__ reps, int r, int nblocks, int thermo) {
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const int lane = threadIdx.x;
  double su = 0.0, sk = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    su += S.red[(size_t)r * kPlainRed + b];
    sk += S.red[(size_t)r * kPlainRed + kPlainRed / 2 + b];
  }
  su = warp_sum(su);
  sk = warp_sum(sk);
  if (lane == 0) {
    const double U = 0.5 * su, Kn = 0.5 * sk;
    int st = S.status[r];
    double alpha = 1.0, Kp = Kn;
    if (thermo && E.tau > 0.0) {
      const int nf = 3 * E.N - 3;
      int capped = 0;
      const double2 nz = svr_noise(nf, E.seed, (uint64_t)rd.stream, (uint64_t)S.step[r], &capped);
      if (capped) st |= kStRngCap;
      alpha = svr_alpha(Kn, 0.5 * nf * S.T[r], nf, exp(-E.dt / E.tau), nz.x, nz.y, &Kp);
      S.econs[r] += Kn - Kp;
    }
    if (!isfinite(U) || !isfinite(Kp)) st |= kStNumeric;
    S.U[r] = U;
    S.K[r] = Kp;
    if (thermo) {
      S.vscale[r] = alpha;
      S.step[r] += 1;
    }
    S.status[r] = st;
  }
}

// ------------------------------------------------------------------ exchange
// Sorted order of R distinct positive keys (ascending; ties, which the API
// excludes, by index): a bitonic sort of (key, index) pairs over the next
// power of two m >= R in shared memory -- keyd and order hold m entries, the
// first R keys set by the caller, the padding sorts last.  Positive doubles
// order like their IEEE bit patterns read as 64-bit integers, so the
// comparisons run on the integer units instead of the (1/64-rate) FP64 unit.
__device__ void sort_keys(double* keyd, int* order, int R) {
  long long* key = reinterpret_cast<long long*>(keyd);
  int m = 1;
  while (m < R) m <<= 1;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    if (t >= R) key[t] = LLONG_MAX;
    order[t] = t;
  }
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const bool up = (t & k) == 0;
          const long long ka = key[t], kb = key[u];
          const int ia = order[t], ib = order[u];
          if ((ka > kb || (ka == kb && ia > ib)) == up) {
            key[t] = kb;
            key[u] = ka;
            order[t] = ib;
            order[u] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
}

// shared memory of sort_keys for R keys
__host__ __device__ inline size_t sort_keys_bytes(int R) {
  size_t m = 1;
  while (m < (size_t)R) m <<= 1;
  return m * (sizeof(double) + sizeof(int));
}

// Ladders up to this size are ordered by one CTA counting ranks (every thread
// scans all keys, broadcast reads, no barriers); longer ones by
// exchange_cluster_kernel.
constexpr int kRankSortMax = 256;

// shared memory of exchange_kernel for R replicas: sort_keys' area (12 bytes
// per key slot: not a multiple of 8 for a one-replica ladder), then, from the
// next 16-byte boundary, per replica the quotients lam/T and U/lam, the
// exchange uniform, T and lam
__host__ __device__ inline size_t exchange_dbl_offset(int R) {
  return (sort_keys_bytes(R) + 15) / 16 * 16;
}
__host__ __device__ inline size_t exchange_smem_bytes(int R) {
  return exchange_dbl_offset(R) + (size_t)R * 5 * sizeof(double);
}

// One exchange attempt per ensemble (one CTA each; contexts whose longest
// ladder exceeds kRankSortMax use exchange_cluster_kernel): ladder keys T/lam sorted,
// pairs (q, q + d) of the ladder (d = 1: sorted neighbours), the Metropolis
// rule, and on acceptance the parameter sets (T, lam) are swapped: the
// velocities take the pending factor sqrt(T_new/T_old), the forces
// lam_new/lam_old, K and U follow and econs absorbs both changes.
// The kernel is a short chain of dependent steps on one CTA, so it is laid
// out for latency: one load phase, every per-replica quotient and uniform
// computed once and in parallel (the same operations as the pair formula, so
// the decisions are those of metropolis()), and what an accepted pair
// changes read before the decision.
// rec (may be null): the cycle's record row, per replica id of all rtot
// replicas T, U, K and econs after the attempt at rec[0..4 rtot).
__global__ void exchange_kernel(StateDev S, const EnsDev* __restrict__ ens, int32_t* partner_out,
                                uint8_t* acc_out, double* rec, int rtot) {
  extern __shared__ __align__(16) unsigned char sh[];
  const int R = ens[blockIdx.x].R, base = ens[blockIdx.x].rep_off;
  const int pair_off = ens[blockIdx.x].pair_off, xdist = ens[blockIdx.x].xdist;
  const int parity_mode = ens[blockIdx.x].parity_mode;
  const uint64_t seed = ens[blockIdx.x].seed;
  const int64_t attempt = S.attempt[blockIdx.x];
  int m = 1;
  while (m < R) m <<= 1;
  double* key = reinterpret_cast<double*>(sh);
  int* order = reinterpret_cast<int*>(key + m);
  double* qt = reinterpret_cast<double*>(sh + exchange_dbl_offset(R));  // lam / T
  double* qu = qt + R;                                               // U / lam
  double* uni = qu + R;                                              // uniform of id a
  double* Tsh = uni + R;
  double* lsh = Tsh + R;
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    const double T = S.T[base + a], lam = S.lam[base + a], U = S.U[base + a];
    const bool one = lam == 1.0;  // x / 1 == x exactly: the divisions are skipped
    key[a] = one ? T : T / lam;
    qt[a] = __ddiv_rn(lam, T);
    qu[a] = one ? U : __ddiv_rn(U, lam);
    uni[a] = uniforms(seed, (uint64_t)a, (uint64_t)attempt, kTagExch, 0ull).u0;
    Tsh[a] = T;
    lsh[a] = lam;
    if (partner_out) partner_out[base + a] = -1;
    if (acc_out) acc_out[base + a] = 0;
  }
  __syncthreads();
  if (R <= kRankSortMax) {
    // positive doubles order like their bit patterns; ties (excluded by the
    // API) by index, as sort_keys
    const long long* ki = reinterpret_cast<const long long*>(key);
    for (int a = threadIdx.x; a < R; a += blockDim.x) {
      const long long ka = ki[a];
      int rank = 0;
#pragma unroll 8
      for (int b = 0; b < R; ++b) {
        const long long kb = ki[b];
        rank += (kb < ka) | ((kb == ka) & (b < a));
      }
      order[rank] = a;
    }
  } else {
    sort_keys(key, order, R);
  }
  __syncthreads();
  const int p = pair_offset(parity_mode, seed, attempt);
  const int d = max(1, xdist);
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    const int qb = ladder_partner(q, R, p, d);
    if (qb <= q) continue;  // unpaired, or the upper member of its pair
    const int a = order[q], b = order[qb];
    const int ga = base + a, gb = base + b;
    // everything an accepted exchange changes, requested before the decision
    const long long n_att = S.pair_att[pair_off + q], n_acc = S.pair_acc[pair_off + q];
    const double Ka = S.K[ga], Kb = S.K[gb], Ea = S.econs[ga], Eb = S.econs[gb];
    const double va = S.vscale[ga], vb = S.vscale[gb];
    const double Ta = Tsh[a], Tb = Tsh[b], la = lsh[a], lb = lsh[b];
    // metropolis(): D = (lam_a/T_a - lam_b/T_b)(U_a/lam_a - U_b/lam_b), accept
    // iff D >= 0 or r < exp(D), r the uniform of the lower replica id
    const double dd = __dmul_rn(__dsub_rn(qt[a], qt[b]), __dsub_rn(qu[a], qu[b]));
    const bool ok = dd >= 0.0 || uni[min(a, b)] < exp(dd);
    if (partner_out) {
      partner_out[ga] = b;
      partner_out[gb] = a;
    }
    S.pair_att[pair_off + q] = n_att + 1;
    if (ok) {
      S.pair_acc[pair_off + q] = n_acc + 1;
      if (acc_out) acc_out[ga] = acc_out[gb] = 1;
      const double sa = sqrt(Tb / Ta), sb = sqrt(Ta / Tb);
      const double Kan = Ka * (sa * sa), Kbn = Kb * (sb * sb);
      S.vscale[ga] = va * sa;
      S.vscale[gb] = vb * sb;
      double ea = Ea + (Ka - Kan), eb = Eb + (Kb - Kbn);
      S.K[ga] = Kan;
      S.K[gb] = Kbn;
      S.T[ga] = Tb;
      S.T[gb] = Ta;
      if (la != lb) {
        const double ua = lb / la, ub = la / lb;
        const double Ua = S.U[ga], Ub = S.U[gb];
        const double Uan = Ua * ua, Ubn = Ub * ub;
        S.fscale[ga] *= ua;
        S.fscale[gb] *= ub;
        ea += Ua - Uan;
        eb += Ub - Ubn;
        S.U[ga] = Uan;
        S.U[gb] = Ubn;
        S.lam[ga] = lb;
        S.lam[gb] = la;
      }
      S.econs[ga] = ea;
      S.econs[gb] = eb;
    }
  }
  __syncthreads();
  if (rec) {
    for (int a = threadIdx.x; a < R; a += blockDim.x) {
      const int g = base + a;
      rec[g] = S.T[g];
      rec[rtot + g] = S.U[g];
      rec[2 * rtot + g] = S.K[g];
      rec[3 * rtot + g] = S.econs[g];
    }
  }
  if (threadIdx.x == 0) S.attempt[blockIdx.x] = attempt + 1;
}

// Ladders longer than kRankSortMax: one cluster of C CTAs per ensemble
// (blocks e*C .. e*C + C - 1).  Every CTA reads the whole ladder's keys and
// ranks its slice of the replicas by counting (G threads per replica, each
// counting over every G-th key, summed by shuffles), writing each replica's
// ladder position into the order array of every CTA of the cluster
// (distributed shared memory); after a cluster barrier each CTA runs the
// pairs whose lower ladder position lies in its slice, with the arithmetic of
// exchange_kernel, so the decisions are the same.  A second barrier makes
// every CTA's updates visible before the record is written and the attempt
// counted.
__global__ void exchange_cluster_kernel(StateDev S, const EnsDev* __restrict__ ens,
                                        int32_t* partner_out, uint8_t* acc_out, double* rec,
                                        int rtot) {
  extern __shared__ __align__(16) unsigned char sh[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), cr = (int)cl.block_rank();
  const int e = blockIdx.x / C;
  const int R = ens[e].R, base = ens[e].rep_off;
  const int pair_off = ens[e].pair_off, xdist = ens[e].xdist;
  const int parity_mode = ens[e].parity_mode;
  const uint64_t seed = ens[e].seed;
  const int64_t attempt = S.attempt[e];
  long long* key = reinterpret_cast<long long*>(sh);  // R: T/lam as bit patterns
  int* order = reinterpret_cast<int*>(key + R);       // R: replica at each ladder position
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int a = tid; a < R; a += nt) {
    const double T = S.T[base + a], lam = S.lam[base + a];
    key[a] = __double_as_longlong(lam == 1.0 ? T : T / lam);
  }
  const int per = (R + C - 1) / C;
  const int a0 = min(R, cr * per), a1 = min(R, a0 + per);
  for (int a = a0 + tid; a < a1; a += nt) {
    if (partner_out) partner_out[base + a] = -1;
    if (acc_out) acc_out[base + a] = 0;
  }
  __syncthreads();
  // G threads (consecutive lanes, G a power of two <= 32) per replica
  int G = 1;
  while (G < 32 && G * 2 * per <= nt) G *= 2;
  for (int t0 = 0; t0 < per * G; t0 += nt) {
    const int t = t0 + tid;
    const int a = a0 + t / G, part = t % G;
    const bool mine = t < per * G && a < a1;
    int rank = 0;
    if (mine) {
      const long long ka = key[a];
      for (int b = part; b < R; b += G) {
        const long long kb = key[b];
        rank += (kb < ka) | ((kb == ka) & (b < a));
      }
    }
    for (int o = G / 2; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    if (mine && part == 0)
      for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(order + rank, rk) = a;
  }
  cl.sync();
  const int p = pair_offset(parity_mode, seed, attempt);
  const int d = max(1, xdist);
  for (int q = a0 + tid; q < a1; q += nt) {
    const int qb = ladder_partner(q, R, p, d);
    if (qb <= q) continue;
    const int a = order[q], b = order[qb];
    const int ga = base + a, gb = base + b;
    const long long n_att = S.pair_att[pair_off + q], n_acc = S.pair_acc[pair_off + q];
    const double Ka = S.K[ga], Kb = S.K[gb], Ea = S.econs[ga], Eb = S.econs[gb];
    const double va = S.vscale[ga], vb = S.vscale[gb];
    const double Ta = S.T[ga], Tb = S.T[gb], la = S.lam[ga], lb = S.lam[gb];
    const double Ua = S.U[ga], Ub = S.U[gb];
    const double qta = __ddiv_rn(la, Ta), qtb = __ddiv_rn(lb, Tb);
    const double qua = la == 1.0 ? Ua : __ddiv_rn(Ua, la), qub = lb == 1.0 ? Ub : __ddiv_rn(Ub, lb);
    const double dd = __dmul_rn(__dsub_rn(qta, qtb), __dsub_rn(qua, qub));
    bool ok = dd >= 0.0;
    if (!ok)
      ok = uniforms(seed, (uint64_t)min(a, b), (uint64_t)attempt, kTagExch, 0ull).u0 < exp(dd);
    if (partner_out) {
      partner_out[ga] = b;
      partner_out[gb] = a;
    }
    S.pair_att[pair_off + q] = n_att + 1;
    if (ok) {
      S.pair_acc[pair_off + q] = n_acc + 1;
      if (acc_out) acc_out[ga] = acc_out[gb] = 1;
      const double sa = sqrt(Tb / Ta), sb = sqrt(Ta / Tb);
      const double Kan = Ka * (sa * sa), Kbn = Kb * (sb * sb);
      S.vscale[ga] = va * sa;
      S.vscale[gb] = vb * sb;
      double ea = Ea + (Ka - Kan), eb = Eb + (Kb - Kbn);
      S.K[ga] = Kan;
      S.K[gb] = Kbn;
      S.T[ga] = Tb;
      S.T[gb] = Ta;
      if (la != lb) {
        const double ua = lb / la, ub = la / lb;
        const double Uan = Ua * ua, Ubn = Ub * ub;
        S.fscale[ga] *= ua;
        S.fscale[gb] *= ub;
        ea += Ua - Uan;
        eb += Ub - Ubn;
        S.U[ga] = Uan;
        S.U[gb] = Ubn;
        S.lam[ga] = lb;
        S.lam[gb] = la;
      }
      S.econs[ga] = ea;
      S.econs[gb] = eb;
    }
  }
  __threadfence();  // the pairs' global updates, before the record reads them
  cl.sync();
  if (rec) {
    for (int a = a0 + tid; a < a1; a += nt) {
      const int g = base + a;
      rec[g] = S.T[g];
      rec[rtot + g] = S.U[g];
      rec[2 * rtot + g] = S.K[g];
      rec[3 * rtot + g] = S.econs[g];
    }
  }
  if (cr == 0 && tid == 0) S.attempt[e] = attempt + 1;
}

__global__ void exchange_raw_kernel(int R, const double* __restrict__ T,
                                    const double* __restrict__ lam,
                                    const double* __restrict__ U, uint64_t seed, int64_t attempt,
                                    int mode, int distance, double* T_out, double* lam_out,
                                    int32_t* partner, uint8_t* acc, double* vscale,
                                    double* uscale) {
  extern __shared__ __align__(16) unsigned char sh[];
  int m = 1;
  while (m < R) m <<= 1;
  double* key = reinterpret_cast<double*>(sh);
  int* order = reinterpret_cast<int*>(key + m);
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    const double l = lam ? lam[a] : 1.0;
    key[a] = T[a] / l;
    T_out[a] = T[a];
    if (lam_out) lam_out[a] = l;
    partner[a] = -1;
    acc[a] = 0;
    vscale[a] = 1.0;
    if (uscale) uscale[a] = 1.0;
  }
  __syncthreads();
  sort_keys(key, order, R);
  __syncthreads();
  const int p = pair_offset(mode, seed, attempt);
  const int d = max(1, distance);
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    const int qb = ladder_partner(q, R, p, d);
    if (qb <= q) continue;
    const int a = order[q], b = order[qb];
    const double Ta = T[a], Tb = T[b];
    const double la = lam ? lam[a] : 1.0, lb = lam ? lam[b] : 1.0;
    const bool ok = metropolis(Ta, Tb, la, lb, U[a], U[b], seed, min(a, b), attempt);
    partner[a] = b;
    partner[b] = a;
    if (ok) {
      acc[a] = acc[b] = 1;
      vscale[a] = sqrt(Tb / Ta);
      vscale[b] = sqrt(Ta / Tb);
      T_out[a] = Tb;
      T_out[b] = Ta;
      if (lam_out) {
        lam_out[a] = lb;
        lam_out[b] = la;
      }
      if (uscale) {
        uscale[a] = lb / la;
        uscale[b] = la / lb;
      }
    }
  }
}

// Exchange results decided elsewhere (a ladder sharded over several
// contexts): in = [T_new | lam_new | vscale | uscale], R values each.  The same
// bookkeeping as exchange_kernel for an accepted pair.
__global__ void apply_exchange_kernel(StateDev S, const double* __restrict__ in, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const double vs = in[2 * R + r], us = in[3 * R + r];
  if (vs != 1.0) {
    const double K = S.K[r], Kn = K * (vs * vs);
    S.econs[r] += K - Kn;
    S.K[r] = Kn;
    S.vscale[r] *= vs;
  }
  if (us != 1.0) {
    const double U = S.U[r], Un = U * us;
    S.econs[r] += U - Un;
    S.U[r] = Un;
    S.fscale[r] *= us;
  }
  S.T[r] = in[r];
  S.lam[r] = in[R + r];
}

// ------------------------------------------------------------------ state I/O
__global__ void apply_vscale_kernel(StateDev S, const RepDev* __restrict__ reps,
                                    const EnsDev* __restrict__ ens, int r0) {
  const int r = r0 + blockIdx.y;
  const RepDev rd = reps[r];
  const int N = ens[rd.ens].N;
  const double vs = S.vscale[r];
  const double fs = S.fscale ? S.fscale[r] : 1.0;
  if (vs == 1.0 && fs == 1.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int g = rd.atom_off + i;
    if (S.vfix) {
      // the same words and rounding as the batched kernel's launch start
      vfix_put(S.vx, g, vfix_scale(vfix_get(S.vx, g), vs));
      vfix_put(S.vy, g, vfix_scale(vfix_get(S.vy, g), vs));
      vfix_put(S.vz, g, vfix_scale(vfix_get(S.vz, g), vs));
      hfix_put(S.fx, g, hfix_scale(hfix_get(S.fx, g), fs));
      hfix_put(S.fy, g, hfix_scale(hfix_get(S.fy, g), fs));
      hfix_put(S.fz, g, hfix_scale(hfix_get(S.fz, g), fs));
      continue;
    }
    S.vx[g] *= vs;
    S.vy[g] *= vs;
    S.vz[g] *= vs;
    S.fx[g] *= fs;
    S.fy[g] *= fs;
    S.fz[g] *= fs;
  }
}

// resets the pending velocity and force factors (after apply_vscale_kernel)
__global__ void reset_vscale_kernel(StateDev S, int r0, int n_rep) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_rep) {
    S.vscale[r0 + r] = 1.0;
    if (S.fscale) S.fscale[r0 + r] = 1.0;
  }
}

__global__ void export_kernel(StateDev S, const EnsDev* __restrict__ ens,
                              const RepDev* __restrict__ reps, double* x, double* v, double* f) {
  const int r = blockIdx.y;
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < E.N; i += gridDim.x * blockDim.x) {
    const int g = rd.atom_off + i;
    // original order (no permutation array: slots are the original order)
    const size_t o = (size_t)rd.atom_off + (S.perm ? S.perm[g] : i);
    if (x) {
      const uint64_t q[3] = {S.qx[g], S.qy[g], S.qz[g]};
      for (int d = 0; d < 3; ++d) {
        double xv = fix_to_double(q[d], E.L);
        if (xv >= E.L) xv -= E.L;  // rounding of a word just below 2^64
        x[3 * o + d] = xv;
      }
    }
    if (v) {
      v[3 * o + 0] = S.vfix ? vfix_to_double(vfix_get(S.vx, g)) : S.vx[g];
      v[3 * o + 1] = S.vfix ? vfix_to_double(vfix_get(S.vy, g)) : S.vy[g];
      v[3 * o + 2] = S.vfix ? vfix_to_double(vfix_get(S.vz, g)) : S.vz[g];
    }
    if (f) {
      // mixed path: F = (dt/2 F) / (dt/2), the half-kick increment scaled back
      f[3 * o + 0] = S.vfix ? (double)hfix_get(S.fx, g) * E.kc.inv_hdt : S.fx[g];
      f[3 * o + 1] = S.vfix ? (double)hfix_get(S.fy, g) * E.kc.inv_hdt : S.fy[g];
      f[3 * o + 2] = S.vfix ? (double)hfix_get(S.fz, g) * E.kc.inv_hdt : S.fz[g];
    }
  }
}

__global__ void import_kernel(StateDev S, const EnsDev* __restrict__ ens,
                              const RepDev* __restrict__ reps, const double* x, const double* v) {
  const int r = blockIdx.y;
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const double inv_l = 1.0 / E.L;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < E.N; i += gridDim.x * blockDim.x) {
    const int g = rd.atom_off + i;
    // original order (no permutation array: slots are the original order)
    const size_t o = (size_t)rd.atom_off + (S.perm ? S.perm[g] : i);
    if (x) {
      S.qx[g] = fix_from_double(x[3 * o + 0], inv_l);
      S.qy[g] = fix_from_double(x[3 * o + 1], inv_l);
      S.qz[g] = fix_from_double(x[3 * o + 2], inv_l);
    }
    if (v) {
      if (S.vfix) {
        vfix_put(S.vx, g, vfix_from_double(v[3 * o + 0]));
        vfix_put(S.vy, g, vfix_from_double(v[3 * o + 1]));
        vfix_put(S.vz, g, vfix_from_double(v[3 * o + 2]));
      } else {
        S.vx[g] = v[3 * o + 0];
        S.vy[g] = v[3 * o + 1];
        S.vz[g] = v[3 * o + 2];
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.valid[r] = 0;
    S.vscale[r] = 1.0;
    if (S.fscale) S.fscale[r] = 1.0;
    S.status[r] = 0;
  }
}

// ------------------------------------------------------------------ spatial sort
// Order of the atoms of one replica by cell (the list cells, or 4 per side
// when the replica has none), ties by current slot: the same counting sort as
// the list build.  One CTA per replica.
__global__ void sort_order_kernel(StateDev S, const EnsDev* __restrict__ ens,
                                  const RepDev* __restrict__ reps, int max_ncell) {
  extern __shared__ __align__(16) unsigned char sh[];
  __shared__ int scr[64];
  const int r = blockIdx.x;
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const int N = E.N;
  const int nc = E.nc > 0 ? E.nc : 4;
  uint4* spos = reinterpret_cast<uint4*>(sh);
  Hi3* hp = reinterpret_cast<Hi3*>(spos + N);
  int* cstart = reinterpret_cast<int*>(hp + N);
  int* ccnt = cstart + (max_ncell + 1);
  uint16_t* acell = reinterpret_cast<uint16_t*>(ccnt + (max_ncell + 1));
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int g = rd.atom_off + i;
    hp[i] = Hi3{(uint32_t)(S.qx[g] >> 32), (uint32_t)(S.qy[g] >> 32), (uint32_t)(S.qz[g] >> 32)};
  }
  __syncthreads();
  auto hi_of = [&](int i) { return hp[i]; };
  cta_build_cells(hi_of, N, nc, cstart, ccnt, spos, acell, scr);
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    S.order[rd.atom_off + k] = rd.atom_off + (int)spos[k].w;
}

__global__ void identity_perm_kernel(StateDev S, const EnsDev* __restrict__ ens,
                                     const RepDev* __restrict__ reps) {
  const int r = blockIdx.y;
  const RepDev rd = reps[r];
  const int N = ens[rd.ens].N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    S.perm[rd.atom_off + i] = i;
}

// staging copy in the new order: positions, velocities, permutation
__global__ void sort_gather_kernel(StateDev S, int64_t n_atoms) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_atoms) return;
  const int src = S.order[g];
  S.sbuf[7 * g + 0] = S.qx[src];
  S.sbuf[7 * g + 1] = S.qy[src];
  S.sbuf[7 * g + 2] = S.qz[src];
  S.sbuf[7 * g + 3] = (uint64_t)__double_as_longlong(S.vx[src]);
  S.sbuf[7 * g + 4] = (uint64_t)__double_as_longlong(S.vy[src]);
  S.sbuf[7 * g + 5] = (uint64_t)__double_as_longlong(S.vz[src]);
  S.sbuf[7 * g + 6] = (uint64_t)(uint32_t)S.perm[src];
}

__global__ void sort_scatter_kernel(StateDev S, int64_t n_atoms, int n_rep) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n_atoms) {
    S.qx[g] = S.sbuf[7 * g + 0];
    S.qy[g] = S.sbuf[7 * g + 1];
    S.qz[g] = S.sbuf[7 * g + 2];
    S.vx[g] = __longlong_as_double((long long)S.sbuf[7 * g + 3]);
    S.vy[g] = __longlong_as_double((long long)S.sbuf[7 * g + 4]);
    S.vz[g] = __longlong_as_double((long long)S.sbuf[7 * g + 5]);
    S.perm[g] = (int32_t)(uint32_t)S.sbuf[7 * g + 6];
  }
  if (g < n_rep) S.valid[g] = 0;  // lists and forces are rebuilt by the next launch
}

}  // namespace

// ====================================================================== host
cudaError_t launch_init_lattice(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, int max_threads, cudaStream_t st) {
  if (n_rep <= 0) return cudaSuccess;
  init_lattice_kernel<<<n_rep, max_threads, 0, st>>>(s, d_ens, d_rep);
  return cudaGetLastError();
}

size_t batched_smem_bytes(int max_n, int max_ncell, int threads, bool fp64, size_t list_elems) {
  return batched_layout(max_n, max_ncell, threads, fp64, list_elems, nullptr, nullptr);
}


int batched_max_active_clusters(bool fp64, const LaunchCfg& cfg, int max_n, int max_ncell) {
#define RE_MC(F, PP)                                                                   \
  return cfg.threads <= kNarrowThreads                                                   \
             ? max_active_clusters_t<F, PP, false, kNarrowThreads>(cfg, max_n, max_ncell, 0) \
             : max_active_clusters_t<F, PP, false, 1024>(cfg, max_n, max_ncell, 0);
#define RE_MCP(F)             \
  switch (cfg.atom_threads) { \
    case 1: RE_MC(F, 1)       \
    case 2: RE_MC(F, 2)       \
    case 4: RE_MC(F, 4)       \
    case 8: RE_MC(F, 8)       \
  }
  if (fp64) {
    RE_MCP(true)
  } else {
    RE_MCP(false)
  }
#undef RE_MCP
#undef RE_MC
  return 0;
}

__global__ void split_work_kernel(const double* __restrict__ T, int R, int wide_n, int* work) {
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    const double t = T[a];
    int rank = 0;  // replicas hotter than a (ties: lower index first)
    for (int b = 0; b < R; ++b) {
      const double u = T[b];
      rank += (u > t) || (u == t && b < a);
    }
    work[rank < wide_n ? R - wide_n + rank : rank - wide_n] = a;
  }
}

cudaError_t launch_split_work(const double* T, int R, int wide_n, int* work, cudaStream_t st) {
  split_work_kernel<<<1, 256, 0, st>>>(T, R, wide_n, work);
  return cudaGetLastError();
}

// Longest job first: the replicas of [r0, r0 + n) ordered by decreasing
// budget x atoms, ties by index; work[r0 + rank] = replica.  One block: the
// (key, replica) pairs are bitonic-sorted in shared memory (n <= kOrderMax).
constexpr int kOrderMax = 4096;

__global__ void __launch_bounds__(1024) order_work_kernel(const int32_t* __restrict__ budget,
                                                          const RepDev* __restrict__ reps,
                                                          const EnsDev* __restrict__ ens, int r0,
                                                          int n, int* work) {
  __shared__ long long key[kOrderMax];
  __shared__ int idx[kOrderMax];
  int m = 1;
  while (m < n) m <<= 1;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    // larger work first: sort ascending on the negated work; padding last
    key[t] = t < n ? -(long long)budget[r0 + t] * ens[reps[r0 + t].ens].N : LLONG_MAX;
    idx[t] = r0 + t;
  }
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const bool up = (t & k) == 0;  // this block of k sorts ascending
          const long long ka = key[t], kb = key[u];
          const int ia = idx[t], ib = idx[u];
          const bool greater = ka > kb || (ka == kb && ia > ib);
          if (greater == up) {
            key[t] = kb;
            key[u] = ka;
            idx[t] = ib;
            idx[u] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) work[r0 + t] = idx[t];
}

cudaError_t launch_order_work(const int32_t* budget, const RepDev* d_rep, const EnsDev* d_ens,
                              int r0, int n, int* work, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kOrderMax) return cudaErrorInvalidValue;
  order_work_kernel<<<1, 1024, 0, st>>>(budget, d_rep, d_ens, r0, n, work);
  return cudaGetLastError();
}

__global__ void attempt_add_kernel(StateDev S, int n_ens, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n_ens) S.attempt[e] += n;
}

cudaError_t launch_attempt_add(const StateDev& s, int n_ens, int n, cudaStream_t st) {
  attempt_add_kernel<<<(n_ens + 127) / 128, 128, 0, st>>>(s, n_ens, n);
  return cudaGetLastError();
}

cudaError_t launch_batched(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                           const int* d_work, int n_work, const int32_t* d_budget, bool fp64,
                           const LaunchCfg& cfg, int max_n, int max_ncell, size_t list_elems,
                           int async_nx, cudaStream_t st, const FreeDev* fr) {
  if (n_work <= 0) return cudaSuccess;
  const bool lsm = list_elems > 0;
  const int mode = (fr && fr->nx > 0) ? 2 : (async_nx > 0 ? 1 : 0);
  // the two free-running modes keep the lists in global memory
  if (mode != 0 && lsm) return cudaErrorInvalidValue;
#define RE_LB(F, PP, LS, M)                                                                   \
  return cfg.threads <= kNarrowThreads                                                         \
             ? launch_batched_t<F, PP, LS, M, kNarrowThreads>(s, d_ens, d_rep, d_work, n_work, \
                                                              d_budget, cfg, max_n, max_ncell, \
                                                              list_elems, async_nx, st, fr)    \
             : launch_batched_t<F, PP, LS, M, 1024>(s, d_ens, d_rep, d_work, n_work, d_budget, \
                                                    cfg, max_n, max_ncell, list_elems,         \
                                                    async_nx, st, fr);
#define RE_LBP(F, LS, M)                           \
  switch (cfg.atom_threads) {                      \
    case 1: RE_LB(F, 1, LS, M)                     \
    case 2: RE_LB(F, 2, LS, M)                     \
    case 4: RE_LB(F, 4, LS, M)                     \
    case 8: RE_LB(F, 8, LS, M)                     \
  }
  if (mode == 1) {
    if (fp64) { RE_LBP(true, false, 1) } else { RE_LBP(false, false, 1) }
  } else if (mode == 2) {
    if (fp64) { RE_LBP(true, false, 2) } else { RE_LBP(false, false, 2) }
  } else if (fp64) {
    if (lsm) { RE_LBP(true, true, 0) } else { RE_LBP(true, false, 0) }
  } else {
    if (lsm) { RE_LBP(false, true, 0) } else { RE_LBP(false, false, 0) }
  }
#undef RE_LBP
#undef RE_LB
  return cudaErrorInvalidValue;
}

cudaError_t launch_plain_advance(const StateDev& s, const EnsDev& e, const RepDev& rd, int r,
                                 const EnsDev* d_ens, const RepDev* d_rep, int steps,
                                 int max_ncell, cudaStream_t st, int refresh) {
  const int N = e.N;
  const int tb = 128;
  const int nb = (N + tb - 1) / tb;
  const int ncell = e.nc > 0 ? e.nc * e.nc * e.nc : 0;
  (void)max_ncell;
  (void)rd;
  const size_t rsmem = (size_t)N * (16 + sizeof(Hi3)) + (size_t)(ncell + 1) * 8 + (size_t)N * 2 + 64;
  cudaError_t err = cudaFuncSetAttribute(plain_rebuild, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rsmem);
  if (err != cudaSuccess) return err;
  if (refresh) {
    // Prologue after creation or an external state change: lists (the list
    // is invalid, so plain_rebuild rebuilds), forces, U and K.
    plain_rebuild<<<1, 1024, rsmem, st>>>(s, d_ens, d_rep, r, ncell);
    plain_forces<<<nb, tb, 0, st>>>(s, d_ens, d_rep, r);
    plain_kick<<<nb, tb, 0, st>>>(s, d_ens, d_rep, r, 0);
    plain_thermo<<<1, 32, 0, st>>>(s, d_ens, d_rep, r, nb, 0);
  }
  for (int k = 0; k < steps; ++k) {
    plain_kick_drift<<<(N + 255) / 256, 256, 0, st>>>(s, d_ens, d_rep, r);
    plain_rebuild<<<1, 1024, rsmem, st>>>(s, d_ens, d_rep, r, ncell);
    plain_forces<<<nb, tb, 0, st>>>(s, d_ens, d_rep, r);
    plain_kick<<<nb, tb, 0, st>>>(s, d_ens, d_rep, r, 1);
    plain_thermo<<<1, 32, 0, st>>>(s, d_ens, d_rep, r, nb, 1);
  }
  if (steps > 0) {
    // the last thermostat factor becomes part of the stored velocities
    apply_vscale_kernel<<<dim3((N + 255) / 256, 1), 256, 0, st>>>(s, d_rep, d_ens, r);
    reset_vscale_kernel<<<1, 32, 0, st>>>(s, r, 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_exchange(const StateDev& s, const double* d_in, int R, cudaStream_t st) {
  apply_exchange_kernel<<<(R + 127) / 128, 128, 0, st>>>(s, d_in, R);
  return cudaGetLastError();
}

cudaError_t launch_exchange(const StateDev& s, const EnsDev* d_ens, int n_ens, int max_r,
                            int32_t* d_partner, uint8_t* d_acc, cudaStream_t st, double* d_rec,
                            int rtot) {
  if (max_r > kRankSortMax) {
    // one cluster per ensemble: about 128 replicas per CTA, at most 8 CTAs
    const int C = std::min(8, (max_r + 127) / 128);
    const int threads = 512;
    const size_t smem = (size_t)max_r * (sizeof(long long) + sizeof(int));
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(exchange_cluster_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3((unsigned)(n_ens * C));
    lc.blockDim = dim3((unsigned)threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, exchange_cluster_kernel, s, d_ens, d_partner, d_acc, d_rec,
                              rtot);
  }
  const size_t smem = exchange_smem_bytes(max_r);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(exchange_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int threads = max_r >= 512 ? 512 : ((max_r + 31) / 32) * 32;
  exchange_kernel<<<n_ens, threads, smem, st>>>(s, d_ens, d_partner, d_acc, d_rec, rtot);
  return cudaGetLastError();
}

cudaError_t launch_apply_vscale(const StateDev& s, const RepDev* d_rep, const EnsDev* d_ens,
                                int n_rep, cudaStream_t st) {
  if (n_rep <= 0) return cudaSuccess;
  apply_vscale_kernel<<<dim3(64, n_rep), 256, 0, st>>>(s, d_rep, d_ens, 0);
  reset_vscale_kernel<<<(n_rep + 255) / 256, 256, 0, st>>>(s, 0, n_rep);
  return cudaGetLastError();
}

cudaError_t launch_export_state(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, double* d_x, double* d_v, double* d_f,
                                cudaStream_t st) {
  if (n_rep <= 0) return cudaSuccess;
  export_kernel<<<dim3(32, n_rep), 256, 0, st>>>(s, d_ens, d_rep, d_x, d_v, d_f);
  return cudaGetLastError();
}

cudaError_t launch_import_state(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, const double* d_x, const double* d_v,
                                cudaStream_t st) {
  if (n_rep <= 0) return cudaSuccess;
  import_kernel<<<dim3(32, n_rep), 256, 0, st>>>(s, d_ens, d_rep, d_x, d_v);
  return cudaGetLastError();
}

cudaError_t launch_identity_perm(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                 int n_rep, cudaStream_t st) {
  if (n_rep <= 0 || !s.perm) return cudaSuccess;
  identity_perm_kernel<<<dim3(16, n_rep), 256, 0, st>>>(s, d_ens, d_rep);
  return cudaGetLastError();
}

cudaError_t launch_spatial_sort(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, int max_n, int max_ncell, int64_t n_atoms,
                                cudaStream_t st) {
  if (n_rep <= 0) return cudaSuccess;
  const int mc = std::max(max_ncell, 64);
  const size_t smem = (size_t)max_n * (16 + sizeof(Hi3)) + (size_t)(mc + 1) * 8 +
                      (size_t)max_n * 2 + 64;
  cudaError_t e = cudaFuncSetAttribute(sort_order_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  sort_order_kernel<<<n_rep, 1024, smem, st>>>(s, d_ens, d_rep, mc);
  const int nb = (int)((n_atoms + 255) / 256);
  sort_gather_kernel<<<nb, 256, 0, st>>>(s, n_atoms);
  sort_scatter_kernel<<<std::max(nb, (n_rep + 255) / 256), 256, 0, st>>>(s, n_atoms, n_rep);
  return cudaGetLastError();
}

cudaError_t launch_exchange_raw(int R, const double* T, const double* lam, const double* U,
                                uint64_t seed, int64_t attempt, int parity_mode, int distance,
                                double* T_out, double* lam_out, int32_t* partner,
                                uint8_t* accepted, double* vscale, double* uscale,
                                cudaStream_t st) {
  const size_t smem = sort_keys_bytes(R);
  const int threads = R >= 512 ? 512 : ((R + 31) / 32) * 32;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(exchange_raw_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  exchange_raw_kernel<<<1, threads, smem, st>>>(R, T, lam, U, seed, attempt, parity_mode, distance,
                                               T_out, lam_out, partner, accepted, vscale, uscale);
  return cudaGetLastError();
}

}  // namespace re
