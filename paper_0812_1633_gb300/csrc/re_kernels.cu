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
#include <cooperative_groups.h>

#include "re_device.cuh"
#include "re_internal.h"

namespace cg = cooperative_groups;

namespace re {

namespace {

constexpr int kMaxCluster = 8;
constexpr int kMaxWarps = 32;
constexpr int kPlainRed = 1024;  // per-replica reduction slots of the plain path

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
    S.qx[g] = fix_from_double(x, inv_l);
    S.qy[g] = fix_from_double(y, inv_l);
    S.qz[g] = fix_from_double(z, inv_l);
    const Uni4 u = uniforms(E.seed, (uint64_t)rd.id, (uint64_t)i, kTagVel, 0ull);
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
    S.vx[g] *= scale;
    S.vy[g] *= scale;
    S.vz[g] *= scale;
  }
  if (threadIdx.x == 0) {
    S.K[r] = K * scale * scale;
    S.U[r] = 0.0;
    S.econs[r] = 0.0;
    S.vscale[r] = 1.0;
    S.step[r] = 0;
    S.nreb[r] = 0;
    S.status[r] = 0;
    S.valid[r] = 0;
  }
}

// ------------------------------------------------------------------ cells
// Top 32 bits of a position (enough for binning and list radii).
struct Hi3 {
  uint32_t x, y, z;
};

__device__ __forceinline__ int cell_of(Hi3 p, int nc) {
  return ((int)__umulhi(p.x, (uint32_t)nc) * nc + (int)__umulhi(p.y, (uint32_t)nc)) * nc +
         (int)__umulhi(p.z, (uint32_t)nc);
}

// Exclusive scan of cnt[0..n) into start[0..n], start[n] = total.  Whole block.
__device__ void block_exclusive_scan(const int* cnt, int* start, int n, int* scratch) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (T + 31) >> 5;
  const int per = (n + T - 1) / T;
  const int lo = min(n, tid * per), hi = min(n, lo + per);
  int s = 0;
  for (int c = lo; c < hi; ++c) s += cnt[c];
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < warp; ++w) off += scratch[w];
  int run = off + incl - s;
  for (int c = lo; c < hi; ++c) {
    start[c] = run;
    run += cnt[c];
  }
  if (tid == T - 1) {
    int tot = 0;
    for (int w = 0; w < nw; ++w) tot += scratch[w];
    start[n] = tot;
  }
  __syncthreads();
}

// Cell binning and counting sort of all N atoms of a replica (whole block):
// cstart[c]..cstart[c+1] index catoms, the atoms of cell c in increasing
// index order (cells x-major, as ((cx * nc) + cy) * nc + cz).
template <class PosFn>
__device__ void cta_build_cells(PosFn pos_hi, int N, int nc, int* cstart, int* ccnt,
                                uint16_t* catoms, uint16_t* acell, int* scratch) {
  const int T = blockDim.x, tid = threadIdx.x;
  const int ncell = nc * nc * nc;
  for (int c = tid; c < ncell; c += T) ccnt[c] = 0;
  __syncthreads();
  for (int i = tid; i < N; i += T) {
    const int c = cell_of(pos_hi(i), nc);
    acell[i] = (uint16_t)c;
    atomicAdd(&ccnt[c], 1);
  }
  __syncthreads();
  block_exclusive_scan(ccnt, cstart, ncell, scratch);
  for (int c = tid; c < ncell; c += T) ccnt[c] = cstart[c];
  __syncthreads();
  for (int i = tid; i < N; i += T) {
    const int k = atomicAdd(&ccnt[acell[i]], 1);
    catoms[k] = (uint16_t)i;
  }
  __syncthreads();
  for (int c = tid; c < ncell; c += T) {
    const int b = cstart[c], e = cstart[c + 1];
    for (int k = b + 1; k < e; ++k) {
      const uint16_t v = catoms[k];
      int j = k - 1;
      while (j >= b && catoms[j] > v) {
        catoms[j + 1] = catoms[j];
        --j;
      }
      catoms[j + 1] = v;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float sep2_hi(Hi3 a, Hi3 b) {
  const float dx = (float)(int)(b.x - a.x), dy = (float)(int)(b.y - a.y),
              dz = (float)(int)(b.z - a.z);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Verlet list of atom i: every j != i closer than the list radius (squared,
// in units of (L / 2^32)^2), scanned over the (2m+1)^3 neighbour cells (or
// all atoms when nc == 0).  Entry k goes to nb[((k/4) * N + i) * 4 + k%4].
// Returns the count; sets *overflow when more than cap were found.
template <class PosFn>
__device__ int build_atom_list(int i, PosFn pos_hi, int N, int nc, int m, const int* cstart,
                               const uint16_t* catoms, float rl2u, uint16_t* nb, int cap,
                               int* overflow) {
  const Hi3 pi = pos_hi(i);
  int cnt = 0;
  if (nc == 0) {
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      if (sep2_hi(pi, pos_hi(j)) < rl2u) {
        if (cnt < cap) nb[((size_t)(cnt >> 2) * N + i) * 4 + (cnt & 3)] = (uint16_t)j;
        ++cnt;
      }
    }
  } else {
    const int cx = (int)__umulhi(pi.x, (uint32_t)nc), cy = (int)__umulhi(pi.y, (uint32_t)nc),
              cz = (int)__umulhi(pi.z, (uint32_t)nc);
    for (int ox = -m; ox <= m; ++ox) {
      const int x = (cx + ox + nc) % nc;
      for (int oy = -m; oy <= m; ++oy) {
        const int y = (cy + oy + nc) % nc;
        for (int oz = -m; oz <= m; ++oz) {
          const int z = (cz + oz + nc) % nc;
          const int c = (x * nc + y) * nc + z;
          const int e = cstart[c + 1];
          for (int k = cstart[c]; k < e; ++k) {
            const int j = catoms[k];
            if (j == i) continue;
            if (sep2_hi(pi, pos_hi(j)) < rl2u) {
              if (cnt < cap) nb[((size_t)(cnt >> 2) * N + i) * 4 + (cnt & 3)] = (uint16_t)j;
              ++cnt;
            }
          }
        }
      }
    }
  }
  if (cnt > cap) {
    *overflow = 1;
    cnt = cap;
  }
  return cnt;
}

// ------------------------------------------------------------------ forces
// Mixed precision pair loop of atom i.  Separations are exact 32-bit integer
// minimum images (units lam = L / 2^32) converted to FP32 once; the pair force
// and energy are FP32; the per-atom sums are FP32 over this atom's list and
// are folded into FP64 by the caller.  Force on i from j = fs * d with
// fs = s^4 (24 - 48 s^3), s = 1/r^2 (sigma units); pair energy 4 s^3 (s^3 - 1).
struct MixedAcc {
  float fx, fy, fz, e;
  int nin;
};

__device__ __forceinline__ void mixed_pair(uint4 pi, uint4 pj, float rc2u, float inv_lam2,
                                           MixedAcc& a) {
  const float dx = i32_to_f32_split((int)(pj.x - pi.x));
  const float dy = i32_to_f32_split((int)(pj.y - pi.y));
  const float dz = (float)(int)(pj.z - pi.z);
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  if (r2 < rc2u) {
    const float s = rcp_approx(r2) * inv_lam2;
    const float s3 = s * s * s;
    const float fs = (s * s3) * fmaf(-48.0f, s3, 24.0f);
    a.fx = fmaf(fs, dx, a.fx);
    a.fy = fmaf(fs, dy, a.fy);
    a.fz = fmaf(fs, dz, a.fz);
    a.e = fmaf(s3, fmaf(4.0f, s3, -4.0f), a.e);
    a.nin += 1;
  }
}

__device__ __forceinline__ MixedAcc mixed_atom_forces(int i, const uint4* __restrict__ pos,
                                                      const uint16_t* __restrict__ nb, int N,
                                                      int cnt, float rc2u, float inv_lam2) {
  MixedAcc a{0.f, 0.f, 0.f, 0.f, 0};
  const uint4 pi = pos[i];
  const int nblk = (cnt + 3) >> 2;
  for (int kb = 0; kb < nblk; ++kb) {
    const uint2 w = *reinterpret_cast<const uint2*>(nb + ((size_t)kb * N + i) * 4);
    const int rem = cnt - 4 * kb;
    const uint4 p0 = pos[w.x & 0xFFFFu];
    const uint4 p1 = pos[rem > 1 ? (w.x >> 16) : i];
    const uint4 p2 = pos[rem > 2 ? (w.y & 0xFFFFu) : i];
    const uint4 p3 = pos[rem > 3 ? (w.y >> 16) : i];
    mixed_pair(pi, p0, rc2u, inv_lam2, a);
    if (rem > 1) mixed_pair(pi, p1, rc2u, inv_lam2, a);
    if (rem > 2) mixed_pair(pi, p2, rc2u, inv_lam2, a);
    if (rem > 3) mixed_pair(pi, p3, rc2u, inv_lam2, a);
  }
  return a;
}

// FP64 pair loop of atom i: separations are exact 64-bit minimum images
// converted to double (units L / 2^64), pair force and energy in FP64.
struct Pos64 {
  uint64_t x, y, z, w;
};

__device__ __forceinline__ void fp64_atom_forces(int i, Pos64 pi, const Pos64* pos,
                                                 const uint16_t* nb, int N, int cnt, double lam64,
                                                 double rc2, double uc, double& fx, double& fy,
                                                 double& fz, double& e) {
  fx = fy = fz = e = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const int j = nb[((size_t)(k >> 2) * N + i) * 4 + (k & 3)];
    const Pos64 pj = pos[j];
    const double dx = (double)(long long)(pj.x - pi.x) * lam64;
    const double dy = (double)(long long)(pj.y - pi.y) * lam64;
    const double dz = (double)(long long)(pj.z - pi.z) * lam64;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < rc2) {
      const double s = 1.0 / r2;
      const double s3 = s * s * s;
      const double fs = 48.0 * s3 * s3 * s - 24.0 * s3 * s;
      fx -= fs * dx;
      fy -= fs * dy;
      fz -= fs * dz;
      e += 4.0 * (s3 * s3 - s3) - uc;
    }
  }
}

// ------------------------------------------------------------------ batched
struct StepConst {
  double lam32, lam64, inv_l, dtq, hdt, uc, rc2, c_th, kbar;
  float rc2u, rl2u, half2u, inv_lam2;
  int nf;
};

__device__ __forceinline__ StepConst step_const(const EnsDev& E, double T) {
  StepConst k;
  k.lam32 = E.L * 0x1.0p-32;
  k.lam64 = E.L * 0x1.0p-64;
  k.inv_l = 1.0 / E.L;
  k.dtq = E.dt * 0x1.0p64 / E.L;
  k.hdt = 0.5 * E.dt;
  const double rc6 = E.rc * E.rc * E.rc * E.rc * E.rc * E.rc;
  k.uc = E.shift ? 4.0 * (1.0 / (rc6 * rc6) - 1.0 / rc6) : 0.0;
  k.rc2 = E.rc * E.rc;
  const double rcu = E.rc / k.lam32;
  k.rc2u = (float)(rcu * rcu);
  const double rlu = E.rlist * (1.0 + 1e-6) / k.lam32;
  k.rl2u = (float)(rlu * rlu);
  const double hu = 0.5 * E.skin * (1.0 - 1e-6) / k.lam32;
  k.half2u = (float)(hu * hu);
  k.inv_lam2 = (float)(1.0 / (k.lam32 * k.lam32));
  k.nf = 3 * E.N - 3;
  k.c_th = E.tau > 0.0 ? exp(-E.dt / E.tau) : 1.0;
  k.kbar = 0.5 * k.nf * T;
  return k;
}

struct BatchedSmem {
  void* pos;      // uint4[N] (mixed) or Pos64[N] (fp64)
  int* cstart;    // ncell + 1
  int* ccnt;      // ncell
  uint16_t* catoms;
  uint16_t* acell;
  double2* noise; // threads
  float* slot_md; // [cluster][warps]
  double* slot_uk;// [cluster][warps][2]
  int* slot_st;   // [cluster]
  double* red;    // 64
  int* iscr;      // 64
  double* bcast;  // 8
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline size_t batched_layout(int max_n, int max_ncell, int threads, bool fp64,
                                                 unsigned char* base, BatchedSmem* out) {
  size_t off = 0;
  auto take = [&](size_t bytes, size_t al) {
    off = align_up(off, al);
    size_t o = off;
    off += bytes;
    return o;
  };
  const size_t o_pos = take((size_t)max_n * (fp64 ? 32 : 16), 32);
  const size_t o_noise = take((size_t)threads * 16, 16);
  const size_t o_uk = take((size_t)kMaxCluster * kMaxWarps * 2 * 8, 16);
  const size_t o_red = take(64 * 8, 8);
  const size_t o_bc = take(8 * 8, 8);
  const size_t o_md = take((size_t)kMaxCluster * kMaxWarps * 4, 4);
  const size_t o_st = take(kMaxCluster * 4, 4);
  const size_t o_isc = take(64 * 4, 4);
  const size_t o_cs = take((size_t)(max_ncell + 1) * 4, 4);
  const size_t o_cc = take((size_t)(max_ncell + 1) * 4, 4);
  const size_t o_ca = take((size_t)max_n * 2, 2);
  const size_t o_ac = take((size_t)max_n * 2, 2);
  if (out) {
    out->pos = base + o_pos;
    out->noise = reinterpret_cast<double2*>(base + o_noise);
    out->slot_uk = reinterpret_cast<double*>(base + o_uk);
    out->red = reinterpret_cast<double*>(base + o_red);
    out->bcast = reinterpret_cast<double*>(base + o_bc);
    out->slot_md = reinterpret_cast<float*>(base + o_md);
    out->slot_st = reinterpret_cast<int*>(base + o_st);
    out->iscr = reinterpret_cast<int*>(base + o_isc);
    out->cstart = reinterpret_cast<int*>(base + o_cs);
    out->ccnt = reinterpret_cast<int*>(base + o_cc);
    out->catoms = reinterpret_cast<uint16_t*>(base + o_ca);
    out->acell = reinterpret_cast<uint16_t*>(base + o_ac);
  }
  return align_up(off, 128);
}

struct KernelDims {
  int max_n, max_ncell;
};

// One thread-block cluster per replica (work item).  CTA `crank` of the
// cluster owns atoms [i0, i1) and keeps the positions of all N atoms of the
// replica in its shared memory; each step it broadcasts its own atoms' new
// positions to every CTA of the cluster.  Two cluster barriers per step: after
// the drift (positions and displacement maxima visible) and after the second
// kick (energy partial sums visible; all position reads of the step done).
template <bool FP64>
__global__ void __launch_bounds__(512, 1) md_batched_kernel(StateDev S,
                                                          const EnsDev* __restrict__ ens,
                                                          const RepDev* __restrict__ reps,
                                                          const int* __restrict__ work,
                                                          const int32_t* __restrict__ budget,
                                                          KernelDims dims) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int r = work[blockIdx.x / C];
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const int N = E.N, T = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nw = (T + 31) >> 5;
  const int B = budget[r];
  const int status0 = S.status[r];
  const int valid0 = S.valid[r];
  double vs = S.vscale[r];
  double econs = S.econs[r];
  const double Ttarget = S.T[r];
  const int64_t step0 = S.step[r];

  extern __shared__ __align__(128) unsigned char smem_raw[];
  BatchedSmem sm;
  batched_layout(dims.max_n, dims.max_ncell, T, FP64, smem_raw, &sm);
  uint4* posm = reinterpret_cast<uint4*>(sm.pos);
  Pos64* pos64 = reinterpret_cast<Pos64*>(sm.pos);

  // Every CTA has read the replica's flags before any CTA may change them.
  cl.sync();
  if (status0 != 0 || (B <= 0 && valid0)) return;  // uniform over the cluster

  const StepConst K = step_const(E, Ttarget);
  const int per = (N + C - 1) / C;
  const int i0 = min(N, crank * per), i1 = min(N, i0 + per);
  const int aoff = rd.atom_off;
  uint16_t* nb = S.nbr + rd.nbr_off;

  auto hi_of = [&](int i) -> Hi3 {
    if (FP64) {
      const Pos64 p = pos64[i];
      return Hi3{(uint32_t)(p.x >> 32), (uint32_t)(p.y >> 32), (uint32_t)(p.z >> 32)};
    } else {
      const uint4 p = posm[i];
      return Hi3{p.x, p.y, p.z};
    }
  };
  auto publish = [&](int i, uint64_t qx, uint64_t qy, uint64_t qz) {
    if (FP64) {
      const Pos64 p{qx, qy, qz, 0ull};
      for (int q = 0; q < C; ++q) cl.map_shared_rank(pos64, q)[i] = p;
    } else {
      const uint4 p = make_uint4((uint32_t)(qx >> 32), (uint32_t)(qy >> 32),
                                 (uint32_t)(qz >> 32), 0u);
      for (int q = 0; q < C; ++q) cl.map_shared_rank(posm, q)[i] = p;
    }
  };

  // Rebuild of the lists of this CTA's atoms (cells built redundantly per CTA).
  int overflow = 0;
  int nreb = 0;
  auto rebuild = [&]() {
    if (E.nc > 0)
      cta_build_cells(hi_of, N, E.nc, sm.cstart, sm.ccnt, sm.catoms, sm.acell, sm.iscr);
    for (int i = i0 + tid; i < i1; i += T) {
      const int g = aoff + i;
      const int cnt = build_atom_list(i, hi_of, N, E.nc, E.m, sm.cstart, sm.catoms, K.rl2u, nb,
                                      E.cap, &overflow);
      S.ncnt[g] = cnt;
      const Hi3 p = hi_of(i);
      S.rx[g] = p.x;
      S.ry[g] = p.y;
      S.rz[g] = p.z;
    }
    ++nreb;
  };

  // Forces of this CTA's atoms (and optionally the second half kick); returns
  // this thread's partial U (per-atom energies, full list) and K (sum v^2).
  auto forces = [&](bool kick, double& u_part, double& k_part) {
    u_part = 0.0;
    k_part = 0.0;
    for (int i = i0 + tid; i < i1; i += T) {
      const int g = aoff + i;
      const int cnt = S.ncnt[g];
      double fx, fy, fz, e;
      if (FP64) {
        fp64_atom_forces(i, pos64[i], pos64, nb, N, cnt, K.lam64, K.rc2, K.uc, fx, fy, fz, e);
      } else {
        const MixedAcc a = mixed_atom_forces(i, posm, nb, N, cnt, K.rc2u, K.inv_lam2);
        fx = (double)a.fx * K.lam32;
        fy = (double)a.fy * K.lam32;
        fz = (double)a.fz * K.lam32;
        e = (double)a.e - K.uc * (double)a.nin;
      }
      S.fx[g] = fx;
      S.fy[g] = fy;
      S.fz[g] = fz;
      u_part += e;
      double vx = S.vx[g], vy = S.vy[g], vz = S.vz[g];
      if (kick) {
        vx += K.hdt * fx;
        vy += K.hdt * fy;
        vz += K.hdt * fz;
        S.vx[g] = vx;
        S.vy[g] = vy;
        S.vz[g] = vz;
      }
      k_part += vx * vx + vy * vy + vz * vz;
    }
  };

  // Publish per-warp partial sums to every CTA, then (after the barrier) warp 0
  // of each CTA sums them in a fixed order.
  auto publish_uk = [&](double u, double kk, int st) {
    u = warp_sum(u);
    kk = warp_sum(kk);
    st = warp_or(st);
    if (lane == 0) {
      for (int q = 0; q < C; ++q) {
        double* uk = cl.map_shared_rank(sm.slot_uk, q);
        uk[(crank * kMaxWarps + warp) * 2 + 0] = u;
        uk[(crank * kMaxWarps + warp) * 2 + 1] = kk;
        if (st) atomicOr(cl.map_shared_rank(sm.slot_st, q) + crank, st);
      }
    }
  };

  if (tid < C) sm.slot_st[tid] = 0;

  double U = S.U[r], Kin = S.K[r];
  int status = 0;

  if (!valid0) {
    // Prologue: apply any pending velocity factor, build lists, forces, U, K.
    for (int i = i0 + tid; i < i1; i += T) {
      const int g = aoff + i;
      if (vs != 1.0) {
        S.vx[g] *= vs;
        S.vy[g] *= vs;
        S.vz[g] *= vs;
      }
      publish(i, S.qx[g], S.qy[g], S.qz[g]);
    }
    vs = 1.0;
    cl.sync();
    rebuild();
    double u, kk;
    forces(false, u, kk);
    publish_uk(u, kk, overflow ? kStOverflow : 0);
    cl.sync();
    if (warp == 0) {
      double su = 0.0, sk = 0.0;
      for (int idx = lane; idx < C * kMaxWarps; idx += 32) {
        const int q = idx / kMaxWarps, w = idx % kMaxWarps;
        if (w < nw) {
          su += sm.slot_uk[(q * kMaxWarps + w) * 2 + 0];
          sk += sm.slot_uk[(q * kMaxWarps + w) * 2 + 1];
        }
      }
      su = warp_sum(su);
      sk = warp_sum(sk);
      if (lane == 0) {
        sm.bcast[0] = 0.5 * su;
        sm.bcast[1] = 0.5 * sk;
        int st = 0;
        for (int q = 0; q < C; ++q) st |= sm.slot_st[q];
        sm.bcast[2] = (double)st;
      }
    }
    __syncthreads();
    U = sm.bcast[0];
    Kin = sm.bcast[1];
    status = (int)sm.bcast[2];
    if (!isfinite(U) || !isfinite(Kin)) status |= kStNumeric;
  }

  int done = 0;
  for (int s = 0; s < B && status == 0; ++s) {
    const int64_t n = step0 + s;
    if (E.tau > 0.0 && (s % T) == 0 && s + tid < B) {
      int capped = 0;
      sm.noise[tid] = svr_noise(K.nf, E.seed, (uint64_t)rd.id, (uint64_t)(n + tid), &capped);
      if (capped) sm.noise[tid].y = -1.0;
    }
    // kick + drift + displacement since the last rebuild
    float md = 0.0f;
    for (int i = i0 + tid; i < i1; i += T) {
      const int g = aoff + i;
      const double vx = fma(S.vx[g], vs, K.hdt * S.fx[g]);
      const double vy = fma(S.vy[g], vs, K.hdt * S.fy[g]);
      const double vz = fma(S.vz[g], vs, K.hdt * S.fz[g]);
      S.vx[g] = vx;
      S.vy[g] = vy;
      S.vz[g] = vz;
      const uint64_t qx = S.qx[g] + (uint64_t)__double2ll_rn(vx * K.dtq);
      const uint64_t qy = S.qy[g] + (uint64_t)__double2ll_rn(vy * K.dtq);
      const uint64_t qz = S.qz[g] + (uint64_t)__double2ll_rn(vz * K.dtq);
      S.qx[g] = qx;
      S.qy[g] = qy;
      S.qz[g] = qz;
      publish(i, qx, qy, qz);
      const Hi3 ref{S.rx[g], S.ry[g], S.rz[g]};
      const Hi3 now{(uint32_t)(qx >> 32), (uint32_t)(qy >> 32), (uint32_t)(qz >> 32)};
      md = fmaxf(md, sep2_hi(ref, now));
    }
    vs = 1.0;
    md = warp_max(md);
    if (lane == 0)
      for (int q = 0; q < C; ++q) cl.map_shared_rank(sm.slot_md, q)[crank * kMaxWarps + warp] = md;
    cl.sync();  // B1
    float mdall = 0.0f;
    for (int idx = lane; idx < C * kMaxWarps; idx += 32)
      if (idx % kMaxWarps < nw) mdall = fmaxf(mdall, sm.slot_md[idx]);
    mdall = warp_max(mdall);
    if (mdall > K.half2u) rebuild();
    double u, kk;
    forces(true, u, kk);
    publish_uk(u, kk, overflow ? kStOverflow : 0);
    cl.sync();  // B2
    if (warp == 0) {
      double su = 0.0, sk = 0.0;
      for (int idx = lane; idx < C * kMaxWarps; idx += 32) {
        const int q = idx / kMaxWarps, w = idx % kMaxWarps;
        if (w < nw) {
          su += sm.slot_uk[(q * kMaxWarps + w) * 2 + 0];
          sk += sm.slot_uk[(q * kMaxWarps + w) * 2 + 1];
        }
      }
      su = warp_sum(su);
      sk = warp_sum(sk);
      if (lane == 0) {
        const double Un = 0.5 * su, Kn = 0.5 * sk;
        int st = 0;
        for (int q = 0; q < C; ++q) st |= sm.slot_st[q];
        double alpha = 1.0, Kp = Kn;
        if (E.tau > 0.0) {
          const double2 nz = sm.noise[s % T];
          if (nz.y < 0.0) st |= kStRngCap;
          alpha = svr_alpha(Kn, K.kbar, K.nf, K.c_th, nz.x, nz.y, &Kp);
        }
        if (!isfinite(Un) || !isfinite(Kp)) st |= kStNumeric;
        sm.bcast[0] = Un;
        sm.bcast[1] = Kp;
        sm.bcast[2] = alpha;
        sm.bcast[3] = Kn - Kp;
        sm.bcast[4] = (double)st;
      }
    }
    __syncthreads();
    U = sm.bcast[0];
    Kin = sm.bcast[1];
    vs = sm.bcast[2];
    econs += sm.bcast[3];
    status = (int)sm.bcast[4];
    ++done;
  }
  // Apply the last thermostat factor so that the stored velocities are final.
  if (vs != 1.0) {
    for (int i = i0 + tid; i < i1; i += T) {
      const int g = aoff + i;
      S.vx[g] *= vs;
      S.vy[g] *= vs;
      S.vz[g] *= vs;
    }
  }
  if (crank == 0 && tid == 0) {
    S.U[r] = U;
    S.K[r] = Kin;
    S.econs[r] = econs;
    S.step[r] = step0 + done;
    S.nreb[r] += nreb;
    S.vscale[r] = 1.0;
    S.status[r] = status;
    S.valid[r] = (status & kStOverflow) ? 0 : 1;
  }
  cl.sync();  // no CTA leaves while another may still touch its shared memory
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
  const StepConst K = step_const(E, 1.0);
  const double vs = S.vscale[r];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float md = 0.0f;
  if (i < E.N) {
    const int g = rd.atom_off + i;
    const double vx = fma(S.vx[g], vs, K.hdt * S.fx[g]);
    const double vy = fma(S.vy[g], vs, K.hdt * S.fy[g]);
    const double vz = fma(S.vz[g], vs, K.hdt * S.fz[g]);
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
  const StepConst K = step_const(E, 1.0);
  const bool need = !S.valid[r] || __uint_as_float(S.dmax[r]) > K.half2u;
  __syncthreads();
  if (threadIdx.x == 0) {
    S.dmax[r] = 0u;
    ovf = 0;
  }
  if (!need) return;
  const int N = E.N;
  Hi3* hp = reinterpret_cast<Hi3*>(sh);
  int* cstart = reinterpret_cast<int*>(hp + N);
  int* ccnt = cstart + (max_ncell + 1);
  uint16_t* catoms = reinterpret_cast<uint16_t*>(ccnt + (max_ncell + 1));
  uint16_t* acell = catoms + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int g = rd.atom_off + i;
    hp[i] = Hi3{(uint32_t)(S.qx[g] >> 32), (uint32_t)(S.qy[g] >> 32), (uint32_t)(S.qz[g] >> 32)};
  }
  __syncthreads();
  auto hi_of = [&](int i) { return hp[i]; };
  if (E.nc > 0) cta_build_cells(hi_of, N, E.nc, cstart, ccnt, catoms, acell, scr);
  int overflow = 0;
  uint16_t* nb = S.nbr + rd.nbr_off;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int g = rd.atom_off + i;
    S.ncnt[g] = build_atom_list(i, hi_of, N, E.nc, E.m, cstart, catoms, K.rl2u, nb, E.cap,
                                &overflow);
    S.rx[g] = hp[i].x;
    S.ry[g] = hp[i].y;
    S.rz[g] = hp[i].z;
  }
  if (overflow) atomicOr(&ovf, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    S.valid[r] = ovf ? 0 : 1;
    S.nreb[r] += 1;
    if (ovf) S.status[r] |= kStOverflow;
  }
}

// FP64 forces of one replica from its list, positions read from global memory;
// per-block energy partials to red[r][block].
__global__ void plain_forces(StateDev S, const EnsDev* __restrict__ ens,
                             const RepDev* __restrict__ reps, int r) {
  __shared__ double scr[kMaxWarps];
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  const StepConst K = step_const(E, 1.0);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < E.N) {
    const int g = rd.atom_off + i;
    const uint64_t xi = S.qx[g], yi = S.qy[g], zi = S.qz[g];
    const int cnt = S.ncnt[g];
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
    S.fx[g] = fx;
    S.fy[g] = fy;
    S.fz[g] = fz;
  }
  e = block_sum(e, scr);
  if (threadIdx.x == 0) S.red[(size_t)r * kPlainRed + blockIdx.x] = e;
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
      const double2 nz = svr_noise(nf, E.seed, (uint64_t)rd.id, (uint64_t)S.step[r], &capped);
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
// Metropolis rule of the Implementation section for the pair (a colder, b
// hotter): D = (1/T_a - 1/T_b)(U_a - U_b); accept iff D >= 0 or r < exp(D),
// r the uniform of the lower replica id for this attempt.
__device__ __forceinline__ bool metropolis(double Ta, double Tb, double Ua, double Ub,
                                           uint64_t seed, int id_lo, int64_t attempt) {
  const double d = __dmul_rn(__dsub_rn(__ddiv_rn(1.0, Ta), __ddiv_rn(1.0, Tb)), __dsub_rn(Ua, Ub));
  if (d >= 0.0) return true;
  const Uni4 u = uniforms(seed, (uint64_t)id_lo, (uint64_t)attempt, kTagExch, 0ull);
  return u.u0 < exp(d);
}

__device__ __forceinline__ int pair_offset(int mode, uint64_t seed, int64_t attempt) {
  if (mode == 0) return (int)(attempt & 1);
  const Uni4 u = uniforms(seed, ~0ull, (uint64_t)attempt, kTagParity, 0ull);
  return u.u0 < 0.5 ? 0 : 1;
}

// Sorted order of R distinct temperatures by counting (rank = number of
// smaller values, ties broken by index).  Ts, order in shared memory.
__device__ void rank_sort(const double* Ts, int* order, int R) {
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    const double t = Ts[a];
    int rank = 0;
    for (int b = 0; b < R; ++b) {
      const double u = Ts[b];
      rank += (u < t) || (u == t && b < a);
    }
    order[rank] = a;
  }
}

__global__ void exchange_kernel(StateDev S, const EnsDev* __restrict__ ens, int32_t* partner_out,
                                uint8_t* acc_out) {
  extern __shared__ __align__(16) unsigned char sh[];
  const EnsDev E = ens[blockIdx.x];
  const int R = E.R, base = E.rep_off;
  double* Ts = reinterpret_cast<double*>(sh);
  int* order = reinterpret_cast<int*>(Ts + R);
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    Ts[a] = S.T[base + a];
    if (partner_out) partner_out[base + a] = -1;
    if (acc_out) acc_out[base + a] = 0;
  }
  __syncthreads();
  rank_sort(Ts, order, R);
  __syncthreads();
  const int64_t attempt = S.attempt[blockIdx.x];
  const int p = pair_offset(E.parity_mode, E.seed, attempt);
  for (int k = p + 2 * threadIdx.x; k + 1 < R; k += 2 * blockDim.x) {
    const int a = order[k], b = order[k + 1];
    const int ga = base + a, gb = base + b;
    const double Ta = Ts[a], Tb = Ts[b];
    const bool ok = metropolis(Ta, Tb, S.U[ga], S.U[gb], E.seed, min(a, b), attempt);
    if (partner_out) {
      partner_out[ga] = b;
      partner_out[gb] = a;
    }
    S.pair_att[E.pair_off + k] += 1;
    if (ok) {
      S.pair_acc[E.pair_off + k] += 1;
      if (acc_out) acc_out[ga] = acc_out[gb] = 1;
      const double sa = sqrt(Tb / Ta), sb = sqrt(Ta / Tb);
      const double Ka = S.K[ga], Kb = S.K[gb];
      const double Kan = Ka * (sa * sa), Kbn = Kb * (sb * sb);
      S.vscale[ga] *= sa;
      S.vscale[gb] *= sb;
      S.econs[ga] += Ka - Kan;
      S.econs[gb] += Kb - Kbn;
      S.K[ga] = Kan;
      S.K[gb] = Kbn;
      S.T[ga] = Tb;
      S.T[gb] = Ta;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) S.attempt[blockIdx.x] = attempt + 1;
}

__global__ void exchange_raw_kernel(int R, const double* __restrict__ T,
                                    const double* __restrict__ U, uint64_t seed, int64_t attempt,
                                    int mode, double* T_out, int32_t* partner, uint8_t* acc,
                                    double* vscale) {
  extern __shared__ __align__(16) unsigned char sh[];
  double* Ts = reinterpret_cast<double*>(sh);
  int* order = reinterpret_cast<int*>(Ts + R);
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    Ts[a] = T[a];
    T_out[a] = T[a];
    partner[a] = -1;
    acc[a] = 0;
    vscale[a] = 1.0;
  }
  __syncthreads();
  rank_sort(Ts, order, R);
  __syncthreads();
  const int p = pair_offset(mode, seed, attempt);
  for (int k = p + 2 * threadIdx.x; k + 1 < R; k += 2 * blockDim.x) {
    const int a = order[k], b = order[k + 1];
    const double Ta = Ts[a], Tb = Ts[b];
    const bool ok = metropolis(Ta, Tb, U[a], U[b], seed, min(a, b), attempt);
    partner[a] = b;
    partner[b] = a;
    if (ok) {
      acc[a] = acc[b] = 1;
      vscale[a] = sqrt(Tb / Ta);
      vscale[b] = sqrt(Ta / Tb);
      T_out[a] = Tb;
      T_out[b] = Ta;
    }
  }
}

// ------------------------------------------------------------------ state I/O
__global__ void apply_vscale_kernel(StateDev S, const RepDev* __restrict__ reps,
                                    const EnsDev* __restrict__ ens, int r0) {
  const int r = r0 + blockIdx.y;
  const RepDev rd = reps[r];
  const int N = ens[rd.ens].N;
  const double vs = S.vscale[r];
  if (vs == 1.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int g = rd.atom_off + i;
    S.vx[g] *= vs;
    S.vy[g] *= vs;
    S.vz[g] *= vs;
  }
}

__global__ void reset_vscale_kernel(StateDev S, int r0, int n_rep) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_rep) S.vscale[r0 + r] = 1.0;
}

__global__ void export_kernel(StateDev S, const EnsDev* __restrict__ ens,
                              const RepDev* __restrict__ reps, double* x, double* v, double* f) {
  const int r = blockIdx.y;
  const RepDev rd = reps[r];
  const EnsDev E = ens[rd.ens];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < E.N; i += gridDim.x * blockDim.x) {
    const int g = rd.atom_off + i;
    if (x) {
      const uint64_t q[3] = {S.qx[g], S.qy[g], S.qz[g]};
      for (int d = 0; d < 3; ++d) {
        double xv = fix_to_double(q[d], E.L);
        if (xv >= E.L) xv -= E.L;  // rounding of a word just below 2^64
        x[3 * (size_t)g + d] = xv;
      }
    }
    if (v) {
      v[3 * (size_t)g + 0] = S.vx[g];
      v[3 * (size_t)g + 1] = S.vy[g];
      v[3 * (size_t)g + 2] = S.vz[g];
    }
    if (f) {
      f[3 * (size_t)g + 0] = S.fx[g];
      f[3 * (size_t)g + 1] = S.fy[g];
      f[3 * (size_t)g + 2] = S.fz[g];
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
    if (x) {
      S.qx[g] = fix_from_double(x[3 * (size_t)g + 0], inv_l);
      S.qy[g] = fix_from_double(x[3 * (size_t)g + 1], inv_l);
      S.qz[g] = fix_from_double(x[3 * (size_t)g + 2], inv_l);
    }
    if (v) {
      S.vx[g] = v[3 * (size_t)g + 0];
      S.vy[g] = v[3 * (size_t)g + 1];
      S.vz[g] = v[3 * (size_t)g + 2];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.valid[r] = 0;
    S.vscale[r] = 1.0;
    S.status[r] = 0;
  }
}

}  // namespace

// ====================================================================== host
cudaError_t launch_init_lattice(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                int n_rep, int max_threads, cudaStream_t st) {
  if (n_rep <= 0) return cudaSuccess;
  init_lattice_kernel<<<n_rep, max_threads, 0, st>>>(s, d_ens, d_rep);
  return cudaGetLastError();
}

size_t batched_smem_bytes(int max_n, int max_ncell, int threads, bool fp64) {
  return batched_layout(max_n, max_ncell, threads, fp64, nullptr, nullptr);
}

cudaError_t launch_batched(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                           const int* d_work, int n_work, const int32_t* d_budget, bool fp64,
                           const LaunchCfg& cfg, int max_n, int max_ncell, cudaStream_t st) {
  if (n_work <= 0) return cudaSuccess;
  const size_t smem = batched_smem_bytes(max_n, max_ncell, cfg.threads, fp64);
  const void* fn = fp64 ? (const void*)md_batched_kernel<true> : (const void*)md_batched_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)(n_work * cfg.cluster));
  lc.blockDim = dim3((unsigned)cfg.threads);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cfg.cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  KernelDims dims{max_n, max_ncell};
  if (fp64)
    e = cudaLaunchKernelEx(&lc, md_batched_kernel<true>, s, d_ens, d_rep, d_work, d_budget, dims);
  else
    e = cudaLaunchKernelEx(&lc, md_batched_kernel<false>, s, d_ens, d_rep, d_work, d_budget, dims);
  return e;
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
  const size_t rsmem = (size_t)N * sizeof(Hi3) + (size_t)(ncell + 1) * 8 + (size_t)N * 4 + 64;
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

cudaError_t launch_exchange(const StateDev& s, const EnsDev* d_ens, int n_ens, int max_r,
                            int32_t* d_partner, uint8_t* d_acc, cudaStream_t st) {
  const size_t smem = (size_t)max_r * (sizeof(double) + sizeof(int));
  const int threads = max_r >= 512 ? 512 : ((max_r + 31) / 32) * 32;
  exchange_kernel<<<n_ens, threads, smem, st>>>(s, d_ens, d_partner, d_acc);
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

cudaError_t launch_exchange_raw(int R, const double* T, const double* U, uint64_t seed,
                                int64_t attempt, int parity_mode, double* T_out,
                                int32_t* partner, uint8_t* accepted, double* vscale,
                                cudaStream_t st) {
  const size_t smem = (size_t)R * (sizeof(double) + sizeof(int));
  const int threads = R >= 512 ? 512 : ((R + 31) / 32) * 32;
  exchange_raw_kernel<<<1, threads, smem, st>>>(R, T, U, seed, attempt, parity_mode, T_out,
                                                partner, accepted, vscale);
  return cudaGetLastError();
}

}  // namespace re
