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

#include <algorithm>

#include "re_device.cuh"
#include "re_internal.h"

namespace cg = cooperative_groups;

namespace re {

namespace {

constexpr int kMaxCluster = 8;
constexpr int kMaxWarps = 32;
constexpr int kPlainRed = 1024;  // per-replica reduction slots of the plain path
constexpr int kNoiseChunk = 64;  // thermostat records prepared at a time (double buffered)
constexpr int kSvrStepBytes = 32;  // sizeof(SvrStep)

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
    S.vx[g] *= scale;
    S.vy[g] *= scale;
    S.vz[g] *= scale;
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
// cstart[c]..cstart[c+1] index spos, the atoms of cell c in increasing index
// order (cells x-major, as ((cx * nc) + cy) * nc + cz); spos[k] holds the top
// 32 bits of the position and, in .w, the atom index, so that the list build
// scans contiguous ranges with one load per candidate.
template <class PosFn>
__device__ void cta_build_cells(PosFn pos_hi, int N, int nc, int* cstart, int* ccnt, uint4* spos,
                                uint16_t* acell, int* scratch) {
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
    const Hi3 p = pos_hi(i);
    spos[k] = make_uint4(p.x, p.y, p.z, (uint32_t)i);
  }
  __syncthreads();
  for (int c = tid; c < ncell; c += T) {
    const int b = cstart[c], e = cstart[c + 1];
    for (int k = b + 1; k < e; ++k) {
      const uint4 v = spos[k];
      int j = k - 1;
      while (j >= b && spos[j].w > v.w) {
        spos[j + 1] = spos[j];
        --j;
      }
      spos[j + 1] = v;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float sep2_hi(Hi3 a, Hi3 b) {
  const float dx = (float)(int)(b.x - a.x), dy = (float)(int)(b.y - a.y),
              dz = (float)(int)(b.z - a.z);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
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

template <bool ENERGY, bool MAYBE_SELF>
__device__ __forceinline__ void mixed_pair(uint4 pi, uint4 pj, float rc2u, float inv_lam2,
                                           MixedAcc& a) {
  const float dx = (float)(int)(pj.x - pi.x);
  const float dy = (float)(int)(pj.y - pi.y);
  const float dz = (float)(int)(pj.z - pi.z);
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  // r2 == 0 only for the atom itself (sub-list padding, last block only);
  // distinct atoms at distance 0 are reported by the list build
  if (r2 < rc2u && (!MAYBE_SELF || r2 > 0.0f)) {
    const float s = rcp_approx(r2) * inv_lam2;
    const float s3 = s * s * s;
    const float fs = (s * s3) * fmaf(-48.0f, s3, 24.0f);
    a.fx = fmaf(fs, dx, a.fx);
    a.fy = fmaf(fs, dy, a.fy);
    a.fz = fmaf(fs, dz, a.fz);
    if (ENERGY) {
      a.e = fmaf(s3, fmaf(4.0f, s3, -4.0f), a.e);
      a.nin += 1;
    }
  }
}

// Positions of the FP64 path: 64-bit fixed-point words (units L / 2^64).
struct Pos64 {
  uint64_t x, y, z, w;
};

// ------------------------------------------------------------------ batched
struct BatchedSmem {
  uint16_t* nb_sm;  // this CTA's neighbour sub-lists when they fit in shared memory
  void* pos;       // uint4[N] (mixed: top 32 bits of x, y, z) or Pos64[N] (fp64)
  int* cstart;     // ncell + 1
  int* ccnt;       // ncell
  uint4* spos;     // cell-sorted positions (.w = atom index)
  int* wscan;      // 2 x (threads + 1): block scan of own atoms in cell order
  uint16_t* own_sorted;  // threads: sorted slots of this CTA's atoms
  int* cnt_sh;     // threads: sub-list counts handed to the owners
  long long* rec_k;  // kNoiseChunk: 2K of each step (fixed point), CTA 0
  float* rec_e;      // kNoiseChunk: alpha - 1 of each step
  uint16_t* acell;
  double2* noise;  // 2 x kNoiseChunk thermostat records (double buffered)
  float* slot_md;  // [cluster][warps]
  double* slot_uk; // [cluster][warps][2]
  int* slot_st;    // [cluster]
  int* iscr;       // 64
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline size_t batched_layout(int max_n, int max_ncell, int threads, bool fp64,
                                                 size_t list_elems, unsigned char* base,
                                                 BatchedSmem* out) {
  size_t off = 0;
  auto take = [&](size_t bytes, size_t al) {
    off = align_up(off, al);
    size_t o = off;
    off += bytes;
    return o;
  };
  const size_t o_nbs = take(list_elems * 2, 16);
  const size_t o_pos = take((size_t)max_n * (fp64 ? 32 : 16), 32);
  const size_t o_sp = take((size_t)max_n * 16, 16);
  const size_t o_noise = take((size_t)kNoiseChunk * 2 * kSvrStepBytes, 16);
  const size_t o_uk = take((size_t)kMaxCluster * kMaxWarps * 2 * 8, 16);
  const size_t o_md = take((size_t)kMaxCluster * kMaxWarps * 4, 4);
  const size_t o_st = take(kMaxCluster * 4, 4);
  const size_t o_isc = take(64 * 4, 4);
  const size_t o_rk = take((size_t)kNoiseChunk * 8, 8);
  const size_t o_re = take((size_t)kNoiseChunk * 4, 4);
  const size_t o_cs = take((size_t)(max_ncell + 1) * 4, 4);
  const size_t o_cc = take((size_t)(max_ncell + 1) * 4, 4);
  // one region, two lifetimes: the atoms' cell ids during the cell sort, then
  // the block scan, the own-slot list and the hand-over counts of the list build
  const size_t scan_bytes = (size_t)2 * (threads + 1) * 4 + (size_t)threads * 4 + (size_t)threads * 2;
  const size_t o_un = take(scan_bytes > (size_t)max_n * 2 ? scan_bytes : (size_t)max_n * 2, 4);
  const size_t o_ws = o_un;
  const size_t o_cn = o_un + (size_t)2 * (threads + 1) * 4;
  const size_t o_os = o_cn + (size_t)threads * 4;
  const size_t o_ac = o_un;
  if (out) {
    out->nb_sm = reinterpret_cast<uint16_t*>(base + o_nbs);
    out->pos = base + o_pos;
    out->noise = reinterpret_cast<double2*>(base + o_noise);
    out->slot_uk = reinterpret_cast<double*>(base + o_uk);
    out->slot_md = reinterpret_cast<float*>(base + o_md);
    out->slot_st = reinterpret_cast<int*>(base + o_st);
    out->iscr = reinterpret_cast<int*>(base + o_isc);
    out->rec_k = reinterpret_cast<long long*>(base + o_rk);
    out->rec_e = reinterpret_cast<float*>(base + o_re);
    out->cstart = reinterpret_cast<int*>(base + o_cs);
    out->ccnt = reinterpret_cast<int*>(base + o_cc);
    out->spos = reinterpret_cast<uint4*>(base + o_sp);
    out->wscan = reinterpret_cast<int*>(base + o_ws);
    out->cnt_sh = reinterpret_cast<int*>(base + o_cn);
    out->own_sorted = reinterpret_cast<uint16_t*>(base + o_os);
    out->acell = reinterpret_cast<uint16_t*>(base + o_ac);
  }
  return align_up(off, 128);
}

struct KernelDims {
  int max_n, max_ncell;
  size_t list_elems;  // shared-memory list entries per CTA (0: lists in global memory)
  int async_nx;       // > 0: free-running mode with this many master steps
};

// free-running mode: step cap of the non-master replicas (a bound, not a budget)
constexpr int kAsyncCapFactor = 16;

__device__ __forceinline__ uint64_t* qcomp(const StateDev& S, int d) {
  return d == 0 ? S.qx : (d == 1 ? S.qy : S.qz);
}
__device__ __forceinline__ double* vcomp(const StateDev& S, int d) {
  return d == 0 ? S.vx : (d == 1 ? S.vy : S.vz);
}
__device__ __forceinline__ double* fcomp(const StateDev& S, int d) {
  return d == 0 ? S.fx : (d == 1 ? S.fy : S.fz);
}
__device__ __forceinline__ uint32_t* rcomp(const StateDev& S, int d) {
  return d == 0 ? S.rx : (d == 1 ? S.ry : S.rz);
}

// Sub-list of lane q (of P) of atom i: candidates of every scanned range are
// dealt to the P lanes in turn (candidate k of a range goes to lane k % P).
// Entry k of sub-list (i, q) sits at nb[((k/4) * N*P + i*P + q) * 4 + k%4].
// The sub-list of column `col` of a list with `ncols` columns: entry k at
// element ((k / 4) * ncols + col) * 4 + k % 4 of nb.
template <int P, class PosFn>
__device__ int build_sublist(int i, int q, PosFn pos_hi, int N, int nc, int m, const int* cstart,
                             const uint4* spos, float rl2u, uint16_t* nb, uint32_t col,
                             uint32_t ncols, int cap_sub, int* overflow) {
  const Hi3 pi = pos_hi(i);
  // a running offset: +1 inside a block of four, + ncols*4 - 3 across blocks
  uint32_t wofs = col * 4;
  const uint32_t jump = ncols * 4 - 3u;
  int cnt = 0;
  bool coincident = false;
  auto accept = [&](int j, Hi3 pj) {
    const float r2 = sep2_hi(pi, pj);
    if (j != i && r2 < rl2u) {
      // two distinct atoms at one point (closer than L / 2^32): the pair loop
      // treats distance 0 as the sub-list padding, so report it (below)
      coincident |= (r2 == 0.0f);
      if (cnt < cap_sub) {
        nb[wofs] = (uint16_t)j;
        wofs += ((cnt & 3) == 3) ? jump : 1u;
      }
      ++cnt;
    }
  };
  if (nc == 0) {
    for (int j = q; j < N; j += P) accept(j, pos_hi(j));
  } else {
    const int cx = (int)__umulhi(pi.x, (uint32_t)nc), cy = (int)__umulhi(pi.y, (uint32_t)nc),
              cz = (int)__umulhi(pi.z, (uint32_t)nc);
    // cells z in [cz - m, cz + m] (periodic) are at most two contiguous ranges
    // of the cell order: [lo1, hi1) and [0, hi2) (empty when hi2 == 0).
    // (Pruning columns and z ranges to the sphere with the atom's exact offset
    // scans fewer candidates but was not faster: the per-column work and the
    // lane divergence it adds cost as much as the candidates it saves.)
    const int zlo = cz - m, zhi = cz + m;
    const int lo1 = zlo < 0 ? zlo + nc : zlo;
    const int hi1 = (zlo < 0 || zhi >= nc) ? nc : zhi + 1;
    const int hi2 = zlo < 0 ? zhi + 1 : (zhi >= nc ? zhi - nc + 1 : 0);
    for (int ox = -m; ox <= m; ++ox) {
      int x = cx + ox;
      x += (x < 0) ? nc : 0;
      x -= (x >= nc) ? nc : 0;
      for (int oy = -m; oy <= m; ++oy) {
        int y = cy + oy;
        y += (y < 0) ? nc : 0;
        y -= (y >= nc) ? nc : 0;
        const int base = (x * nc + y) * nc;
        const int b1 = cstart[base + lo1], e1 = cstart[base + hi1];
        const int b2 = cstart[base], e2 = cstart[base + hi2];
        const int n1 = e1 - b1, n = n1 + (e2 - b2);
        // two candidates per iteration: both loads issue before either test
        int t = q;
        for (; t + P < n; t += 2 * P) {
          const int t2 = t + P;
          const uint4 v = spos[t < n1 ? b1 + t : b2 + (t - n1)];
          const uint4 w = spos[t2 < n1 ? b1 + t2 : b2 + (t2 - n1)];
          accept((int)v.w, Hi3{v.x, v.y, v.z});
          accept((int)w.w, Hi3{w.x, w.y, w.z});
        }
        if (t < n) {
          const uint4 v = spos[t < n1 ? b1 + t : b2 + (t - n1)];
          accept((int)v.w, Hi3{v.x, v.y, v.z});
        }
      }
    }
  }
  if (coincident) *overflow |= kStNumeric;
  if (cnt > cap_sub) {
    *overflow |= kStOverflow;
    cnt = cap_sub;
  }
  // pad to a whole block of four with the atom's own index (skipped by r2 > 0)
  for (int k = cnt; k & 3; ++k) nb[wofs++] = (uint16_t)i;
  return cnt;
}

// Mixed-precision sub-list loop of lane (i, q); see mixed_pair.
// Sub-lists are padded with the atom's own index up to a whole block of four;
// only the last block can hold padding, so only it tests for the atom itself.
// ENERGY: also sum the pair energies (needed only when U is reported).
template <bool ENERGY>
__device__ __forceinline__ MixedAcc mixed_sublist_forces(uint4 pi, const uint4* __restrict__ pos,
                                                         const uint16_t* __restrict__ nb,
                                                         uint32_t col, uint32_t ncols, int cnt,
                                                         float rc2u, float inv_lam2) {
  MixedAcc a{0.f, 0.f, 0.f, 0.f, 0};
  const size_t stride4 = (size_t)ncols * 4;
  const uint16_t* base = nb + (size_t)col * 4;
  const int nblk = (cnt + 3) >> 2;
  const int nfull = cnt >> 2;
  uint2 w = nblk > 0 ? *reinterpret_cast<const uint2*>(base) : make_uint2(0u, 0u);
  for (int kb = 0; kb < nfull; ++kb) {
    // the next block of indices is requested before this block is used
    const uint2 wn = kb + 1 < nblk ? *reinterpret_cast<const uint2*>(base + (size_t)(kb + 1) * stride4) : w;
    const uint4 p0 = pos[w.x & 0xFFFFu];
    const uint4 p1 = pos[w.x >> 16];
    const uint4 p2 = pos[w.y & 0xFFFFu];
    const uint4 p3 = pos[w.y >> 16];
    mixed_pair<ENERGY, false>(pi, p0, rc2u, inv_lam2, a);
    mixed_pair<ENERGY, false>(pi, p1, rc2u, inv_lam2, a);
    mixed_pair<ENERGY, false>(pi, p2, rc2u, inv_lam2, a);
    mixed_pair<ENERGY, false>(pi, p3, rc2u, inv_lam2, a);
    w = wn;
  }
  if (nblk > nfull) {
    const uint4 p0 = pos[w.x & 0xFFFFu];
    const uint4 p1 = pos[w.x >> 16];
    const uint4 p2 = pos[w.y & 0xFFFFu];
    const uint4 p3 = pos[w.y >> 16];
    mixed_pair<ENERGY, true>(pi, p0, rc2u, inv_lam2, a);
    mixed_pair<ENERGY, true>(pi, p1, rc2u, inv_lam2, a);
    mixed_pair<ENERGY, true>(pi, p2, rc2u, inv_lam2, a);
    mixed_pair<ENERGY, true>(pi, p3, rc2u, inv_lam2, a);
  }
  return a;
}

__device__ __forceinline__ void fp64_sublist_forces(Pos64 pi, const Pos64* pos, const uint16_t* nb,
                                                    uint32_t col, uint32_t ncols, int cnt,
                                                    double lam64, double rc2, double uc,
                                                    double& fx, double& fy, double& fz,
                                                    double& e) {
  fx = fy = fz = e = 0.0;
  const size_t stride = ncols;
  for (int k = 0; k < cnt; ++k) {
    const int j = nb[((size_t)(k >> 2) * stride + col) * 4 + (k & 3)];
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

template <int P>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = 1; o < P; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int P>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = 1; o < P; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int P>
__device__ __forceinline__ int group_sum(int v) {
#pragma unroll
  for (int o = 1; o < P; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-step thermostat draws, generated ahead of the step (off the critical
// path).  With K the kinetic energy after the second half kick, the SVR update
// is K'/K = 1 + delta with delta = (c - 1) + (a + b sqrt(K)) / K, where
// a = (1 - c) Kbar (R1^2 + S) / Nf and b = 2 R1 sqrt(c (1 - c) Kbar / Nf); the
// factor alpha = +-sqrt(1 + delta) is negative when R1 + g sqrt(K) < 0,
// g = sqrt(c Nf / ((1 - c) Kbar)).
struct SvrStep {
  double r1, s;  // the draws (FP64 path)
  float r1f, sf; // the draws (mixed path)
  int bad;       // the Gamma sampler hit its trial cap
  int pad;
};
static_assert(sizeof(SvrStep) == kSvrStepBytes, "thermostat record size");

__device__ inline SvrStep svr_step(bool fp64, const StepConst& K, uint64_t seed, uint64_t stream,
                                   uint64_t n, int* capped) {
  SvrStep t;
  t.bad = 0;
  t.pad = 0;
  if (fp64) {
    const double2 z = svr_noise(K.nf, seed, stream, n, capped);
    t.r1 = z.x;
    t.s = z.y;
    t.r1f = (float)z.x;
    t.sf = (float)z.y;
  } else {
    const float2 z = svr_noise_f32(K.nf, seed, stream, n, capped);
    t.r1 = z.x;
    t.s = z.y;
    t.r1f = z.x;
    t.sf = z.y;
  }
  return t;
}

// alpha - 1 in FP32 without cancellation: sqrt(1 + delta) - 1 = delta / (1 + sqrt(1 + delta)).
// The temperature-dependent constants are read from K at the step (the
// target may change within a launch).
__device__ __forceinline__ float svr_eps(const SvrStep& t, float Kf, const StepConst& K) {
  const float a = K.af * fmaf(t.r1f, t.r1f, t.sf);
  const float b = K.bf * t.r1f;
  const float sk = sqrtf(Kf);
  const float delta = K.cm1f + (a + b * sk) / Kf;
  const float root = sqrtf(1.0f + delta);
  if (t.r1f + K.gf * sk < 0.0f) return -1.0f - root;  // alpha = -sqrt(1 + delta)
  return delta / (1.0f + root);
}

// Fixed-point scales of the mixed path: velocities in units of 2^-48 (64-bit,
// |v| < 2^15), energy partial sums in units of 2^-28 (64-bit, |sum| < 2^35).
constexpr float kVelScale = 281474976710656.0f;        // 2^48
constexpr float kVelUnit = 3.5527136788005009e-15f;   // 2^-48
constexpr float kEnScale = 268435456.0f;              // 2^28
constexpr double kEnUnit = 3.7252902984619140625e-09; // 2^-28

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Metropolis rule of the Implementation section for the pair (a before b in
// ladder order), generalised to parameter sets (T, lam) whose Hamiltonians
// are K + lam U_LJ: D = (lam_a/T_a - lam_b/T_b)(U_a/lam_a - U_b/lam_b) with U
// the stored (scaled) potential energies; lam = 1 gives
// D = (1/T_a - 1/T_b)(U_a - U_b).  Accept iff D >= 0 or r < exp(D), r the
// uniform of the lower replica id for this attempt.
__device__ __forceinline__ bool metropolis(double Ta, double Tb, double la, double lb, double Ua,
                                           double Ub, uint64_t seed, int id_lo, int64_t attempt) {
  const double d = __dmul_rn(__dsub_rn(__ddiv_rn(la, Ta), __ddiv_rn(lb, Tb)),
                             __dsub_rn(__ddiv_rn(Ua, la), __ddiv_rn(Ub, lb)));
  if (d >= 0.0) return true;
  const Uni4 u = uniforms(seed, (uint64_t)id_lo, (uint64_t)attempt, kTagExch, 0ull);
  return u.u0 < exp(d);
}

// Partner position of ladder position q: pairs (q, q + d) for q - o in
// [0, d) modulo 2d, o = p d (p the parity offset); -1 when unpaired.
__device__ __forceinline__ int ladder_partner(int q, int R, int p, int d) {
  const int o = p * d;
  if (q < o) return -1;
  if ((q - o) % (2 * d) < d) return q + d < R ? q + d : -1;
  return q - d;
}

__device__ __forceinline__ int pair_offset(int mode, uint64_t seed, int64_t attempt) {
  if (mode == 0) return (int)(attempt & 1);
  const Uni4 u = uniforms(seed, ~0ull, (uint64_t)attempt, kTagParity, 0ull);
  return u.u0 < 0.5 ? 0 : 1;
}

// ------------------------------------------------------ free-running exchange
// The asynchronous scheme of the Implementation section inside one persistent
// launch: every replica integrates without stopping; the master of pattern k
// (member (attempt + k) mod R, so the role rotates with every attempt), after
// nx of its own steps since it took part in pattern k - 1, waits until every
// member has taken part in pattern k - 1, sorts the members' temperatures and
// publishes pattern k.  Each replica checks for a new pattern after every
// step; when one is there it publishes (T, U), waits for its partner's pair,
// and both take the same Metropolis decision with the lower id's uniform.
// Every wait is bounded (kWaitNs, and an iteration cap) and watches the
// ensemble's abort flag; a replica that gives up or fails raises that flag.
constexpr uint64_t kWaitNs = 1000000000ull;

__device__ bool wait_at_least(const int* p, int want, const int* abort_flag) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (ld_acquire(p) >= want) return true;
    if (*reinterpret_cast<const volatile int*>(abort_flag)) return false;
    if ((it & 63u) == 63u && global_ns() - t0 > kWaitNs) return false;
    __nanosleep(32);
  }
  return false;
}

// The master's part, by one warp: pattern k of ensemble e.  Returns false when
// a wait gave up.
__device__ bool issue_pattern(const FreeDev& fr, const StateDev& S, const EnsDev& E, int e, int k,
                              int64_t attempt) {
  const int lane = threadIdx.x & 31;
  const int R = E.R, base = E.rep_off;
  bool ok = true;
  if (k > 0)
    for (int m = lane; m < R && ok; m += 32) ok = wait_at_least(fr.done + base + m, k, fr.abort_ + e);
  ok = __all_sync(0xffffffffu, ok);
  if (!ok) return false;
  __threadfence();
  // ladder keys T/lam (positive: their bit patterns order like the values)
  for (int m = lane; m < R; m += 32)
    fr.key[base + m] = __ldcg(S.T + base + m) / __ldcg(S.lam + base + m);
  __syncwarp();
  const long long* key = reinterpret_cast<const long long*>(fr.key + base);
  for (int m = lane; m < R; m += 32) {
    const long long t = key[m];
    int rank = 0;
    for (int b = 0; b < R; ++b) {
      const long long u = key[b];
      rank += (u < t) || (u == t && b < m);
    }
    fr.order[base + rank] = m;
    fr.pos[base + m] = rank;
  }
  __syncwarp();
  const int p = pair_offset(E.parity_mode, E.seed, attempt);
  const int d = max(1, E.xdist);
  for (int m = lane; m < R; m += 32) {
    const int q = ladder_partner(fr.pos[base + m], R, p, d);
    fr.partner[base + m] = q < 0 ? -1 : fr.order[base + q];
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    st_release(fr.issue + e, k + 1);
  }
  return true;
}

// A replica's part of pattern k (one thread), parameters (Tcur, lcur).
// Returns the velocity scale sqrt(T_new / T_old) and sets *us =
// lam_new / lam_old (both 1 when not accepted); *ok = false when the wait
// gave up.
__device__ double pair_exchange(const FreeDev& fr, const StateDev& S, const EnsDev& E,
                                const RepDev& rd, int r, int k, int64_t attempt, double Tcur,
                                double lcur, double U, double* Tnew, double* lnew, double* us,
                                int* partner_out, int* acc_out, bool* ok) {
  const int p = __ldcg(fr.partner + r);
  *Tnew = Tcur;
  *lnew = lcur;
  *us = 1.0;
  *partner_out = p;
  *acc_out = 0;
  *ok = true;
  if (p < 0) return 1.0;
  fr.slot[3 * r] = Tcur;
  fr.slot[3 * r + 1] = U;
  fr.slot[3 * r + 2] = lcur;
  __threadfence();
  st_release(fr.flag + r, k + 1);
  const int gp = E.rep_off + p;
  if (!wait_at_least(fr.flag + gp, k + 1, fr.abort_ + rd.ens)) {
    *ok = false;
    return 1.0;
  }
  __threadfence();
  const double Tp = __ldcg(fr.slot + 3 * gp), Up = __ldcg(fr.slot + 3 * gp + 1),
               lp = __ldcg(fr.slot + 3 * gp + 2);
  const int q = __ldcg(fr.pos + r), qp = __ldcg(fr.pos + gp);
  const bool lower = q < qp;  // this replica comes first in ladder order
  const int id_lo = min(rd.id, p);
  const bool accept = lower ? metropolis(Tcur, Tp, lcur, lp, U, Up, E.seed, id_lo, attempt)
                            : metropolis(Tp, Tcur, lp, lcur, Up, U, E.seed, id_lo, attempt);
  if (lower) {
    atomicAdd(reinterpret_cast<unsigned long long*>(S.pair_att + E.pair_off + q), 1ull);
    if (accept) atomicAdd(reinterpret_cast<unsigned long long*>(S.pair_acc + E.pair_off + q), 1ull);
  }
  if (!accept) return 1.0;
  *acc_out = 1;
  *Tnew = Tp;
  *lnew = lp;
  *us = lp / lcur;
  return sqrt(Tp / Tcur);
}

// One thread-block cluster per replica (work item).  CTA `crank` owns atoms
// [i0, i1); P consecutive lanes serve one atom: lane q keeps the state of the
// coordinates d = q, q + P, ... in registers for the whole launch and owns one
// sub-list of the atom's Verlet list.  Every CTA keeps the positions of all N
// atoms of the replica in shared memory (top 32 bits, or all 64 bits on the
// FP64 path); each step the owners broadcast their new coordinates to every
// CTA of the cluster.  Two cluster barriers per step: after the drift
// (positions and displacement maxima visible) and after the second kick
// (energy partial sums visible; all position reads of the step done).
//
// Mixed path: positions and velocities are 64-bit fixed-point master copies
// updated with FP32 increments (exact accumulation; FP64 arithmetic runs at
// 1/64 of the FP32 rate on this GPU); pair forces FP32; energy sums 64-bit
// integers (exact, order independent).  The second half kick, the thermostat
// factor and the next first half kick form one increment per coordinate.
// FP64 path: FP64 state arithmetic and FP64 pair forces throughout.
// MODE 0: per-replica step budgets; 1: master-stop (dims.async_nx); 2:
// free-running with exchanges inside the launch (fr).
template <bool FP64, int P, bool LSM, int MODE>
__global__ void __launch_bounds__(1024, 1) md_batched_kernel(StateDev S,
                                                             const EnsDev* __restrict__ ens,
                                                             const RepDev* __restrict__ reps,
                                                             const int* __restrict__ work,
                                                             const int32_t* __restrict__ budget,
                                                             KernelDims dims, FreeDev fr) {
  constexpr int ND = (3 + P - 1) / P;  // coordinates per lane
  // replica constants live in shared memory, not in registers
  __shared__ EnsDev E;
  __shared__ StepConst K;
  __shared__ double alpha_sh, kp_sh;
  __shared__ float eps_sh;
  __shared__ int st_sh;
  // free-running exchange: the result handed to the cluster (velocity scale,
  // new T, status), the replica's current T and the launch's first attempt
  // number (thread 0), own steps since the last pattern (warp 0 of CTA 0)
  __shared__ double xs_sh, xT_sh, xl_sh, xu_sh, Tcur_sh;
  __shared__ long long A0_sh;
  __shared__ int xst_sh, since_sh, fold0_sh;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int r = work[blockIdx.x / C];
  const RepDev rd = reps[r];
  if (threadIdx.x == 0) {
    E = ens[rd.ens];
    K = E.kc;
    set_thermo_target(K, S.T[r]);
    set_potential_scale(K, S.lam[r]);
    Tcur_sh = S.T[r];
    A0_sh = S.attempt[rd.ens];
    since_sh = 0;
    fold0_sh = 0;
  }
  const int T = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nw = (T + 31) >> 5;
  const int q = tid & (P - 1);
  // Budget mode: budget[r] steps.  Free-running mode (Implementation section):
  // the ensemble's master (replica attempt mod R, rotating with every attempt)
  // does async_nx steps and then raises the ensemble's stop flag; every other
  // replica checks the flag after each step and stops after the step in which
  // it sees it (at most kAsyncCapFactor * async_nx + 16 steps).  No thread waits.
  const int async_nx = MODE == 1 ? dims.async_nx : 0;
  constexpr bool freerun = MODE == 2;
  bool is_master = false;
  int B;
  if (freerun) {
    B = (fr.n_att + 1) * (kAsyncCapFactor * fr.nx + 16);  // step cap of the launch
  } else if (async_nx > 0) {
    const int Rens = ens[rd.ens].R;
    is_master = rd.id == (int)(S.attempt[rd.ens] % Rens);
    B = is_master ? async_nx : kAsyncCapFactor * async_nx + 16;
  } else {
    B = budget[r];
  }
  const int status0 = S.status[r];
  const int valid0 = S.valid[r];
  const double vs0 = S.vscale[r];
  const double fs0 = S.fscale[r];
  double econs = S.econs[r];
  const int64_t step0 = S.step[r];

  extern __shared__ __align__(128) unsigned char smem_raw[];
  BatchedSmem sm;
  batched_layout(dims.max_n, dims.max_ncell, T, FP64, dims.list_elems, smem_raw, &sm);
  uint4* posm = reinterpret_cast<uint4*>(sm.pos);
  Pos64* pos64 = reinterpret_cast<Pos64*>(sm.pos);

  // Every CTA has read the replica's flags before any CTA may change them
  // (the barrier also publishes E and K to the whole CTA).
  cl.sync();
  if (status0 != 0 || (B <= 0 && valid0)) {  // uniform over the cluster
    // a replica that cannot run must not leave its partners waiting
    if (freerun && crank == 0 && threadIdx.x == 0) atomicExch(fr.abort_ + rd.ens, 1);
    return;
  }
  // a one-CTA replica synchronises with the cheaper block barrier
  auto csync = [&]() {
    if (C > 1)
      cl.sync();
    else
      __syncthreads();
  };

  const int N = E.N;
  const int per = (N + C - 1) / C;
  const int i0 = min(N, crank * per), i1 = min(N, i0 + per);
  const int i = i0 + tid / P;
  const bool own = i < i1;
  const int g = rd.atom_off + i;
  const int cap_sub = E.capsub[P == 1 ? 0 : (P == 2 ? 1 : (P == 4 ? 2 : 3))];
  uint16_t* nbg = S.nbr + rd.nbr_off;  // global lists: columns i * P + q of N * P
  // lists used by the step loop: in shared memory (columns (i - i0) * P + q of
  // per * P) when they fit, else the global ones
  uint16_t* nb = LSM ? sm.nb_sm : nbg;
  const uint32_t ncols = LSM ? (uint32_t)(per * P) : (uint32_t)(N * P);
  const uint32_t mycol = LSM ? (uint32_t)((i - i0) * P + q) : (uint32_t)(i * P + q);
  int32_t* ncnt = S.ncnt + (size_t)rd.atom_off * 8;
  const float dtqf = (float)K.dtq;
  const float ucf = (float)K.uc;
  const bool thermo = E.tau > 0.0;  // decided once; no FP64 tests inside the step loop

  // per-lane state in registers
  uint64_t xq[ND];
  double v[ND], f[ND];       // FP64 path
  long long vq[ND];          // mixed path: velocity, fixed point
  float vf[ND], hf[ND];      // mixed path: FP32 velocity copy, half-kick increment
  uint32_t ref[ND];
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int d = q + j * P;
    xq[j] = 0;
    v[j] = f[j] = 0.0;
    vq[j] = 0;
    vf[j] = hf[j] = 0.0f;
    ref[j] = 0;
    if (own && d < 3) {
      xq[j] = qcomp(S, d)[g];
      const double vv = vcomp(S, d)[g] * vs0;
      const double ff = fcomp(S, d)[g] * fs0;
      ref[j] = rcomp(S, d)[g];
      if (FP64) {
        v[j] = vv;
        f[j] = ff;
      } else {
        vq[j] = __double2ll_rn(vv * 0x1.0p48);  // once per launch
        vf[j] = (float)vv;
        hf[j] = (float)(ff * K.hdt);
      }
    }
  }
  if (own) cnt = ncnt[(size_t)i * P + q];

  auto hi_of = [&](int a) -> Hi3 {
    if (FP64) {
      const Pos64 p = pos64[a];
      return Hi3{(uint32_t)(p.x >> 32), (uint32_t)(p.y >> 32), (uint32_t)(p.z >> 32)};
    } else {
      const uint4 p = posm[a];
      return Hi3{p.x, p.y, p.z};
    }
  };
  // broadcast this lane's coordinates of atom i to every CTA of the cluster
  auto publish = [&]() {
    if (!own) return;
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int d = q + j * P;
      if (d >= 3) continue;
      if (FP64) {
        uint64_t* dst = reinterpret_cast<uint64_t*>(&pos64[i]) + d;
        for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(dst, rk) = xq[j];
      } else {
        uint32_t* dst = reinterpret_cast<uint32_t*>(&posm[i]) + d;
        const uint32_t hv = (uint32_t)(xq[j] >> 32);
        for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(dst, rk) = hv;
      }
    }
  };

  int overflow = 0;
  int nreb = 0;
  // Rebuild of the lists of this CTA's atoms.  With cells, the lane groups take
  // this CTA's atoms in cell order (neighbouring lanes then scan the same cell
  // ranges) and hand the sub-list counts to the owners through shared memory.
  auto rebuild = [&]() {
    if (E.nc > 0) {
      cta_build_cells(hi_of, N, E.nc, sm.cstart, sm.ccnt, sm.spos, sm.acell, sm.iscr);
      int n_own = i1 - i0;
      if (C > 1) {
        const int pt = (N + T - 1) / T;
        const int lo = min(N, tid * pt), hi = min(N, lo + pt);
        int c = 0;
        for (int k = lo; k < hi; ++k) {
          const int a = (int)sm.spos[k].w;
          c += (a >= i0 && a < i1);
        }
        sm.wscan[tid] = c;
        __syncthreads();
        block_exclusive_scan(sm.wscan, sm.wscan + T + 1, T, sm.iscr);
        int at = sm.wscan[T + 1 + tid];
        for (int k = lo; k < hi; ++k) {
          const int a = (int)sm.spos[k].w;
          if (a >= i0 && a < i1) sm.own_sorted[at++] = (uint16_t)k;
        }
        __syncthreads();
      }
      const int gi = tid / P;
      if (gi < n_own) {
        // one CTA: every sorted slot is its own; several: the compacted slots
        const int a = (int)sm.spos[C == 1 ? gi : (int)sm.own_sorted[gi]].w;
        const uint32_t col = LSM ? (uint32_t)((a - i0) * P + q) : (uint32_t)(a * P + q);
        const int c = build_sublist<P>(a, q, hi_of, N, E.nc, E.m, sm.cstart, sm.spos, K.rl2u, nb,
                                       col, ncols, cap_sub, &overflow);
        sm.cnt_sh[(a - i0) * P + q] = c;
      }
      __syncthreads();
      if (own) cnt = sm.cnt_sh[(i - i0) * P + q];
    } else if (own) {
      cnt = build_sublist<P>(i, q, hi_of, N, E.nc, E.m, sm.cstart, sm.spos, K.rl2u, nb, mycol,
                             ncols, cap_sub, &overflow);
    }
    if (own) {
#pragma unroll
      for (int j = 0; j < ND; ++j) ref[j] = (uint32_t)(xq[j] >> 32);
    }
    ++nreb;
  };

  // Forces on this lane's atom (sub-list sums combined over the P lanes) and
  // the second half kick when `kick`.  Publishes this warp's partial sums of
  // U and of v^2 (after the kick) to every CTA; returns the lanes' numeric flag.
  auto forces_and_publish = [&](bool kick, bool energy, int st_in) {
    int st = st_in;
    long long iu = 0, ik = 0;  // mixed: fixed-point partial sums
    double du = 0.0, dk = 0.0; // FP64 path
    if (FP64) {
      double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
      if (own)
        fp64_sublist_forces(pos64[i], pos64, nb, mycol, ncols, cnt, K.lam64, K.rc2, K.uc, fx, fy,
                            fz, e);
      fx = group_sum<P>(fx);
      fy = group_sum<P>(fy);
      fz = group_sum<P>(fz);
      e = group_sum<P>(e);
      if (own) {
        if (q == 0) du = e;
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          const int d = q + j * P;
          if (d >= 3) continue;
          f[j] = K.lamv * (d == 0 ? fx : (d == 1 ? fy : fz));
          if (kick) v[j] += K.hdt * f[j];
          dk += v[j] * v[j];
        }
      }
      du = warp_sum(du);
      dk = warp_sum(dk);
    } else {
      MixedAcc a{0.f, 0.f, 0.f, 0.f, 0};
      if (own) {
        if (energy)
          a = mixed_sublist_forces<true>(posm[i], posm, nb, mycol, ncols, cnt, K.rc2u, K.inv_lam2);
        else
          a = mixed_sublist_forces<false>(posm[i], posm, nb, mycol, ncols, cnt, K.rc2u, K.inv_lam2);
      }
      const float ax = group_sum<P>(a.fx), ay = group_sum<P>(a.fy), az = group_sum<P>(a.fz);
      float ae = 0.0f;
      if (energy) ae = group_sum<P>(a.e) - ucf * (float)group_sum<P>(a.nin);  // uniform flag
      if (own) {
        if (!isfinite(ax) || !isfinite(ay) || !isfinite(az)) st |= kStNumeric;
        if (energy && q == 0) {
          if (!isfinite(ae)) st |= kStNumeric;
          iu = f2ll_split(ae * kEnScale);
        }
        float kl = 0.0f;
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          const int d = q + j * P;
          if (d >= 3) continue;
          hf[j] = (d == 0 ? ax : (d == 1 ? ay : az)) * K.hlf;
          const float w = kick ? vf[j] + hf[j] : vf[j];
          kl = fmaf(w, w, kl);
        }
        if (!isfinite(kl)) st |= kStNumeric;
        ik = f2ll_split(kl * kEnScale);
      }
      if (energy) iu = warp_sum_i64(iu);  // U is summed only when it is reported
      ik = warp_sum_i64(ik);
    }
    st = warp_or(st);
    if (lane == 0) {
      for (int rk = 0; rk < C; ++rk) {
        long long* uk = reinterpret_cast<long long*>(cl.map_shared_rank(sm.slot_uk, rk));
        uk[(crank * kMaxWarps + warp) * 2 + 0] = FP64 ? __double_as_longlong(du) : iu;
        uk[(crank * kMaxWarps + warp) * 2 + 1] = FP64 ? __double_as_longlong(dk) : ik;
        if (st) atomicOr(cl.map_shared_rank(sm.slot_st, rk) + crank, st);
      }
    }
  };
  // Every warp sums the published partials in the same fixed order and reads
  // the status bits of every CTA.  FP64 path: sums of FP64 values.  Mixed
  // path: exact 64-bit integer sums of the fixed-point partials.
  auto totals_fp64 = [&](double& su, double& sk, int& st) {
    const long long* uk = reinterpret_cast<const long long*>(sm.slot_uk);
    su = 0.0;
    sk = 0.0;
    for (int idx = lane; idx < C * kMaxWarps; idx += 32)
      if (idx % kMaxWarps < nw) {
        su += __longlong_as_double(uk[idx * 2 + 0]);
        sk += __longlong_as_double(uk[idx * 2 + 1]);
      }
    su = warp_sum(su);
    sk = warp_sum(sk);
    st = 0;
    for (int rk = 0; rk < C; ++rk) st |= sm.slot_st[rk];
  };
  auto totals_int = [&](long long& iu, long long& ik, int& st, bool energy) {
    const long long* uk = reinterpret_cast<const long long*>(sm.slot_uk);
    long long a = 0, b = 0;
    for (int idx = lane; idx < C * kMaxWarps; idx += 32)
      if (idx % kMaxWarps < nw) {
        if (energy) a += uk[idx * 2 + 0];
        b += uk[idx * 2 + 1];
      }
    iu = energy ? warp_sum_i64(a) : 0ll;
    ik = warp_sum_i64(b);
    st = 0;
    for (int rk = 0; rk < C; ++rk) st |= sm.slot_st[rk];
  };

  if (tid < C) sm.slot_st[tid] = 0;
  // shared-memory lists: bring this CTA's valid lists in (blocks of four entries)
  const int nblk_sub = cap_sub / 4;
  if (LSM && valid0) {
    // asynchronous copies, all in flight at once (the loop issues, one wait)
    const int cols = per * P, own_cols = (i1 - i0) * P;
    uint2* dst = reinterpret_cast<uint2*>(nb);
    const uint2* src = reinterpret_cast<const uint2*>(nbg) + (size_t)i0 * P;
    for (int kb = 0; kb < nblk_sub; ++kb)
      for (int c = tid; c < own_cols; c += T)
        cp_async8(dst + (size_t)kb * cols + c, src + (size_t)kb * N * P + c);
    cp_async_wait_all();
    __syncthreads();
  }

  double U = S.U[r], Kin = S.K[r];
  int status = 0;

  if (!valid0) {
    // Prologue: lists, forces, U and K at the current positions.
    publish();
    csync();
    rebuild();
    forces_and_publish(false, true, overflow);
    csync();
    if (FP64) {
      double su, sk;
      totals_fp64(su, sk, status);
      U = 0.5 * su * K.lamv;
      Kin = 0.5 * sk;
      if (!isfinite(U) || !isfinite(Kin)) status |= kStNumeric;
    } else {
      long long iu, ik;
      totals_int(iu, ik, status, true);
      U = 0.5 * (double)iu * kEnUnit * K.lamv;  // FP64 only for the stored energies
      Kin = 0.5 * (double)ik * kEnUnit;
    }
  }

  int k_next = 0;           // free-running: next pattern to take part in (uniform)
  bool first_kick = true;  // the step starts with a first half kick

  int done = 0;
  for (int s = 0; s < B && status == 0 && !(freerun && k_next >= fr.n_att); ++s) {
    const int64_t n = step0 + s;
    SvrStep* sv = reinterpret_cast<SvrStep*>(sm.noise) + ((s / kNoiseChunk) & 1) * kNoiseChunk;
    // The thermostat records of the next kNoiseChunk steps.  Every CTA of the
    // cluster makes its own identical copy and every record a step may read
    // is written whatever the block size: the CTAs of a replica must take the
    // same decisions (a CTA that left the step loop early would leave its
    // partners writing into the shared memory of an exited block).
    if (thermo && (s % kNoiseChunk) == 0) {
      for (int t = tid; t < kNoiseChunk && s + t < B; t += T) {
        int capped = 0;
        SvrStep z = svr_step(FP64, K, E.seed, (uint64_t)rd.stream, (uint64_t)(n + t), &capped);
        z.bad = capped;
        sv[t] = z;
      }
    }
    // (first half kick of the launch) + drift + displacement since the last rebuild
    float d2 = 0.0f;
    if (own) {
#pragma unroll
      for (int j = 0; j < ND; ++j) {
        const int d = q + j * P;
        if (d >= 3) continue;
        if (FP64) {
          if (first_kick) v[j] += K.hdt * f[j];
          xq[j] += (uint64_t)__double2ll_rn(v[j] * K.dtq);
        } else {
          if (first_kick) {
            vq[j] += f2ll_split(hf[j] * kVelScale);
            vf[j] = ll2f_split(vq[j]) * kVelUnit;
          }
          xq[j] += (uint64_t)f2ll_split(vf[j] * dtqf);
        }
        const float dd = (float)(int)((uint32_t)(xq[j] >> 32) - ref[j]);
        d2 = fmaf(dd, dd, d2);
      }
    }
    publish();
    d2 = group_sum<P>(d2);
    float md = warp_max(d2);
    if (lane == 0)
      for (int rk = 0; rk < C; ++rk)
        cl.map_shared_rank(sm.slot_md, rk)[crank * kMaxWarps + warp] = md;
    csync();  // B1
    float mdall = 0.0f;
    for (int idx = lane; idx < C * kMaxWarps; idx += 32)
      if (idx % kMaxWarps < nw) mdall = fmaxf(mdall, sm.slot_md[idx]);
    mdall = warp_max(mdall);
    if (mdall > K.half2u) rebuild();
    // the pair energies are summed only when U is reported (the last step;
    // every step in free-running mode, where the last step is not known ahead)
    const bool energy = async_nx > 0 || freerun || s + 1 == B;
    forces_and_publish(true, energy, overflow);
    // master-stop mode: CTA 0 reads the master's flag and tells every CTA of
    // the cluster (through the status slots) that this step is the last
    if (async_nx > 0 && !is_master && crank == 0 && tid == 0) {
      if (*reinterpret_cast<volatile int32_t*>(S.stop + rd.ens))
        for (int rk = 0; rk < C; ++rk) atomicOr(cl.map_shared_rank(sm.slot_st, rk), (int)kStStop);
    }
    if (freerun) {
      // the master of the next pattern issues it after nx of its own steps
      if (crank == 0 && warp == 0 && k_next < fr.n_att && since_sh + 1 >= fr.nx &&
          rd.id == (int)((A0_sh + k_next) % E.R)) {
        if (!issue_pattern(fr, S, E, rd.ens, k_next, A0_sh + k_next) && lane == 0)
          atomicExch(fr.abort_ + rd.ens, 1);
      }
      // CTA 0 looks for a new pattern (or an abort) and tells every CTA
      if (crank == 0 && tid == 0) {
        int bits = 0;
        if (ld_acquire(fr.issue + rd.ens) > k_next) bits |= kStXchg;
        if (*reinterpret_cast<volatile int32_t*>(fr.abort_ + rd.ens)) bits |= kStStop;
        if (bits)
          for (int rk = 0; rk < C; ++rk) atomicOr(cl.map_shared_rank(sm.slot_st, rk), bits);
      }
    }
    csync();  // B2
    int st;
    const SvrStep z = thermo ? sv[s % kNoiseChunk] : SvrStep{0.0, 0.0, 0.f, 0.f, 0, 0};
    // the stop and exchange bits are in every CTA's slots after B2: read them
    // before the update
    const bool stop_seen = (sm.slot_st[0] & kStStop) != 0;
    const bool xchg = freerun && (sm.slot_st[0] & kStXchg) != 0;
    const bool last = (s + 1 == B) || stop_seen;
    // the step ends on a materialised step boundary (velocities at full step)
    const bool bnd = last || xchg;
    if (FP64) {
      double su, sk;
      totals_fp64(su, sk, st);
      st &= ~(int)kStXchg;
      if (z.bad) st |= kStRngCap;
      const double Un = 0.5 * su * K.lamv, Kn = 0.5 * sk;
      // one lane forms the FP64 factor and K'; the CTA reads both after the
      // barrier, so every thread takes the same decisions below
      if (tid == 0) {
        double alpha = 1.0, kp = Kn;
        if (thermo) alpha = svr_alpha(Kn, K.kbar, K.nf, K.c_th, z.r1, z.s, &kp);
        alpha_sh = alpha;
        kp_sh = kp;
      }
      __syncthreads();
      const double alpha = alpha_sh;
      const double Kp = kp_sh;
      if (!isfinite(alpha) || !isfinite(Un) || !isfinite(Kp)) st |= kStNumeric;
      if (own) {
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          v[j] *= alpha;
          if (!bnd) v[j] += K.hdt * f[j];  // first half kick of the next step
        }
      }
      U = Un;
      Kin = Kp;
      econs += Kn - Kp;
    } else {
      // warp 0 forms the integer totals and alpha - 1 (FP32); the block reads
      // them after a block barrier (far cheaper than every warp repeating it)
      long long iu = 0, ik = 0;
      if (warp == 0) {
        totals_int(iu, ik, st, energy);
        st &= ~(int)kStXchg;
        if (z.bad) st |= kStRngCap;
        const float Kf = ll2f_split(ik) * (float)(0.5 * kEnUnit);
        const float e0 = thermo ? svr_eps(z, Kf, K) : 0.0f;
        if (!isfinite(e0)) st |= kStNumeric;
        if (lane == 0) {
          eps_sh = e0;
          st_sh = st;
        }
      }
      __syncthreads();
      const float eps = eps_sh;
      st = st_sh;
      if (own) {
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          const int d = q + j * P;
          if (d >= 3) continue;
          const float w = vf[j] + hf[j];
          // second half kick + thermostat factor (+ next first half kick)
          const float inc = fmaf(eps, w, bnd ? hf[j] : 2.0f * hf[j]);
          vq[j] += f2ll_split(inc * kVelScale);
          vf[j] = ll2f_split(vq[j]) * kVelUnit;
        }
      }
      // FP64 bookkeeping of the stored energies, off the step's critical path:
      // the step's (2K, alpha - 1) are recorded; warp 0 of CTA 0 folds the
      // records into econs every kNoiseChunk steps and after the last step
      if (crank == 0 && warp == 0) {
        const int slot = s % kNoiseChunk;
        if (lane == 0) {
          sm.rec_k[slot] = ik;
          sm.rec_e[slot] = eps;
        }
        if (slot == kNoiseChunk - 1 || bnd) {
          __syncwarp();
          double dsum = 0.0, kp = 0.0;
          const int fold0 = fold0_sh;
          for (int t = fold0 + lane; t <= slot; t += 32) {
            const double Kn = 0.5 * (double)sm.rec_k[t] * kEnUnit;
            const double a1 = 1.0 + (double)sm.rec_e[t];
            dsum += Kn - Kn * a1 * a1;
            if (t == slot) kp = Kn * a1 * a1;
          }
          econs += warp_sum(dsum);
          kp = __shfl_sync(0xffffffffu, kp, (slot - fold0) & 31);
          Kin = kp;
          if (energy) U = 0.5 * (double)iu * kEnUnit * K.lamv;
          __syncwarp();
          if (lane == 0) fold0_sh = slot + 1 == kNoiseChunk ? 0 : slot + 1;
          __syncwarp();
        }
      }
    }
    status = st;
    ++done;
    // the master, having finished its steps, raises the ensemble's stop flag
    if (is_master && s + 1 == B && crank == 0 && tid == 0) {
      __threadfence();
      atomicExch(S.stop + rd.ens, 1);
    }
    if (xchg) {
      // this replica's part of the pattern: CTA 0 runs the pair protocol and
      // hands the result to every CTA of the cluster
      if (crank == 0 && tid == 0) {
        double Tn, ln, us;
        int pid, acc;
        bool ok;
        const double sc = pair_exchange(fr, S, E, rd, r, k_next, A0_sh + k_next, Tcur_sh, K.lamv,
                                        U, &Tn, &ln, &us, &pid, &acc, &ok);
        if (k_next < fr.log_cap) {
          const size_t li = (size_t)k_next * fr.rtot + r;
          fr.log_step[li] = step0 + done;
          fr.log_T[li] = Tn;
          fr.log_partner[li] = pid;
          fr.log_acc[li] = acc;
        }
        if (Tn != Tcur_sh) S.T[r] = Tn;
        if (ln != K.lamv) S.lam[r] = ln;
        for (int rk = 0; rk < C; ++rk) {
          *cl.map_shared_rank(&xs_sh, rk) = sc;
          *cl.map_shared_rank(&xT_sh, rk) = Tn;
          *cl.map_shared_rank(&xl_sh, rk) = ln;
          *cl.map_shared_rank(&xu_sh, rk) = us;
          *cl.map_shared_rank(&xst_sh, rk) = ok ? 0 : (int)kStTimeout;
        }
      }
      csync();  // B3
      const double sc = xs_sh, Tn = xT_sh, ln = xl_sh, us = xu_sh;
      status |= xst_sh;
      if (tid == 0) atomicAnd(&sm.slot_st[0], ~(int)kStXchg);
      if (own && sc != 1.0) {
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          const int d = q + j * P;
          if (d >= 3) continue;
          if (FP64) {
            v[j] *= sc;
          } else {
            vq[j] = __double2ll_rn((double)vq[j] * sc);
            vf[j] = ll2f_split(vq[j]) * kVelUnit;
          }
        }
      }
      if (own && us != 1.0) {
        // the new Hamiltonian's forces: scale by lam_new / lam_old
#pragma unroll
        for (int j = 0; j < ND; ++j) {
          if (FP64) f[j] *= us;
          else hf[j] *= (float)us;
        }
      }
      const double Ks = Kin * (sc * sc);
      econs += Kin - Ks;
      Kin = Ks;
      const double Us = U * us;
      econs += U - Us;
      U = Us;
      // read by the other threads only after the next barriers; the lam
      // comparison reads K before thread 0 may change it
      const bool new_lam = ln != K.lamv;
      __syncthreads();
      if (tid == 0) {
        if (Tn != Tcur_sh) {
          set_thermo_target(K, Tn);
          Tcur_sh = Tn;
        }
        if (new_lam) set_potential_scale(K, ln);
        since_sh = 0;
      }
      if (crank == 0 && tid == 0) {
        __threadfence();
        st_release(fr.done + r, k_next + 1);
      }
      ++k_next;
    } else if (freerun && tid == 0) {
      ++since_sh;
    }
    first_kick = bnd;
  }
  if (freerun && k_next < fr.n_att) {
    // left before the last pattern: the partners' waits must not run out
    if (crank == 0 && tid == 0) atomicExch(fr.abort_ + rd.ens, 1);
    if ((status & ~(int)kStStop) == 0) status |= kStTimeout;
  }
  // shared-memory lists go back to global memory for the next launch
  if (LSM) {
    __syncthreads();
    const int cols = per * P, own_cols = (i1 - i0) * P;
    const uint2* src = reinterpret_cast<const uint2*>(nb);
    uint2* dst = reinterpret_cast<uint2*>(nbg) + (size_t)i0 * P;
    for (int kb = 0; kb < nblk_sub; ++kb)
      for (int c = tid; c < own_cols; c += T) dst[(size_t)kb * N * P + c] = src[(size_t)kb * cols + c];
  }
  // write the state back
  if (own) {
#pragma unroll
    for (int j = 0; j < ND; ++j) {
      const int d = q + j * P;
      if (d >= 3) continue;
      qcomp(S, d)[g] = xq[j];
      rcomp(S, d)[g] = ref[j];
      if (FP64) {
        vcomp(S, d)[g] = v[j];
        fcomp(S, d)[g] = f[j];
      } else {
        vcomp(S, d)[g] = (double)vq[j] * 0x1.0p-48;
        fcomp(S, d)[g] = (double)hf[j] * K.inv_hdt;
      }
    }
    ncnt[(size_t)i * P + q] = cnt;
  }
  if (crank == 0 && tid == 0) {
    S.U[r] = U;
    S.K[r] = Kin;
    S.econs[r] = econs;
    S.step[r] = step0 + done;
    S.nreb[r] += nreb;
    S.vscale[r] = 1.0;
    S.fscale[r] = 1.0;
    S.status[r] = status & ~(int)(kStStop | kStXchg);
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
// Sorted order of R distinct temperatures by counting (rank = number of
// smaller values, ties broken by index).  Ts, order in shared memory.  The
// temperatures are positive, so their IEEE bit patterns read as 64-bit
// integers order exactly like the values: the comparisons run on the integer
// units instead of the (1/64-rate) FP64 unit.
__device__ void rank_sort(const double* Ts, int* order, int R) {
  const long long* key = reinterpret_cast<const long long*>(Ts);
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    const long long t = key[a];
    int rank = 0;
    for (int b = 0; b < R; ++b) {
      const long long u = key[b];
      rank += (u < t) || (u == t && b < a);
    }
    order[rank] = a;
  }
}

// One exchange attempt per ensemble (one CTA each): ladder keys T/lam sorted,
// pairs (q, q + d) of the ladder (d = 1: sorted neighbours), the Metropolis
// rule, and on acceptance the parameter sets (T, lam) are swapped: the
// velocities take the pending factor sqrt(T_new/T_old), the forces
// lam_new/lam_old, K and U follow and econs absorbs both changes.
__global__ void exchange_kernel(StateDev S, const EnsDev* __restrict__ ens, int32_t* partner_out,
                                uint8_t* acc_out) {
  extern __shared__ __align__(16) unsigned char sh[];
  const EnsDev E = ens[blockIdx.x];
  const int R = E.R, base = E.rep_off;
  double* key = reinterpret_cast<double*>(sh);
  int* order = reinterpret_cast<int*>(key + R);
  for (int a = threadIdx.x; a < R; a += blockDim.x) {
    key[a] = S.T[base + a] / S.lam[base + a];
    if (partner_out) partner_out[base + a] = -1;
    if (acc_out) acc_out[base + a] = 0;
  }
  __syncthreads();
  rank_sort(key, order, R);
  __syncthreads();
  const int64_t attempt = S.attempt[blockIdx.x];
  const int p = pair_offset(E.parity_mode, E.seed, attempt);
  const int d = max(1, E.xdist);
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    const int qb = ladder_partner(q, R, p, d);
    if (qb <= q) continue;  // unpaired, or the upper member of its pair
    const int a = order[q], b = order[qb];
    const int ga = base + a, gb = base + b;
    const double Ta = S.T[ga], Tb = S.T[gb], la = S.lam[ga], lb = S.lam[gb];
    const bool ok = metropolis(Ta, Tb, la, lb, S.U[ga], S.U[gb], E.seed, min(a, b), attempt);
    if (partner_out) {
      partner_out[ga] = b;
      partner_out[gb] = a;
    }
    S.pair_att[E.pair_off + q] += 1;
    if (ok) {
      S.pair_acc[E.pair_off + q] += 1;
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
      if (la != lb) {
        const double ua = lb / la, ub = la / lb;
        const double Ua = S.U[ga], Ub = S.U[gb];
        const double Uan = Ua * ua, Ubn = Ub * ub;
        S.fscale[ga] *= ua;
        S.fscale[gb] *= ub;
        S.econs[ga] += Ua - Uan;
        S.econs[gb] += Ub - Ubn;
        S.U[ga] = Uan;
        S.U[gb] = Ubn;
        S.lam[ga] = lb;
        S.lam[gb] = la;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) S.attempt[blockIdx.x] = attempt + 1;
}

__global__ void exchange_raw_kernel(int R, const double* __restrict__ T,
                                    const double* __restrict__ lam,
                                    const double* __restrict__ U, uint64_t seed, int64_t attempt,
                                    int mode, int distance, double* T_out, double* lam_out,
                                    int32_t* partner, uint8_t* acc, double* vscale,
                                    double* uscale) {
  extern __shared__ __align__(16) unsigned char sh[];
  double* key = reinterpret_cast<double*>(sh);
  int* order = reinterpret_cast<int*>(key + R);
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
  rank_sort(key, order, R);
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
      v[3 * o + 0] = S.vx[g];
      v[3 * o + 1] = S.vy[g];
      v[3 * o + 2] = S.vz[g];
    }
    if (f) {
      f[3 * o + 0] = S.fx[g];
      f[3 * o + 1] = S.fy[g];
      f[3 * o + 2] = S.fz[g];
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
      S.vx[g] = v[3 * o + 0];
      S.vy[g] = v[3 * o + 1];
      S.vz[g] = v[3 * o + 2];
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

template <bool FP64, int P, bool LSM, int MODE>
static cudaError_t launch_batched_t(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                   const int* d_work, int n_work, const int32_t* d_budget,
                                   const LaunchCfg& cfg, int max_n, int max_ncell,
                                   size_t list_elems, int async_nx, cudaStream_t st,
                                   const FreeDev* fr) {
  const size_t smem = batched_smem_bytes(max_n, max_ncell, cfg.threads, FP64, list_elems);
  auto fn = md_batched_kernel<FP64, P, LSM, MODE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the rest of the SM's 256 KB serves as L1 (lists in global memory, state)
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, cfg.threads, smem);
  per_sm = std::max(1, per_sm);
  const int carve = (int)std::min<size_t>(100, (per_sm * (smem + 1024) * 100 + 232447) / 232448);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
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
  KernelDims dims{max_n, max_ncell, list_elems, async_nx};
  FreeDev f{};
  if (fr) f = *fr;
  return cudaLaunchKernelEx(&lc, fn, s, d_ens, d_rep, d_work, d_budget, dims, f);
}

template <bool FP64, int P, bool LSM>
static int max_active_clusters_t(const LaunchCfg& cfg, int max_n, int max_ncell,
                                 size_t list_elems) {
  const size_t smem = batched_smem_bytes(max_n, max_ncell, cfg.threads, FP64, list_elems);
  auto fn = md_batched_kernel<FP64, P, LSM, 2>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)cfg.cluster);
  lc.blockDim = dim3((unsigned)cfg.threads);
  lc.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cfg.cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &lc) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int batched_max_active_clusters(bool fp64, const LaunchCfg& cfg, int max_n, int max_ncell) {
#define RE_MC(F, PP) return max_active_clusters_t<F, PP, false>(cfg, max_n, max_ncell, 0);
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
  return launch_batched_t<F, PP, LS, M>(s, d_ens, d_rep, d_work, n_work, d_budget, cfg,      \
                                        max_n, max_ncell, list_elems, async_nx, st, fr);
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
  const size_t smem = (size_t)R * (sizeof(double) + sizeof(int));
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
