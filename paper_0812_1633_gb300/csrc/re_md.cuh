// re_md.cuh -- device building blocks of the sm_103a replica-exchange LJ MD
// kernels shared by every translation unit of the library: cell binning,
// neighbour-list build, pair forces, thermostat records, the exchange rule
// and the free-running exchange protocol.  Internal header.
#pragma once
#include <cooperative_groups.h>

#include <algorithm>

#include "re_device.cuh"
#include "re_internal.h"

namespace re {
namespace cg = cooperative_groups;

namespace {

constexpr int kMaxCluster = 8;
constexpr int kMaxWarps = 32;
constexpr int kPlainRed = 1024;  // per-replica reduction slots of the plain path
constexpr int kNoiseChunk = 64;  // thermostat records prepared at a time (double buffered)
constexpr int kSvrStepBytes = 32;  // sizeof(SvrStep)

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
//
// The cutoff test.  The force is truncated at rc (Example section), so it
// jumps there by F(rc) ~ 0.04: a pair put on the wrong side of rc costs its
// atoms a force error of ~1e-3 of the rms force, and the FP32 r^2 (relative
// error below 3e-7) would do that for pairs within ~1e-7 of rc -- about one
// pair per ten evaluations of a 4000-atom replica.  So FP32 decides every
// pair outside a relative band of 2e-6 around rc^2, and pairs inside the band
// are decided in FP64 on 42-bit separations: the top 32 bits and the next 10
// bits of each coordinate (kept in .w of the shared-memory position, 10 bits
// per coordinate).  The result equals the FP64 test on the full positions
// except for pairs within ~1e-11 of rc.
struct MixedAcc {
  float fx, fy, fz, e;
  int nin;
  float r2max;  // largest r^2 counted inside ...
  int jmax;     // ... and its atom (checked exactly when r2max lies in the band)
};

// The cutoff constants the pair loop keeps in registers; the band's lower
// edge and rc^2 in 42-bit units are read from the step constants (shared
// memory) only after the loop, so that they hold no register during it.
struct MixedCut {
  float hi;         // rc^2 (1 + 2e-6), units (L / 2^32)^2
  float inv_lam2;   // (2^32 / L)^2
};

// 42-bit minimum-image separation of one coordinate: top 32 bits (hj, hi) and
// the next 10 bits (lj, li) of the two positions.
__device__ __forceinline__ double sep42(uint32_t hj, uint32_t hi, uint32_t lj, uint32_t li) {
  return (double)(((long long)(int)(hj - hi) << 10) + ((long long)lj - (long long)li));
}

__device__ __forceinline__ bool inside_cutoff_42(uint4 pi, uint4 pj, double x42) {
  const double dx = sep42(pj.x, pi.x, (pj.w >> 20) & 1023u, (pi.w >> 20) & 1023u);
  const double dy = sep42(pj.y, pi.y, (pj.w >> 10) & 1023u, (pi.w >> 10) & 1023u);
  const double dz = sep42(pj.z, pi.z, pj.w & 1023u, pi.w & 1023u);
  return fma(dx, dx, fma(dy, dy, dz * dz)) < x42;
}

// The pair force on i from j: fs * d with fs = s^4 (24 - 48 s^3), s = 1/r^2
// (sigma units), d = (dx, dy, dz); energy 4 s^3 (s^3 - 1).
template <bool ENERGY>
__device__ __forceinline__ void mixed_pair_add(float r2, float dx, float dy, float dz,
                                               float inv_lam2, float sign, MixedAcc& a) {
  const float s = rcp_approx(r2) * inv_lam2;
  const float s3 = s * s * s;
  const float fs = sign * (s * s3) * fmaf(-48.0f, s3, 24.0f);
  a.fx = fmaf(fs, dx, a.fx);
  a.fy = fmaf(fs, dy, a.fy);
  a.fz = fmaf(fs, dz, a.fz);
  if (ENERGY) {
    a.e = fmaf(sign * s3, fmaf(4.0f, s3, -4.0f), a.e);
    a.nin += (int)sign;
  }
}

// Every pair with FP32 r^2 < cut.hi is counted inside; a.r2max and a.jmax
// remember the largest such r^2 and its atom.  The caller then checks that
// pair exactly when it lies in the band (mixed_cut_fix).
template <bool ENERGY, bool MAYBE_SELF>
__device__ __forceinline__ void mixed_pair(uint4 pi, uint4 pj, int j, const MixedCut& cut,
                                           MixedAcc& a) {
  const float dx = (float)(int)(pj.x - pi.x);
  const float dy = (float)(int)(pj.y - pi.y);
  const float dz = (float)(int)(pj.z - pi.z);
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  // r2 == 0 only for the atom itself (sub-list padding, last block only);
  // distinct atoms at distance 0 are reported by the list build
  if (r2 < cut.hi && (!MAYBE_SELF || r2 > 0.0f)) {
    if (r2 > a.r2max) {
      a.r2max = r2;
      a.jmax = j;
    }
    mixed_pair_add<ENERGY>(r2, dx, dy, dz, cut.inv_lam2, 1.0f, a);
  }
}

// After the sub-list: if the largest r^2 counted lies in the band and the
// 42-bit separations put that pair outside rc, take its contribution out
// again.  (A second band pair in one sub-list -- about one sub-list in 1e8 --
// stays counted as the FP32 test decided.)
template <bool ENERGY>
__device__ __forceinline__ void mixed_cut_fix(const uint4* pos, int i, const StepConst& K,
                                              MixedAcc& a) {
  if (a.r2max > K.rc2u_lo) {
    const uint4 pi = pos[i], pj = pos[a.jmax];
    if (!inside_cutoff_42(pi, pj, K.rc2x)) {
      const float dx = (float)(int)(pj.x - pi.x);
      const float dy = (float)(int)(pj.y - pi.y);
      const float dz = (float)(int)(pj.z - pi.z);
      mixed_pair_add<ENERGY>(a.r2max, dx, dy, dz, K.inv_lam2, -1.0f, a);
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
  uint32_t* ref;     // 3 per own atom: top 32 bits of the coordinates at the last list build
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
  const size_t o_ref = take(fp64 ? 0 : (size_t)threads * 3 * 4, 4);  // own atoms <= threads
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
    out->ref = reinterpret_cast<uint32_t*>(base + o_ref);
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
        // (four were measured slower)
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
__device__ __forceinline__ MixedAcc mixed_sublist_forces(int i, const uint4* __restrict__ pos,
                                                         const uint16_t* __restrict__ nb,
                                                         uint32_t col, uint32_t ncols, int cnt,
                                                         const StepConst& K) {
  MixedAcc a{0.f, 0.f, 0.f, 0.f, 0, 0.f, 0};
  const MixedCut cut{K.rc2u_hi, K.inv_lam2};
  const uint4 pi = pos[i];
  const size_t stride4 = (size_t)ncols * 4;
  const uint16_t* base = nb + (size_t)col * 4;
  const int nblk = (cnt + 3) >> 2;
  const int nfull = cnt >> 2;
  uint2 w = nblk > 0 ? *reinterpret_cast<const uint2*>(base) : make_uint2(0u, 0u);
  for (int kb = 0; kb < nfull; ++kb) {
    // the next block of indices is requested before this block is used
    const uint2 wn = kb + 1 < nblk ? *reinterpret_cast<const uint2*>(base + (size_t)(kb + 1) * stride4) : w;
    const int j0 = w.x & 0xFFFFu, j1 = w.x >> 16, j2 = w.y & 0xFFFFu, j3 = w.y >> 16;
    const uint4 p0 = pos[j0];
    const uint4 p1 = pos[j1];
    const uint4 p2 = pos[j2];
    const uint4 p3 = pos[j3];
    mixed_pair<ENERGY, false>(pi, p0, j0, cut, a);
    mixed_pair<ENERGY, false>(pi, p1, j1, cut, a);
    mixed_pair<ENERGY, false>(pi, p2, j2, cut, a);
    mixed_pair<ENERGY, false>(pi, p3, j3, cut, a);
    w = wn;
  }
  if (nblk > nfull) {
    const int j0 = w.x & 0xFFFFu, j1 = w.x >> 16, j2 = w.y & 0xFFFFu, j3 = w.y >> 16;
    const uint4 p0 = pos[j0];
    const uint4 p1 = pos[j1];
    const uint4 p2 = pos[j2];
    const uint4 p3 = pos[j3];
    mixed_pair<ENERGY, true>(pi, p0, j0, cut, a);
    mixed_pair<ENERGY, true>(pi, p1, j1, cut, a);
    mixed_pair<ENERGY, true>(pi, p2, j2, cut, a);
    mixed_pair<ENERGY, true>(pi, p3, j3, cut, a);
  }
  mixed_cut_fix<ENERGY>(pos, i, K, a);
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
// Every wait is bounded (fr.wait_ns of the global timer, and an iteration
// cap); a replica that gives up or fails raises the ensemble's abort flag.
// The master's collection of temperatures also ends when that flag is up.  A
// replica waiting for its partner's pair message does not: the partner has
// already seen the pattern (it is issued before any abort can follow from
// it), so it either publishes or has stopped answering, and ending the wait
// early on the flag could leave one member of a pair swapped and the other
// not.

// true when *p >= want; false when the wait ran out or abort_flag (if not
// null) was raised
__device__ bool wait_at_least(const int* p, int want, const int* abort_flag, uint64_t wait_ns) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (ld_acquire(p) >= want) return true;
    if (abort_flag && *reinterpret_cast<const volatile int*>(abort_flag)) return false;
    if ((it & 63u) == 63u && global_ns() - t0 > wait_ns) return false;
    __nanosleep(32);
  }
  return false;
}

// The master's part, by one warp: pattern k of ensemble e.  Returns false when
// a wait gave up.
__device__ bool issue_pattern(const FreeDev& fr, const StateDev& S, const EnsHdr& E, int e, int k,
                              int64_t attempt) {
  const int lane = threadIdx.x & 31;
  const int R = E.R, base = E.rep_off;
  bool ok = true;
  if (k > 0)
    for (int m = lane; m < R && ok; m += 32) ok = wait_at_least(fr.done + base + m, k, fr.abort_ + e, fr.wait_ns);
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
__device__ double pair_exchange(const FreeDev& fr, const StateDev& S, const EnsHdr& E,
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
  if (!wait_at_least(fr.flag + gp, k + 1, nullptr, fr.wait_ns)) {
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

}  // namespace
}  // namespace re
