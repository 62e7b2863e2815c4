// re_batched.cuh -- the persistent batched MD kernel (one thread-block cluster
// per replica) and its launch helpers, instantiated per precision and mode in
// the re_batched_*.cu translation units so that they compile in parallel.
#pragma once
#include "re_md.cuh"

namespace re {
namespace {

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
// MAXT: the most threads per CTA of this instantiation; it sets the register
// budget (1024: 64 registers per thread; kNarrowThreads = 896: 72), and the
// launcher picks the narrowest instantiation that holds the launch's CTAs.
template <bool FP64, int P, bool LSM, int MODE, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) md_batched_kernel(StateDev S,
                                                             const EnsDev* __restrict__ ens,
                                                             const RepDev* __restrict__ reps,
                                                             const int* __restrict__ work,
                                                             const int32_t* __restrict__ budget,
                                                             KernelDims dims, FreeDev fr) {
  constexpr int ND = (3 + P - 1) / P;  // coordinates per lane
  // replica constants live in shared memory, not in registers
  __shared__ EnsHdr E;
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
    E = static_cast<const EnsHdr&>(ens[rd.ens]);
    K = ens[rd.ens].kc;
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
  // factors of exactly 1 (the rule), tested on the integer units
  const bool vs_one = __double_as_longlong(vs0) == 0x3FF0000000000000LL;
  const bool fs_one = __double_as_longlong(fs0) == 0x3FF0000000000000LL;
  // the replica's stored energies (U, K, econs), kept by thread 0 of each CTA
  // in shared memory (CTA 0's are written back); registers are kept for the
  // per-atom state
  __shared__ double U_sh, K_sh, econs_sh;
  if (threadIdx.x == 0) {
    U_sh = S.U[r];
    K_sh = S.K[r];
    econs_sh = S.econs[r];
  }
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

  // per-lane state in registers (the FP32 velocity of the mixed path is
  // formed from the fixed-point word when needed, and the positions at the
  // last list build are kept in shared memory: registers are the scarce
  // resource of this kernel, which holds the state for a whole launch)
  uint64_t xq[ND];
  double v[ND], f[ND];       // FP64 path
  long long vq[ND];          // mixed path: velocity, fixed point
  float hf[ND];              // mixed path: half-kick increment
  // top 32 bits of the coordinates at the last list build: in shared memory
  // on the mixed path (3 words per own atom), in registers on the FP64 path
  // (whose shared memory holds 64-bit positions)
  uint32_t ref_r[ND];
  uint32_t* ref_sm = FP64 ? nullptr : sm.ref + (size_t)(i - i0) * 3;
  auto ref = [&](int j) -> uint32_t& { return FP64 ? ref_r[j] : ref_sm[q + j * P]; };
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < ND; ++j) {
    const int d = q + j * P;
    xq[j] = 0;
    v[j] = f[j] = 0.0;
    vq[j] = 0;
    hf[j] = 0.0f;
    ref_r[j] = 0;
    if (own && d < 3) {
      xq[j] = qcomp(S, d)[g];
      ref(j) = rcomp(S, d)[g];
      if (FP64) {
        v[j] = vcomp(S, d)[g] * vs0;
        f[j] = fcomp(S, d)[g] * fs0;
      } else {
        // the state is stored in these words: FP64 only for a pending factor
        const long long vb = vfix_get(vcomp(S, d), g);
        const float hb = hfix_get(fcomp(S, d), g);
        vq[j] = vs_one ? vb : vfix_scale(vb, vs0);
        hf[j] = fs_one ? hb : hfix_scale(hb, fs0);
      }
    }
  }
  // FP32 copy of velocity word j (mixed path)
  auto vf = [&](int j) { return ll2f_split(vq[j]) * kVelUnit; };
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
  // broadcast this lane's coordinates of atom i to every CTA of the cluster.
  // Mixed path: the top 32 bits of each coordinate, and in .w the next 10 bits
  // of x, y, z (bits 20-29, 10-19, 0-9), gathered from the atom's lanes by
  // lane q == 0, for the exact cutoff test of mixed_pair.
  auto publish = [&]() {
    uint32_t low = 0;
    if (!FP64) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const uint32_t b = __shfl_sync(0xffffffffu, (uint32_t)(xq[d / P] >> 22) & 1023u,
                                       (lane & ~(P - 1)) | (d % P));
        low |= b << (20 - 10 * d);
      }
    }
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
    if (!FP64 && q == 0) {
      uint32_t* dst = reinterpret_cast<uint32_t*>(&posm[i]) + 3;
      for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(dst, rk) = low;
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
      for (int j = 0; j < ND; ++j)
        if (q + j * P < 3) ref(j) = (uint32_t)(xq[j] >> 32);
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
      MixedAcc a{0.f, 0.f, 0.f, 0.f, 0, 0.f, 0};
      if (own) {
        if (energy)
          a = mixed_sublist_forces<true>(i, posm, nb, mycol, ncols, cnt, K);
        else
          a = mixed_sublist_forces<false>(i, posm, nb, mycol, ncols, cnt, K);
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
          const float w = kick ? vf(j) + hf[j] : vf(j);
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
      const double U0 = 0.5 * su * K.lamv, K0 = 0.5 * sk;
      if (!isfinite(U0) || !isfinite(K0)) status |= kStNumeric;
      if (tid == 0) {
        U_sh = U0;
        K_sh = K0;
      }
    } else {
      long long iu, ik;
      totals_int(iu, ik, status, true);
      if (tid == 0) {
        U_sh = 0.5 * (double)iu * kEnUnit * K.lamv;  // FP64 only for the stored energies
        K_sh = 0.5 * (double)ik * kEnUnit;
      }
    }
  }

  int k_next = 0;           // free-running: next pattern to take part in (uniform)
  bool stalled = false;     // free-running: stopped answering (fault injection)
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
          if (first_kick) vq[j] += f2ll_split(hf[j] * kVelScale);
          xq[j] += (uint64_t)f2ll_split(vf(j) * dtqf);
        }
        const float dd = (float)(int)((uint32_t)(xq[j] >> 32) - ref(j));
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
      if (tid == 0) {
        U_sh = Un;
        K_sh = Kp;
        econs_sh += Kn - Kp;
      }
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
          const float w = vf(j) + hf[j];
          // second half kick + thermostat factor (+ next first half kick)
          const float inc = fmaf(eps, w, bnd ? hf[j] : 2.0f * hf[j]);
          vq[j] += f2ll_split(inc * kVelScale);
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
          dsum = warp_sum(dsum);
          kp = __shfl_sync(0xffffffffu, kp, (slot - fold0) & 31);
          if (lane == 0) {
            econs_sh += dsum;
            K_sh = kp;
            if (energy) U_sh = 0.5 * (double)iu * kEnUnit * K.lamv;
          }
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
    if (xchg && r == fr.stall_rep && k_next >= fr.stall_from) {
      // host-side fault injection: from this pattern on the replica stops
      // answering (no pair message, no "done", no abort flag), as a stalled
      // process would; it leaves the launch at this step boundary
      stalled = true;
      break;
    }
    if (xchg) {
      // this replica's part of the pattern: CTA 0 runs the pair protocol and
      // hands the result to every CTA of the cluster
      if (crank == 0 && tid == 0) {
        double Tn, ln, us;
        int pid, acc;
        bool ok;
        const double sc = pair_exchange(fr, S, E, rd, r, k_next, A0_sh + k_next, Tcur_sh, K.lamv,
                                        U_sh, &Tn, &ln, &us, &pid, &acc, &ok);
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
      if (tid == 0) {
        const double Ks = K_sh * (sc * sc);
        econs_sh += K_sh - Ks;
        K_sh = Ks;
        const double Us = U_sh * us;
        econs_sh += U_sh - Us;
        U_sh = Us;
      }
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
  if (stalled) {
    status |= kStTimeout;
  } else if (freerun && k_next < fr.n_att) {
    // left before the last pattern: the others stop too (waits on this
    // replica would otherwise run to their limit)
    if (crank == 0 && tid == 0) atomicExch(fr.abort_ + rd.ens, 1);
    if ((status & ~(int)kStStop) == 0) status |= kStAborted;
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
      rcomp(S, d)[g] = ref(j);
      if (FP64) {
        vcomp(S, d)[g] = v[j];
        fcomp(S, d)[g] = f[j];
      } else {
        vfix_put(vcomp(S, d), g, vq[j]);
        hfix_put(fcomp(S, d), g, hf[j]);
      }
    }
    ncnt[(size_t)i * P + q] = cnt;
  }
  if (crank == 0 && tid == 0) {
    S.U[r] = U_sh;
    S.K[r] = K_sh;
    S.econs[r] = econs_sh;
    S.step[r] = step0 + done;
    S.nreb[r] += nreb;
    S.vscale[r] = 1.0;
    S.fscale[r] = 1.0;
    S.status[r] = status & ~(int)(kStStop | kStXchg);
    S.valid[r] = (status & kStOverflow) ? 0 : 1;
  }
  cl.sync();  // no CTA leaves while another may still touch its shared memory
}

}  // namespace

template <bool FP64, int P, bool LSM, int MODE, int MAXT>
cudaError_t launch_batched_t(const StateDev& s, const EnsDev* d_ens, const RepDev* d_rep,
                                   const int* d_work, int n_work, const int32_t* d_budget,
                                   const LaunchCfg& cfg, int max_n, int max_ncell,
                                   size_t list_elems, int async_nx, cudaStream_t st,
                                   const FreeDev* fr) {
  const size_t smem = batched_smem_bytes(max_n, max_ncell, cfg.threads, FP64, list_elems);
  auto fn = md_batched_kernel<FP64, P, LSM, MODE, MAXT>;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  if (fa.sharedSizeBytes > kBatchedStaticSmem) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
  e = cudaLaunchKernelEx(&lc, fn, s, d_ens, d_rep, d_work, d_budget, dims, f);
  if (e != cudaSuccess) cudaGetLastError();  // a refused launch leaves no error behind
  return e;
}

template <bool FP64, int P, bool LSM, int MAXT>
int max_active_clusters_t(const LaunchCfg& cfg, int max_n, int max_ncell,
                                 size_t list_elems) {
  const size_t smem = batched_smem_bytes(max_n, max_ncell, cfg.threads, FP64, list_elems);
  auto fn = md_batched_kernel<FP64, P, LSM, 2, MAXT>;
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
}  // namespace re
