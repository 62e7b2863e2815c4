// re_noalloc.cu -- LJ forces of caller-given positions without any device or
// host allocation, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or under a fixed memory budget, a plug-in that may
// not touch the allocator, or a path that must not add allocation latency.
// re_lj_forces_device_noalloc serves them: it computes what
// re_lj_forces_device computes (FP64 pair forces; same cell binning,
// neighbour-list and force kernels, those of the plain path) but keeps every
// intermediate array (fixed-point positions, lists, counters, reduction
// partials, tables) in one file-scope device array, g_scratch, of fixed size.
//
// Limits: N <= kMaxAtoms atoms and at most kMaxNeighbours list entries per
// atom (density times the list-sphere volume, with margin).  The array lives
// on every device that loads this library until the process exits.  The
// first call on a device looks up the array's device address
// (cudaGetSymbolAddress) and caches it; make that first call before any
// stream capture.  All calls share the array: it keeps the previous call's
// contents, the call clears what must start at zero, and calls that overlap
// on the GPU (different streams, or threads without ordering) race.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "re.h"
#include "re_internal.h"

namespace {

constexpr int kMaxAtoms = 4096;
constexpr int kMaxNeighbours = 256;
constexpr int kMaxDevices = 64;
constexpr size_t kAlign = 256;

constexpr size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch array for up to kMaxAtoms atoms (one replica).
struct Layout {
  size_t q, v, f, r, ncnt, nbr, scal, red, tab, total;
};
constexpr Layout layout() {
  Layout l{};
  size_t o = 0;
  l.q = o;    o += up(3 * 8 * (size_t)kMaxAtoms);
  l.v = o;    o += up(3 * 8 * (size_t)kMaxAtoms);
  l.f = o;    o += up(3 * 8 * (size_t)kMaxAtoms);
  l.r = o;    o += up(3 * 4 * (size_t)kMaxAtoms);
  l.ncnt = o; o += up(8 * 4 * (size_t)kMaxAtoms);
  l.nbr = o;  o += up(2 * (size_t)kMaxNeighbours * kMaxAtoms);
  l.scal = o; o += up(16 * 8);
  l.red = o;  o += up(1024 * 8);
  l.tab = o;  o += up(sizeof(re::EnsDev)) + up(sizeof(re::RepDev));
  l.total = o;
  return l;
}
constexpr Layout kL = layout();

// device address of g_scratch, per device; every thread that fills an entry
// stores the same value, so relaxed atomic accesses suffice
std::atomic<void*> g_scratch_dev[kMaxDevices];

// errors are reported by return code only (a message would need allocation)
int fail(int code, const char*) { return code; }

}  // namespace

// The scratch array: one per device that loads the library, for its lifetime.
static __device__ __align__(256) unsigned char g_scratch[kL.total];

extern "C" int re_lj_forces_device_noalloc(int N, double L, double rc, int shift, const double* x,
                                           double* f, double* U, void* stream) {
  if (N < 2 || N > kMaxAtoms) return fail(RE_EINVAL, "N must be in [2, 4096]");
  if (!x || !f || !U) return fail(RE_EINVAL, "NULL device pointer");
  if (!(L > 0) || !(rc > 0) || rc + 0.5 >= 0.5 * L) return fail(RE_EINVAL, "need rc + 0.5 < L/2");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(RE_ECUDA, "no usable current device");
  // once per device, with that device current: the array's device address
  void* sp = g_scratch_dev[dev].load(std::memory_order_relaxed);
  if (!sp) {
    const cudaError_t e = cudaGetSymbolAddress(&sp, g_scratch);
    if (e != cudaSuccess || !sp) return fail(RE_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    g_scratch_dev[dev].store(sp, std::memory_order_relaxed);
  }
  unsigned char* base = static_cast<unsigned char*>(sp);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // the ensemble table of one replica (list radius rc + 0.5)
  re::EnsDev e{};
  e.N = N;
  e.R = 1;
  e.L = L;
  e.rc = rc;
  e.skin = 0.5;
  e.rlist = rc + 0.5;
  e.dt = 0.005;
  e.tau = 0.0;
  e.shift = shift ? 1 : 0;
  re::set_capacity(e, 0);
  re::finish_ens(e);
  if (e.capsub[0] > kMaxNeighbours)
    return fail(RE_EOVERFLOW, "density too high for the fixed neighbour capacity (256 per atom)");
  re::choose_cells(L, e.rlist, N, 0, &e.nc, &e.m);
  // the plain list build keeps cells in shared memory: fall back to all pairs
  // when the cell table would not fit
  const size_t fixed = (size_t)N * 30 + 64;
  if (e.nc > 0 && fixed + (size_t)(e.nc * e.nc * e.nc + 1) * 8 > 200 * 1024) e.nc = e.m = 0;
  re::RepDev rd{};
  rd.ens = 0;
  rd.id = 0;
  rd.stream = 0;
  rd.atom_off = 0;
  rd.nbr_off = 0;

  re::StateDev s{};
  s.qx = reinterpret_cast<uint64_t*>(base + kL.q);
  s.qy = s.qx + N;
  s.qz = s.qy + N;
  s.vx = reinterpret_cast<double*>(base + kL.v);
  s.vy = s.vx + N;
  s.vz = s.vy + N;
  s.fx = reinterpret_cast<double*>(base + kL.f);
  s.fy = s.fx + N;
  s.fz = s.fy + N;
  s.rx = reinterpret_cast<uint32_t*>(base + kL.r);
  s.ry = s.rx + N;
  s.rz = s.ry + N;
  s.ncnt = reinterpret_cast<int32_t*>(base + kL.ncnt);
  s.nbr = reinterpret_cast<uint16_t*>(base + kL.nbr);
  double* sd = reinterpret_cast<double*>(base + kL.scal);
  s.T = sd + 0;
  s.U = sd + 1;
  s.K = sd + 2;
  s.econs = sd + 3;
  s.vscale = sd + 4;
  s.step = reinterpret_cast<int64_t*>(sd + 5);
  s.nreb = reinterpret_cast<int64_t*>(sd + 6);
  s.attempt = reinterpret_cast<int64_t*>(sd + 7);
  s.pair_att = reinterpret_cast<int64_t*>(sd + 8);
  s.pair_acc = reinterpret_cast<int64_t*>(sd + 9);
  s.status = reinterpret_cast<int32_t*>(sd + 10);
  s.valid = s.status + 1;
  s.dmax = reinterpret_cast<uint32_t*>(sd + 11);
  s.red = reinterpret_cast<double*>(base + kL.red);
  re::EnsDev* d_ens = reinterpret_cast<re::EnsDev*>(base + kL.tab);
  re::RepDev* d_rep = reinterpret_cast<re::RepDev*>(base + kL.tab + up(sizeof(re::EnsDev)));

  // clear what must start at zero (the array keeps the previous call's data)
  cudaError_t ce;
  if ((ce = cudaMemsetAsync(base + kL.scal, 0, 16 * 8, st)) ||
      (ce = cudaMemsetAsync(base + kL.v, 0, 3 * 8 * (size_t)N, st)) ||
      (ce = cudaMemcpyAsync(d_ens, &e, sizeof e, cudaMemcpyHostToDevice, st)) ||
      (ce = cudaMemcpyAsync(d_rep, &rd, sizeof rd, cudaMemcpyHostToDevice, st)))
    return fail(RE_ECUDA, cudaGetErrorString(ce));
  // positions -> fixed point (also marks the list invalid), list build,
  // forces and energy, forces back to the caller
  if ((ce = re::launch_import_state(s, d_ens, d_rep, 1, x, nullptr, st)) ||
      (ce = re::launch_plain_advance(s, e, rd, 0, d_ens, d_rep, 0, 0, st, 1)) ||
      (ce = re::launch_export_state(s, d_ens, d_rep, 1, nullptr, nullptr, f, st)) ||
      (ce = cudaMemcpyAsync(U, s.U, sizeof(double), cudaMemcpyDeviceToDevice, st)))
    return fail(RE_ECUDA, cudaGetErrorString(ce));
  int32_t status = 0;
  if ((ce = cudaMemcpyAsync(&status, s.status, sizeof status, cudaMemcpyDeviceToHost, st)) ||
      (ce = cudaStreamSynchronize(st)))
    return fail(RE_ECUDA, cudaGetErrorString(ce));
  if (status & re::kStOverflow) return fail(RE_EOVERFLOW, "neighbour list capacity exceeded");
  if (status) return fail(RE_ENUMERIC, "non-finite energy (overlapping atoms?)");
  return RE_OK;
}
