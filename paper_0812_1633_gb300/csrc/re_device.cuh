// re_device.cuh -- device helpers of the sm_103a replica-exchange LJ MD kernels.
//
// Counter-based random numbers (Philox4x64-10, Salmon et al., SC'11), the
// Box-Muller transform, Marsaglia-Tsang Gamma variates (ACM TOMS 2000), the
// stochastic-velocity-rescaling factor (Bussi, Donadio, Parrinello, JCP 126,
// 014101, 2007: the thermostat of the paper's Example section), fixed-point
// positions and block reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace re {

// Philox stream tags; the layout is part of the library contract (re.h).
constexpr uint64_t kTagVel = 1, kTagSvrR1 = 2, kTagSvrGamma = 3, kTagExch = 4, kTagParity = 5;

struct U64x4 {
  uint64_t a, b, c, d;
};

// Philox4x64-10: ten rounds; each round multiplies words 0 and 2 by the two
// round constants (128-bit products), xors the high halves with the other
// words and the round key, and the key advances by the Weyl increments.
__device__ __forceinline__ U64x4 philox4x64_10(U64x4 x, uint64_t k0, uint64_t k1) {
  constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t h0 = __umul64hi(M0, x.a), l0 = M0 * x.a;
    const uint64_t h1 = __umul64hi(M1, x.c), l1 = M1 * x.c;
    x = U64x4{h1 ^ x.b ^ k0, l1, h0 ^ x.d ^ k1, l0};
  }
  return x;
}

__device__ __forceinline__ double to_unit(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

struct Uni4 {
  double u0, u1, u2, u3;
};

__device__ __forceinline__ Uni4 uniforms(uint64_t seed, uint64_t stream, uint64_t index,
                                         uint64_t tag, uint64_t sub) {
  const U64x4 o = philox4x64_10(U64x4{index, tag, sub, 0ull}, seed, stream);
  return Uni4{to_unit(o.a), to_unit(o.b), to_unit(o.c), to_unit(o.d)};
}

// Box-Muller: radius sqrt(-2 ln(1 - u0)) (1 - u0 in (0, 1]), angle 2 pi u1.
__device__ __forceinline__ void box_muller(double u0, double u1, double* g_cos, double* g_sin) {
  const double rho = sqrt(-2.0 * log(1.0 - u0));
  double s, c;
  sincospi(2.0 * u1, &s, &c);
  *g_cos = rho * c;
  *g_sin = rho * s;
}

// Gamma(a, 1) for a >= 1 by Marsaglia & Tsang: with d = a - 1/3 and
// c = 1/sqrt(9 d), propose d (1 + c x)^3 for standard normal x, accept on the
// squeeze u < 1 - 0.0331 x^4 or on log u < x^2/2 + d (1 - v + log v).  Trial
// t consumes Philox block (index, tag, t).  The loop is capped; past the cap
// (probability far below 1e-100 for a >= 1) the mean a is returned and *capped
// is set.
__device__ inline double gamma_marsaglia_tsang(double a, uint64_t seed, uint64_t stream,
                                               uint64_t index, int* capped) {
  const double d = a - 1.0 / 3.0;
  const double c = 1.0 / sqrt(9.0 * d);
  for (int t = 0; t < 256; ++t) {
    const Uni4 u = uniforms(seed, stream, index, kTagSvrGamma, (uint64_t)t);
    double x, unused;
    box_muller(u.u0, u.u1, &x, &unused);
    const double w = 1.0 + c * x;
    if (w <= 0.0) continue;
    const double v = w * w * w;
    const double x2 = x * x;
    if (u.u2 < 1.0 - 0.0331 * x2 * x2) return d * v;
    if (log(u.u2) < 0.5 * x2 + d * (1.0 - v + log(v))) return d * v;
  }
  *capped = 1;
  return a;
}

// Thermostat noise of one step: R1 ~ N(0,1) and S ~ chi^2 with nf - 1 degrees.
__device__ inline double2 svr_noise(int nf, uint64_t seed, uint64_t stream, uint64_t step,
                                    int* capped) {
  const Uni4 u = uniforms(seed, stream, step, kTagSvrR1, 0ull);
  double r1, unused;
  box_muller(u.u0, u.u1, &r1, &unused);
  const double s = 2.0 * gamma_marsaglia_tsang(0.5 * (double)(nf - 1), seed, stream, step, capped);
  return make_double2(r1, s);
}

// The same draws in FP32 (mixed path): the top 24 bits of the same Philox
// words, Box-Muller and Marsaglia-Tsang in single precision.
__device__ __forceinline__ float to_unit_f(uint64_t w) { return (float)(w >> 40) * 5.9604644775390625e-08f; }

__device__ inline float2 svr_noise_f32(int nf, uint64_t seed, uint64_t stream, uint64_t step,
                                       int* capped) {
  const U64x4 o = philox4x64_10(U64x4{step, kTagSvrR1, 0ull, 0ull}, seed, stream);
  float s0, c0;
  sincospif(2.0f * to_unit_f(o.b), &s0, &c0);
  const float r1 = sqrtf(-2.0f * logf(1.0f - to_unit_f(o.a))) * c0;
  const float a = 0.5f * (float)(nf - 1);
  const float d = a - 1.0f / 3.0f;
  const float c = rsqrtf(9.0f * d);
  for (int t = 0; t < 256; ++t) {
    const U64x4 g = philox4x64_10(U64x4{step, kTagSvrGamma, (uint64_t)t, 0ull}, seed, stream);
    float sn, cs;
    sincospif(2.0f * to_unit_f(g.b), &sn, &cs);
    const float x = sqrtf(-2.0f * logf(1.0f - to_unit_f(g.a))) * cs;
    const float w = 1.0f + c * x;
    if (w <= 0.0f) continue;
    const float v = w * w * w;
    const float u = to_unit_f(g.c);
    const float x2 = x * x;
    if (u < 1.0f - 0.0331f * x2 * x2 || logf(u) < 0.5f * x2 + d * (1.0f - v + logf(v)))
      return make_float2(r1, 2.0f * d * v);
  }
  *capped = 1;
  return make_float2(r1, 2.0f * a);
}

// Stochastic velocity rescaling over one step: the new kinetic energy is
//   K' = c K + (1 - c) Kbar (R1^2 + S)/Nf + 2 R1 sqrt(c (1 - c) Kbar K / Nf)
// (c = exp(-dt/tau), Kbar = Nf T/2) and velocities scale by
// alpha = +-sqrt(K'/K), negative when R1 + sqrt(c Nf K / ((1 - c) Kbar)) < 0.
__device__ inline double svr_alpha(double K, double Kbar, int nf, double c, double r1, double s,
                                   double* Knew) {
  const double f = (double)nf;
  const double kp = c * K + (1.0 - c) * Kbar * (r1 * r1 + s) / f +
                    2.0 * r1 * sqrt(c * (1.0 - c) * Kbar * K / f);
  double alpha = sqrt(kp / K);
  if (r1 + sqrt(c * f * K / ((1.0 - c) * Kbar)) < 0.0) alpha = -alpha;
  *Knew = kp;
  return alpha;
}

// ------------------------------------------------------------- fixed point
// A coordinate x in the periodic box [0, L) is stored as q = x/L * 2^64
// (uint64, wrapping).  The difference of two such words read as a signed
// integer is the minimum-image separation, exactly; the top 32 bits give a
// 32-bit copy for single-precision pair arithmetic.
__device__ __forceinline__ uint64_t fix_from_double(double x, double inv_l) {
  double t = x * inv_l;
  t -= floor(t);
  const double q = t * 0x1.0p64;
  return q >= 0x1.0p64 ? 0ull : __double2ull_rn(q);
}

__device__ __forceinline__ double fix_to_double(uint64_t q, double l) {
  return __ull2double_rn(q) * (l * 0x1.0p-64);
}

// exact conversion of a signed 32-bit integer to the nearest float without the
// conversion unit: split into a high and a low 16-bit part, each made exact by
// the 2^23 exponent trick, and join them with one rounding in an FMA.
__device__ __forceinline__ float i32_to_f32_split(int v) {
  const float hi = __int_as_float(0x4B400000 + (v >> 16)) - 12582912.0f;       // v >> 16 in [-2^15, 2^15)
  const float lo = __int_as_float(0x4B000000 | (v & 0xFFFF)) - 8388608.0f;     // low 16 bits
  return fmaf(hi, 65536.0f, lo);
}

// 64-bit integer <-> float conversions through two 32-bit conversions (the
// 64-bit forms run on the FP64 unit, about 2 per clock per SM on this GPU;
// the 32-bit forms run at more than 50 per clock).
// nearest int64 to y, |y| < 2^62 (within one unit)
__device__ __forceinline__ long long f2ll_split(float y) {
  const int hi = __float2int_rn(y * 2.3283064365386963e-10f);  // y / 2^32
  const float rem = fmaf((float)hi, -4294967296.0f, y);        // exact
  const int lo = __float2int_rn(rem);
  return ((long long)hi << 32) + (long long)lo;
}
// float nearest to v (one extra rounding of the low word, below 2^-24 relative)
__device__ __forceinline__ float ll2f_split(long long v) {
  const int hi = (int)(v >> 32);
  const unsigned lo = (unsigned)(v & 0xFFFFFFFFll);
  return fmaf((float)hi, 4294967296.0f, (float)lo);
}

// ------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_or(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order (lane tree, then warps in order);
// every thread gets the result.  scratch: >= 32 doubles of shared memory.
__device__ inline double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += scratch[w];
  return t;
}

__device__ inline float block_max(float v, float* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  float t = 0.0f;
  for (int w = 0; w < nw; ++w) t = fmaxf(t, scratch[w]);
  return t;
}

__device__ inline int block_or(int v, int* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_or(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  int t = 0;
  for (int w = 0; w < nw; ++w) t |= scratch[w];
  return t;
}

// ------------------------------------------------- inter-CTA signalling
// Release/acquire accesses at GPU scope (PTX memory model) for the flags of
// the free-running exchange, and a wall clock for bounded waits.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 8-byte asynchronous global -> shared copy (both addresses 8-byte aligned);
// completes at cp_async_wait_all.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Velocity and force words of the mixed path's native state (StateDev::vfix):
// v as 64-bit fixed point in units of 2^-48, the half-kick increment as FP32.
__device__ __forceinline__ long long vfix_get(const double* a, size_t g) {
  return reinterpret_cast<const long long*>(a)[g];
}
__device__ __forceinline__ void vfix_put(double* a, size_t g, long long vq) {
  reinterpret_cast<long long*>(a)[g] = vq;
}
__device__ __forceinline__ float hfix_get(const double* a, size_t g) {
  return __uint_as_float((uint32_t)reinterpret_cast<const unsigned long long*>(a)[g]);
}
__device__ __forceinline__ void hfix_put(double* a, size_t g, float h) {
  reinterpret_cast<unsigned long long*>(a)[g] = __float_as_uint(h);
}
__device__ __forceinline__ double vfix_to_double(long long vq) { return (double)vq * 0x1.0p-48; }
__device__ __forceinline__ long long vfix_from_double(double v) {
  return __double2ll_rn(v * 0x1.0p48);
}
// pending factors: v <- v * vs, the half-kick increment (and the force) <- * fs
__device__ __forceinline__ long long vfix_scale(long long vq, double vs) {
  return __double2ll_rn((double)vq * vs);
}
__device__ __forceinline__ float hfix_scale(float h, double fs) { return (float)((double)h * fs); }

}  // namespace re
