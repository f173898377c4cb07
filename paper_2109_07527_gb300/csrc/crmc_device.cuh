// crmc_device.cuh -- device primitives of the CR-MC kernels: Philox4x32-10,
// the FP32 cell and insertion-coordinate rules, DSF and WCA pair terms, and
// warp-level list helpers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "crmc_common.h"

namespace crmc {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the
// two 32x32->64 multiplications with the key bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                          uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// integer in [0, n): floor(w * n / 2^32)
__device__ __forceinline__ int pick32(uint32_t w, int n) {
  return (int)(((unsigned long long)w * (unsigned long long)(unsigned)n) >> 32);
}

// uniform in (0, 1) with 53 bits; every operation is exact
__device__ __forceinline__ double unif53(uint32_t whi, uint32_t wlo) {
  const double a = (double)(whi >> 5), b = (double)(wlo >> 6);
  return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0);
}

// Cell of a coordinate: floor(fl32(x * nc/L)), clamped.  Taken in FP32
// (explicitly rounded multiply, no contraction) because it decides which
// domain owns a particle.
__device__ __forceinline__ int cell_of(float x, float scf, int nc) {
  const float t = __fmul_rn(x, scf);
  const int c = (int)floorf(t);
  return min(max(c, 0), nc - 1);
}

// Insertion coordinate in a domain whose first cell is c0, in FP32 with
// explicitly rounded operations: f = top 24 bits of w times 2^-24,
// u = fl32(c0 + k f) wrapped into [0, nc), x = fl32(u * a) wrapped into [0, L).
__device__ __forceinline__ float insert_coord(int c0, uint32_t w, int k, int nc, float af, float Lf) {
  const float f = __fmul_rn((float)(w >> 8), 1.0f / 16777216.0f);
  const float kf = __fmul_rn((float)k, f);
  float u = __fadd_rn((float)c0, kf);
  if (u >= (float)nc) u = __fsub_rn(u, (float)nc);
  float xf = __fmul_rn(u, af);
  if (xf >= Lf) xf = __fsub_rn(xf, Lf);
  return xf;
}

// round(v * 2^32) as a 64-bit integer for |v| < 2^20, from two 32-bit
// conversions (the direct float->int64 conversion is several times slower):
// v = hi + lo with hi = trunc(v) and lo exact, lo * 2^31 rounded to int32.
__device__ __forceinline__ long long fix32(float v) {
  const float hi = truncf(v);
  const float lo = v - hi;
  const int l = __float2int_rn(lo * 2147483648.0f);
  return ((long long)(int)hi << 32) + ((long long)l << 1);
}

// the same at scale 2^24 for |v| < 2^30 (MD forces)
__device__ __forceinline__ long long fix24(float v) {
  v = fminf(fmaxf(v, -1073741824.0f), 1073741824.0f);
  const float hi = truncf(v);
  const float lo = v - hi;
  const int l = __float2int_rn(lo * 8388608.0f);
  return ((long long)(int)hi << 24) + ((long long)l << 1);
}

// kind of a slot for the eligibility lists, from its info word
__device__ __forceinline__ int kind_of(int info) {
  const int t = info & INFO_TYPE_MASK;
  const int ion = (info >> 6) & 1;
  // (type, ionised) -> kind; table nibbles for index 2*type + ionised, types
  // bead, acid, base, X+, X-, core, S+, S-
  const unsigned long long tab = 0x7766885544321088ull;
  const int idx = 2 * t + ion;
  return idx < 16 ? (int)((tab >> (4 * idx)) & 15ull) : K_OTHER;
}


// Minimum-image difference a - b of two coordinates in [0, L) without the
// large intermediate a - b ~ L: across the boundary the coordinate above L/2
// is shifted by L first, which is exact (Sterbenz).
__device__ __forceinline__ float wrap_diff(float a, float b, float L, float halfL) {
  const float d = a - b;
  if (d > halfL) return (a - L) - b;
  if (d < -halfL) return a - (b - L);
  return d;
}
__device__ __forceinline__ double wrap_diff_d(float a, float b, double L, double halfL) {
  double d = (double)a - (double)b;
  if (d > halfL) d -= L;
  else if (d < -halfL) d += L;
  return d;
}

// WCA change of an inserted (dp > 0) or deleted (dp < 0) particle against a
// bystander, in FP64 from the exact float positions: the steep (sigma/s)^12
// would amplify FP32 distance rounding twelvefold.  Returns the change and
// its gross magnitude; flags an overlap when an inserted particle comes
// closer than half a diameter.
__device__ __forceinline__ bool wca_change_d(const WcaEntry &w, int dp, float cx, float cy, float cz, float xj,
                                             float yj, float zj, double L, double halfL, double &du, double &gs,
                                             int &ov) {
  const double dx = wrap_diff_d(xj, cx, L, halfL), dy = wrap_diff_d(yj, cy, L, halfL),
               dz = wrap_diff_d(zj, cz, L, halfL);
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  if (!(r < w.wcut_d)) return false;
  const double s = r - w.del_d;
  if (dp > 0 && s < 0.5 * w.sig_d) {
    ov = 1;
    return false;
  }
  const double t = w.sig_d / s;
  const double t2 = t * t;
  const double t6 = t2 * t2 * t2;
  du = (double)dp * (4.0 * w.eps_d * (t6 * t6 - t6) + w.eps_d);
  gs = w.eps_d * (4.0 * t6 * t6 + 4.0 * t6 + 1.0);
  return true;
}

// int64 sum over the warp (mod 2^64, exact), result in every lane: v = a 2^42
// + b 2^21 + c with b, c in [0, 2^21) and a in [-2^21, 2^21), each part
// summed by one 32-bit warp reduction (partial sums below 2^26 in magnitude)
__device__ __forceinline__ long long warp_sum_i64(long long v) {
  const unsigned c = (unsigned)v & 0x1FFFFFu, b = (unsigned)(v >> 21) & 0x1FFFFFu;
  const int a = (int)(v >> 42);
  const unsigned sc = __reduce_add_sync(0xffffffffu, c), sb = __reduce_add_sync(0xffffffffu, b);
  const int sa = (int)__reduce_add_sync(0xffffffffu, (unsigned)a);
  return (long long)sa * (1ll << 42) + (long long)sb * (1ll << 21) + (long long)sc;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace crmc
