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

// Insertion coordinate in a domain whose first cell is c0: u = c0 + k f
// (exact), wrapped to [0, nc), times the FP64 cell side, rounded once to FP32.
__device__ __forceinline__ float insert_coord(int c0, uint32_t w, int k, int nc, double a, float Lf) {
  const double f = (double)(w >> 8) * (1.0 / 16777216.0);
  double u = (double)c0 + (double)k * f;
  if (u >= (double)nc) u -= (double)nc;
  const double xd = __dmul_rn(u, a);
  float xf = __double2float_rn(xd);
  if (xf >= Lf) xf = __fsub_rn(xf, Lf);
  return xf;
}

// kind of a slot for the eligibility lists, from its info word
__device__ __forceinline__ int kind_of(int info) {
  const int t = info & INFO_TYPE_MASK;
  const int ion = (info >> 6) & 1;
  // (type, ionised) -> kind; table nibbles for index 2*type + ionised
  const unsigned long long tab = 0x665544321066ull;
  const int idx = 2 * t + ion;
  return idx < 12 ? (int)((tab >> (4 * idx)) & 15ull) : K_OTHER;
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

// One pair change of a changed particle c against a bystander j:
//   du = lB dq_c q_j phi(r) [r < rc] + dp_c U_wca(r)
// accumulated in 2^-32 kT fixed point: the Coulomb part in FP32, the WCA part
// of inserted / deleted particles in FP64.  Inserted particles closer than
// half a WCA diameter, and any |du| >= 2^20 kT, flag an overlap.
template <bool WITH_S>
__device__ __forceinline__ void pair_change(const SysParams &P, float cx, float cy, float cz, float dqlB, int dp,
                                            int ccls, float xj, float yj, float zj, float qj, int jcls,
                                            long long &acc, unsigned long long &sacc, int &ov) {
  const float dx = wrap_diff(xj, cx, P.Lf, P.halfL);
  const float dy = wrap_diff(yj, cy, P.Lf, P.halfL);
  const float dz = wrap_diff(zj, cz, P.Lf, P.halfL);
  const float r2 = dx * dx + dy * dy + dz * dz;
  double du = 0.0, gs = 0.0;
  bool any = false;
  if (r2 < P.rc2 && dqlB != 0.0f && qj != 0.0f) {
    const float r = sqrtf(r2);
    const float e = erfcf(P.alpha * r) / r;
    du = (double)(dqlB * qj * (e - P.c1 + P.c2 * (r - P.rcf)));
    if (WITH_S) gs = (double)(fabsf(dqlB * qj) * (e + P.c1 + P.c2 * fabsf(r - P.rcf)));
    any = true;
  }
  double dw = 0.0, gw = 0.0;
  bool wany = false;
  if (dp != 0) {
    const WcaEntry &w = P.wca[ccls * 4 + jcls];
    if (w.on && r2 < 1.0001f * w.wcut2)
      wany = wca_change_d(w, dp, cx, cy, cz, xj, yj, zj, P.Ld, P.halfLd, dw, gw, ov);
  }
  if (any || wany) {
    if (!(fabs(du + dw) < (double)BIG_TERM)) {
      ov = 1;
    } else {
      // the FP32 Coulomb part and the FP64 WCA part enter the fixed-point sum separately
      if (any) acc += __float2ll_rn((float)du * FIX_SCALE);
      if (wany) acc += __double2ll_rn(dw * (double)FIX_SCALE);
      if (WITH_S) sacc += (unsigned long long)__double2ll_rn(fmin(gs + gw, (double)BIG_TERM) * (double)FIX_SCALE);
    }
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace crmc
