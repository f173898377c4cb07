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

__device__ __forceinline__ float min_image(float d, float L, float invL) { return d - L * rintf(d * invL); }

// One pair change of a changed particle c against a bystander j:
//   du = lB dq_c q_j phi(r) [r < rc] + dp_c U_wca(r)
// accumulated in 2^-32 kT fixed point.  Inserted particles (dp > 0) that come
// closer than half a WCA diameter, and any |du| >= 2^20 kT, flag an overlap.
template <bool WITH_S>
__device__ __forceinline__ void pair_change(const SysParams &P, float cx, float cy, float cz, float dqlB, int dp,
                                            int ccls, float xj, float yj, float zj, float qj, int jcls,
                                            long long &acc, unsigned long long &sacc, int &ov) {
  const float dx = min_image(xj - cx, P.Lf, P.invL);
  const float dy = min_image(yj - cy, P.Lf, P.invL);
  const float dz = min_image(zj - cz, P.Lf, P.invL);
  const float r2 = dx * dx + dy * dy + dz * dz;
  float du = 0.0f;
  bool any = false;
  if (r2 < P.rc2 && dqlB != 0.0f && qj != 0.0f) {
    const float r = sqrtf(r2);
    du = dqlB * qj * (erfcf(P.alpha * r) / r - P.c1 + P.c2 * (r - P.rcf));
    any = true;
  }
  if (dp != 0) {
    const WcaEntry &w = P.wca[ccls * 4 + jcls];
    if (w.on && r2 < w.wcut2) {
      const float s = sqrtf(r2) - w.del;
      if (dp > 0 && s < 0.5f * w.sig) {
        ov = 1;
      } else {
        const float t = w.sig / s;
        const float t2 = t * t;
        const float t6 = t2 * t2 * t2;
        du += (float)dp * (4.0f * w.eps * (t6 * t6 - t6) + w.eps);
        any = true;
      }
    }
  }
  if (any) {
    if (!(fabsf(du) < BIG_TERM)) {
      ov = 1;
    } else {
      acc += __float2ll_rn(du * FIX_SCALE);
      if (WITH_S) sacc += (unsigned long long)__float2ll_rn(fabsf(du) * FIX_SCALE);
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
