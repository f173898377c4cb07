// crmc_phase.cu -- the colour-phase kernel of the CR-MC stage (sm_103a).
//
// k_cr_phase: one CTA per active domain of one colour of the 8-colour
// checkerboard, for one or several replicas (blockIdx.x) in one launch; the
// domains of a colour are launched densest first (blockIdx.y is the rank in
// the order k_domain_order computes at the start of every sweep), so that the
// long CTAs do not form the tail of the launch.
// The CTA
//   1. stages the domain's particles into a list kept in canonical order
//      (in-domain cell rank, then id) -- in shared memory, or in a global
//      scratch region when the domain is unusually dense -- and the halo
//      particles around it into registers (they do not change in the phase);
//   2. draws the phase's random numbers for a chunk of trials at once
//      (Philox4x32-10, counter (trial, domain, phase, purpose));
//   3. runs the m trials of the domain one after another: warp 0 selects the
//      participants (ballot scans of the list); every thread sums its share of
//      the pair changes -- FP32 Coulomb, FP64 WCA of inserted/deleted ions --
//      into 64-bit fixed point, exact and therefore independent of the thread
//      count; warp 0 takes the FP64 Metropolis decision and commits the move;
//   4. writes the domain's cells back (id-sorted) and adds its count changes.
// The move rules are those of Sec. II.C of the paper applied to the domain
// (the domain's volume and counts).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "crmc_device.cuh"
#include "crmc_kernels.h"

namespace crmc {

namespace {

constexpr int MAX_WARPS = 16;  // up to 512 threads per CTA

struct TrialPre {
  uint32_t w0, w1, w2, w3;  // move, site choice, first ion, second ion
  float ax, ay, az, bx, by, bz;
  int rankA, rankB;  // in-domain cell rank of the insertion points, -1 = outside
  uint32_t uhi, ulo; // the two words of the Metropolis uniform
  float lnu_f;       // FP32 ln u (decides unless within LNU_BAND of lnA)
  int pad;
  double lnu;        // FP64 ln u (trial records only)
  // delayed acceptance: the stage-2 uniform (Philox purpose 3)
  uint32_t u2hi, u2lo;
  float lnu2_f;
  int pad2;
  double lnu2;
};

struct Desc {
  float x, y, z, dqlB;  // position, lB * (q_new - q_old)
  int dp, cls, skip;    // WCA presence change, class, list index (-1 inserted)
};

struct TrialCtl {
  Desc c[2];
  int nch;    // changed particles needing the energy sweep (0 = decided)
  int flags;  // CR_TRIAL_* bits known before the sweep
  int move;
  int site, ionA, ionB;  // list indices (-1 none)
  unsigned long long id_a, id_b, newid;
  long long ln_ratio_fx, dself_fx;  // 2^-48 fixed point
  float qa_o, qa_n, qb_o, qb_n;  // effective charges of the two changed particles
  int pa_o, pa_n, pb_o, pb_n;    // presence before / after
  // delayed acceptance: in-domain cell ranks of a and b, charge and presence
  // changes, feature group of a (0 ion, 8 site), stage-1 outcome
  int rka, rkb, dqa, dqb, eta_a, eta_b, cat_a, go;
  int ewacc;             // Ewald: the trial was accepted (S(k) follows)
  float sur;             // surrogate dE~ (DA)
  long long sur_fx;      // dE~ clamped, 2^-48 fixed point (DA)
};

struct DomList {
  float4 *pos, *vel;
  unsigned long long *id;
  long long *lnk;  // site constant ln10 (pH - pK - pI_X) at 2^-48, 0 for non-sites
  int *info, *rank;
};

// FP32 constants of the pair sweep, kept in registers
struct PairK {
  float Lf, halfL, rc2, alpha, c1, c2, rcf, lBf;
  double Ld, halfLd;
};

__device__ __forceinline__ int region_coord(int i, int org, int k, int h, int nr, int nc) {
  int c = (i < k + h) ? org + i : org + i - nr;
  c %= nc;
  if (c < 0) c += nc;
  return c;
}

// Exclusive scan of n ints (shared memory) into pre[0..n]; all threads call.
__device__ void block_scan(const int *vals, int n, int *pre, int *tmp) {
  const int T = blockDim.x, t = threadIdx.x, lane = t & 31, w = t >> 5, nw = T >> 5;
  const int per = (n + T - 1) / T;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += vals[i];
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[w] = x;
  __syncthreads();
  if (w == 0) {
    int v = lane < nw ? tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) tmp[lane] = v;
  }
  __syncthreads();
  int run = x - s + (w > 0 ? tmp[w - 1] : 0);
  for (int i = lo; i < hi; ++i) {
    pre[i] = run;
    run += vals[i];
  }
  if (t == T - 1) pre[n] = run;
  __syncthreads();
}

// largest i with pre[i] <= j (pre ascending, pre[0] = 0, j < pre[n])
__device__ __forceinline__ int upper_idx(const int *pre, int n, int j) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// warp: index of the kth (0-based) list entry of a kind, -1 if none
__device__ __forceinline__ int warp_kth(const int *info, int n, int kind, int kth) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < n; base += 32) {
    const int j = base + lane;
    const bool m = j < n && kind_of(info[j]) == kind;
    const unsigned b = __ballot_sync(0xffffffffu, m);
    const int c = __popc(b);
    if (kth < c) {
      const unsigned lt = b & ((1u << lane) - 1u);
      const unsigned hit = __ballot_sync(0xffffffffu, m && __popc(lt) == kth);
      return base + __ffs(hit) - 1;
    }
    kth -= c;
  }
  return -1;
}

// warp: number of entries with rank < r and rank == r (four chunks per round)
__device__ __forceinline__ void warp_rank_count(const int *rank, int n, int r, int &below, int &same) {
  const int lane = threadIdx.x & 31;
  below = 0;
  same = 0;
  for (int base = 0; base < n; base += 128) {
    int rk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = base + 32 * u + lane;
      rk[u] = j < n ? rank[j] : INT_MAX;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      below += __popc(__ballot_sync(0xffffffffu, rk[u] < r));
      same += __popc(__ballot_sync(0xffffffffu, rk[u] == r));
    }
  }
}

// one list entry held in registers while the list shifts
struct EntryRegs {
  float4 a, v;
  unsigned long long b;
  long long e;
  int c, d;
};
__device__ __forceinline__ EntryRegs entry_load(const DomList &L, int j) {
  return EntryRegs{L.pos[j], L.vel[j], L.id[j], L.lnk[j], L.info[j], L.rank[j]};
}
__device__ __forceinline__ void entry_store(const DomList &L, int j, const EntryRegs &x) {
  L.pos[j] = x.a; L.vel[j] = x.v; L.id[j] = x.b; L.lnk[j] = x.e; L.info[j] = x.c; L.rank[j] = x.d;
}

// warp: open a hole at p (entries [p, n) move up by one), 64 entries per
// round from the top down: every load of a round before its stores
__device__ void warp_insert_gap(DomList L, int n, int p) {
  const int lane = threadIdx.x & 31;
  for (int hi = n; hi > p; hi -= 64) {
    const int lo = max(p, hi - 64);
    const int j0 = lo + lane, j1 = lo + 32 + lane;
    const bool a0 = j0 < hi, a1 = j1 < hi;
    EntryRegs x0{}, x1{};
    if (a0) x0 = entry_load(L, j0);
    if (a1) x1 = entry_load(L, j1);
    __syncwarp();
    if (a0) entry_store(L, j0 + 1, x0);
    if (a1) entry_store(L, j1 + 1, x1);
    __syncwarp();
  }
}

// warp: remove entry p (entries (p, n) move down by one), 64 entries per
// round from the bottom up
__device__ void warp_remove(DomList L, int n, int p) {
  const int lane = threadIdx.x & 31;
  for (int lo = p + 1; lo < n; lo += 64) {
    const int j0 = lo + lane, j1 = lo + 32 + lane;
    const bool a0 = j0 < n, a1 = j1 < n;
    EntryRegs x0{}, x1{};
    if (a0) x0 = entry_load(L, j0);
    if (a1) x1 = entry_load(L, j1);
    __syncwarp();
    if (a0) entry_store(L, j0 - 1, x0);
    if (a1) entry_store(L, j1 - 1, x1);
    __syncwarp();
  }
}

// pair change between the two changed particles: u_new - u_old, Coulomb in
// FP32 and WCA in FP64, into fixed point (without a WCA term the FP64 sum
// reduces to the FP32 change, taken directly)
template <bool WITH_S>
__device__ __forceinline__ void cc_change_impl(const PairK &K, const WcaEntry *wca, const TrialCtl &t, long long &acc,
                                               unsigned long long &sacc, int &ov) {
  const Desc &A = t.c[0], &B = t.c[1];
  const float dx = wrap_diff(B.x, A.x, K.Lf, K.halfL);
  const float dy = wrap_diff(B.y, A.y, K.Lf, K.halfL);
  const float dz = wrap_diff(B.z, A.z, K.Lf, K.halfL);
  const float r2 = dx * dx + dy * dy + dz * dz;
  const WcaEntry &w = wca[A.cls * 4 + B.cls];
  float uc[2] = {0.0f, 0.0f};
  double uw[2] = {0.0, 0.0};
  double gs = 0.0;
  bool hit = false;
  for (int s = 0; s < 2; ++s) {
    const bool pres = s ? (t.pa_n && t.pb_n) : (t.pa_o && t.pb_o);
    if (!pres) continue;
    const float qa = s ? t.qa_n : t.qa_o, qb = s ? t.qb_n : t.qb_o;
    if (r2 < K.rc2 && qa != 0.0f && qb != 0.0f) {
      const float rinv = rsqrtf(r2);
      const float r = r2 * rinv;
      const float e = erfcf(K.alpha * r) * rinv;
      uc[s] = K.lBf * qa * qb * (e - K.c1 + K.c2 * (r - K.rcf));
      if (WITH_S) gs += (double)(fabsf(K.lBf * qa * qb) * (e + K.c1 + K.c2 * fabsf(r - K.rcf)));
    }
    if (w.on && r2 < 1.0001f * w.wcut2) {
      const double ddx = wrap_diff_d(B.x, A.x, K.Ld, K.halfLd), ddy = wrap_diff_d(B.y, A.y, K.Ld, K.halfLd),
                   ddz = wrap_diff_d(B.z, A.z, K.Ld, K.halfLd);
      const double r = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
      if (r < w.wcut_d) {
        const double sv = r - w.del_d;
        const bool inserted = s == 1 && ((t.pa_n && !t.pa_o) || (t.pb_n && !t.pb_o));
        if (inserted && sv < 0.5 * w.sig_d) {
          ov = 1;
        } else {
          const double tt = w.sig_d / sv;
          const double t2 = tt * tt;
          const double t6 = t2 * t2 * t2;
          uw[s] = 4.0 * w.eps_d * (t6 * t6 - t6) + w.eps_d;
          if (WITH_S) gs += w.eps_d * (4.0 * t6 * t6 + 4.0 * t6 + 1.0);
          hit = true;
        }
      }
    }
  }
  const float dc = uc[1] - uc[0];
  if (!hit) {  // dw = 0: |dc| < 2^20 decides, fix32(dc) is the sum
    if (dc != 0.0f) {
      if (!(fabsf(dc) < BIG_TERM)) {
        ov = 1;
      } else {
        acc += fix32(dc);
        if (WITH_S) sacc += (unsigned long long)__double2ll_rn(fmin(gs, (double)BIG_TERM) * (double)FIX_SCALE);
      }
    }
    return;
  }
  const double dw = uw[1] - uw[0];
  if (dc != 0.0f || dw != 0.0) {
    if (!(fabs((double)dc + dw) < (double)BIG_TERM)) {
      ov = 1;
    } else {
      acc += fix32(dc) + __double2ll_rn(dw * (double)FIX_SCALE);
      if (WITH_S) sacc += (unsigned long long)__double2ll_rn(fmin(gs, (double)BIG_TERM) * (double)FIX_SCALE);
    }
  }
}

// Sums of pair terms returned by value from the out-of-line helpers, so that
// the callers' accumulators stay in registers.
struct PairSum {
  long long acc;
  unsigned long long sacc;
  int ov;
};

constexpr unsigned FULL = 0xffffffffu;
constexpr int QCAP = 96;  // per-warp queue of Coulomb pair terms (up to 31 waiting + 64 new)

// Metropolis comparison ln u < lnA with lnA in 2^-48 fixed point: the FP32
// ln u decides outside LNU_BAND, the FP64 ln u inside it
// (the FP64 logarithm of the band is out of line: rare, and large)
__device__ __noinline__ bool accept_band(long long lnA_fx, uint32_t uhi, uint32_t ulo) {
  return __double2ll_rn(log(unif53(uhi, ulo)) * LNFIX) < lnA_fx;
}
__device__ __forceinline__ bool accept_fx(long long lnA_fx, float lnu_f, uint32_t uhi, uint32_t ulo) {
  const long long lnu_apx = (long long)__float2int_rn(lnu_f * 16777216.0f) << 24;
  const long long diff = lnA_fx - lnu_apx;
  if (diff > LNU_BAND) return true;
  if (diff < -LNU_BAND) return false;
  return accept_band(lnA_fx, uhi, ulo);
}

// Maxwell-Boltzmann velocity of an inserted ion (unit mass, kT = 1): Box-Muller
// on the four 24-bit uniforms of Philox block (trial, domain, phase, purpose),
// purpose 6 for the first inserted ion of a trial and 7 for the second
__device__ __noinline__ float4 ion_velocity(uint32_t k, uint32_t d, uint32_t phi, uint32_t purpose, uint32_t key0,
                                           uint32_t key1) {
  const uint4 w = philox10(k, d, phi, purpose, key0, key1);
  const float u0 = ((float)(w.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u1 = ((float)(w.y >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u2 = ((float)(w.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u3 = ((float)(w.w >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float r1 = sqrtf(-2.0f * logf(u0)), r2 = sqrtf(-2.0f * logf(u2));
  float s1, c1, s3, c3;
  sincospif(2.0f * u1, &s1, &c1);
  sincospif(2.0f * u3, &s3, &c3);
  return make_float4(r1 * c1, r1 * s1, r2 * c3, 0.0f);
}

__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7ff8000000000000ll); }

// ---- delayed-acceptance surrogate
__device__ __forceinline__ float bf16_value(uint16_t w) { return __uint_as_float((uint32_t)w << 16); }

// shell of a squared integer cell offset inside the 5^3 stencil:
// {0},{1},{2},{3},{4},{5},{6},{8,9,12}
__device__ __forceinline__ int shell_of_n2(int n2) { return n2 <= 6 ? n2 : 7; }

// shell of in-domain cell rank rb relative to rank ra (-1 outside the stencil)
__device__ __forceinline__ int shell_ranks(int ra, int rb, int k) {
  const int dx = rb % k - ra % k, dy = (rb / k) % k - (ra / k) % k, dz = rb / (k * k) - ra / (k * k);
  if (abs(dx) > 2 || abs(dy) > 2 || abs(dz) > 2) return -1;
  return shell_of_n2(dx * dx + dy * dy + dz * dz);
}

// region cell of in-domain rank r shifted by (dx, dy, dz) in [-2, 2]^3
__device__ __forceinline__ int region_of(int r, int dx, int dy, int dz, int k, int nr) {
  int x = r % k + dx, y = (r / k) % k + dy, z = r / (k * k) + dz;
  x += x < 0 ? nr : 0;
  y += y < 0 ? nr : 0;
  z += z < 0 ? nr : 0;
  return x + nr * (y + nr * z);
}

// one dense layer with ReLU for the two input vectors x[2][n_in] -> y[2][128]:
// each output is its bias plus one FP32 fused multiply-add per weight, in
// input order (weights transposed, WT[k][o], so that a warp's loads coalesce)
template <int T>
__device__ __forceinline__ void mlp_layer(const uint16_t *__restrict__ WT, const float *__restrict__ b,
                                          const float *x, int n_in, float *y) {
  for (int o = threadIdx.x; o < 2 * MLP_H; o += T) {
    const int v = o / MLP_H, i = o % MLP_H;
    const float *xv = x + v * n_in;
    float a = __ldg(&b[i]);
#pragma unroll 8
    for (int kk = 0; kk < n_in; ++kk) a = __fmaf_rn(bf16_value(__ldg(&WT[kk * MLP_H + i])), xv[kk], a);
    y[o] = a > 0.0f ? a : 0.0f;
  }
}

// DSF Coulomb change of one queued pair: qp * phi(r), qp = lB dq_c q_j
template <bool WITH_S>
__device__ __forceinline__ void coul_eval(const PairK &K, float r2, float qp, long long &acc,
                                          unsigned long long &sacc, int &ov) {
  const float rinv = rsqrtf(r2);
  const float r = r2 * rinv;
  const float e = erfcf(K.alpha * r) * rinv;
  const float du = qp * (e - K.c1 + K.c2 * (r - K.rcf));
  if (!(fabsf(du) < BIG_TERM)) {
    ov = 1;
  } else {
    acc += fix32(du);
    if (WITH_S) sacc += (unsigned long long)fix32(fminf(fabsf(qp) * (e + K.c1 + K.c2 * fabsf(r - K.rcf)), BIG_TERM));
  }
}

// WCA pre-check radii of a changed particle against the four classes
// (1.0001 x squared cutoff, or -1 when it is not inserted / deleted or the
// pair does not interact), kept in registers for the whole trial
__device__ __forceinline__ float4 wca_radii(const WcaEntry *wca, const Desc &c) {
  float r[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const WcaEntry &w = wca[c.cls * 4 + j];
    r[j] = (c.dp != 0 && w.on) ? 1.0001f * w.wcut2 : -1.0f;
  }
  return make_float4(r[0], r[1], r[2], r[3]);
}

__device__ __forceinline__ float sel4(const float4 v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// A pair within the WCA range of an inserted / deleted changed particle:
// Coulomb in FP32 and WCA in FP64, evaluated at once (rare).  Not inlined, to
// keep the sweep's loop small; everything it needs comes by value or from
// shared memory (P, w), and its sums come back by value.
template <bool WITH_S>
__device__ __noinline__ PairSum near_pair(const SysParams &P, const WcaEntry &w, float cx, float cy, float cz,
                                          float cdq, int cdp, float xj, float yj, float zj, float qj, float r2) {
  PairSum out{0, 0ull, 0};
  float du = 0.0f, gs = 0.0f;
  const bool any = r2 < P.rc2 && cdq != 0.0f && qj != 0.0f;
  if (any) {
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float e = erfcf(P.alpha * r) * rinv;
    du = cdq * qj * (e - P.c1 + P.c2 * (r - P.rcf));
    if (WITH_S) gs = fabsf(cdq * qj) * (e + P.c1 + P.c2 * fabsf(r - P.rcf));
  }
  double du_w = 0.0, gs_w = 0.0;
  int ovw = 0;
  const bool hit = wca_change_d(w, cdp, cx, cy, cz, xj, yj, zj, P.Ld, P.halfLd, du_w, gs_w, ovw);
  if (ovw) {
    out.ov = 1;
  } else if (hit) {
    if (!(fabs((double)du + du_w) < (double)BIG_TERM)) {
      out.ov = 1;
    } else {
      if (any) out.acc += fix32(du);
      out.acc += __double2ll_rn(du_w * (double)FIX_SCALE);
      if (WITH_S) out.sacc += (unsigned long long)__double2ll_rn(fmin((double)gs + gs_w, (double)BIG_TERM) * (double)FIX_SCALE);
    }
  } else if (any) {  // beyond the WCA cutoff after all: Coulomb only
    if (!(fabsf(du) < BIG_TERM)) out.ov = 1;
    else {
      out.acc += fix32(du);
      if (WITH_S) out.sacc += (unsigned long long)fix32(fminf(gs, BIG_TERM));
    }
  }
  return out;
}

// the pair between the two changed particles (one thread per trial; out of
// line, with its FP64 WCA branch)
template <bool WITH_S>
__device__ __noinline__ PairSum cc_change(const SysParams &P, const TrialCtl &t) {
  PairK K;
  K.Lf = P.Lf; K.halfL = P.halfL; K.rc2 = P.rc2; K.alpha = P.alpha; K.c1 = P.c1; K.c2 = P.c2; K.rcf = P.rcf;
  K.lBf = P.lBf; K.Ld = P.Ld; K.halfLd = P.halfLd;
  PairSum out{0, 0ull, 0};
  cc_change_impl<WITH_S>(K, P.wca, t, out.acc, out.sacc, out.ov);
  return out;
}

// Flat frame of a region that spans less than half the box: along an axis
// whose region wraps around the periodic boundary (bit i of strad), a
// coordinate x >= L/2 becomes x - L (exact: L/2 <= x < L).  Between two points
// of the region the plain difference in this frame then equals the
// minimum-image difference bit for bit, whichever of the two had been shifted.
__device__ __forceinline__ float frame_x(float x, int strad, int axis, float halfL, float L) {
  return ((strad >> axis) & 1) && x >= halfL ? x - L : x;
}

// every full 32 queued Coulomb pairs of the warp are evaluated with all lanes
// busy; the rest (fewer than 32) stays queued
template <bool WITH_S>
__device__ __forceinline__ void queue_flush(const PairK &K, float *qr2, float *qqp, int &qn, long long &acc,
                                            unsigned long long &sacc, int &ov) {
  const int lane = threadIdx.x & 31;
  while (qn >= 32) {
    __syncwarp();
    coul_eval<WITH_S>(K, qr2[lane], qqp[lane], acc, sacc, ov);
    const int rest = qn - 32;
    float a0 = 0.f, b0 = 0.f, a1 = 0.f, b1 = 0.f;
    if (lane < rest) {
      a0 = qr2[32 + lane];
      b0 = qqp[32 + lane];
    }
    if (lane + 32 < rest) {
      a1 = qr2[64 + lane];
      b1 = qqp[64 + lane];
    }
    __syncwarp();
    if (lane < rest) {
      qr2[lane] = a0;
      qqp[lane] = b0;
    }
    if (lane + 32 < rest) {
      qr2[32 + lane] = a1;
      qqp[32 + lane] = b1;
    }
    __syncwarp();
    qn = rest;
  }
}

// Both changed particles A and B against one candidate j (lane-parallel):
// the two distance tests are independent, pairs near an inserted / deleted
// particle are evaluated at once, the in-range Coulomb pairs of A and B join
// the warp's queue with one compaction step, and every full 32 queued pairs
// are evaluated with all lanes busy.
// FLAT: the candidate's coordinates and As, Bs (those of A and B) are in the
// region's flat frame (below), where plain differences are the minimum-image
// ones; the raw coordinates, for the FP64 WCA of a near pair, come back
// exactly as x + L for a shifted (negative) x.
template <bool WITH_S, bool FLAT = false>
__device__ __forceinline__ void offer2(const SysParams &P, const PairK &K, const WcaEntry *wca, const Desc &A,
                                       const Desc &B,
                                       const float4 wrA, const float4 wrB, bool valid, float xj, float yj, float zj,
                                       float qj, int jcls, float *qr2, float *qqp, int &qn, long long &acc,
                                       unsigned long long &sacc, int &ov, const float3 As = float3{},
                                       const float3 Bs = float3{}) {
  const int lane = threadIdx.x & 31;
  float ax, ay, az, bx, by, bz;
  if (FLAT) {
    ax = xj - As.x; ay = yj - As.y; az = zj - As.z;
    bx = xj - Bs.x; by = yj - Bs.y; bz = zj - Bs.z;
  } else {
    ax = wrap_diff(xj, A.x, K.Lf, K.halfL); ay = wrap_diff(yj, A.y, K.Lf, K.halfL); az = wrap_diff(zj, A.z, K.Lf, K.halfL);
    bx = wrap_diff(xj, B.x, K.Lf, K.halfL); by = wrap_diff(yj, B.y, K.Lf, K.halfL); bz = wrap_diff(zj, B.z, K.Lf, K.halfL);
  }
  const float rA = ax * ax + ay * ay + az * az, rB = bx * bx + by * by + bz * bz;
  const bool nearA = valid && rA < sel4(wrA, jcls), nearB = valid && rB < sel4(wrB, jcls);
  if (nearA || nearB) {
    float xr = xj, yr = yj, zr = zj;
    if (FLAT) {
      xr = xj < 0.0f ? xj + K.Lf : xj;
      yr = yj < 0.0f ? yj + K.Lf : yj;
      zr = zj < 0.0f ? zj + K.Lf : zj;
    }
    if (nearA) {
      const PairSum p = near_pair<WITH_S>(P, wca[A.cls * 4 + jcls], A.x, A.y, A.z, A.dqlB, A.dp, xr, yr, zr, qj, rA);
      acc += p.acc;
      sacc += p.sacc;
      ov |= p.ov;
    }
    if (nearB) {
      const PairSum p = near_pair<WITH_S>(P, wca[B.cls * 4 + jcls], B.x, B.y, B.z, B.dqlB, B.dp, xr, yr, zr, qj, rB);
      acc += p.acc;
      sacc += p.sacc;
      ov |= p.ov;
    }
  }
  const bool inA = valid && !nearA && rA < K.rc2 && A.dqlB != 0.0f && qj != 0.0f;
  const bool inB = valid && !nearB && rB < K.rc2 && B.dqlB != 0.0f && qj != 0.0f;
  const unsigned mA = __ballot_sync(FULL, inA), mB = __ballot_sync(FULL, inB);
  if ((mA | mB) == 0u) return;
  const unsigned lt = (1u << lane) - 1u;
  const int nA = __popc(mA);
  if (inA) {
    const int p = qn + __popc(mA & lt);
    qr2[p] = rA;
    qqp[p] = A.dqlB * qj;
  }
  if (inB) {
    const int p = qn + nA + __popc(mB & lt);
    qr2[p] = rB;
    qqp[p] = B.dqlB * qj;
  }
  qn += nA + __popc(mB);
  queue_flush<WITH_S>(K, qr2, qqp, qn, acc, sacc, ov);
}


template <int T>
__device__ __forceinline__ void cta_sync() {
  if (T == 32) __syncwarp();
  else __syncthreads();
}

// int64 sum over the warp, result in every lane
__device__ __forceinline__ long long warp_allsum(long long v) { return warp_sum_i64(v); }

// Random numbers of a chunk of trials (Philox purposes 0-3 and 6-7; thread i0
// of a group of `stride` threads takes every stride-th task): the move and
// its choices, both insertion points with their in-domain cell ranks, the
// Metropolis uniform, for delayed acceptance the stage-2 uniform, and the
// velocities of the ions an insertion would add.
template <bool LOG, bool DA>
__device__ __noinline__ void draw_chunk(TrialPre *tp, float4 *tvel, int k0, int nchunk, int i0, int stride, int d,
                                        uint32_t phi, int org0, int org1, int org2, int off0, int off1, int off2,
                                        int dd0, int dd1, int dd2, int k, int nc, float af, float Lf, float scf,
                                        uint32_t key0, uint32_t key1) {
  const int org[3] = {org0, org1, org2}, off[3] = {off0, off1, off2}, dd[3] = {dd0, dd1, dd2};
  for (int u = i0; u < 3 * nchunk; u += stride) {
    if (u >= nchunk) {  // the Maxwell-Boltzmann velocities an accepted insertion gives its ions (purposes 6, 7)
      const int t = u % nchunk, which = u / nchunk - 1;
      tvel[2 * t + which] = ion_velocity((uint32_t)(k0 + t), (uint32_t)d, phi, 6u + (uint32_t)which, key0, key1);
      continue;
    }
    const int t = u;
    const uint32_t kk = (uint32_t)(k0 + t);
    const uint4 a = philox10(kk, (uint32_t)d, phi, 0u, key0, key1);
    const uint4 b = philox10(kk, (uint32_t)d, phi, 1u, key0, key1);
    const uint4 c = philox10(kk, (uint32_t)d, phi, 2u, key0, key1);
    TrialPre q;
    q.w0 = a.x; q.w1 = a.y; q.w2 = a.z; q.w3 = a.w;
    q.ax = insert_coord(org[0], b.x, k, nc, af, Lf);
    q.ay = insert_coord(org[1], b.y, k, nc, af, Lf);
    q.az = insert_coord(org[2], b.z, k, nc, af, Lf);
    q.bx = insert_coord(org[0], b.w, k, nc, af, Lf);
    q.by = insert_coord(org[1], c.x, k, nc, af, Lf);
    q.bz = insert_coord(org[2], c.y, k, nc, af, Lf);
    const float xs[2][3] = {{q.ax, q.ay, q.az}, {q.bx, q.by, q.bz}};
    int rk[2];
    for (int s = 0; s < 2; ++s) {
      int l[3];
      bool in = true;
      for (int i = 0; i < 3; ++i) {
        const int cc = cell_of(xs[s][i], scf, nc);
        const int sh = ((cc - off[i]) % nc + nc) % nc;
        in = in && (sh / k == dd[i]);
        l[i] = sh % k;
      }
      rk[s] = in ? l[0] + k * (l[1] + k * l[2]) : -1;
    }
    q.rankA = rk[0];
    q.rankB = rk[1];
    q.uhi = c.z;
    q.ulo = c.w;
    q.lnu_f = logf((float)(c.z >> 5) * 7.450580596923828e-09f + ((float)(c.w >> 6) + 0.5f) * 1.1102230246251565e-16f);
    q.pad = 0;
    q.lnu = LOG ? log(unif53(c.z, c.w)) : 0.0;
    q.u2hi = q.u2lo = 0u;
    q.lnu2_f = 0.0f;
    q.pad2 = 0;
    q.lnu2 = 0.0;
    if (DA) {
      const uint4 e = philox10(kk, (uint32_t)d, phi, 3u, key0, key1);
      q.u2hi = e.x;
      q.u2lo = e.y;
      q.lnu2_f = logf((float)(e.x >> 5) * 7.450580596923828e-09f + ((float)(e.y >> 6) + 0.5f) * 1.1102230246251565e-16f);
      q.lnu2 = LOG ? log(unif53(e.x, e.y)) : 0.0;
    }
    tp[t] = q;
  }
}

// Proposal of trial kk on the current list (Sec. II.C applied to the domain):
// the move, its participants, the log of the acceptance ratio without the
// energy, the self-energy change and the two changed particles.  Every lane
// of the calling warp computes the same values (the list scans are ballots).
template <bool DA>
__device__ __forceinline__ void select_trial(const SysParams &P, const DomList &L, const int *misc,
                                             const long long *lnt, const TrialPre &q, int d, int m, int kk,
                                             uint32_t phi, TrialCtl &C) {
  const int lane = threadIdx.x & 31;
  const int n = misc[0];
  const int mv = pick32(q.w0, 2 * P.n_react);
  const int r = P.react[mv >> 1];
  const bool fwd = (mv & 1) == 0;
  int flags = 0, site = -1, ionA = -1, ionB = -1, nch = 0;
  bool bad = false;
  long long ln_ratio = 0;
  const unsigned long long newid = ((unsigned long long)(phi + 1u) << 32) |
                                   (unsigned long long)(2u * ((uint32_t)d * (uint32_t)m + (uint32_t)kk));
  unsigned long long id_a = ~0ull, id_b = ~0ull;
  Desc c0 = {}, c1 = {};
  float qa_o = 0.f, qa_n = 0.f, qb_o = 0.f, qb_n = 0.f;
  int pa_o = 0, pa_n = 0, pb_o = 0, pb_n = 0;
  if (r == R_ACID || r == R_BASE) {
    const int kn = r == R_ACID ? K_A0 : K_B0, ki = r == R_ACID ? K_A1 : K_B1;
    const int kx = r == R_ACID ? P.kxp : P.kxm;
    const float qs = r == R_ACID ? -1.0f : 1.0f;
    const int n0 = misc[1 + kn], n1 = misc[1 + ki], nx = misc[1 + kx];
    if (fwd) {
      if (n0 == 0) flags |= CR_TRIAL_NO_ELIGIBLE;
      else {
        site = warp_kth(L.info, n, kn, pick32(q.w1, n0));
        if (q.rankA < 0) flags |= CR_TRIAL_EDGE;
        if (site < 0) { site = 0; bad = true; }
        id_a = L.id[site];
        id_b = newid;
        const float4 sp4 = L.pos[site];
        const int sinfo = L.info[site];
        c0 = Desc{sp4.x, sp4.y, sp4.z, P.lBf * qs, 0, (sinfo >> INFO_CLS_SHIFT) & 3, site};
        c1 = Desc{q.ax, q.ay, q.az, P.lBf * (-qs * P.ion_q), 1, P.ion_cls, -1};
        qa_o = 0.f; qa_n = qs; qb_o = 0.f; qb_n = -qs * P.ion_q;
        pa_o = pa_n = 1; pb_o = 0; pb_n = 1;
        nch = 2;
        ln_ratio = lnt[n0] + P.lnz1_fx - lnt[n1 + 1];
        ln_ratio -= lnt[nx + 1];
        ln_ratio += L.lnk[site];
      }
    } else {
      if (n1 == 0 || nx == 0) flags |= CR_TRIAL_NO_ELIGIBLE;
      else {
        site = warp_kth(L.info, n, ki, pick32(q.w1, n1));
        ionA = warp_kth(L.info, n, kx, pick32(q.w2, nx));
        if (site < 0 || ionA < 0) { site = max(site, 0); ionA = max(ionA, 0); bad = true; }
        id_a = L.id[site];
        id_b = L.id[ionA];
        const float4 sp4 = L.pos[site], ip4 = L.pos[ionA];
        const int sinfo = L.info[site], iinfo = L.info[ionA];
        c0 = Desc{sp4.x, sp4.y, sp4.z, P.lBf * (-qs), 0, (sinfo >> INFO_CLS_SHIFT) & 3, site};
        c1 = Desc{ip4.x, ip4.y, ip4.z, P.lBf * (-ip4.w), -1, (iinfo >> INFO_CLS_SHIFT) & 3, ionA};
        qa_o = qs; qa_n = 0.f; qb_o = ip4.w; qb_n = 0.f;
        pa_o = pa_n = 1; pb_o = 1; pb_n = 0;
        nch = 2;
        ln_ratio = lnt[n1] - lnt[n0 + 1] - P.lnz1_fx;
        ln_ratio += lnt[nx];
        ln_ratio -= L.lnk[site];
      }
    }
  } else {
    const int nxp = misc[1 + P.kxp], nxm = misc[1 + P.kxm];
    if (fwd) {
      if (q.rankA < 0 || q.rankB < 0) flags |= CR_TRIAL_EDGE;
      id_a = newid;
      id_b = newid + 1u;
      c0 = Desc{q.ax, q.ay, q.az, P.lBf * P.ion_q, 1, P.ion_cls, -1};
      c1 = Desc{q.bx, q.by, q.bz, P.lBf * (-P.ion_q), 1, P.ion_cls, -1};
      qa_o = 0.f; qa_n = P.ion_q; qb_o = 0.f; qb_n = -P.ion_q;
      pa_o = 0; pa_n = 1; pb_o = 0; pb_n = 1;
      nch = 2;
      ln_ratio = 2 * P.lnz1_fx + P.lnsalt_fx;
      ln_ratio -= lnt[nxp + 1] + lnt[nxm + 1];
    } else {
      if (nxp == 0 || nxm == 0) flags |= CR_TRIAL_NO_ELIGIBLE;
      else {
        ionA = warp_kth(L.info, n, P.kxp, pick32(q.w2, nxp));
        ionB = warp_kth(L.info, n, P.kxm, pick32(q.w3, nxm));
        if (ionA < 0 || ionB < 0) { ionA = max(ionA, 0); ionB = max(ionB, 0); bad = true; }
        id_a = L.id[ionA];
        id_b = L.id[ionB];
        const float4 a4 = L.pos[ionA], b4 = L.pos[ionB];
        c0 = Desc{a4.x, a4.y, a4.z, P.lBf * (-a4.w), -1, (L.info[ionA] >> INFO_CLS_SHIFT) & 3, ionA};
        c1 = Desc{b4.x, b4.y, b4.z, P.lBf * (-b4.w), -1, (L.info[ionB] >> INFO_CLS_SHIFT) & 3, ionB};
        qa_o = a4.w; qa_n = 0.f; qb_o = b4.w; qb_n = 0.f;
        pa_o = 1; pa_n = 0; pb_o = 1; pb_n = 0;
        nch = 2;
        ln_ratio = -2 * P.lnz1_fx - P.lnsalt_fx;
        ln_ratio += lnt[nxp] + lnt[nxm];
      }
    }
  }
  // a failed selection would mean the kind counts and the list disagree:
  // record it and reject instead of touching memory outside the list
  if (bad) {
    flags |= CR_TRIAL_NO_ELIGIBLE;
    if (lane == 0) atomicOr(P.err, ERRB_ARG);
  }
  nch = (flags & (CR_TRIAL_NO_ELIGIBLE | CR_TRIAL_EDGE)) ? 0 : nch;
  // self-energy change: lB s_self (sum of q_new^2 - q_old^2), an integer multiple
  const int sq = (pa_n ? (int)(qa_n * qa_n) : 0) - (pa_o ? (int)(qa_o * qa_o) : 0) +
                 (pb_n ? (int)(qb_n * qb_n) : 0) - (pb_o ? (int)(qb_o * qb_o) : 0);
  // lane 0 publishes the selection (C lives in shared memory; every lane
  // holds the same values)
  int rka = 0, rkb = 0;
  if (DA && nch) {
    if (r == R_SALT) {
      rka = fwd ? q.rankA : L.rank[ionA];
      rkb = fwd ? q.rankB : L.rank[ionB];
    } else {
      rka = L.rank[site];
      rkb = fwd ? q.rankA : L.rank[ionA];
    }
  }
  if (lane == 0) {
    C.c[0] = c0;
    C.c[1] = c1;
    C.nch = nch;
    C.move = 2 * r + (fwd ? 0 : 1);
    C.flags = flags;
    C.site = site;
    C.ionA = ionA;
    C.ionB = ionB;
    C.ln_ratio_fx = ln_ratio;
    C.dself_fx = P.lBself_fx * (long long)sq;
    C.id_a = id_a;
    C.id_b = id_b;
    C.newid = newid;
    C.sur = 0.0f;
    C.sur_fx = 0;
    C.qa_o = qa_o; C.qa_n = qa_n; C.qb_o = qb_o; C.qb_n = qb_n;
    C.pa_o = pa_o; C.pa_n = pa_n; C.pb_o = pb_o; C.pb_n = pb_n;
    C.rka = rka;
    C.rkb = rkb;
    C.dqa = C.dqb = C.eta_a = C.eta_b = C.cat_a = 0;
    C.go = 1;
    if (DA) {
      C.dqa = (pa_n ? __float2int_rn(qa_n) : 0) - (pa_o ? __float2int_rn(qa_o) : 0);
      C.dqb = (pb_n ? __float2int_rn(qb_n) : 0) - (pb_o ? __float2int_rn(qb_o) : 0);
      C.eta_a = pa_n - pa_o;
      C.eta_b = pb_n - pb_o;
      C.cat_a = r == R_SALT ? 0 : 8;
    }
  }
}

// One candidate of the merged stream of a region's particles that are not
// held in registers: u < nhc the on-chip halo (shared memory, already in the
// flat frame when the region is flat, w = q + 8 cls), u < NH the halo beyond
// it (global memory), then the domain list.  FLAT: coordinates are returned
// in the region's flat frame.
template <bool FLAT>
__device__ __forceinline__ bool stream_cand(const SysParams &P, const DomList &L, const Desc &A, const Desc &B,
                                            const float4 *hpos, int nhc, int NH, int n, const int *hpre,
                                            const int *hcell, int NR, int strad, int u, float &x, float &y,
                                            float &z, float &q, int &cls) {
  if (u < nhc) {
    const float4 p = hpos[u];
    cls = __float2int_rd((p.w + 2.0f) * 0.125f);
    q = p.w - 8.0f * (float)cls;
    x = p.x;
    y = p.y;
    z = p.z;
    return true;
  }
  float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
  bool v = false;
  cls = 0;
  if (u < NH) {  // halo beyond what is held on chip (dense regions): straight from global memory
    const int i = upper_idx(hpre, NR, u);
    const int g = hcell[i] * P.cap + (u - hpre[i]);
    p = P.pos[g];
    cls = (P.info[g] >> INFO_CLS_SHIFT) & 3;
    v = true;
  } else if (u < NH + n) {
    const int j = u - NH;
    p = L.pos[j];
    cls = (L.info[j] >> INFO_CLS_SHIFT) & 3;
    v = j != A.skip && j != B.skip;
  }
  q = p.w;
  if (FLAT) {
    x = frame_x(p.x, strad, 0, P.halfL, P.Lf);
    y = frame_x(p.y, strad, 1, P.halfL, P.Lf);
    z = frame_x(p.z, strad, 2, P.halfL, P.Lf);
  } else {
    x = p.x;
    y = p.y;
    z = p.z;
  }
  return v;
}

// The region's stream (all of it, or from `from` on) against A and B without
// the flat frame: regions wider than 0.4 L, i.e. small boxes.  Out of line,
// so that the flat loop is the only pair sweep in the trial loop's code; its
// sums come back by value.
template <bool LOG>
__device__ __noinline__ PairSum sweep_general(const SysParams &P, const TrialCtl &C, const float4 *lpos,
                                              const int *linfo, const float4 *hpos, int nhc, int NH, int n,
                                              const int *hpre, const int *hcell, int NR, int from, int i0, int stride,
                                              float *qr2, float *qqp) {
  const Desc A = C.c[0], B = C.c[1];
  DomList L{};
  L.pos = const_cast<float4 *>(lpos);
  L.info = const_cast<int *>(linfo);
  PairK K;
  K.Lf = P.Lf; K.halfL = P.halfL; K.rc2 = P.rc2; K.alpha = P.alpha; K.c1 = P.c1; K.c2 = P.c2; K.rcf = P.rcf;
  K.lBf = P.lBf; K.Ld = P.Ld; K.halfLd = P.halfLd;
  const WcaEntry *wca = P.wca;
  const float4 wrA = wca_radii(wca, A), wrB = wca_radii(wca, B);
  const int lane = threadIdx.x & 31;
  PairSum out{0, 0ull, 0};
  int qn = 0;
  for (int base = from; base < NH + n; base += stride) {
    float x, y, z, q;
    int cls;
    const int u = base + i0;
    const bool v = stream_cand<false>(P, L, A, B, hpos, nhc, NH, n, hpre, hcell, NR, 0, u, x, y, z, q, cls);
    offer2<LOG>(P, K, wca, A, B, wrA, wrB, v, x, y, z, q, cls, qr2, qqp, qn, out.acc, out.sacc, out.ov);
  }
  __syncwarp();
  if (lane < qn) coul_eval<LOG>(K, qr2[lane], qqp[lane], out.acc, out.sacc, out.ov);
  return out;
}

// The pair changes of the two changed particles A and B against the halo and
// the domain list, summed by a group of threads (thread i0 of `stride`; each
// thread keeps its part in acc / sacc / ov; the warp's queued Coulomb pairs
// are evaluated at the end).  The pair between A and B is not included.
// Flat regions (the common case) take every candidate in the flat frame in
// one loop over the merged stream; halo particles held in registers come
// first.
template <bool LOG, int R, int RR>
__device__ __forceinline__ void sweep_pairs(const PairK &K, const WcaEntry *wca, const SysParams &P, const DomList &L,
                                            const Desc &A, const Desc &B, const float4 (&hreg)[RR], int nmine,
                                            const float4 *hpos, int NH, int hcap, const int *hpre, const int *hcell,
                                            int NR, int n, int i0, int stride, float *qr2, float *qqp, long long &acc,
                                            unsigned long long &sacc, int &ov, bool flat, int strad,
                                            const TrialCtl *ctl) {
  const int lane = threadIdx.x & 31;
  const float4 wrA = wca_radii(wca, A), wrB = wca_radii(wca, B);
  int qn = 0;
  // the on-chip halo is stored in the flat frame when the region allows it
  const float3 As = make_float3(frame_x(A.x, strad, 0, K.halfL, K.Lf), frame_x(A.y, strad, 1, K.halfL, K.Lf),
                                frame_x(A.z, strad, 2, K.halfL, K.Lf));
  const float3 Bs = make_float3(frame_x(B.x, strad, 0, K.halfL, K.Lf), frame_x(B.y, strad, 1, K.halfL, K.Lf),
                                frame_x(B.z, strad, 2, K.halfL, K.Lf));
  if (R > 0) {
    if (flat) {
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const float4 p = hreg[r];
        const int cls = __float2int_rd((p.w + 2.0f) * 0.125f);
        const float q = p.w - 8.0f * (float)cls;
        offer2<LOG, true>(P, K, wca, A, B, wrA, wrB, r < nmine, p.x, p.y, p.z, q, cls, qr2, qqp, qn, acc, sacc, ov,
                          As, Bs);
      }
    } else {
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const float4 p = hreg[r];
        const int cls = __float2int_rd((p.w + 2.0f) * 0.125f);
        const float q = p.w - 8.0f * (float)cls;
        offer2<LOG>(P, K, wca, A, B, wrA, wrB, r < nmine, p.x, p.y, p.z, q, cls, qr2, qqp, qn, acc, sacc, ov);
      }
    }
  }
  // the rest of the stream: for R == 0 the halo in shared memory from 0, for
  // R > 0 the part of the halo beyond the registers, then the list
  const int nhc = R > 0 ? 0 : min(NH, hcap);
  const int from = R > 0 ? min(NH, hcap) : 0;
  if (flat) {
    for (int base = from; base < NH + n; base += stride) {
      float x, y, z, q;
      int cls;
      const bool v = stream_cand<true>(P, L, A, B, hpos, nhc, NH, n, hpre, hcell, NR, strad, base + i0, x, y, z, q,
                                       cls);
      offer2<LOG, true>(P, K, wca, A, B, wrA, wrB, v, x, y, z, q, cls, qr2, qqp, qn, acc, sacc, ov, As, Bs);
    }
    __syncwarp();
    if (lane < qn) coul_eval<LOG>(K, qr2[lane], qqp[lane], acc, sacc, ov);
  } else {
    __syncwarp();
    if (lane < qn) coul_eval<LOG>(K, qr2[lane], qqp[lane], acc, sacc, ov);  // the registers' queue
    const PairSum g =
        sweep_general<LOG>(P, *ctl, L.pos, L.info, hpos, nhc, NH, n, hpre, hcell, NR, from, i0, stride, qr2, qqp);
    acc += g.acc;
    sacc += g.sacc;
    ov |= g.ov;
  }
}

// ---- Ewald reciprocal part (global schedule): the change of
// sum_k A_k |S(k)|^2 when the changed particles' charges dq enter S(k).  The
// phase exp(i 2 pi n u), u = x / L, is reduced exactly in integers: U = u in
// 0.32 fixed point (FP64), n U mod 2^32 is the fraction of n u; FP32 sincospi
// of that fraction gives the factor.  A reciprocal vector's factor is the
// product of its three axes' factors (the conjugate for negative n).
__device__ __forceinline__ uint32_t ew_frac32(float x, double invL) {
  return (uint32_t)(unsigned long long)llrint((double)x * invL * 4294967296.0);
}
__device__ __forceinline__ float2 ew_factor(uint32_t U, int n) {
  const uint32_t t = (uint32_t)n * U;
  float sn, cs;
  sincospif((float)t * (2.0f / 4294967296.0f), &sn, &cs);
  return make_float2(cs, sn);
}
__device__ __forceinline__ float2 ew_cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 ew_axis(const float2 *f, int n) {
  const float2 v = f[n < 0 ? -n : n];
  return make_float2(v.x, n < 0 ? -v.y : v.y);
}
__device__ __forceinline__ void ew_decode(int code, int &nx, int &ny, int &nz) {
  nx = (int)(signed char)(code & 255);
  ny = (int)(signed char)((code >> 8) & 255);
  nz = (int)(signed char)((code >> 16) & 255);
}

// the axis factors of the trial's two changed particles (f[c][axis][n], n <=
// kmax) and their charge changes dq[c] (0 where absent); threads tid of T
__device__ __noinline__ void ewald_factors(const SysParams &P, const TrialCtl &C, float2 *f, float *dq, int ewk, int tid,
                                           int T) {
  for (int i = tid; i < 6 * ewk; i += T) {
    const int c = i / (3 * ewk), ax = (i / ewk) % 3, n = i % ewk;
    const Desc &D = C.c[c];
    const float x = ax == 0 ? D.x : (ax == 1 ? D.y : D.z);
    f[i] = ew_factor(ew_frac32(x, P.invLd), n);
  }
  if (tid == 0) {
    dq[0] = (C.pa_n ? C.qa_n : 0.0f) - (C.pa_o ? C.qa_o : 0.0f);
    dq[1] = (C.pb_n ? C.qb_n : 0.0f) - (C.pb_o ? C.qb_o : 0.0f);
  }
}

// dS(k) of the trial for the reciprocal vector of code `code`
__device__ __forceinline__ float2 ewald_dS(const float2 *f, const float *dq, int ewk, int code) {
  int nx, ny, nz;
  ew_decode(code, nx, ny, nz);
  const float2 ea = ew_cmul(ew_cmul(ew_axis(f, nx), ew_axis(f + ewk, ny)), ew_axis(f + 2 * ewk, nz));
  const float2 eb = ew_cmul(ew_cmul(ew_axis(f + 3 * ewk, nx), ew_axis(f + 4 * ewk, ny)), ew_axis(f + 5 * ewk, nz));
  return make_float2(dq[0] * ea.x + dq[1] * eb.x, dq[0] * ea.y + dq[1] * eb.y);
}

// this thread's share of the reciprocal energy change, into 2^-32 fixed point
// (vectors tid, tid + T, ...; four loaded ahead at a time)
template <bool WITH_S>
__device__ __noinline__ PairSum ewald_dE(const SysParams &P, const float2 *f, const float *dq, int ewk, int tid,
                                         int T) {
  PairSum out{0, 0ull, 0};
  const int nk = P.ewald_nk;
  const int2 *nA = P.ek_nA;
  const float2 *S32 = P.ek_Shi;
  for (int i0 = tid; i0 < nk; i0 += 4 * T) {
    int2 v[4];
    float2 sv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * T;
      v[u] = i < nk ? nA[i] : make_int2(0, 0);
      sv[u] = i < nk ? S32[i] : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (i0 + u * T >= nk) continue;
      const float2 d = ewald_dS(f, dq, ewk, v[u].x);
      const float term = __int_as_float(v[u].y) * (2.0f * (sv[u].x * d.x + sv[u].y * d.y) + (d.x * d.x + d.y * d.y));
      if (!(fabsf(term) < BIG_TERM)) {
        out.ov = 1;
      } else {
        out.acc += fix32(term);
        if (WITH_S) out.sacc += (unsigned long long)fix32(fabsf(term));
      }
    }
  }
  return out;
}

// hi + lo += d in FP32 with the rounding error kept (Knuth's two-sum, then
// Dekker's fast two-sum to renormalise: hi stays the FP32 value of the sum)
__device__ __forceinline__ void ew_add2(float &hi, float &lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(d, bp));
  const float l = __fadd_rn(lo, err);
  const float h = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(h, s));
  hi = h;
}

// an accepted trial: S(k) += dS(k) for this thread's reciprocal vectors (the
// same vectors ewald_dE gave it)
__device__ __noinline__ void ewald_update(const SysParams &P, const float2 *f, const float *dq, int ewk, int tid,
                                          int T) {
  for (int i = tid; i < P.ewald_nk; i += T) {
    const float2 d = ewald_dS(f, dq, ewk, P.ek_nA[i].x);
    float2 hi = P.ek_Shi[i], lo = P.ek_Slo[i];
    ew_add2(hi.x, lo.x, d.x);
    ew_add2(hi.y, lo.y, d.y);
    P.ek_Shi[i] = hi;
    P.ek_Slo[i] = lo;
  }
}

// room for the ions an accepted insertion adds: their cells below the cell
// capacity and the list below its capacity (belowA / sameA: entries of the
// list before and in the first ion's cell, where it goes)
__device__ __forceinline__ bool insert_room(const SysParams &P, const DomList &L, int n, int list_cap, int r,
                                            const TrialPre &q, int &belowA, int &sameA) {
  warp_rank_count(L.rank, n, q.rankA, belowA, sameA);
  bool full = sameA + 1 > P.cap;
  if (r == R_SALT) {
    int below2, same2;
    warp_rank_count(L.rank, n, q.rankB, below2, same2);
    full = full || same2 + 1 + (q.rankB == q.rankA ? 1 : 0) > P.cap;
  }
  return !(full || n + 2 > list_cap);
}

// Commit of an accepted trial by one warp: the site's charge state, the ion
// inserted (after every entry of its cell, as new ids are the largest) or
// deleted in the list, the kind counts.  Returns the new list size.
__device__ __forceinline__ int commit_trial(const SysParams &P, const DomList &L, int *misc, const TrialCtl &C,
                                            const TrialPre &q, const float4 *vel, int n, int belowA, int sameA) {
  const int lane = threadIdx.x & 31;
  const int r = C.move >> 1;
  const bool fwd = (C.move & 1) == 0;
  if (r == R_ACID || r == R_BASE) {
    const float qs = r == R_ACID ? -1.0f : 1.0f;
    const int s_site = C.site;
    if (lane == 0) {
      L.info[s_site] ^= INFO_ION_BIT;
      L.pos[s_site].w = fwd ? qs : 0.0f;
    }
    __syncwarp();
    if (fwd) {
      const int p = belowA + sameA;  // after every entry of its cell rank
      warp_insert_gap(L, n, p);
      if (lane == 0) {
        L.pos[p] = make_float4(q.ax, q.ay, q.az, -qs * P.ion_q);
        L.vel[p] = vel[0];
        L.id[p] = C.newid;
        L.lnk[p] = 0;
        L.info[p] = (r == R_ACID ? P.txp : P.txm) | (P.ion_cls << INFO_CLS_SHIFT);
        L.rank[p] = q.rankA;
      }
      n += 1;
    } else {
      warp_remove(L, n, C.ionA);
      n -= 1;
    }
    if (lane == 0) {
      const int kn = r == R_ACID ? K_A0 : K_B0, ki = kn + 1, kx = r == R_ACID ? P.kxp : P.kxm;
      const int dlt = fwd ? 1 : -1;
      misc[1 + kn] -= dlt;
      misc[1 + ki] += dlt;
      misc[1 + kx] += dlt;
    }
  } else {
    if (fwd) {
      int p = belowA + sameA;
      warp_insert_gap(L, n, p);
      if (lane == 0) {
        L.pos[p] = make_float4(q.ax, q.ay, q.az, P.ion_q);
        L.vel[p] = vel[0];
        L.id[p] = C.newid;
        L.lnk[p] = 0;
        L.info[p] = P.txp | (P.ion_cls << INFO_CLS_SHIFT);
        L.rank[p] = q.rankA;
      }
      __syncwarp();
      n += 1;
      int below, same;
      warp_rank_count(L.rank, n, q.rankB, below, same);
      p = below + same;
      warp_insert_gap(L, n, p);
      if (lane == 0) {
        L.pos[p] = make_float4(q.bx, q.by, q.bz, -P.ion_q);
        L.vel[p] = vel[1];
        L.id[p] = C.newid + 1u;
        L.lnk[p] = 0;
        L.info[p] = P.txm | (P.ion_cls << INFO_CLS_SHIFT);
        L.rank[p] = q.rankB;
      }
      n += 1;
    } else {
      const int hi = max(C.ionA, C.ionB), lo = min(C.ionA, C.ionB);
      warp_remove(L, n, hi);
      n -= 1;
      warp_remove(L, n, lo);
      n -= 1;
    }
    if (lane == 0) {
      const int dlt = fwd ? 1 : -1;
      misc[1 + P.kxp] += dlt;
      misc[1 + P.kxm] += dlt;
    }
  }
  __syncwarp();
  return n;
}

// An accepted trial, by warp 0: room for the ions an insertion adds (else
// -1 and nothing changes), then the commit; returns the new list size.  Out
// of line: it runs only for accepted trials and is large.
__device__ __noinline__ int try_commit(const SysParams &P, float4 *lpos, float4 *lvel, unsigned long long *lid,
                                       long long *llnk, int *linfo, int *lrank, int *misc, const TrialCtl &C,
                                       const TrialPre &q, const float4 *vel, int n, int list_cap) {
  DomList L;
  L.pos = lpos; L.vel = lvel; L.id = lid; L.lnk = llnk; L.info = linfo; L.rank = lrank;
  const int r = C.move >> 1;
  const bool fwd = (C.move & 1) == 0;
  int belowA = 0, sameA = 0;
  if (fwd && !insert_room(P, L, n, list_cap, r, q, belowA, sameA)) return -1;
  return commit_trial(P, L, misc, C, q, vel, n, belowA, sameA);
}

}  // namespace

// ---------------------------------------------------------------------------
// One domain of one colour phase of replica `rep`: `rank` is its place in
// the colour's launch order.  Every thread of the CTA calls it; smem is the
// CTA's dynamic shared memory, carved up as phase_smem_bytes describes.
template <int T, int R, bool LOG, bool DA>
__device__ __forceinline__ void phase_task(unsigned char *smem, const SysParams *__restrict__ reps,
                                           const PhaseShape &S, uint32_t sweep, uint32_t sweep0, int colour,
                                           uint32_t key0, uint32_t key1_base, int rep, int rank) {
  constexpr int NW = T / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- shared memory carve-up (launch-wide shape); every array starts on
  // a 16-byte boundary (phase_smem_bytes mirrors this order and padding)
  unsigned char *sp = smem;
  auto take = [&](size_t bytes) {
    unsigned char *p = sp;
    sp += (bytes + 15) / 16 * 16;
    return p;
  };
  SysParams &P = *(SysParams *)take(sizeof(SysParams));
  DomList Ls;
  Ls.pos = (float4 *)take(sizeof(float4) * S.dcs);
  Ls.vel = (float4 *)take(sizeof(float4) * S.dcs);
  Ls.id = (unsigned long long *)take(sizeof(unsigned long long) * S.dcs);
  Ls.lnk = (long long *)take(sizeof(long long) * S.dcs);
  Ls.info = (int *)take(sizeof(int) * S.dcs);
  Ls.rank = (int *)take(sizeof(int) * S.dcs);
  float4 *hpos = (float4 *)take(sizeof(float4) * S.hcs);  // halo (R == 0): x, y, z, q + 8 cls
  long long *lntab_s = (long long *)take(sizeof(long long) * S.lns);
  TrialPre *tp = (TrialPre *)take(sizeof(TrialPre) * S.chunk);
  float4 *tvel = (float4 *)take(sizeof(float4) * 2 * S.chunk);  // velocities of inserted ions
  TrialCtl *ctl = (TrialCtl *)take(sizeof(TrialCtl));
  long long *red = (long long *)take(sizeof(long long) * MAX_WARPS);
  unsigned long long *reds = (unsigned long long *)take(sizeof(unsigned long long) * MAX_WARPS);
  unsigned long long *st = (unsigned long long *)take(sizeof(unsigned long long) * 16);
  float *qbuf = (float *)take(sizeof(float) * 2 * QCAP * NW);
  int *redov = (int *)take(sizeof(int) * MAX_WARPS);
  int *scan_tmp = (int *)take(sizeof(int) * 32);
  int *misc = (int *)take(sizeof(int) * MISC_N);  // [0] list size, [1 + kind] counts, [MISC_INIT + kind] at start
  int *hcnt = (int *)take(sizeof(int) * (S.nr3 + 1));
  int *hcell = (int *)take(sizeof(int) * (S.nr3 + 1));
  int *hpre = (int *)take(sizeof(int) * (S.nr3 + 1));
  int *dcnt = (int *)take(sizeof(int) * (S.kc3 + 1));
  int *dpre = (int *)take(sizeof(int) * (S.kc3 + 1));
  float *qr2 = qbuf + warp * 2 * QCAP, *qqp = qr2 + QCAP;
  // Ewald: the changed particles' axis factors and charge changes
  float2 *ewf = (float2 *)take(sizeof(float2) * 6 * S.ewk);
  float *ewq = (float *)take(sizeof(float) * 4);
  // delayed acceptance: region cell aggregates (ion charge, site charge,
  // particles), feature bins, the two surrogate inputs and hidden layers
  int *aQi = nullptr, *aQs = nullptr, *aN = nullptr, *dfeat = nullptr;
  float *fv = nullptr, *hb0 = nullptr, *hb1 = nullptr;
  if (DA) {
    aQi = (int *)take(sizeof(int) * (S.nr3 + 1));
    aQs = (int *)take(sizeof(int) * (S.nr3 + 1));
    aN = (int *)take(sizeof(int) * (S.nr3 + 1));
    dfeat = (int *)take(sizeof(int) * MLP_IN);
    fv = (float *)take(sizeof(float) * 2 * MLP_IN);
    hb0 = (float *)take(sizeof(float) * 2 * MLP_H);
    hb1 = (float *)take(sizeof(float) * 2 * MLP_H);
  }

  {
    const int *src = (const int *)&reps[rep];
    int *dst = (int *)&P;
    for (int i = tid; i < (int)(sizeof(SysParams) / 4); i += T) dst[i] = src[i];
  }
  __syncthreads();
  if (rank >= P.nact) return;  // uniform over the CTA
  const int bdom = P.order ? P.order[colour * P.nact + rank] : rank;  // active-domain index
  const int k = P.k, h = P.h, nc = P.nc, nr = P.nr, m = P.m;
  const int KC = k * k * k, NR = nr * nr * nr;
  const uint32_t key1 = key1_base ^ P.key_xor;
  PairK K;
  K.Lf = P.Lf; K.halfL = P.halfL; K.rc2 = P.rc2; K.alpha = P.alpha; K.c1 = P.c1; K.c2 = P.c2; K.rcf = P.rcf;
  K.lBf = P.lBf; K.Ld = P.Ld; K.halfLd = P.halfLd;
  const WcaEntry *wca = P.wca;

  // ---- which domain
  int dd[3];
  if (P.global) {
    dd[0] = dd[1] = dd[2] = 0;
  } else {
    const int hn = P.nd >> 1;
    const int b = bdom;
    dd[0] = 2 * (b % hn) + (colour & 1);
    dd[1] = 2 * ((b / hn) % hn) + ((colour >> 1) & 1);
    dd[2] = 2 * (b / (hn * hn)) + ((colour >> 2) & 1);
  }
  const int d = dd[0] + P.nd * (dd[1] + P.nd * dd[2]);
  const uint32_t phi = sweep * (uint32_t)P.ncol + (uint32_t)colour;
  int off[3] = {0, 0, 0};
  if (!P.global) {
    const uint4 w = philox10(0u, 0u, sweep, 4u, key0, key1);
    off[0] = pick32(w.x, nc);
    off[1] = pick32(w.y, nc);
    off[2] = pick32(w.z, nc);
  }
  int org[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) org[i] = (off[i] + dd[i] * k) % nc;

  // ---- cell counts of the domain and of its halo (cell indices kept)
  for (int r = tid; r < KC; r += T) {
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    dcnt[r] = P.cnt[(org[0] + lx) % nc + nc * ((org[1] + ly) % nc + nc * ((org[2] + lz) % nc))];
  }
  for (int i = tid; i < NR; i += T) {
    const int ix = i % nr, iy = (i / nr) % nr, iz = i / (nr * nr);
    int c = 0, cell = 0;
    if (!(ix < k && iy < k && iz < k)) {
      cell = region_coord(ix, org[0], k, h, nr, nc) +
             nc * (region_coord(iy, org[1], k, h, nr, nc) + nc * region_coord(iz, org[2], k, h, nr, nc));
      c = P.cnt[cell];
    }
    hcnt[i] = c;
    hcell[i] = cell;
  }
  if (tid < MISC_N) misc[tid] = 0;
  if (tid < 16) st[tid] = 0ull;
  __syncthreads();
  block_scan(dcnt, KC, dpre, scan_tmp);
  block_scan(hcnt, NR, hpre, scan_tmp);
  const int ND = dpre[KC], NH = hpre[NR];
  // the list lives in shared memory unless the domain is unusually dense
  const bool in_smem = ND + 2 * m <= S.dcs;
  DomList L = Ls;
  if (!in_smem) {
    const size_t o = (size_t)(colour * P.nact + rank) * P.dcap_glob;  // this domain's region of the replica's scratch
    L.pos = P.gs_pos + o; L.vel = P.gs_vel + o; L.id = P.gs_id + o; L.lnk = P.gs_lnk + o;
    L.info = P.gs_info + o; L.rank = P.gs_rank + o;
    if (ND + 2 * m > P.dcap_glob) {  // cannot happen: a cell holds at most cap particles
      if (tid == 0) atomicOr(P.err, ERRB_CELL_OVERFLOW);
      return;
    }
  }
  const int lnmax_need = min(P.lnmax, ND + 2 * m + 2);
  const bool ln_in_smem = lnmax_need <= S.lns;
  const long long *lnt = ln_in_smem ? lntab_s : P.lntab_fx;
  if (ln_in_smem)
    for (int i = tid; i < lnmax_need; i += T) lntab_s[i] = P.lntab_fx[i];
  for (int j = tid; j < ND; j += T) {
    const int r = upper_idx(dpre, KC, j);
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    const int cell = (org[0] + lx) % nc + nc * ((org[1] + ly) % nc + nc * ((org[2] + lz) % nc));
    const int g = cell * P.cap + (j - dpre[r]);
    const int info = P.info[g];
    const int t = info & INFO_TYPE_MASK;
    L.pos[j] = P.pos[g];
    L.vel[j] = P.vel[g];
    L.id[j] = P.pid[g];
    L.lnk[j] = (t == CR_ACID || t == CR_BASE) ? P.lnK_fx[info >> INFO_SITE_SHIFT] : 0ll;
    L.info[j] = info;
    L.rank[j] = r;
    atomicAdd(&misc[1 + min(kind_of(info), (int)K_OTHER)], 1);
  }
  // flat frame (frame_x): a region spanning less than half the box along
  // every axis is compared without minimum-image tests; strad marks the
  // axes along which it wraps around the periodic boundary
  const bool flat = !P.global && 2.5f * (float)nr * P.af < P.Lf;
  int strad = 0;
  if (flat)
    for (int i = 0; i < 3; ++i) strad |= (org[i] < h || org[i] + k + h > nc) ? 1 << i : 0;
  // halo particles (they do not change during the phase): w = q + 8 * cls
  constexpr int RR = R > 0 ? R : 1;
  float4 hreg[RR];
  int nmine = 0;
  const int hcap = R > 0 ? R * T : S.hcs;  // halo entries held on chip
  if (R > 0) {
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const int j = tid + r * T;
      hreg[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < NH) {
        const int i = upper_idx(hpre, NR, j);
        const int g = hcell[i] * P.cap + (j - hpre[i]);
        const float4 p = P.pos[g];
        hreg[r] = make_float4(frame_x(p.x, strad, 0, P.halfL, P.Lf), frame_x(p.y, strad, 1, P.halfL, P.Lf),
                              frame_x(p.z, strad, 2, P.halfL, P.Lf),
                              p.w + 8.0f * (float)((P.info[g] >> INFO_CLS_SHIFT) & 3));
        nmine = r + 1;
      }
    }
  } else {
    for (int j = tid; j < min(NH, hcap); j += T) {
      const int i = upper_idx(hpre, NR, j);
      const int g = hcell[i] * P.cap + (j - hpre[i]);
      const float4 p = P.pos[g];
      hpos[j] = make_float4(frame_x(p.x, strad, 0, P.halfL, P.Lf), frame_x(p.y, strad, 1, P.halfL, P.Lf),
                            frame_x(p.z, strad, 2, P.halfL, P.Lf),
                            p.w + 8.0f * (float)((P.info[g] >> INFO_CLS_SHIFT) & 3));
    }
  }
  if (DA) {  // region cell aggregates at the start of the phase
    for (int i = tid; i < NR; i += T) {
      const int ix = i % nr, iy = (i / nr) % nr, iz = i / (nr * nr);
      const int cell = region_coord(ix, org[0], k, h, nr, nc) +
                       nc * (region_coord(iy, org[1], k, h, nr, nc) + nc * region_coord(iz, org[2], k, h, nr, nc));
      const int cn = P.cnt[cell];
      int qi = 0, qs = 0;
      for (int sl = 0; sl < cn; ++sl) {
        const int g = cell * P.cap + sl;
        const int t = P.info[g] & INFO_TYPE_MASK;
        const int q = __float2int_rn(P.pos[g].w);
        if (is_ion_type(t)) qi += q;
        else if (t == CR_ACID || t == CR_BASE) qs += q;
      }
      aQi[i] = qi;
      aQs[i] = qs;
      aN[i] = cn;
    }
  }
  if (tid == 0) misc[0] = ND;
  __syncthreads();
  if (tid < N_KIND) misc[MISC_INIT + tid] = misc[1 + tid];
  const int cc_thread = NW > 1 ? 32 : 0;  // the thread that adds the changed-pair term
  const long long log_dom = (long long)(sweep - sweep0) * P.per_sweep + (long long)colour * P.nact * m +
                            (long long)bdom * m;

  for (int k0 = 0; k0 < m; k0 += S.chunk) {
    const int nchunk = min(S.chunk, m - k0);
    // ---- random numbers of the chunk
    draw_chunk<LOG, DA>(tp, tvel, k0, nchunk, tid, T, d, phi, org[0], org[1], org[2], off[0], off[1], off[2], dd[0],
                        dd[1], dd[2], k, nc, P.af, P.Lf, P.scf, key0, key1);
    __syncthreads();

    for (int t = 0; t < nchunk; ++t) {
      const int kk = k0 + t;
      // ---- warp 0: proposal and participants; the selection lives in
      // shared memory (*ctl) across the sweep
      if (warp == 0) select_trial<DA>(P, L, misc, lnt, tp[t], d, m, kk, phi, *ctl);
      cta_sync<T>();
      // Ewald (global schedule): the changed particles' phase factors
      const bool ew = !DA && P.ewald_nk > 0 && ctl->nch;
      if (ew) {
        ewald_factors(P, *ctl, ewf, ewq, S.ewk, tid, T);
        cta_sync<T>();
      }
      // ---- delayed acceptance, stage 1: surrogate features and MLP (all
      // threads), decision in warp 0; a rejection skips the pair sweep
      if (DA && ctl->nch) {
        if (tid < MLP_IN) dfeat[tid] = 0;
        cta_sync<T>();
        const int rka = ctl->rka, rkb = ctl->rkb;
        const int dqa = ctl->dqa, dqb = ctl->dqb, ea = ctl->eta_a, eb = ctl->eta_b;
        for (int it = tid; it < 250; it += T) {  // 2 changed particles x 125 stencil cells
          const int sb = it >= 125 ? 1 : 0;
          const int c = it - 125 * sb;
          const int dx = c % 5 - 2, dy = (c / 5) % 5 - 2, dz = c / 25 - 2;
          const int ri = region_of(sb ? rkb : rka, dx, dy, dz, k, nr);
          const int sh = shell_of_n2(dx * dx + dy * dy + dz * dz);
          const int dq = sb ? dqb : dqa, eta = sb ? eb : ea;
          if (dq != 0) {
            const int qi = aQi[ri], qs = aQs[ri];
            if (qi) atomicAdd(&dfeat[24 * sb + sh], dq * qi);
            if (qs) atomicAdd(&dfeat[24 * sb + 8 + sh], dq * qs);
          }
          if (eta != 0 && aN[ri]) atomicAdd(&dfeat[24 * sb + 16 + sh], eta * aN[ri]);
        }
        cta_sync<T>();
        if (tid == 0) {  // the changed particles themselves do not count; the a-b pair term
          const TrialCtl &C = *ctl;
          const int qao = __float2int_rn(C.qa_o), qan = __float2int_rn(C.qa_n);
          const int qbo = __float2int_rn(C.qb_o), qbn = __float2int_rn(C.qb_n);
          for (int sb = 0; sb < 2; ++sb) {
            const int rs = sb ? rkb : rka, dq = sb ? dqb : dqa, eta = sb ? eb : ea;
            for (int x = 0; x < 2; ++x) {
              if (!(x ? C.pb_o : C.pa_o)) continue;
              const int sh = shell_ranks(rs, x ? rkb : rka, k);
              if (sh < 0) continue;
              dfeat[24 * sb + (x ? 0 : C.cat_a) + sh] -= dq * (x ? qbo : qao);
              dfeat[24 * sb + 16 + sh] -= eta;
            }
          }
          const int sh = shell_ranks(rka, rkb, k);
          if (sh >= 0) dfeat[sh] += (C.pa_n && C.pb_n ? qan * qbn : 0) - (C.pa_o && C.pb_o ? qao * qbo : 0);
        }
        cta_sync<T>();
        if (tid < MLP_IN) {
          const float f = (float)dfeat[tid];
          fv[tid] = f;
          fv[MLP_IN + tid] = -f;
          if (LOG && P.feat_log) P.feat_log[(size_t)(log_dom + kk) * MLP_IN + tid] = f;
        }
        cta_sync<T>();
        mlp_layer<T>(P.mlp_w + MLPW_W1, P.mlp_b, fv, MLP_IN, hb0);
        cta_sync<T>();
        mlp_layer<T>(P.mlp_w + MLPW_W2, P.mlp_b + MLP_H, hb0, MLP_H, hb1);
        cta_sync<T>();
        mlp_layer<T>(P.mlp_w + MLPW_W3, P.mlp_b + 2 * MLP_H, hb1, MLP_H, hb0);
        cta_sync<T>();
        if (warp == 0) {
          float y = 0.0f;
          if (lane < 2) {
            y = __ldg(&P.mlp_b[3 * MLP_H]);
            const uint16_t *w4 = P.mlp_w + MLPW_W4;
            const float *hv = hb0 + lane * MLP_H;
#pragma unroll 8
            for (int kk2 = 0; kk2 < MLP_H; ++kk2) y = __fmaf_rn(bf16_value(__ldg(&w4[kk2])), hv[kk2], y);
          }
          const float y0 = __shfl_sync(FULL, y, 0), y1 = __shfl_sync(FULL, y, 1);
          const float sur = 0.5f * (y0 - y1);
          bool s1 = false;  // NaN: rejected, as a comparison with NaN is false
          long long sur_fx = 0;
          if (sur == sur) {
            sur_fx = __double2ll_rn((double)fminf(fmaxf(sur, -16384.0f), 16384.0f) * LNFIX);
            s1 = accept_fx(ctl->ln_ratio_fx - ctl->dself_fx - sur_fx, tp[t].lnu_f, tp[t].uhi, tp[t].ulo);
          }
          if (lane == 0) {
            ctl->go = s1 ? 1 : 0;
            ctl->sur = sur;
            ctl->sur_fx = sur_fx;
          }
        }
        cta_sync<T>();
      } else if (DA && LOG && P.feat_log && tid < MLP_IN) {
        P.feat_log[(size_t)(log_dom + kk) * MLP_IN + tid] = 0.0f;
      }
      // ---- all threads: the pair-change sweep
      const int nch = (DA && !LOG && !ctl->go) ? 0 : ctl->nch;
      long long acc = 0;
      unsigned long long sacc = 0;
      int ov = 0;
      if (nch) {
        const Desc A = ctl->c[0], B = ctl->c[1];
        sweep_pairs<LOG, R, RR>(K, wca, P, L, A, B, hreg, nmine, hpos, NH, hcap, hpre, hcell, NR, misc[0], tid, T,
                                qr2, qqp, acc, sacc, ov, flat, strad, ctl);
        if (tid == cc_thread) {
          const PairSum cc = cc_change<LOG>(P, *ctl);
          acc += cc.acc;
          sacc += cc.sacc;
          ov |= cc.ov;
        }
        if (ew) {
          const PairSum e = ewald_dE<LOG>(P, ewf, ewq, S.ewk, tid, T);
          acc += e.acc;
          sacc += e.sacc;
          ov |= e.ov;
        }
        acc = warp_allsum(acc);
        if (LOG) sacc = (unsigned long long)warp_allsum((long long)sacc);
        ov = __any_sync(FULL, ov) ? 1 : 0;
        if (NW > 1 && lane == 0) {
          red[warp] = acc;
          reds[warp] = sacc;
          redov[warp] = ov;
        }
      }
      if (NW > 1) __syncthreads();
      // ---- warp 0: decision and commit
      if (warp == 0) {
        const TrialPre &q = tp[t];
        const int s_move = ctl->move, s_nch = ctl->nch;
        const long long s_ln_ratio = ctl->ln_ratio_fx, s_dself = ctl->dself_fx;
        const unsigned long long s_id_a = ctl->id_a, s_id_b = ctl->id_b;
        const bool s1 = !DA || ctl->go != 0;
        const float sur = DA ? ctl->sur : 0.0f;
        const long long sur_fx = DA ? ctl->sur_fx : 0ll;
        int flags = ctl->flags;
        bool accept = false;
        double dE = 0.0, Ssum = 0.0, lnA = -INFINITY, lnA2r = quiet_nan();
        if (DA && LOG && s_nch) lnA = (double)s_ln_ratio / LNFIX - (double)s_dself / LNFIX - (double)sur;
        if (s_nch && (!DA || LOG || s1)) {
          long long tot = acc;
          unsigned long long stot = sacc;
          int anyov = ov;
          if (NW > 1) {
            tot = warp_allsum(lane < NW ? red[lane] : 0ll);
            if (LOG) stot = (unsigned long long)warp_allsum(lane < NW ? (long long)reds[lane] : 0ll);
            anyov = __any_sync(FULL, lane < NW && redov[lane]) ? 1 : 0;
          }
          if (anyov) {
            if (!DA || s1) flags |= CR_TRIAL_OVERLAP;  // DA: only an exact evaluation that decides
            dE = INFINITY;
          } else {
            const long long totc = tot > DE_CLAMP32 ? DE_CLAMP32 : (tot < -DE_CLAMP32 ? -DE_CLAMP32 : tot);
            if (DA) {  // stage 2: ln u2 < dE~ - dE_pair
              if (s1) accept = accept_fx(sur_fx - (totc << 16), q.lnu2_f, q.u2hi, q.u2lo);
            } else {
              accept = accept_fx(s_ln_ratio - ((totc << 16) + s_dself), q.lnu_f, q.uhi, q.ulo);
            }
            if (LOG) {
              dE = (double)tot * FIX_INV + (double)s_dself / LNFIX;
              Ssum = (double)stot * FIX_INV + fabs((double)s_dself / LNFIX);
              if (!DA) lnA = (double)s_ln_ratio / LNFIX - dE;  // unclamped, for the record
              else lnA2r = (double)sur - (double)tot * FIX_INV;
            }
          }
        }
        const int r = s_move >> 1;
        const bool fwd = (s_move & 1) == 0;
        int n = misc[0];
        if (accept) {  // commit, unless an insertion finds no room (checked before anything changes)
          const int n2 = try_commit(P, L.pos, L.vel, L.id, L.lnk, L.info, L.rank, misc, *ctl, q, tvel + 2 * t, n,
                                    in_smem ? S.dcs : P.dcap_glob);
          if (n2 < 0) {
            accept = false;
            if (lane == 0) atomicOr(P.err, ERRB_CELL_OVERFLOW);
          } else {
            n = n2;
          }
        }
        (void)r;
        (void)fwd;
        if (lane == 0) ctl->ewacc = accept ? 1 : 0;
        if (accept) {
          flags |= CR_TRIAL_ACCEPTED;
          if (DA && lane == 0) {  // region aggregates follow the committed change
            const TrialCtl &C = *ctl;
            for (int x = 0; x < 2; ++x) {
              const int ri = region_of(x ? C.rkb : C.rka, 0, 0, 0, k, nr);
              int *aq = (x == 0 && C.cat_a == 8) ? aQs : aQi;
              if (x ? C.pb_o : C.pa_o) {
                aq[ri] -= __float2int_rn(x ? C.qb_o : C.qa_o);
                aN[ri] -= 1;
              }
              if (x ? C.pb_n : C.pa_n) {
                aq[ri] += __float2int_rn(x ? C.qb_n : C.qa_n);
                aN[ri] += 1;
              }
            }
          }
        }
        if (lane == 0) {
          misc[0] = n;
          st[s_move] += 1;
          if (flags & CR_TRIAL_ACCEPTED) st[6 + s_move] += 1;
          if (flags & CR_TRIAL_NO_ELIGIBLE) st[12] += 1;
          if (flags & CR_TRIAL_EDGE) st[13] += 1;
          if (flags & CR_TRIAL_OVERLAP) st[14] += 1;
          st[15] += 1;
          if (LOG && P.log) {
            cr_trial rec;
            rec.move = s_move;
            rec.flags = flags;
            rec.id_a = s_id_a;
            rec.id_b = s_id_b;
            rec.dE = dE;
            rec.S = Ssum;
            rec.lnA = lnA;
            rec.lnu = q.lnu;
            P.log[log_dom + kk] = rec;
            if (DA && P.dlog) {
              cr_trial_da dr;
              dr.dE_sur = s_nch ? sur : 0.0f;
              dr.stage = s_nch ? (s1 ? 2 : 1) : 0;
              dr.lnA2 = lnA2r;
              dr.lnu2 = s_nch ? q.lnu2 : quiet_nan();
              P.dlog[log_dom + kk] = dr;
            }
          }
        }
      }
      cta_sync<T>();
      if (ew && ctl->ewacc) ewald_update(P, ewf, ewq, S.ewk, tid, T);
    }
  }
  // ---- write the domain back (id-sorted cells) and publish counts
  __syncthreads();
  const int n = misc[0];
  for (int r = tid; r < KC; r += T) {
    int lo = 0, hi = n;  // first entry with rank >= r
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (L.rank[mid] < r) lo = mid + 1; else hi = mid; }
    int lo2 = lo, hi2 = n;  // first entry with rank > r
    while (lo2 < hi2) { const int mid = (lo2 + hi2) >> 1; if (L.rank[mid] <= r) lo2 = mid + 1; else hi2 = mid; }
    dcnt[r] = lo;
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    P.cnt[(org[0] + lx) % nc + nc * ((org[1] + ly) % nc + nc * ((org[2] + lz) % nc))] = lo2 - lo;
  }
  __syncthreads();
  for (int j = tid; j < n; j += T) {
    const int r = L.rank[j];
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    const int cell = (org[0] + lx) % nc + nc * ((org[1] + ly) % nc + nc * ((org[2] + lz) % nc));
    const int g = cell * P.cap + (j - dcnt[r]);
    const unsigned long long id = L.id[j];
    P.pos[g] = L.pos[j];
    P.vel[g] = L.vel[j];
    P.pid[g] = id;
    P.info[g] = L.info[j];
    if (id < (unsigned long long)P.n_perm) P.perm_slot[id] = g;
  }
  if (tid < 16 && st[tid]) atomicAdd(&P.stats[tid], st[tid]);
  if (tid < N_KIND && misc[1 + tid] != misc[MISC_INIT + tid])
    atomicAdd((unsigned long long *)&P.counts[tid],
              (unsigned long long)(long long)(misc[1 + tid] - misc[MISC_INIT + tid]));
}

// ---------------------------------------------------------------------------
// the phase kernel: one CTA per active domain of one colour
//   T threads per domain (T == 32: one warp, no block barriers);
//   R > 0: halo particles in R registers per thread, R == 0: in shared memory
// ---------------------------------------------------------------------------
template <int T, int R, bool LOG, bool DA>
__global__ void __launch_bounds__(T, (T <= 32 ? 16 : (T <= 64 ? 8 : (T <= 128 ? 4 : (T <= 256 ? 2 : 1)))))
    k_cr_phase(const SysParams *__restrict__ reps, PhaseShape S, uint32_t sweep, uint32_t sweep0, int colour,
               uint32_t key0, uint32_t key1_base, const StepDyn *dyn) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (dyn) {  // a captured cycle: this step's sweep counter and key
    const unsigned long long step = dyn->step, seed = dyn->sweep_seed0 + step;
    sweep = dyn->sweep0 + (uint32_t)step;
    key0 = (uint32_t)seed;
    key1_base = (uint32_t)(seed >> 32);
  }
  phase_task<T, R, LOG, DA>(smem, reps, S, sweep, sweep0, colour, key0, key1_base, (int)blockIdx.x,
                            (int)blockIdx.y);
}

// ---------------------------------------------------------------------------
// The persistent sweep: every colour of every replica of a batch in one
// launch.  CTAs claim tasks (colour c, replica r, domain rank i) in that
// order from a counter.  A domain's phase reads its region -- its own cells
// and the halo, which lies inside its 26 neighbouring domains -- and writes
// only its own cells, so the colour-by-colour schedule is reproduced exactly
// when each task starts after its neighbours of lower colours have finished
// (per-domain completion flags; Q.fine) or, for geometries whose halo reaches
// beyond the neighbouring domains, after its replica's whole previous colour
// (per-(replica, colour) counters).  Tasks of later colours thus start while
// distant domains of earlier colours still run, and no colour waits for the
// slowest domain of the batch.  A task is claimed only after every task it
// depends on was claimed, so the claims always make progress; each wait is
// nevertheless bounded in time, and a wait that runs out marks the replica's
// error word (ERRB_TIMEOUT), raises the launch's abort flag and skips the
// task, after which every remaining task is skipped without waiting.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// linear index of the domain of active rank i in colour c of replica P
__device__ __forceinline__ int task_domain(const SysParams &P, int c, int i, int (&dd)[3]) {
  const int b = P.order ? P.order[c * P.nact + i] : i;
  const int hn = P.nd >> 1;
  dd[0] = 2 * (b % hn) + (c & 1);
  dd[1] = 2 * ((b / hn) % hn) + ((c >> 1) & 1);
  dd[2] = 2 * (b / (hn * hn)) + ((c >> 2) & 1);
  return dd[0] + P.nd * (dd[1] + P.nd * dd[2]);
}

// bounded wait of one lane until *p >= need; false when the time ran out or
// the launch was aborted
__device__ __forceinline__ bool wait_at_least(const unsigned *p, unsigned need, const SweepSched &Q, int &timed_out) {
  const unsigned long long t0 = global_ns();
  while (ld_acquire_u32(p) < need) {
    if (*(volatile int *)Q.abort) return false;
    if (global_ns() - t0 > Q.wait_ns) {
      timed_out = 1;
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

template <int T, int R, bool DA>
__global__ void __launch_bounds__(T, (T <= 32 ? 16 : (T <= 64 ? 8 : (T <= 128 ? 4 : (T <= 256 ? 2 : 1)))))
    k_cr_sweep(const SysParams *__restrict__ reps, PhaseShape S, uint32_t sweep, uint32_t sweep0, uint32_t key0,
               uint32_t key1_base, SweepSched Q, const StepDyn *dyn) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (dyn) {  // a captured cycle: this step's sweep counter and key
    const unsigned long long step = dyn->step, seed = dyn->sweep_seed0 + step;
    sweep = dyn->sweep0 + (uint32_t)step;
    key0 = (uint32_t)seed;
    key1_base = (uint32_t)(seed >> 32);
  }
  __shared__ int s_task, s_run, s_dom;
  const int lane = threadIdx.x & 31;
  const int per_colour = Q.rep_first[Q.n_rep];
  const int total = per_colour * Q.ncol;
  for (;;) {
    if (threadIdx.x < 32) {  // warp 0: claim a task and wait for what it depends on
      int t = 0;
      if (lane == 0) t = (int)atomicAdd(Q.next, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      int run = 0, dom = -1;
      if (t < total) {
        const int c = t / per_colour, q = t - c * per_colour;
        int r = 0;
        while (Q.rep_first[r + 1] <= q) ++r;
        const SysParams &P = reps[r];
        int dd[3] = {0, 0, 0};
        if (Q.fine) dom = task_domain(P, c, q - Q.rep_first[r], dd);
        int ok = *(volatile int *)Q.abort ? 0 : 1, timed_out = 0;
        if (ok && c > 0) {
          if (Q.fine) {  // lane l < 26: neighbour l of the 3^3 block around the domain
            const int nd = P.nd;
            if (lane < 26) {
              const int o = lane < 13 ? lane : lane + 1;
              const int nx = (dd[0] + o % 3 - 1 + nd) % nd, ny = (dd[1] + (o / 3) % 3 - 1 + nd) % nd,
                        nz = (dd[2] + o / 9 - 1 + nd) % nd;
              const int col = (nx & 1) | ((ny & 1) << 1) | ((nz & 1) << 2);
              if (col < c) ok = wait_at_least(Q.flags + Q.dom_first[r] + nx + nd * (ny + nd * nz), 1u, Q, timed_out);
            }
          } else if (lane == 0) {  // the replica's whole previous colour
            const unsigned need = (unsigned)(Q.rep_first[r + 1] - Q.rep_first[r]);
            ok = wait_at_least(Q.done + r * Q.ncol + (c - 1), need, Q, timed_out);
          }
          ok = __all_sync(0xffffffffu, ok);
          if (__any_sync(0xffffffffu, timed_out) && lane == 0) {
            atomicOr(P.err, ERRB_TIMEOUT);
            atomicExch(Q.abort, 1);
          }
        }
        run = ok;
      }
      if (lane == 0) {
        s_task = t;
        s_run = run;
        s_dom = dom;
      }
    }
    __syncthreads();
    const int t = s_task;
    if (t >= total) break;
    const int c = t / per_colour, q = t - c * per_colour;
    int r = 0;
    while (Q.rep_first[r + 1] <= q) ++r;
    if (s_run)
      phase_task<T, R, false, DA>(smem, reps, S, sweep, sweep0, c, key0, key1_base, r, q - Q.rep_first[r]);
    __syncthreads();  // the task's stores are done, its shared memory is free
    if (threadIdx.x == 0 && !(r == Q.withhold_rep && c == 0)) {
      __threadfence();
      if (Q.fine) st_release_u32(Q.flags + Q.dom_first[r] + s_dom, 1u);
      else atomicAdd(Q.done + r * Q.ncol + c, 1u);
    }
  }
}

template <int T, int R, bool DA>
static cudaError_t launch_sweep_t(const SysParams *d_reps, PhaseShape S, cudaStream_t s, uint32_t sweep,
                                  uint32_t sweep0, uint32_t k0, uint32_t k1, const SweepSched &Q, int max_ctas,
                                  const StepDyn *dyn) {
  if (R > 0) S.hcs = 0;  // halo in registers
  static size_t attr_bytes = 0;
  static int per_sm = 0;
  static size_t per_sm_bytes = ~(size_t)0;
  const size_t smem = phase_smem_bytes(S, T, DA);
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_cr_sweep<T, R, DA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  if (smem != per_sm_bytes) {  // resident CTAs per SM at this shared-memory size
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cr_sweep<T, R, DA>, T, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(nb, 1);
    per_sm_bytes = smem;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int total = Q.tasks_total;
  int grid = std::min(total, per_sm * std::max(sms, 1));
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  if (grid <= 0) return cudaSuccess;
  k_cr_sweep<T, R, DA><<<grid, T, smem, s>>>(d_reps, S, sweep, sweep0, k0, k1, Q, dyn);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const SysParams *d_reps, const PhaseShape &S, int threads, int R, bool da, cudaStream_t s,
                         uint32_t sweep, uint32_t sweep0, uint32_t k0, uint32_t k1, const SweepSched &Q,
                         int max_ctas, const StepDyn *dyn) {
#define CRMC_SW(TT, RR, DD)                                                                   \
  if (da == DD && threads == TT && R == RR)                                                    \
    return launch_sweep_t<TT, RR, DD>(d_reps, S, s, sweep, sweep0, k0, k1, Q, max_ctas, dyn);
  CRMC_SW(32, 0, false)
  CRMC_SW(64, 0, false)
  CRMC_SW(128, 0, false)
  CRMC_SW(128, 4, false)
  CRMC_SW(256, 0, false)
  CRMC_SW(256, 2, false)
  CRMC_SW(512, 0, false)
  CRMC_SW(512, 1, false)
  CRMC_SW(128, 0, true)
  CRMC_SW(256, 0, true)
  CRMC_SW(512, 0, true)
#undef CRMC_SW
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Launch order of the domains of one colour for one sweep: the particles in
// each domain's region (its cells and the halo around them, counted at the
// start of the sweep; one warp sums a region's cell counts) and the domains
// ranked by decreasing count (ties by index).  Only the order of independent
// CTAs changes, never a result.  One CTA per (replica, colour); colours of
// more than ORDER_MAX_NACT domains keep the natural order (P.order is null).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_domain_order(const SysParams *__restrict__ reps, uint32_t sweep, uint32_t key0,
                                                      uint32_t key1_base, const StepDyn *dyn) {
  if (dyn) {  // a captured cycle: this step's sweep counter and key
    const unsigned long long step = dyn->step, seed = dyn->sweep_seed0 + step;
    sweep = dyn->sweep0 + (uint32_t)step;
    key0 = (uint32_t)seed;
    key1_base = (uint32_t)(seed >> 32);
  }
  const SysParams &P = reps[blockIdx.x];
  if (!P.order) return;
  __shared__ int cost[ORDER_MAX_NACT];
  const int c = blockIdx.y;
  if (c >= P.ncol) return;
  const int nc = P.nc, nr = P.nr, h = P.h, k = P.k, nact = P.nact;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const uint32_t key1 = key1_base ^ P.key_xor;
  const uint4 w = philox10(0u, 0u, sweep, 4u, key0, key1);
  const int off[3] = {pick32(w.x, nc), pick32(w.y, nc), pick32(w.z, nc)};
  const int hn = P.nd >> 1, nr3 = nr * nr * nr;
  for (int b = wid; b < nact; b += nwarp) {
    const int dd[3] = {2 * (b % hn) + (c & 1), 2 * ((b / hn) % hn) + ((c >> 1) & 1), 2 * (b / (hn * hn)) + ((c >> 2) & 1)};
    int o[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = ((off[i] + dd[i] * k - h) % nc + nc) % nc;  // region origin
    int sum = 0;
    for (int i = lane; i < nr3; i += 32) {
      const int ix = i % nr, iy = (i / nr) % nr, iz = i / (nr * nr);
      sum += P.cnt[(o[0] + ix) % nc + nc * ((o[1] + iy) % nc + nc * ((o[2] + iz) % nc))];
    }
#pragma unroll
    for (int x = 16; x > 0; x >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, x);
    if (lane == 0) cost[b] = sum;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nact; b += blockDim.x) {
    const int cb = cost[b];
    int rank = 0;
    for (int j = 0; j < nact; ++j) {
      const int cj = cost[j];
      rank += (cj > cb || (cj == cb && j < b)) ? 1 : 0;
    }
    P.order[c * nact + rank] = b;
  }
}

cudaError_t launch_domain_order(const SysParams *d_reps, int n_rep, int ncol, int nact, cudaStream_t s, uint32_t sweep,
                                uint32_t k0, uint32_t k1, const StepDyn *dyn) {
  if (nact > ORDER_MAX_NACT) return cudaSuccess;  // contexts keep P.order null then
  k_domain_order<<<dim3(n_rep, ncol), 512, 0, s>>>(d_reps, sweep, k0, k1, dyn);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ewald structure factor S(k) = sum_j q_j exp(i k.r_j) of every replica from
// scratch (at every sweep): k_ewald_list lists each replica's occupied slots
// (one CTA per replica, cells in order), k_ewald_sk gives each reciprocal
// vector a thread, the particles in tiles of 32 whose axis factors the CTA
// computes together in shared memory (FP32 products summed per tile, tiles
// summed in FP64).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ewald_list(const SysParams *__restrict__ reps) {
  const SysParams &P = reps[blockIdx.x];
  if (P.ewald_nk <= 0) return;
  __shared__ int warp_tot[8];
  __shared__ int base_s;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  for (int c0 = 0; c0 < P.ncell; c0 += 256) {
    const int c = c0 + (int)threadIdx.x;
    const int n = c < P.ncell ? P.cnt[c] : 0;
    int x = n;  // inclusive scan over the CTA
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    int before = base_s;
    for (int i = 0; i < w; ++i) before += warp_tot[i];
    const int start = before + x - n;
    for (int sl = 0; sl < n; ++sl) {
      if (start + sl < P.ek_cap) P.ek_list[start + sl] = c * P.cap + sl;
      else atomicOr(P.err, ERRB_CAPACITY);  // more particles than the context's capacity
    }
    __syncthreads();
    if (threadIdx.x == 255) base_s = start + n;
    __syncthreads();
  }
  if (threadIdx.x == 0) *P.ek_np = min(base_s, P.ek_cap);
}

constexpr int EW_TILE = 32;
constexpr int EW_KMAX = 32;

__global__ void __launch_bounds__(256) k_ewald_sk(const SysParams *__restrict__ reps) {
  const SysParams &P = reps[blockIdx.y];
  const int nk = P.ewald_nk;
  if (nk <= 0 || (int)blockIdx.x * 256 >= nk) return;  // uniform over the CTA
  __shared__ float2 fac[EW_TILE][3][EW_KMAX + 1];
  __shared__ float qt[EW_TILE];
  __shared__ uint32_t ut[EW_TILE][3];
  const int ewk = P.ewald_kmax + 1, np = *P.ek_np;
  const int i = (int)blockIdx.x * 256 + (int)threadIdx.x;
  int nx = 0, ny = 0, nz = 0;
  if (i < nk) ew_decode(P.ek_nA[i].x, nx, ny, nz);
  double re = 0.0, im = 0.0;
  for (int t0 = 0; t0 < np; t0 += EW_TILE) {
    const int nt = min(EW_TILE, np - t0);
    if (threadIdx.x < 3 * nt) {  // the tile's coordinates as 0.32 fixed-point fractions of L
      const int p = threadIdx.x / 3, ax = threadIdx.x % 3;
      const float4 r = P.pos[P.ek_list[t0 + p]];
      ut[p][ax] = ew_frac32(ax == 0 ? r.x : (ax == 1 ? r.y : r.z), P.invLd);
      if (ax == 0) qt[p] = r.w;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < nt * 3 * ewk; v += 256) {
      const int p = v / (3 * ewk), ax = (v / ewk) % 3, n = v % ewk;
      fac[p][ax][n] = ew_factor(ut[p][ax], n);
    }
    __syncthreads();
    if (i < nk) {
      float tr = 0.0f, ti = 0.0f;
      for (int p = 0; p < nt; ++p) {
        const float q = qt[p];
        if (q == 0.0f) continue;
        const float2 e = ew_cmul(ew_cmul(ew_axis(fac[p][0], nx), ew_axis(fac[p][1], ny)), ew_axis(fac[p][2], nz));
        tr += q * e.x;
        ti += q * e.y;
      }
      re += (double)tr;
      im += (double)ti;
    }
    __syncthreads();
  }
  if (i < nk) {
    const float hr = (float)re, hm = (float)im;
    P.ek_Shi[i] = make_float2(hr, hm);
    P.ek_Slo[i] = make_float2((float)(re - (double)hr), (float)(im - (double)hm));
  }
}

cudaError_t launch_ewald_sk(const SysParams *d_reps, int n_rep, int max_nk, cudaStream_t s) {
  if (n_rep <= 0 || max_nk <= 0) return cudaSuccess;
  k_ewald_list<<<n_rep, 256, 0, s>>>(d_reps);
  k_ewald_sk<<<dim3((unsigned)((max_nk + 255) / 256), (unsigned)n_rep), 256, 0, s>>>(d_reps);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t phase_smem_bytes(const PhaseShape &S, int threads, bool da) {
  const size_t sizes[] = {sizeof(SysParams),
                          sizeof(float4) * S.dcs,
                          sizeof(float4) * S.dcs,
                          sizeof(unsigned long long) * S.dcs,
                          sizeof(long long) * S.dcs,
                          sizeof(int) * S.dcs,
                          sizeof(int) * S.dcs,
                          sizeof(float4) * S.hcs,
                          sizeof(long long) * S.lns,
                          sizeof(TrialPre) * S.chunk,
                          sizeof(float4) * 2 * S.chunk,
                          sizeof(TrialCtl),
                          sizeof(long long) * MAX_WARPS,
                          sizeof(unsigned long long) * MAX_WARPS,
                          sizeof(unsigned long long) * 16,
                          sizeof(float) * 2 * QCAP * (threads / 32),
                          sizeof(int) * MAX_WARPS,
                          sizeof(int) * 32,
                          sizeof(int) * MISC_N,
                          sizeof(int) * (S.nr3 + 1),
                          sizeof(int) * (S.nr3 + 1),
                          sizeof(int) * (S.nr3 + 1),
                          sizeof(int) * (S.kc3 + 1),
                          sizeof(int) * (S.kc3 + 1),
                          sizeof(float2) * 6 * S.ewk,
                          sizeof(float) * 4};
  size_t b = 0;
  for (size_t x : sizes) b += (x + 15) / 16 * 16;
  if (da) {
    const size_t dsz[] = {sizeof(int) * (S.nr3 + 1), sizeof(int) * (S.nr3 + 1), sizeof(int) * (S.nr3 + 1),
                          sizeof(int) * MLP_IN,      sizeof(float) * 2 * MLP_IN, sizeof(float) * 2 * MLP_H,
                          sizeof(float) * 2 * MLP_H};
    for (size_t x : dsz) b += (x + 15) / 16 * 16;
  }
  return b;
}

template <int T, int R, bool LOG, bool DA>
static cudaError_t launch_phase_t(const SysParams *d_reps, int n_rep, int grid_x, PhaseShape S, cudaStream_t s,
                                  uint32_t sweep, uint32_t sweep0, int colour, uint32_t k0, uint32_t k1,
                                  const StepDyn *dyn) {
  if (R > 0) S.hcs = 0;  // halo in registers
  static size_t attr_bytes = 0;
  const size_t smem = phase_smem_bytes(S, T, DA);
  if (smem > attr_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(k_cr_phase<T, R, LOG, DA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  k_cr_phase<T, R, LOG, DA><<<dim3(n_rep, grid_x), T, smem, s>>>(d_reps, S, sweep, sweep0, colour, k0, k1, dyn);
  return cudaGetLastError();
}

// variants the autotuner picks from: (threads per CTA, halo registers per
// thread (0: the halo in shared memory), compact).  Compact variants size the
// shared-memory list and halo for most domains rather than the densest
// (denser ones spill to global memory), so that more CTAs fit on an SM.
static const int kShapes[][3] = {{32, 0, 0},  {64, 0, 0},  {128, 0, 0}, {128, 4, 0}, {256, 0, 0}, {256, 2, 0},
                                 {512, 0, 0}, {512, 1, 0}, {32, 0, 1},  {64, 0, 1},  {128, 0, 1}, {256, 0, 1}};

// shapes with a delayed-acceptance variant (the surrogate runs on >= 128 threads)
static const int kShapesDA[][3] = {{128, 0, 0}, {256, 0, 0}, {512, 0, 0}, {128, 0, 1}, {256, 0, 1}};

int phase_shape_count(bool da) {
  return da ? (int)(sizeof(kShapesDA) / sizeof(kShapesDA[0])) : (int)(sizeof(kShapes) / sizeof(kShapes[0]));
}
void phase_shape(int i, int *threads, int *regs, bool da) {
  *threads = da ? kShapesDA[i][0] : kShapes[i][0];
  *regs = da ? kShapesDA[i][1] : kShapes[i][1];
}
bool phase_shape_compact(int i, bool da) { return (da ? kShapesDA[i][2] : kShapes[i][2]) != 0; }

size_t phase_shape_smem(const PhaseShape &S, int threads, int regs, bool da) {
  PhaseShape Q = S;
  if (regs > 0) Q.hcs = 0;
  return phase_smem_bytes(Q, threads, da);
}

cudaError_t launch_phase(const SysParams *d_reps, int n_rep, int grid_x, const PhaseShape &S, int threads, int R,
                         bool log, bool da, cudaStream_t s, uint32_t sweep, uint32_t sweep0, int colour,
                         uint32_t k0, uint32_t k1, const StepDyn *dyn) {
#define CRMC_CASE(TT, RR)                                                                                      \
  if (!da && threads == TT && R == RR)                                                                         \
    return log ? launch_phase_t<TT, RR, true, false>(d_reps, n_rep, grid_x, S, s, sweep, sweep0, colour, k0, k1, dyn) \
               : launch_phase_t<TT, RR, false, false>(d_reps, n_rep, grid_x, S, s, sweep, sweep0, colour, k0, k1, dyn);
#define CRMC_CASE_DA(TT, RR)                                                                                   \
  if (da && threads == TT && R == RR)                                                                          \
    return log ? launch_phase_t<TT, RR, true, true>(d_reps, n_rep, grid_x, S, s, sweep, sweep0, colour, k0, k1, dyn)  \
               : launch_phase_t<TT, RR, false, true>(d_reps, n_rep, grid_x, S, s, sweep, sweep0, colour, k0, k1, dyn);
  CRMC_CASE(32, 0)
  CRMC_CASE(64, 0)
  CRMC_CASE(128, 0)
  CRMC_CASE(128, 4)
  CRMC_CASE(256, 0)
  CRMC_CASE(256, 2)
  CRMC_CASE(512, 0)
  CRMC_CASE(512, 1)
  CRMC_CASE_DA(128, 0)
  CRMC_CASE_DA(256, 0)
  CRMC_CASE_DA(512, 0)
#undef CRMC_CASE
#undef CRMC_CASE_DA
  return cudaErrorInvalidValue;
}

}  // namespace crmc
