// crmc_kernels.cu -- CUDA kernels of the CR-MC stage (sm_103a).
//
// k_cr_phase: one CTA per active domain of one colour of the 8-colour
// checkerboard.  The CTA
//   1. stages the domain's particles into a shared-memory list kept in
//      canonical order (in-domain cell rank, then id) and the surrounding halo
//      particles into registers (they do not change during the phase);
//   2. draws the phase's random numbers for a chunk of trials at once
//      (Philox4x32-10, counter (trial, domain, phase, purpose));
//   3. runs the m trials of the domain one after another: warp 0 selects the
//      participants (ballot scans of the list), every thread sums its share of
//      the pair changes in FP32 into 64-bit fixed point (exact, so the sum does
//      not depend on the thread count), warp 0 takes the FP64 Metropolis
//      decision and commits the move to the list;
//   4. writes the domain's cells back (id-sorted) and adds its count changes.
// The move rules are those of Sec. II.C of the paper applied to the domain
// (volume v of the domain, counts of the domain).
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "crmc_device.cuh"
#include "crmc_kernels.h"

namespace crmc {

struct TrialPre {
  uint32_t w0, w1, w2, w3;  // move, site choice, first ion, second ion
  float ax, ay, az, bx, by, bz;
  int rankA, rankB;  // in-domain cell rank of the insertion points, -1 = outside
  double lnu;
};

struct Desc {
  float x, y, z, dqlB;  // position, lB * (q_new - q_old)
  int dp, cls, skip;    // WCA presence change, class, list index (-1 inserted)
};

struct TrialCtl {
  Desc c[2];
  int nch;        // changed particles needing the energy sweep (0 = decided)
  int flags;      // CR_TRIAL_* bits known before the sweep
  int move;
  int site, ionA, ionB;  // list indices (-1 none)
  unsigned long long id_a, id_b, newid;
  double ln_ratio;
  long long cc;   // changed-changed pair change (fixed point)
  unsigned long long cc_s;
  int cc_ov;
  double dself;
};

// region cell along one dimension: i < k + h -> org + i, else org + i - nr
__device__ __forceinline__ int region_coord(int i, int org, int k, int h, int nr, int nc) {
  int c = (i < k + h) ? org + i : org + i - nr;
  c %= nc;
  if (c < 0) c += nc;
  return c;
}

// Exclusive scan of n ints in shared memory (vals) into pre[0..n] (all threads).
__device__ void block_scan(const int *vals, int n, int *pre, int *tmp) {
  const int T = blockDim.x, t = threadIdx.x;
  const int per = (n + T - 1) / T;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += vals[i];
  tmp[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < T; ++i) {
      const int v = tmp[i];
      tmp[i] = run;
      run += v;
    }
    pre[n] = run;
  }
  __syncthreads();
  int run = tmp[t];
  for (int i = lo; i < hi; ++i) {
    pre[i] = run;
    run += vals[i];
  }
  __syncthreads();
}

// largest i with pre[i] <= j (pre ascending, pre[0] = 0, j < pre[n])
__device__ __forceinline__ int upper_idx(const int *pre, int n, int j) {
  int lo = 0, hi = n;  // pre[lo] <= j < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= j) lo = mid; else hi = mid;
  }
  return lo;
}

// warp: index of the kth (0-based) list entry of a kind, -1 if none
__device__ __forceinline__ int warp_kth(const int *dinfo, int n, int kind, int kth) {
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < n; base += 32) {
    const int j = base + lane;
    const bool m = j < n && kind_of(dinfo[j]) == kind;
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

// warp: number of entries with rank < r and rank == r
__device__ __forceinline__ void warp_rank_count(const int *drank, int n, int r, int &below, int &same) {
  const int lane = threadIdx.x & 31;
  below = 0;
  same = 0;
  for (int base = 0; base < n; base += 32) {
    const int j = base + lane;
    const int rk = j < n ? drank[j] : INT_MAX;
    below += __popc(__ballot_sync(0xffffffffu, rk < r));
    same += __popc(__ballot_sync(0xffffffffu, rk == r));
  }
}

struct DomList {
  float4 *pos, *vel;
  unsigned long long *id;
  int *info;
  int *rank;
};

// warp: open a hole at p (entries [p, n) move up by one)
__device__ void warp_insert_gap(DomList L, int n, int p) {
  const int lane = threadIdx.x & 31;
  for (int hi = n; hi > p; hi -= 32) {
    const int lo = max(p, hi - 32);
    const int j = lo + lane;
    const bool act = j < hi;
    float4 a, v;
    unsigned long long b = 0;
    int c = 0, d = 0;
    if (act) { a = L.pos[j]; v = L.vel[j]; b = L.id[j]; c = L.info[j]; d = L.rank[j]; }
    __syncwarp();
    if (act) { L.pos[j + 1] = a; L.vel[j + 1] = v; L.id[j + 1] = b; L.info[j + 1] = c; L.rank[j + 1] = d; }
    __syncwarp();
  }
}

// warp: remove entry p (entries (p, n) move down by one)
__device__ void warp_remove(DomList L, int n, int p) {
  const int lane = threadIdx.x & 31;
  for (int lo = p + 1; lo < n; lo += 32) {
    const int j = lo + lane;
    const bool act = j < n;
    float4 a, v;
    unsigned long long b = 0;
    int c = 0, d = 0;
    if (act) { a = L.pos[j]; v = L.vel[j]; b = L.id[j]; c = L.info[j]; d = L.rank[j]; }
    __syncwarp();
    if (act) { L.pos[j - 1] = a; L.vel[j - 1] = v; L.id[j - 1] = b; L.info[j - 1] = c; L.rank[j - 1] = d; }
    __syncwarp();
  }
}

__device__ __forceinline__ float dqlB_of(const SysParams &P, float dq) { return P.lBf * dq; }

// pair change between the two changed particles: u_new - u_old, the Coulomb
// part in FP32 and the WCA part in FP64 (as for bystanders), into fixed point
__device__ void cc_change(const SysParams &P, const TrialCtl &t, float qa_o, float qa_n, float qb_o, float qb_n,
                          int pa_o, int pa_n, int pb_o, int pb_n, long long &acc, unsigned long long &sacc, int &ov) {
  const Desc &A = t.c[0], &B = t.c[1];
  const float dx = wrap_diff(B.x, A.x, P.Lf, P.halfL);
  const float dy = wrap_diff(B.y, A.y, P.Lf, P.halfL);
  const float dz = wrap_diff(B.z, A.z, P.Lf, P.halfL);
  const float r2 = dx * dx + dy * dy + dz * dz;
  const WcaEntry &w = P.wca[A.cls * 4 + B.cls];
  float uc[2] = {0.0f, 0.0f};  // Coulomb, old / new
  double uw[2] = {0.0, 0.0};   // WCA, old / new
  double gs = 0.0;             // gross magnitude (tolerance scale)
  for (int s = 0; s < 2; ++s) {
    const bool pres = s ? (pa_n && pb_n) : (pa_o && pb_o);
    if (!pres) continue;
    const float qa = s ? qa_n : qa_o, qb = s ? qb_n : qb_o;
    if (r2 < P.rc2 && qa != 0.0f && qb != 0.0f) {
      const float r = sqrtf(r2);
      const float e = erfcf(P.alpha * r) / r;
      uc[s] = P.lBf * qa * qb * (e - P.c1 + P.c2 * (r - P.rcf));
      gs += (double)(fabsf(P.lBf * qa * qb) * (e + P.c1 + P.c2 * fabsf(r - P.rcf)));
    }
    if (w.on && r2 < 1.0001f * w.wcut2) {
      const double ddx = wrap_diff_d(B.x, A.x, P.Ld, P.halfLd), ddy = wrap_diff_d(B.y, A.y, P.Ld, P.halfLd),
                   ddz = wrap_diff_d(B.z, A.z, P.Ld, P.halfLd);
      const double r = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
      if (r < w.wcut_d) {
        const double sv = r - w.del_d;
        const bool inserted = s == 1 && ((pa_n && !pa_o) || (pb_n && !pb_o));
        if (inserted && sv < 0.5 * w.sig_d) {
          ov = 1;
        } else {
          const double tt = w.sig_d / sv;
          const double t2 = tt * tt;
          const double t6 = t2 * t2 * t2;
          uw[s] = 4.0 * w.eps_d * (t6 * t6 - t6) + w.eps_d;
          gs += w.eps_d * (4.0 * t6 * t6 + 4.0 * t6 + 1.0);
        }
      }
    }
  }
  const float dc = uc[1] - uc[0];
  const double dw = uw[1] - uw[0];
  if (dc != 0.0f || dw != 0.0) {
    if (!(fabs((double)dc + dw) < (double)BIG_TERM)) ov = 1;
    else {
      acc += __float2ll_rn(dc * FIX_SCALE) + __double2ll_rn(dw * (double)FIX_SCALE);
      sacc += (unsigned long long)__double2ll_rn(fmin(gs, (double)BIG_TERM) * (double)FIX_SCALE);
    }
  }
}

template <int R, bool LOG>
__global__ void __launch_bounds__(256) k_cr_phase(SysParams P, uint32_t sweep, int colour, uint32_t key0,
                                                   uint32_t key1) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  const int k = P.k, h = P.h, nc = P.nc, nr = P.nr;
  const int KC = k * k * k, NR = nr * nr * nr;

  // ---- shared memory carve-up
  unsigned char *sp = smem;
  DomList L;
  L.pos = (float4 *)sp; sp += sizeof(float4) * P.dcap;
  L.vel = (float4 *)sp; sp += sizeof(float4) * P.dcap;
  L.id = (unsigned long long *)sp; sp += sizeof(unsigned long long) * P.dcap;
  L.info = (int *)sp; sp += sizeof(int) * P.dcap;
  L.rank = (int *)sp; sp += sizeof(int) * P.dcap;
  TrialPre *tp = (TrialPre *)sp; sp += sizeof(TrialPre) * TRIAL_CHUNK;
  TrialCtl *ctl = (TrialCtl *)sp; sp += (sizeof(TrialCtl) + 15) / 16 * 16;
  long long *red = (long long *)sp; sp += sizeof(long long) * 32;
  unsigned long long *reds = (unsigned long long *)sp; sp += sizeof(unsigned long long) * 32;
  int *redov = (int *)sp; sp += sizeof(int) * 32;
  int *scan_tmp = (int *)sp; sp += sizeof(int) * 256;
  int *misc = (int *)sp; sp += sizeof(int) * 16;  // [0] list size, [1..7] kind counts, [9..15] at start
  unsigned long long *st = (unsigned long long *)sp; sp += sizeof(unsigned long long) * 16;
  int *hcnt = (int *)sp; sp += sizeof(int) * (NR + 1);
  int *hpre = (int *)sp; sp += sizeof(int) * (NR + 1);
  int *dcnt = (int *)sp; sp += sizeof(int) * (KC + 1);
  int *dpre = (int *)sp; sp += sizeof(int) * (KC + 1);

  // ---- which domain
  int dd[3];
  if (P.global) {
    dd[0] = dd[1] = dd[2] = 0;
  } else {
    const int hn = P.nd >> 1;
    const int b = blockIdx.x;
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

  // ---- domain cells: counts, prefix, list
  for (int r = tid; r < KC; r += T) {
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    const int cx = (org[0] + lx) % nc, cy = (org[1] + ly) % nc, cz = (org[2] + lz) % nc;
    dcnt[r] = P.cnt[cx + nc * (cy + nc * cz)];
  }
  // ---- halo cells: counts
  for (int i = tid; i < NR; i += T) {
    const int ix = i % nr, iy = (i / nr) % nr, iz = i / (nr * nr);
    int c = 0;
    if (!(ix < k && iy < k && iz < k)) {
      const int cx = region_coord(ix, org[0], k, h, nr, nc), cy = region_coord(iy, org[1], k, h, nr, nc),
                cz = region_coord(iz, org[2], k, h, nr, nc);
      c = P.cnt[cx + nc * (cy + nc * cz)];
    }
    hcnt[i] = c;
  }
  if (tid < 16) misc[tid] = 0;
  if (tid < 16) st[tid] = 0ull;
  __syncthreads();
  block_scan(dcnt, KC, dpre, scan_tmp);
  block_scan(hcnt, NR, hpre, scan_tmp);
  const int ND = dpre[KC], NH = hpre[NR];
  if (ND > P.dcap) {  // cannot happen with dcap = k^3 * cap; guard anyway
    if (tid == 0) atomicOr(P.err, ERRB_CELL_OVERFLOW);
    return;
  }
  for (int j = tid; j < ND; j += T) {
    const int r = upper_idx(dpre, KC, j);
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    const int cell = (org[0] + lx) % nc + nc * ((org[1] + ly) % nc + nc * ((org[2] + lz) % nc));
    const int g = cell * P.cap + (j - dpre[r]);
    L.pos[j] = P.pos[g];
    L.vel[j] = P.vel[g];
    L.id[j] = P.pid[g];
    L.info[j] = P.info[g];
    L.rank[j] = r;
    atomicAdd(&misc[1 + min(kind_of(P.info[g]), 6)], 1);
  }
  // halo particles into registers: w = q + 8 * cls
  float4 hreg[R];
  int nmine = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j = tid + r * T;
    hreg[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < NH) {
      const int i = upper_idx(hpre, NR, j);
      const int ix = i % nr, iy = (i / nr) % nr, iz = i / (nr * nr);
      const int cx = region_coord(ix, org[0], k, h, nr, nc), cy = region_coord(iy, org[1], k, h, nr, nc),
                cz = region_coord(iz, org[2], k, h, nr, nc);
      const int g = (cx + nc * (cy + nc * cz)) * P.cap + (j - hpre[i]);
      const float4 p = P.pos[g];
      const int cls = (P.info[g] >> INFO_CLS_SHIFT) & 3;
      hreg[r] = make_float4(p.x, p.y, p.z, p.w + 8.0f * (float)cls);
      nmine = r + 1;
    }
  }
  if (tid == 0) misc[0] = ND;
  __syncthreads();
  if (tid < 7) misc[9 + tid] = misc[1 + tid];

  const int m = P.m;
  const long long log_dom = P.log_base + (long long)blockIdx.x * m;

  for (int k0 = 0; k0 < m; k0 += TRIAL_CHUNK) {
    const int nchunk = min(TRIAL_CHUNK, m - k0);
    // ---- random numbers of the chunk
    for (int t = tid; t < nchunk; t += T) {
      const uint32_t kk = (uint32_t)(k0 + t);
      const uint4 a = philox10(kk, (uint32_t)d, phi, 0u, key0, key1);
      const uint4 b = philox10(kk, (uint32_t)d, phi, 1u, key0, key1);
      const uint4 c = philox10(kk, (uint32_t)d, phi, 2u, key0, key1);
      TrialPre q;
      q.w0 = a.x; q.w1 = a.y; q.w2 = a.z; q.w3 = a.w;
      q.ax = insert_coord(org[0], b.x, k, nc, P.a, P.Lf);
      q.ay = insert_coord(org[1], b.y, k, nc, P.a, P.Lf);
      q.az = insert_coord(org[2], b.z, k, nc, P.a, P.Lf);
      q.bx = insert_coord(org[0], b.w, k, nc, P.a, P.Lf);
      q.by = insert_coord(org[1], c.x, k, nc, P.a, P.Lf);
      q.bz = insert_coord(org[2], c.y, k, nc, P.a, P.Lf);
      float xs[2][3] = {{q.ax, q.ay, q.az}, {q.bx, q.by, q.bz}};
      int rk[2];
      for (int s = 0; s < 2; ++s) {
        int l[3];
        bool in = true;
        for (int i = 0; i < 3; ++i) {
          const int cc = cell_of(xs[s][i], P.scf, nc);
          const int sh = ((cc - off[i]) % nc + nc) % nc;
          in = in && (sh / k == dd[i]);
          l[i] = sh % k;
        }
        rk[s] = in ? l[0] + k * (l[1] + k * l[2]) : -1;
      }
      q.rankA = rk[0];
      q.rankB = rk[1];
      q.lnu = log(unif53(c.z, c.w));
      tp[t] = q;
    }
    __syncthreads();

    for (int t = 0; t < nchunk; ++t) {
      const int kk = k0 + t;
      // ---- warp 0: proposal and participants
      if (warp == 0) {
        const TrialPre q = tp[t];
        const int n = misc[0];
        const int mv = pick32(q.w0, 2 * P.n_react);
        const int r = P.react[mv >> 1];
        const bool fwd = (mv & 1) == 0;
        int flags = 0, site = -1, ionA = -1, ionB = -1, nch = 0;
        bool bad = false;
        double ln_ratio = 0.0;
        const unsigned long long newid =
            ((unsigned long long)(phi + 1u) << 32) | (unsigned long long)(2u * ((uint32_t)d * (uint32_t)P.m + (uint32_t)kk));
        unsigned long long id_a = ~0ull, id_b = ~0ull;
        Desc c0 = {}, c1 = {};
        float qa_o = 0.f, qa_n = 0.f, qb_o = 0.f, qb_n = 0.f;
        int pa_o = 0, pa_n = 0, pb_o = 0, pb_n = 0;
        if (r == R_ACID || r == R_BASE) {
          const int kn = r == R_ACID ? K_A0 : K_B0, ki = r == R_ACID ? K_A1 : K_B1;
          const int kx = r == R_ACID ? K_XP : K_XM;
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
              c0 = Desc{sp4.x, sp4.y, sp4.z, dqlB_of(P, qs), 0, (sinfo >> INFO_CLS_SHIFT) & 3, site};
              c1 = Desc{q.ax, q.ay, q.az, dqlB_of(P, -qs * P.ion_q), 1, P.ion_cls, -1};
              qa_o = 0.f; qa_n = qs; qb_o = 0.f; qb_n = -qs * P.ion_q;
              pa_o = pa_n = 1; pb_o = 0; pb_n = 1;
              nch = 2;
              ln_ratio = P.lntab[n0] + P.ln_z1 - P.lntab[n1 + 1];
              ln_ratio -= P.lntab[nx + 1];
              ln_ratio += P.lnK[sinfo >> INFO_SITE_SHIFT];
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
              c0 = Desc{sp4.x, sp4.y, sp4.z, dqlB_of(P, -qs), 0, (sinfo >> INFO_CLS_SHIFT) & 3, site};
              c1 = Desc{ip4.x, ip4.y, ip4.z, dqlB_of(P, -ip4.w), -1, (iinfo >> INFO_CLS_SHIFT) & 3, ionA};
              qa_o = qs; qa_n = 0.f; qb_o = ip4.w; qb_n = 0.f;
              pa_o = pa_n = 1; pb_o = 1; pb_n = 0;
              nch = 2;
              ln_ratio = P.lntab[n1] - P.lntab[n0 + 1] - P.ln_z1;
              ln_ratio += P.lntab[nx];
              ln_ratio -= P.lnK[sinfo >> INFO_SITE_SHIFT];
            }
          }
        } else {
          const int nxp = misc[1 + K_XP], nxm = misc[1 + K_XM];
          if (fwd) {
            if (q.rankA < 0 || q.rankB < 0) flags |= CR_TRIAL_EDGE;
            id_a = newid;
            id_b = newid + 1u;
            c0 = Desc{q.ax, q.ay, q.az, dqlB_of(P, P.ion_q), 1, P.ion_cls, -1};
            c1 = Desc{q.bx, q.by, q.bz, dqlB_of(P, -P.ion_q), 1, P.ion_cls, -1};
            qa_o = 0.f; qa_n = P.ion_q; qb_o = 0.f; qb_n = -P.ion_q;
            pa_o = 0; pa_n = 1; pb_o = 0; pb_n = 1;
            nch = 2;
            ln_ratio = 2.0 * P.ln_z1 + P.ln_salt;
            ln_ratio -= P.lntab[nxp + 1] + P.lntab[nxm + 1];
          } else {
            if (nxp == 0 || nxm == 0) flags |= CR_TRIAL_NO_ELIGIBLE;
            else {
              ionA = warp_kth(L.info, n, K_XP, pick32(q.w2, nxp));
              ionB = warp_kth(L.info, n, K_XM, pick32(q.w3, nxm));
              if (ionA < 0 || ionB < 0) { ionA = max(ionA, 0); ionB = max(ionB, 0); bad = true; }
              id_a = L.id[ionA];
              id_b = L.id[ionB];
              const float4 a4 = L.pos[ionA], b4 = L.pos[ionB];
              c0 = Desc{a4.x, a4.y, a4.z, dqlB_of(P, -a4.w), -1, (L.info[ionA] >> INFO_CLS_SHIFT) & 3, ionA};
              c1 = Desc{b4.x, b4.y, b4.z, dqlB_of(P, -b4.w), -1, (L.info[ionB] >> INFO_CLS_SHIFT) & 3, ionB};
              qa_o = a4.w; qa_n = 0.f; qb_o = b4.w; qb_n = 0.f;
              pa_o = 1; pa_n = 0; pb_o = 1; pb_n = 0;
              nch = 2;
              ln_ratio = -2.0 * P.ln_z1 - P.ln_salt;
              ln_ratio += P.lntab[nxp] + P.lntab[nxm];
            }
          }
        }
        // a failed selection would mean the kind counts and the list disagree:
        // record it and reject instead of touching memory outside the list
        if (bad) {
          flags |= CR_TRIAL_NO_ELIGIBLE;
          if (lane == 0) atomicOr(P.err, ERRB_ARG);
        }
        if (lane == 0) {
          TrialCtl &C = *ctl;
          C.c[0] = c0;
          C.c[1] = c1;
          C.flags = flags;
          C.nch = (flags & (CR_TRIAL_NO_ELIGIBLE | CR_TRIAL_EDGE)) ? 0 : nch;
          C.move = 2 * r + (fwd ? 0 : 1);
          C.site = site;
          C.ionA = ionA;
          C.ionB = ionB;
          C.id_a = id_a;
          C.id_b = id_b;
          C.newid = newid;
          C.ln_ratio = ln_ratio;
          long long acc = 0;
          unsigned long long sacc = 0;
          int ov = 0;
          double dself = 0.0;
          if (C.nch) {
            cc_change(P, C, qa_o, qa_n, qb_o, qb_n, pa_o, pa_n, pb_o, pb_n, acc, sacc, ov);
            const double sq = (double)(pa_n ? qa_n * qa_n : 0.f) - (double)(pa_o ? qa_o * qa_o : 0.f) +
                              (double)(pb_n ? qb_n * qb_n : 0.f) - (double)(pb_o ? qb_o * qb_o : 0.f);
            dself = P.lB_self * sq;
          }
          C.cc = acc;
          C.cc_s = sacc;
          C.cc_ov = ov;
          C.dself = dself;
        }
      }
      __syncthreads();
      // ---- all threads: the pair-change sweep
      const int nch = ctl->nch;
      long long acc = 0;
      unsigned long long sacc = 0;
      int ov = 0;
      if (nch) {
        const Desc A = ctl->c[0], B = ctl->c[1];
        // halo (registers)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r < nmine) {
            const float4 p = hreg[r];
            const int cls = __float2int_rd((p.w + 2.0f) * 0.125f);
            const float q = p.w - 8.0f * (float)cls;
            pair_change<LOG>(P, A.x, A.y, A.z, A.dqlB, A.dp, A.cls, p.x, p.y, p.z, q, cls, acc, sacc, ov);
            pair_change<LOG>(P, B.x, B.y, B.z, B.dqlB, B.dp, B.cls, p.x, p.y, p.z, q, cls, acc, sacc, ov);
          }
        }
        // halo beyond the registers (dense regions): straight from global memory
        for (int j = R * T + tid; j < NH; j += T) {
          const int i = upper_idx(hpre, NR, j);
          const int ix = i % nr, iy = (i / nr) % nr, iz = i / (nr * nr);
          const int cx = region_coord(ix, org[0], k, h, nr, nc), cy = region_coord(iy, org[1], k, h, nr, nc),
                    cz = region_coord(iz, org[2], k, h, nr, nc);
          const int g = (cx + nc * (cy + nc * cz)) * P.cap + (j - hpre[i]);
          const float4 p = P.pos[g];
          const int cls = (P.info[g] >> INFO_CLS_SHIFT) & 3;
          pair_change<LOG>(P, A.x, A.y, A.z, A.dqlB, A.dp, A.cls, p.x, p.y, p.z, p.w, cls, acc, sacc, ov);
          pair_change<LOG>(P, B.x, B.y, B.z, B.dqlB, B.dp, B.cls, p.x, p.y, p.z, p.w, cls, acc, sacc, ov);
        }
        // domain list (shared memory)
        const int n = misc[0];
        for (int j = tid; j < n; j += T) {
          if (j == A.skip || j == B.skip) continue;
          const float4 p = L.pos[j];
          const int cls = (L.info[j] >> INFO_CLS_SHIFT) & 3;
          pair_change<LOG>(P, A.x, A.y, A.z, A.dqlB, A.dp, A.cls, p.x, p.y, p.z, p.w, cls, acc, sacc, ov);
          pair_change<LOG>(P, B.x, B.y, B.z, B.dqlB, B.dp, B.cls, p.x, p.y, p.z, p.w, cls, acc, sacc, ov);
        }
        acc = warp_sum(acc);
        if (LOG) sacc = warp_sum(sacc);
        ov = __any_sync(0xffffffffu, ov) ? 1 : 0;
        if (lane == 0) {
          red[warp] = acc;
          reds[warp] = sacc;
          redov[warp] = ov;
        }
      }
      __syncthreads();
      // ---- warp 0: decision and commit
      if (warp == 0) {
        TrialCtl &C = *ctl;
        const TrialPre &q = tp[t];
        int flags = C.flags;
        bool accept = false;
        double dE = 0.0, S = 0.0, lnA = -INFINITY;
        if (C.nch) {
          long long tot = C.cc;
          unsigned long long stot = C.cc_s;
          int anyov = C.cc_ov;
          for (int w = 0; w < nw; ++w) {
            tot += red[w];
            stot += reds[w];
            anyov |= redov[w];
          }
          if (anyov) {
            flags |= CR_TRIAL_OVERLAP;
            dE = INFINITY;
          } else {
            dE = (double)tot * FIX_INV + C.dself;
            S = (double)stot * FIX_INV + fabs(C.dself);
            lnA = C.ln_ratio - dE;
            accept = q.lnu < lnA;
          }
        }
        // cell capacity for insertions (checked before committing anything)
        const int r = C.move >> 1;
        const bool fwd = (C.move & 1) == 0;
        int n = misc[0];
        if (accept && fwd) {
          int below, same;
          warp_rank_count(L.rank, n, q.rankA, below, same);
          int need_same_b = 0;
          bool full = same + 1 > P.cap;
          if (r == R_SALT) {
            int below2, same2;
            warp_rank_count(L.rank, n, q.rankB, below2, same2);
            need_same_b = same2 + 1 + (q.rankB == q.rankA ? 1 : 0);
            full = full || need_same_b > P.cap;
          }
          if (full || n + 2 > P.dcap) {
            accept = false;
            if (lane == 0) atomicOr(P.err, ERRB_CELL_OVERFLOW);
          }
        }
        if (accept) {
          flags |= CR_TRIAL_ACCEPTED;
          const unsigned long long idA = C.newid;
          if (r == R_ACID || r == R_BASE) {
            const float qs = r == R_ACID ? -1.0f : 1.0f;
            if (lane == 0) {
              const int si = C.site;
              L.info[si] ^= INFO_ION_BIT;
              L.pos[si].w = fwd ? qs : 0.0f;
            }
            __syncwarp();
            if (fwd) {
              int below, same;
              warp_rank_count(L.rank, n, q.rankA, below, same);
              const int p = below + same;
              warp_insert_gap(L, n, p);
              if (lane == 0) {
                L.pos[p] = make_float4(q.ax, q.ay, q.az, -qs * P.ion_q);
                L.vel[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                L.id[p] = idA;
                L.info[p] = (r == R_ACID ? CR_XP : CR_XM) | (P.ion_cls << INFO_CLS_SHIFT);
                L.rank[p] = q.rankA;
              }
              n += 1;
            } else {
              warp_remove(L, n, C.ionA);
              n -= 1;
            }
            if (lane == 0) {
              const int kn = r == R_ACID ? K_A0 : K_B0, ki = kn + 1, kx = r == R_ACID ? K_XP : K_XM;
              const int dlt = fwd ? 1 : -1;
              misc[1 + kn] -= dlt;
              misc[1 + ki] += dlt;
              misc[1 + kx] += dlt;
            }
          } else {
            if (fwd) {
              int below, same;
              warp_rank_count(L.rank, n, q.rankA, below, same);
              int p = below + same;
              warp_insert_gap(L, n, p);
              if (lane == 0) {
                L.pos[p] = make_float4(q.ax, q.ay, q.az, P.ion_q);
                L.vel[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                L.id[p] = idA;
                L.info[p] = CR_XP | (P.ion_cls << INFO_CLS_SHIFT);
                L.rank[p] = q.rankA;
              }
              __syncwarp();
              n += 1;
              warp_rank_count(L.rank, n, q.rankB, below, same);
              p = below + same;
              warp_insert_gap(L, n, p);
              if (lane == 0) {
                L.pos[p] = make_float4(q.bx, q.by, q.bz, -P.ion_q);
                L.vel[p] = make_float4(0.f, 0.f, 0.f, 0.f);
                L.id[p] = idA + 1u;
                L.info[p] = CR_XM | (P.ion_cls << INFO_CLS_SHIFT);
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
              misc[1 + K_XP] += dlt;
              misc[1 + K_XM] += dlt;
            }
          }
          __syncwarp();
        }
        if (lane == 0) {
          misc[0] = n;
          st[C.move] += 1;
          if (flags & CR_TRIAL_ACCEPTED) st[6 + C.move] += 1;
          if (flags & CR_TRIAL_NO_ELIGIBLE) st[12] += 1;
          if (flags & CR_TRIAL_EDGE) st[13] += 1;
          if (flags & CR_TRIAL_OVERLAP) st[14] += 1;
          st[15] += 1;
          if (LOG && P.log) {
            cr_trial rec;
            rec.move = C.move;
            rec.flags = flags;
            rec.id_a = C.id_a;
            rec.id_b = C.id_b;
            rec.dE = dE;
            rec.S = S;
            rec.lnA = lnA;
            rec.lnu = q.lnu;
            P.log[log_dom + kk] = rec;
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- write the domain back (id-sorted cells) and publish counts
  const int n = misc[0];
  for (int r = tid; r < KC; r += T) {
    int lo = 0, hi = n;  // first entry with rank >= r
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (L.rank[mid] < r) lo = mid + 1; else hi = mid; }
    int lo2 = lo, hi2 = n;  // first entry with rank > r
    while (lo2 < hi2) { const int mid = (lo2 + hi2) >> 1; if (L.rank[mid] <= r) lo2 = mid + 1; else hi2 = mid; }
    dcnt[r] = lo;
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    const int cell = (org[0] + lx) % nc + nc * ((org[1] + ly) % nc + nc * ((org[2] + lz) % nc));
    P.cnt[cell] = lo2 - lo;
  }
  __syncthreads();
  for (int j = tid; j < n; j += T) {
    const int r = L.rank[j];
    const int lx = r % k, ly = (r / k) % k, lz = r / (k * k);
    const int cell = (org[0] + lx) % nc + nc * ((org[1] + ly) % nc + nc * ((org[2] + lz) % nc));
    const int g = cell * P.cap + (j - dcnt[r]);
    P.pos[g] = L.pos[j];
    P.vel[g] = L.vel[j];
    P.pid[g] = L.id[j];
    P.info[g] = L.info[j];
    if (L.id[j] < (unsigned long long)P.n_perm) P.perm_slot[L.id[j]] = g;
  }
  if (tid < 16 && st[tid]) atomicAdd(&P.stats[tid], st[tid]);
  if (tid < 6 && misc[1 + tid] != misc[9 + tid])
    atomicAdd((unsigned long long *)&P.counts[tid], (unsigned long long)(long long)(misc[1 + tid] - misc[9 + tid]));
}

}  // namespace crmc

namespace crmc {

// ---------------------------------------------------------------------------
// MD: forces on the particles of a block of kb^3 cells, from the particles of
// the block and its halo (cells within h of the block), one warp per particle.
// Pair forces are FP32 terms summed in 2^-24 fixed point, so the result does
// not depend on the launch shape.  Mode 0: conservative forces into fout;
// mode 1: + Langevin friction/noise; mode 2: + Langevin and the closing half
// kick v += dt/2 f.
// ---------------------------------------------------------------------------
constexpr float FFIX = 16777216.0f;  // 2^24
constexpr float FFIX_INV = 1.0f / 16777216.0f;

__device__ __forceinline__ void force_pair(const SysParams &P, float xi, float yi, float zi, float qi, int ci,
                                           float xj, float yj, float zj, float qj, int cj, long long &fx,
                                           long long &fy, long long &fz) {
  const float dx = wrap_diff(xi, xj, P.Lf, P.halfL);
  const float dy = wrap_diff(yi, yj, P.Lf, P.halfL);
  const float dz = wrap_diff(zi, zj, P.Lf, P.halfL);
  const float r2 = dx * dx + dy * dy + dz * dz;
  float f = 0.0f;  // along (ri - rj) / r, positive = repulsive
  bool any = false;
  if (r2 < P.rc2 && qi != 0.0f && qj != 0.0f) {
    const float r = sqrtf(r2);
    const float ar = P.alpha * r;
    f = P.lBf * qi * qj * (erfcf(ar) / r2 + 1.1283791670955126f * P.alpha * expf(-ar * ar) / r - P.c2);
    any = true;
  }
  const WcaEntry &w = P.wca[ci * 4 + cj];
  if (w.on && r2 < w.wcut2) {
    const float s = sqrtf(r2) - w.del;
    const float t = w.sig / s;
    const float t2 = t * t;
    const float t6 = t2 * t2 * t2;
    f += 24.0f * w.eps * (2.0f * t6 * t6 - t6) / s;
    any = true;
  }
  if (any) {
    const float g = f / sqrtf(r2);
    fx += __float2ll_rn(g * dx * FFIX);
    fy += __float2ll_rn(g * dy * FFIX);
    fz += __float2ll_rn(g * dz * FFIX);
  }
}

__global__ void __launch_bounds__(256) k_md_forces(SysParams P, MdParams M, int kb, int nb_dim, int nrb) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  const int nc = P.nc, h = P.h;
  const int KC = kb * kb * kb, NR = nrb * nrb * nrb;
  unsigned char *sp = smem;
  float4 *rpos = (float4 *)sp; sp += sizeof(float4) * M.rcap;
  int *rcls = (int *)sp; sp += sizeof(int) * M.rcap;
  int *scan_tmp = (int *)sp; sp += sizeof(int) * 256;
  int *cnt = (int *)sp; sp += sizeof(int) * (NR + 1);
  int *pre = (int *)sp; sp += sizeof(int) * (NR + 1);
  int *cell_of_r = (int *)sp; sp += sizeof(int) * (NR + 1);

  const int b = blockIdx.x;
  const int bx = b % nb_dim, by = (b / nb_dim) % nb_dim, bz = b / (nb_dim * nb_dim);
  const int org[3] = {bx * kb, by * kb, bz * kb};
  // region cells: block cells first (region index < KC), then the halo
  // (region_coord ordering along each dimension, block cells skipped)
  for (int i = tid; i < NR; i += T) {
    const int ix = i % nrb, iy = (i / nrb) % nrb, iz = i / (nrb * nrb);
    const int cx = region_coord(ix, org[0], kb, h, nrb, nc), cy = region_coord(iy, org[1], kb, h, nrb, nc),
              cz = region_coord(iz, org[2], kb, h, nrb, nc);
    const int cell = cx + nc * (cy + nc * cz);
    const bool inb = ix < kb && iy < kb && iz < kb;
    // order: block cells get slots [0, KC) in rank order, halo cells follow
    const int slot = inb ? (ix + kb * (iy + kb * iz)) : -1;
    if (inb) {
      cell_of_r[slot] = cell;
      cnt[slot] = P.cnt[cell];
    }
  }
  __syncthreads();
  // halo cells in region order after the block
  if (tid == 0) {
    int s = KC;
    for (int i = 0; i < NR; ++i) {
      const int ix = i % nrb, iy = (i / nrb) % nrb, iz = i / (nrb * nrb);
      if (ix < kb && iy < kb && iz < kb) continue;
      const int cx = region_coord(ix, org[0], kb, h, nrb, nc), cy = region_coord(iy, org[1], kb, h, nrb, nc),
                cz = region_coord(iz, org[2], kb, h, nrb, nc);
      cell_of_r[s++] = cx + nc * (cy + nc * cz);
    }
  }
  __syncthreads();
  for (int i = KC + tid; i < NR; i += T) cnt[i] = P.cnt[cell_of_r[i]];
  __syncthreads();
  block_scan(cnt, NR, pre, scan_tmp);
  const int NB = pre[KC], NT = pre[NR];
  for (int j = tid; j < min(NT, M.rcap); j += T) {
    const int i = upper_idx(pre, NR, j);
    const int g = cell_of_r[i] * P.cap + (j - pre[i]);
    rpos[j] = P.pos[g];
    rcls[j] = (P.info[g] >> INFO_CLS_SHIFT) & 3;
  }
  __syncthreads();
  for (int ci = warp; ci < NB; ci += nw) {
    const int ri = upper_idx(pre, KC, ci);
    const int gi = cell_of_r[ri] * P.cap + (ci - pre[ri]);
    const float4 pi = ci < M.rcap ? rpos[ci] : P.pos[gi];
    const int clsi = ci < M.rcap ? rcls[ci] : (P.info[gi] >> INFO_CLS_SHIFT) & 3;
    long long fx = 0, fy = 0, fz = 0;
    for (int j = lane; j < NT; j += 32) {
      if (j == ci) continue;
      float4 pj;
      int cj;
      if (j < M.rcap) {
        pj = rpos[j];
        cj = rcls[j];
      } else {
        const int i = upper_idx(pre, NR, j);
        const int g = cell_of_r[i] * P.cap + (j - pre[i]);
        pj = P.pos[g];
        cj = (P.info[g] >> INFO_CLS_SHIFT) & 3;
      }
      force_pair(P, pi.x, pi.y, pi.z, pi.w, clsi, pj.x, pj.y, pj.z, pj.w, cj, fx, fy, fz);
    }
    // FENE bonds of permanent particles, U = -K R0^2/2 ln(1 - (r/R0)^2)
    const unsigned long long id = P.pid[gi];
    if (id < (unsigned long long)M.n_perm) {
      const int b0 = M.bond_off[id], b1 = M.bond_off[id + 1];
      for (int bb = b0 + lane; bb < b1; bb += 32) {
        const int gj = M.perm_slot[M.bond_nbr[bb]];
        const float4 pj = P.pos[gj];
        const float dx = wrap_diff(pi.x, pj.x, P.Lf, P.halfL);
        const float dy = wrap_diff(pi.y, pj.y, P.Lf, P.halfL);
        const float dz = wrap_diff(pi.z, pj.z, P.Lf, P.halfL);
        const float x2 = (dx * dx + dy * dy + dz * dz) * M.inv_R02;
        if (x2 >= 1.0f) {
          atomicOr(P.err, ERRB_BOND);
          continue;
        }
        const float g = -M.fene_K / (1.0f - x2);
        fx += __float2ll_rn(g * dx * FFIX);
        fy += __float2ll_rn(g * dy * FFIX);
        fz += __float2ll_rn(g * dz * FFIX);
      }
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    if (lane == 0) {
      float4 f = make_float4((float)fx * FFIX_INV, (float)fy * FFIX_INV, (float)fz * FFIX_INV, 0.0f);
      if (M.mode == 0) {
        M.fout[gi] = f;
      } else {
        // Langevin: -gamma v + sqrt(2 gamma kT / dt) xi, xi from Box-Muller on
        // Philox(counter = (id_lo, id_hi, eval, 5), key = seed)
        float4 v = M.vel[gi];
        const uint4 w = philox10((uint32_t)id, (uint32_t)(id >> 32), M.eval, 5u, M.key0, M.key1);
        const float u0 = (float)(((double)w.x + 0.5) * (1.0 / 4294967296.0));
        const float u1 = (float)(((double)w.y + 0.5) * (1.0 / 4294967296.0));
        const float u2 = (float)(((double)w.z + 0.5) * (1.0 / 4294967296.0));
        const float u3 = (float)(((double)w.w + 0.5) * (1.0 / 4294967296.0));
        const float r1 = sqrtf(-2.0f * logf(u0)), r2 = sqrtf(-2.0f * logf(u2));
        float s1, c1, s3, c3;
        sincospif(2.0f * u1, &s1, &c1);
        sincospif(2.0f * u3, &s3, &c3);
        f.x += -M.gamma * v.x + M.amp * r1 * c1;
        f.y += -M.gamma * v.y + M.amp * r1 * s1;
        f.z += -M.gamma * v.z + M.amp * r2 * c3;
        M.fout[gi] = f;
        if (M.mode == 2) {
          v.x += 0.5f * M.dt * f.x;
          v.y += 0.5f * M.dt * f.y;
          v.z += 0.5f * M.dt * f.z;
          M.vel[gi] = v;
        }
      }
    }
  }
}

// v += dt/2 f; x += dt v; wrap into [0, L)
__global__ void k_md_kick_drift(SysParams P, MdParams M) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P.ncell * P.cap) return;
  const int c = g / P.cap;
  if (g - c * P.cap >= P.cnt[c]) return;
  float4 v = M.vel[g];
  const float4 f = M.fout[g];
  v.x += 0.5f * M.dt * f.x;
  v.y += 0.5f * M.dt * f.y;
  v.z += 0.5f * M.dt * f.z;
  M.vel[g] = v;
  float4 p = P.pos[g];
  float x[3] = {p.x + M.dt * v.x, p.y + M.dt * v.y, p.z + M.dt * v.z};
  for (int i = 0; i < 3; ++i) {
    x[i] -= P.Lf * floorf(x[i] * P.invL);
    if (x[i] >= P.Lf) x[i] -= P.Lf;
    if (x[i] < 0.0f) x[i] = 0.0f;
  }
  P.pos[g] = make_float4(x[0], x[1], x[2], p.w);
}

// rebuild, step 1: scatter every particle into its new cell (unordered)
__global__ void k_rebuild_scatter(SysParams P, RebuildBufs B) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P.ncell * P.cap) return;
  const int c = g / P.cap;
  if (g - c * P.cap >= P.cnt[c]) return;
  const float4 p = P.pos[g];
  const int nc = P.nc;
  const int cell = cell_of(p.x, P.scf, nc) + nc * (cell_of(p.y, P.scf, nc) + nc * cell_of(p.z, P.scf, nc));
  const int s = atomicAdd(&B.cnt[cell], 1);
  if (s >= P.cap) {
    atomicOr(P.err, ERRB_CELL_OVERFLOW);
    return;
  }
  const int o = cell * P.cap + s;
  B.pos[o] = p;
  B.pid[o] = P.pid[g];
  B.info[o] = P.info[g];
  B.vel[o] = B.vel_src[g];
  B.frc[o] = B.frc_src[g];
}

// rebuild, step 2: one warp per cell sorts the cell by id into the primary arrays
__global__ void k_rebuild_sort(SysParams P, RebuildBufs B, int *perm_slot, int n_perm) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= P.ncell) return;
  const int c = warp;
  const int n = min(B.cnt[c], P.cap);
  const int base = c * P.cap;
  for (int e = lane; e < n; e += 32) {
    const unsigned long long id = B.pid[base + e];
    int rank = 0;
    for (int o = 0; o < n; ++o) rank += B.pid[base + o] < id;
    const int dst = base + rank;
    P.pos[dst] = B.pos[base + e];
    P.pid[dst] = id;
    P.info[dst] = B.info[base + e];
    B.vel_src[dst] = B.vel[base + e];
    B.frc_src[dst] = B.frc[base + e];
    if (id < (unsigned long long)n_perm) perm_slot[id] = dst;
  }
  __syncwarp();
  if (lane == 0) {
    P.cnt[c] = n;
    B.cnt[c] = 0;
  }
}

// refresh the slot of every permanent particle
__global__ void k_perm_slots(SysParams P, int *perm_slot, int n_perm) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P.ncell * P.cap) return;
  const int c = g / P.cap;
  if (g - c * P.cap >= P.cnt[c]) return;
  const unsigned long long id = P.pid[g];
  if (id < (unsigned long long)n_perm) perm_slot[id] = g;
}

// dump every particle (unordered) for the state view
__global__ void k_dump(SysParams P, DumpBufs D) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P.ncell * P.cap) return;
  const int c = g / P.cap;
  if (g - c * P.cap >= P.cnt[c]) return;
  const int o = atomicAdd(D.counter, 1);
  if (o >= D.cap) return;
  D.pos[o] = P.pos[g];
  D.pid[o] = P.pid[g];
  D.info[o] = P.info[g];
  if (D.vel_src) D.vel[o] = D.vel_src[g];
  if (D.frc_src) D.frc[o] = D.frc_src[g];
}

// load: place input particles (index = id) into cells, unordered
__global__ void k_load_scatter(SysParams P, LoadBufs I, RebuildBufs B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I.n) return;
  const float x = I.xyz[3 * i], y = I.xyz[3 * i + 1], z = I.xyz[3 * i + 2];
  const int t = I.type[i];
  const int ion = (t == CR_ACID || t == CR_BASE) && I.state[i] ? 1 : 0;
  float q = 0.0f;
  int cl = I.cls[i];
  if (t == CR_ACID) q = ion ? -1.0f : 0.0f;
  else if (t == CR_BASE) q = ion ? 1.0f : 0.0f;
  else if (t == CR_XP) { q = P.ion_q; cl = P.ion_cls; }
  else if (t == CR_XM) { q = -P.ion_q; cl = P.ion_cls; }
  const int site = (i < I.n_site_map && I.site[i] >= 0) ? I.site[i] : 0;
  const int nc = P.nc;
  const int cell = cell_of(x, P.scf, nc) + nc * (cell_of(y, P.scf, nc) + nc * cell_of(z, P.scf, nc));
  const int s = atomicAdd(&B.cnt[cell], 1);
  if (s >= P.cap) {
    atomicOr(P.err, ERRB_CELL_OVERFLOW);
    return;
  }
  const int o = cell * P.cap + s;
  B.pos[o] = make_float4(x, y, z, q);
  B.pid[o] = (unsigned long long)i;
  B.info[o] = t | (cl << INFO_CLS_SHIFT) | (ion ? INFO_ION_BIT : 0) | (site << INFO_SITE_SHIFT);
  B.vel[o] = I.vel ? make_float4(I.vel[3 * i], I.vel[3 * i + 1], I.vel[3 * i + 2], 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
  B.frc[o] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int n,
                         uint4 *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox10(c0 + (uint32_t)i, c1, c2, c3, k0, k1);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
size_t phase_smem_bytes(const SysParams &P) {
  const int KC = P.k * P.k * P.k, NR = P.nr * P.nr * P.nr;
  size_t b = 0;
  b += 2 * sizeof(float4) * P.dcap + sizeof(unsigned long long) * P.dcap + 2 * sizeof(int) * P.dcap;
  b += sizeof(TrialPre) * TRIAL_CHUNK;
  b += (sizeof(TrialCtl) + 15) / 16 * 16;
  b += sizeof(long long) * 32 + sizeof(unsigned long long) * 32 + sizeof(int) * 32;
  b += sizeof(int) * 256 + sizeof(int) * 16 + sizeof(unsigned long long) * 16;
  b += 2 * sizeof(int) * (NR + 1) + 2 * sizeof(int) * (KC + 1);
  return b;
}

size_t md_smem_bytes(int kb, int nrb, int rcap) {
  const int NR = nrb * nrb * nrb;
  return sizeof(float4) * rcap + sizeof(int) * rcap + sizeof(int) * 256 + 3 * sizeof(int) * (NR + 1);
}

template <int R, bool LOG>
static cudaError_t launch_phase_t(const SysParams &P, int grid, int threads, size_t smem, cudaStream_t s,
                                  uint32_t sweep, int colour, uint32_t k0, uint32_t k1) {
  static bool attr_done = false;
  static size_t attr_bytes = 0;
  if (!attr_done || smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_cr_phase<R, LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
    attr_bytes = smem;
  }
  k_cr_phase<R, LOG><<<grid, threads, smem, s>>>(P, sweep, colour, k0, k1);
  return cudaGetLastError();
}

cudaError_t launch_phase(const SysParams &P, int R, bool log, int grid, int threads, size_t smem, cudaStream_t s,
                         uint32_t sweep, int colour, uint32_t k0, uint32_t k1) {
#define CRMC_CASE(RR)                                                                      \
  case RR:                                                                                 \
    return log ? launch_phase_t<RR, true>(P, grid, threads, smem, s, sweep, colour, k0, k1) \
               : launch_phase_t<RR, false>(P, grid, threads, smem, s, sweep, colour, k0, k1);
  switch (R) {
    CRMC_CASE(1)
    CRMC_CASE(2)
    CRMC_CASE(4)
    CRMC_CASE(8)
    CRMC_CASE(16)
    default:
      return cudaErrorInvalidValue;
  }
#undef CRMC_CASE
}

cudaError_t launch_md_forces(const SysParams &P, const MdParams &M, int kb, int nb_dim, int nrb, int threads,
                             cudaStream_t s) {
  const size_t smem = md_smem_bytes(kb, nrb, M.rcap);
  static size_t attr = 0;
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(k_md_forces, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  k_md_forces<<<nb_dim * nb_dim * nb_dim, threads, smem, s>>>(P, M, kb, nb_dim, nrb);
  return cudaGetLastError();
}

cudaError_t launch_kick_drift(const SysParams &P, const MdParams &M, cudaStream_t s) {
  const int n = P.ncell * P.cap;
  k_md_kick_drift<<<(n + 255) / 256, 256, 0, s>>>(P, M);
  return cudaGetLastError();
}

cudaError_t launch_rebuild(const SysParams &P, const RebuildBufs &B, int *perm_slot, int n_perm, cudaStream_t s) {
  const int n = P.ncell * P.cap;
  k_rebuild_scatter<<<(n + 255) / 256, 256, 0, s>>>(P, B);
  k_rebuild_sort<<<(P.ncell * 32 + 255) / 256, 256, 0, s>>>(P, B, perm_slot, n_perm);
  return cudaGetLastError();
}

cudaError_t launch_load(const SysParams &P, const LoadBufs &I, const RebuildBufs &B, int *perm_slot, int n_perm,
                        cudaStream_t s) {
  if (I.n > 0) k_load_scatter<<<(I.n + 255) / 256, 256, 0, s>>>(P, I, B);
  k_rebuild_sort<<<(P.ncell * 32 + 255) / 256, 256, 0, s>>>(P, B, perm_slot, n_perm);
  return cudaGetLastError();
}

cudaError_t launch_perm_slots(const SysParams &P, int *perm_slot, int n_perm, cudaStream_t s) {
  const int n = P.ncell * P.cap;
  k_perm_slots<<<(n + 255) / 256, 256, 0, s>>>(P, perm_slot, n_perm);
  return cudaGetLastError();
}

cudaError_t launch_dump(const SysParams &P, const DumpBufs &D, cudaStream_t s) {
  const int n = P.ncell * P.cap;
  k_dump<<<(n + 255) / 256, 256, 0, s>>>(P, D);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int n,
                          uint4 *out, cudaStream_t s) {
  k_philox<<<(n + 255) / 256, 256, 0, s>>>(c0, c1, c2, c3, k0, k1, n, out);
  return cudaGetLastError();
}

}  // namespace crmc
