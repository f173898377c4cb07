// crmc_md.cu -- MD kernels (DSF + WCA + FENE forces, Langevin velocity Verlet),
// the cell rebuild after particles move, configuration upload and a Philox
// check kernel (sm_103a).
#include <cuda_runtime.h>

#include <cstdint>

#include "crmc_device.cuh"
#include "crmc_kernels.h"

namespace crmc {

// ---------------------------------------------------------------------------
// MD force helpers: FP32 pair forces summed in 2^-24 fixed point, so the
// result does not depend on the launch shape or the order of the particle
// list.  Mode 0: conservative forces into fout; mode 1: + Langevin
// friction/noise; mode 2: + Langevin and the closing half kick v += dt/2 f.
// ---------------------------------------------------------------------------
constexpr float FFIX_INV = 1.0f / 16777216.0f;

// FLAT: i and j are given in the stencil's flat frame (md_frame), where the
// plain difference is the minimum-image one bit for bit
// The pair's force on i in 2^-24 fixed point (zero out of range).  The terms
// are odd in (i, j): exchanging the particles negates dx, dy, dz exactly and
// leaves r^2 and g unchanged (charges are 0 or +-1, the WCA table is
// symmetric), and fix24 rounds symmetrically, so the force on j is exactly
// the negated value.
template <bool FLAT = false>
__device__ __forceinline__ void force_pair(const SysParams &P, float xi, float yi, float zi, float qi, int ci,
                                           float xj, float yj, float zj, float qj, int cj, long long &fx,
                                           long long &fy, long long &fz) {
  const float dx = FLAT ? xi - xj : wrap_diff(xi, xj, P.Lf, P.halfL);
  const float dy = FLAT ? yi - yj : wrap_diff(yi, yj, P.Lf, P.halfL);
  const float dz = FLAT ? zi - zj : wrap_diff(zi, zj, P.Lf, P.halfL);
  const float r2 = dx * dx + dy * dy + dz * dz;
  const WcaEntry &w = P.wca[ci * 4 + cj];
  const bool coul = r2 < P.rc2 && qi != 0.0f && qj != 0.0f;
  const bool wca = w.on && r2 < w.wcut2;
  if (!coul && !wca) return;
  const float rinv = rsqrtf(r2);
  float g = 0.0f;  // force / r along (ri - rj), positive = repulsive
  if (coul) {
    const float r = r2 * rinv;
    const float ar = P.alpha * r;
    g = P.lBf * qi * qj * (erfcf(ar) * rinv * rinv + 1.1283791670955126f * P.alpha * __expf(-ar * ar) * rinv - P.c2) * rinv;
  }
  if (wca) {
    const float s = r2 * rinv - w.del;
    const float is = __fdividef(1.0f, s);
    const float t = w.sig * is;
    const float t2 = t * t;
    const float t6 = t2 * t2 * t2;
    g += 24.0f * w.eps * (2.0f * t6 * t6 - t6) * is * rinv;
  }
  fx += fix24(g * dx);
  fy += fix24(g * dy);
  fz += fix24(g * dz);
}


// FENE bonds, Langevin and the store of the total force, for one particle
// (lane 0 of its warp)
__device__ __forceinline__ void finish_particle(const SysParams &P, const MdParams &M, int gi, float4 pi,
                                                long long fx, long long fy, long long fz) {
  const unsigned long long id = P.pid[gi];
  if (id < (unsigned long long)M.n_perm) {  // FENE, U = -K R0^2/2 ln(1 - (r/R0)^2)
    const int b0 = M.bond_off[id], b1 = M.bond_off[id + 1];
    for (int bb = b0; bb < b1; ++bb) {
      const float4 pj = P.pos[M.perm_slot[M.bond_nbr[bb]]];
      const float dx = wrap_diff(pi.x, pj.x, P.Lf, P.halfL);
      const float dy = wrap_diff(pi.y, pj.y, P.Lf, P.halfL);
      const float dz = wrap_diff(pi.z, pj.z, P.Lf, P.halfL);
      const float x2 = (dx * dx + dy * dy + dz * dz) * M.inv_R02;
      if (x2 >= 1.0f) {
        atomicOr(P.err, ERRB_BOND);
        continue;
      }
      const float g = -M.fene_K / (1.0f - x2);
      fx += fix24(g * dx);
      fy += fix24(g * dy);
      fz += fix24(g * dz);
    }
  }
  float4 f = make_float4((float)fx * FFIX_INV, (float)fy * FFIX_INV, (float)fz * FFIX_INV, 0.0f);
  // mode 0, or a rigid body's member (its body takes the thermostat and the kicks)
  if (M.mode == 0 || (M.n_bodies > 0 && id < (unsigned long long)M.n_perm && M.body_member[id] >= 0)) {
    M.fout[gi] = f;
    return;
  }
  // Langevin: -gamma v + sqrt(2 gamma kT / dt) xi, xi from Box-Muller on
  // Philox(counter = (id_lo, id_hi, eval, 5), key = seed)
  float4 v = M.vel[gi];
  uint32_t key0 = M.key0, key1 = M.key1, eval = M.eval;
  if (M.dyn) {  // a captured cycle: this step's key and evaluation counter
    const unsigned long long step = M.dyn->step, seed = M.dyn->md_seed0 + step;
    key0 = (uint32_t)seed;
    key1 = (uint32_t)(seed >> 32) ^ M.rep;
    eval = M.dyn->eval0 + (uint32_t)step + (uint32_t)M.eval_off;
  }
  const uint4 w = philox10((uint32_t)id, (uint32_t)(id >> 32), eval, 5u, key0, key1);
  const float u0 = ((float)(w.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u1 = ((float)(w.y >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u2 = ((float)(w.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u3 = ((float)(w.w >> 8) + 0.5f) * (1.0f / 16777216.0f);
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

constexpr int MD_THREADS = 128;
constexpr int MD_NW = MD_THREADS / 32;
constexpr int MD_QCAP = 64;
constexpr int MD_CPL = 4;  // stencil cells per lane (125 cells of a 5^3 stencil over 32 lanes)
constexpr int HALF5 = 62;  // the own cell's index in a 5^3 stencil; the higher indices are its upper half

__device__ __forceinline__ int wrap_cell(int c, int nc) { return c < 0 ? c + nc : (c >= nc ? c - nc : c); }

// Flat frame of a stencil narrower than 0.4 L: along an axis where the
// stencil wraps around the periodic boundary (s), x >= L/2 becomes x - L
// (exact for L/2 <= x < L); plain differences between points of the stencil
// then equal the minimum-image ones bit for bit.
__device__ __forceinline__ float md_frame(float x, bool s, float halfL, float L) { return s && x >= halfL ? x - L : x; }

// compact list of occupied slots; one atomic per warp of 32 cells
__global__ void k_plist(SysParams P, int *plist, int *n_out, int max_out, long long *fsum) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
  const int n = c < P.ncell ? P.cnt[c] : 0;
  int x = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  int base = 0;
  if (lane == 31) base = atomicAdd(n_out, x);
  base = __shfl_sync(0xffffffffu, base, 31);
  const int o = base + x - n;
  if (o + n > max_out && n > 0) atomicOr(P.err, ERRB_CAPACITY);  // more particles than the context's capacity
  // entries that fit are written even then, so every entry the force kernel
  // reads (below min(count, max_out)) names a slot of this system
  for (int s = 0; s < n && o + s < max_out; ++s) plist[o + s] = c * P.cap + s;
  if (fsum)  // the occupied slots' force sums start from zero (k_md_forces adds both ends of each pair)
    for (int s = 0; s < n; ++s) {
      fsum[3 * (c * P.cap + s)] = 0;
      fsum[3 * (c * P.cap + s) + 1] = 0;
      fsum[3 * (c * P.cap + s) + 2] = 0;
    }
}

// MD forces: one warp per particle.  The candidates of the (2h+1)^3 stencil of
// neighbour cells (cell side >= rc/h) are numbered consecutively over the
// cells (a warp prefix sum of the cell counts), so the lanes take 32
// consecutive candidates per round whatever the cells' occupancy; every lane
// tests its candidate (cheap), in-range partners are queued and their forces
// evaluated with all lanes busy.  Pair forces are FP32 terms summed in 2^-24
// fixed point, so the result does not depend on the order.
// SPLIT: the warp stores its particle's pair-force sums for k_md_finish (one
// thread per particle) instead of finishing it on lane 0 while 31 lanes idle.
// FLAT (with NBC > 0): the stencil spans less than 0.4 L, distances are taken
// in its flat frame (md_frame) without minimum-image tests.
// One queued pair (i, j = slot g2): the force on i into this lane's sums;
// SPLIT: each pair is evaluated once, and the force on j (the exact negation)
// goes into j's fixed-point sums by 64-bit integer atomics (exact and
// order-free, so the sums equal those of evaluating the pair from both ends).
template <bool SPLIT, bool FLAT>
__device__ __forceinline__ void md_pair(const SysParams &P, const MdParams &M, int g2, float xi, float yi, float zi,
                                        float qi, int clsi, bool sx, bool sy, bool sz, long long &fx, long long &fy,
                                        long long &fz) {
  const float4 pj = P.pos[g2];
  long long vx = 0, vy = 0, vz = 0;
  force_pair<FLAT>(P, xi, yi, zi, qi, clsi, FLAT ? md_frame(pj.x, sx, P.halfL, P.Lf) : pj.x,
                   FLAT ? md_frame(pj.y, sy, P.halfL, P.Lf) : pj.y, FLAT ? md_frame(pj.z, sz, P.halfL, P.Lf) : pj.z,
                   pj.w, (P.info[g2] >> INFO_CLS_SHIFT) & 3, vx, vy, vz);
  fx += vx;
  fy += vy;
  fz += vz;
  if (SPLIT && (vx | vy | vz) != 0) {
    unsigned long long *d = reinterpret_cast<unsigned long long *>(M.fsum) + 3 * g2;
    atomicAdd(d, (unsigned long long)(-vx));
    atomicAdd(d + 1, (unsigned long long)(-vy));
    atomicAdd(d + 2, (unsigned long long)(-vz));
  }
}

template <int NBC, bool SPLIT, bool FLAT = false>  // NBC: 2h+1 when the box has at least that many cells per dimension, else 0
__global__ void __launch_bounds__(MD_THREADS) k_md_forces(SysParams P, MdParams M) {
  __shared__ int queue[MD_NW][MD_QCAP];
  __shared__ int cpre[MD_NW][MD_CPL * 32 + 1];  // exclusive prefix of the stencil cells' counts
  __shared__ int cbs[MD_NW][MD_CPL * 32];       // first slot of each stencil cell
  __shared__ int startcell[MD_NW][32];          // per round: the cell that starts at each candidate position
  const int lane = threadIdx.x & 31;
  const int wl = threadIdx.x >> 5;
  const int w = blockIdx.x * MD_NW + wl;
  if (w >= *M.n_particles || w >= M.max_particles) return;  // whole warp
  const int nc = P.nc, h = P.h, cap = P.cap;
  const int gi = M.plist[w];
  const float4 pi = P.pos[gi];
  const int clsi = (P.info[gi] >> INFO_CLS_SHIFT) & 3;
  const int cell = gi / cap;
  const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
  const int nb = NBC > 0 ? NBC : min(2 * h + 1, nc);
  const bool all = NBC == 0 && nb == nc;  // every cell of the dimension, once
  const int nb3 = nb * nb * nb;
  const bool sx = FLAT && (cx < h || cx + h >= nc), sy = FLAT && (cy < h || cy + h >= nc),
             sz = FLAT && (cz < h || cz + h >= nc);
  const float xi = FLAT ? md_frame(pi.x, sx, P.halfL, P.Lf) : pi.x, yi = FLAT ? md_frame(pi.y, sy, P.halfL, P.Lf) : pi.y,
              zi = FLAT ? md_frame(pi.z, sz, P.halfL, P.Lf) : pi.z;
  // stencil cell o = lane + 32 t: its first slot and count; the candidates of
  // all cells are then numbered consecutively (exclusive prefix over o)
  int run = 0;
  int lpre[MD_CPL], lcnt[MD_CPL];  // this lane's cells: first candidate number and count
#pragma unroll
  for (int t = 0; t < MD_CPL; ++t) {
    const int o = lane + 32 * t;
    int n = 0, base = 0;
    // SPLIT over a 5^3 stencil (at least 5 cells per dimension, so no two
    // offsets name the same cell): only the upper half of the offsets, the
    // own cell (o = 62) with its higher slots; the partner's warp finds the
    // pair through the opposite offset otherwise
    if (o < nb3 && !(SPLIT && NBC == 5 && o < HALF5)) {
      const int ox = o % nb, oy = (o / nb) % nb, oz = o / (nb * nb);
      const int jx = all ? ox : wrap_cell(cx + ox - h, nc);
      const int jy = all ? oy : wrap_cell(cy + oy - h, nc);
      const int jz = all ? oz : wrap_cell(cz + oz - h, nc);
      const int jc = jx + nc * (jy + nc * jz);
      base = jc * cap;
      n = P.cnt[jc];
      if (FLAT && n > 0) {  // a cell whose box lies beyond the interaction reach holds no partner
        const float x0 = (float)(cx + ox - h) * P.af, y0 = (float)(cy + oy - h) * P.af,
                    z0 = (float)(cz + oz - h) * P.af;
        const float ex = fmaxf(0.0f, fmaxf(x0 - pi.x, pi.x - (x0 + P.af)));
        const float ey = fmaxf(0.0f, fmaxf(y0 - pi.y, pi.y - (y0 + P.af)));
        const float ez = fmaxf(0.0f, fmaxf(z0 - pi.z, pi.z - (z0 + P.af)));
        if (ex * ex + ey * ey + ez * ez > M.reach2) n = 0;
      }
    }
    int x = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    cpre[wl][o] = run + x - n;
    cbs[wl][o] = base;
    lpre[t] = run + x - n;
    lcnt[t] = n;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) cpre[wl][MD_CPL * 32] = run;
  __syncwarp();
  const int total = run;
  int *q = queue[wl];
  const int *pre = cpre[wl];
  int qn = 0;
  long long fx = 0, fy = 0, fz = 0;
  int carry = 0;  // the cell that runs on past the previous round's last candidate
  for (int c0 = 0; c0 < total; c0 += 32) {
    const int c = c0 + lane;
    // cell of candidate c: the last non-empty cell that starts at or before
    // it; each lane marks where its own cells start inside this round
    unsigned mk = 0u;
#pragma unroll
    for (int t = 0; t < MD_CPL; ++t) {
      const int st = lpre[t] - c0;
      if (lcnt[t] > 0 && st >= 0 && st < 32) {
        mk |= 1u << st;
        startcell[wl][st] = lane + 32 * t;
      }
    }
    mk = __reduce_or_sync(0xffffffffu, mk);
    __syncwarp();
    const unsigned upto = mk & (0xffffffffu >> (31 - lane));
    const int cell_o = upto ? startcell[wl][31 - __clz(upto)] : carry;
    carry = __shfl_sync(0xffffffffu, cell_o, 31);
    __syncwarp();
    bool in = false;
    int gj = -1;
    if (c < total) {
      gj = cbs[wl][cell_o] + (c - pre[cell_o]);
      // SPLIT: each pair once (the upper half of a 5^3 stencil and the higher
      // slots of the own cell; otherwise every pair from its lower slot)
      if (SPLIT ? ((NBC == 5 && cell_o != HALF5) || gj > gi) : gj != gi) {
        const float4 pj = P.pos[gj];
        const int cj = (P.info[gj] >> INFO_CLS_SHIFT) & 3;
        const float dx = FLAT ? xi - md_frame(pj.x, sx, P.halfL, P.Lf) : wrap_diff(pi.x, pj.x, P.Lf, P.halfL);
        const float dy = FLAT ? yi - md_frame(pj.y, sy, P.halfL, P.Lf) : wrap_diff(pi.y, pj.y, P.Lf, P.halfL);
        const float dz = FLAT ? zi - md_frame(pj.z, sz, P.halfL, P.Lf) : wrap_diff(pi.z, pj.z, P.Lf, P.halfL);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const WcaEntry &wc = P.wca[clsi * 4 + cj];
        in = (r2 < P.rc2 && pi.w != 0.0f && pj.w != 0.0f) || (wc.on && r2 < wc.wcut2);
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (in) q[qn + __popc(m & ((1u << lane) - 1u))] = gj;
    qn += __popc(m);
    if (qn >= 32) {
      __syncwarp();
      md_pair<SPLIT, FLAT>(P, M, q[lane], xi, yi, zi, pi.w, clsi, sx, sy, sz, fx, fy, fz);
      const int rest = qn - 32;
      int keep = 0;
      if (lane < rest) keep = q[32 + lane];
      __syncwarp();
      if (lane < rest) q[lane] = keep;
      __syncwarp();
      qn = rest;
    }
  }
  __syncwarp();
  if (lane < qn) md_pair<SPLIT, FLAT>(P, M, q[lane], xi, yi, zi, pi.w, clsi, sx, sy, sz, fx, fy, fz);
  fx = warp_sum_i64(fx);
  fy = warp_sum_i64(fy);
  fz = warp_sum_i64(fz);
  if (SPLIT) {  // this particle's own pairs join what its partners added
    if (lane < 3)
      atomicAdd(reinterpret_cast<unsigned long long *>(M.fsum) + 3 * gi + lane,
                (unsigned long long)(lane == 0 ? fx : (lane == 1 ? fy : fz)));
  } else if (lane == 0) {
    finish_particle(P, M, gi, pi, fx, fy, fz);
  }
}

// FENE bonds, Langevin and the store of every particle's force (and the
// half kick), one thread per particle, after k_md_forces<., true>
__global__ void k_md_finish(SysParams P, MdParams M) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= *M.n_particles || w >= M.max_particles) return;
  const int gi = M.plist[w];
  finish_particle(P, M, gi, P.pos[gi], M.fsum[3 * gi], M.fsum[3 * gi + 1], M.fsum[3 * gi + 2]);
}

// v += dt/2 f; x += dt v; wrap into [0, L); the particle goes straight into
// its new cell of the scratch arrays (unordered; k_rebuild_sort orders them)
__global__ void k_md_kick_drift_scatter(SysParams P, MdParams M, RebuildBufs B) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P.ncell * P.cap) return;
  const int c = g / P.cap;
  if (g - c * P.cap >= P.cnt[c]) return;
  float4 v = M.vel[g];
  const float4 f = M.fout[g];
  const float4 p = P.pos[g];
  const unsigned long long id = P.pid[g];
  const int mb = (M.n_bodies > 0 && id < (unsigned long long)M.n_perm) ? M.body_member[id] : -1;
  float x[3];
  if (mb >= 0) {  // a rigid body's member: placed by its body (k_body_drift)
    const float4 q = M.body_newpos[mb];
    x[0] = q.x;
    x[1] = q.y;
    x[2] = q.z;
  } else {
    v.x += 0.5f * M.dt * f.x;
    v.y += 0.5f * M.dt * f.y;
    v.z += 0.5f * M.dt * f.z;
    x[0] = p.x + M.dt * v.x;
    x[1] = p.y + M.dt * v.y;
    x[2] = p.z + M.dt * v.z;
    for (int i = 0; i < 3; ++i) {
      x[i] -= P.Lf * floorf(x[i] * P.invL);
      if (x[i] >= P.Lf) x[i] -= P.Lf;
      if (x[i] < 0.0f) x[i] = 0.0f;
    }
  }
  const int nc = P.nc;
  const int cell = cell_of(x[0], P.scf, nc) + nc * (cell_of(x[1], P.scf, nc) + nc * cell_of(x[2], P.scf, nc));
  const int s = atomicAdd(&B.cnt[cell], 1);
  if (s >= P.cap) {
    atomicOr(P.err, ERRB_CELL_OVERFLOW);
    return;
  }
  const int o = cell * P.cap + s;
  B.pos[o] = make_float4(x[0], x[1], x[2], p.w);
  B.pid[o] = id;
  B.info[o] = P.info[g];
  B.vel[o] = v;
  B.frc[o] = f;
}

// rebuild: one warp per cell sorts the cell by id into the primary arrays
__device__ __forceinline__ void rebuild_sort_cell(const SysParams &P, const RebuildBufs &B, int *perm_slot, int n_perm,
                                                  int warp) {
  const int lane = threadIdx.x & 31;
  if (warp >= P.ncell) return;
  const int c = warp;
  const int n = min(B.cnt[c], P.cap);
  const int base = c * P.cap;
  if (n <= 32) {  // the cell's ids in the lanes, ranks by shuffles
    const unsigned long long id = lane < n ? B.pid[base + lane] : ~0ull;
    int rank = 0;
    for (int o = 0; o < n; ++o) rank += __shfl_sync(0xffffffffu, id, o) < id ? 1 : 0;
    if (lane < n) {
      const int dst = base + rank;
      P.pos[dst] = B.pos[base + lane];
      P.pid[dst] = id;
      P.info[dst] = B.info[base + lane];
      B.vel_src[dst] = B.vel[base + lane];
      B.frc_src[dst] = B.frc[base + lane];
      if (id < (unsigned long long)n_perm) perm_slot[id] = dst;
    }
  } else {
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
  }
  __syncwarp();
  if (lane == 0) {
    P.cnt[c] = n;
    B.cnt[c] = 0;
  }
}

__global__ void k_rebuild_sort(SysParams P, RebuildBufs B, int *perm_slot, int n_perm) {
  rebuild_sort_cell(P, B, perm_slot, n_perm, (blockIdx.x * blockDim.x + threadIdx.x) >> 5);
}

// the loaded configuration must be neutral (kind counts of the load)
__global__ void k_load_neutral(SysParams P) {
  if (threadIdx.x != 0) return;
  const long long q = P.counts[K_XP] + P.counts[K_SP] - P.counts[K_XM] - P.counts[K_SM] - P.counts[K_A1] + P.counts[K_B1];
  if (q != 0) atomicOr(P.err, ERRB_NOT_NEUTRAL);
}

// load: place input particles (index = id) into cells, unordered
__device__ __forceinline__ void load_particle(const SysParams &P, const LoadBufs &I, const RebuildBufs &B, int i) {
  if (i >= I.n) return;
  const float x = I.xyz[3 * i], y = I.xyz[3 * i + 1], z = I.xyz[3 * i + 2];
  const int t = I.type[i];
  // particle id: given (a restore; the host checked that the ids are unique
  // and complete) or the index
  const unsigned long long pid = I.id ? I.id[i] : (unsigned long long)i;
  {  // the particle must be valid and a bonded / site particle of cr_init must keep its id and type
    const int ti = pid < (unsigned long long)I.n_site_map ? I.init_type[pid] : CR_XP;
    const bool fixed = !is_ion_type(ti);
    const bool ok = t >= CR_BEAD && t <= CR_SM && I.cls[i] >= 0 && I.cls[i] <= 3 && x >= 0.0f && x < P.Lf &&
                    y >= 0.0f && y < P.Lf && z >= 0.0f && z < P.Lf && (fixed ? t == ti : is_ion_type(t));
    if (!ok) {
      atomicOr(P.err, ERRB_ARG);
      return;
    }
  }
  const int ion = (t == CR_ACID || t == CR_BASE) && I.state[i] ? 1 : 0;
  float q = 0.0f;
  int cl = I.cls[i];
  if (t == CR_ACID) q = ion ? -1.0f : 0.0f;
  else if (t == CR_BASE) q = ion ? 1.0f : 0.0f;
  else if (is_ion_type(t)) { q = (float)ion_sign(t) * P.ion_q; cl = P.ion_cls; }
  {  // global kind counts (zeroed by the host before the launch)
    const int kd = t == CR_ACID ? (ion ? K_A1 : K_A0)
                   : t == CR_BASE ? (ion ? K_B1 : K_B0)
                   : t == CR_XP ? K_XP : t == CR_XM ? K_XM : t == CR_SP ? K_SP : t == CR_SM ? K_SM : K_OTHER;
    if (kd < K_OTHER) atomicAdd((unsigned long long *)&P.counts[kd], 1ull);
  }
  const int site = (pid < (unsigned long long)I.n_site_map && I.site[pid] >= 0) ? I.site[pid] : 0;
  const int nc = P.nc;
  const int cell = cell_of(x, P.scf, nc) + nc * (cell_of(y, P.scf, nc) + nc * cell_of(z, P.scf, nc));
  const int s = atomicAdd(&B.cnt[cell], 1);
  if (s >= P.cap) {
    atomicOr(P.err, ERRB_CELL_OVERFLOW);
    return;
  }
  const int o = cell * P.cap + s;
  B.pos[o] = make_float4(x, y, z, q);
  B.pid[o] = pid;
  B.info[o] = t | (cl << INFO_CLS_SHIFT) | (ion ? INFO_ION_BIT : 0) | (site << INFO_SITE_SHIFT);
  B.vel[o] = I.vel ? make_float4(I.vel[3 * i], I.vel[3 * i + 1], I.vel[3 * i + 2], 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
  B.frc[o] = I.frc ? make_float4(I.frc[3 * i], I.frc[3 * i + 1], I.frc[3 * i + 2], 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_load_scatter(SysParams P, LoadBufs I, RebuildBufs B) {
  load_particle(P, I, B, blockIdx.x * blockDim.x + threadIdx.x);
}

// Loads of every replica of a batch (blockIdx.y = replica): counts zeroed,
// particles placed, cells sorted, neutrality checked, one launch per step.
__global__ void k_load_zero_batch(const SysParams *__restrict__ reps) {
  if (threadIdx.x < N_KIND) reps[blockIdx.x].counts[threadIdx.x] = 0;
}
__global__ void k_load_scatter_batch(const SysParams *__restrict__ reps, const LoadJob *__restrict__ jobs) {
  const LoadJob &J = jobs[blockIdx.y];
  load_particle(reps[blockIdx.y], J.I, J.B, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void k_rebuild_sort_batch(const SysParams *__restrict__ reps, const LoadJob *__restrict__ jobs) {
  const LoadJob &J = jobs[blockIdx.y];
  rebuild_sort_cell(reps[blockIdx.y], J.B, J.perm_slot, J.n_perm, (blockIdx.x * blockDim.x + threadIdx.x) >> 5);
}
__global__ void k_load_neutral_batch(const SysParams *__restrict__ reps) {
  if (threadIdx.x != 0) return;
  const SysParams &P = reps[blockIdx.x];
  const long long q = P.counts[K_XP] + P.counts[K_SP] - P.counts[K_XM] - P.counts[K_SM] - P.counts[K_A1] + P.counts[K_B1];
  if (q != 0) atomicOr(P.err, ERRB_NOT_NEUTRAL);
}

__global__ void k_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int n,
                         uint4 *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox10(c0 + (uint32_t)i, c1, c2, c3, k0, k1);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------

__global__ void k_step_advance(StepDyn *dyn) {
  if (threadIdx.x == 0) dyn->step += 1;
}

// ---------------------------------------------------------------------------
// Rigid bodies (Sec. IV.B: the nanoparticles' sites are rigidly attached to
// the shell; the thermostat acts on each nanoparticle as a whole).
// Newton-Euler equations with Langevin friction and noise on the centre of
// mass (-gamma M V + sqrt(2 gamma M / dt) xi) and on the rotation (lab frame:
// -gamma L + sqrt(2 gamma / dt) R diag(sqrt I) R^T xi', L = R pi), the normals
// xi, xi' from the Philox blocks (body, 0, eval, 8) and (body, 0, eval, 9)
// under the MD key.  Velocity Verlet: half kicks V += dt/2 F/M and
// pi += dt/2 R^T T; the drift X += dt V and the free rotation as exact
// rotations about the body axes 1, 2, 3, 2, 1 for dt/2, dt/2, dt, dt/2, dt/2
// (the symmetric splitting of Dullweber, Leimkuhler and McLachlan, J. Chem.
// Phys. 107, 5840 (1997)).  Members sit at wrap(X + R d) and move with
// V + omega x (R d), omega = R (pi / I); they get no thermostat of their own.
// One CTA per body, FP64 body arithmetic; sums over the members go thread by
// thread in member order, then through a fixed tree, so the result does not
// depend on where the members sit in the cell list.
// ---------------------------------------------------------------------------
constexpr int RB_THREADS = 512;

__device__ __forceinline__ void rb_mul(const double *R, const double *v, double *o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = R[3 * a] * v[0] + R[3 * a + 1] * v[1] + R[3 * a + 2] * v[2];
}
__device__ __forceinline__ void rb_tmul(const double *R, const double *v, double *o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = R[a] * v[0] + R[3 + a] * v[1] + R[6 + a] * v[2];
}
__device__ __forceinline__ void rb_cross(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// the CTA's sums of NV per-thread values (every thread gets them)
template <int NV>
__device__ void rb_sum(double (&v)[NV], double *sh) {
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k * RB_THREADS + t] = v[k];
  __syncthreads();
  for (int h = RB_THREADS / 2; h > 0; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k * RB_THREADS + t] += sh[k * RB_THREADS + t + h];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sh[k * RB_THREADS];
  __syncthreads();
}

// symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van
// Loan, Matrix Computations, Sec. 8.5): w the eigenvalues, the columns of V
// the eigenvectors
__device__ void rb_eigen(double *A, double *w, double *V) {
  for (int i = 0; i < 9; ++i) V[i] = (i == 0 || i == 4 || i == 8) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (off == 0.0 || off <= 1e-32 * (A[0] * A[0] + A[4] * A[4] + A[8] * A[8])) break;
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
      const double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      const double tau = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      for (int k = 0; k < 3; ++k) {  // columns p, q of A and V: times the rotation
        const double x = A[3 * k + p], y = A[3 * k + q];
        A[3 * k + p] = c * x - s * y;
        A[3 * k + q] = s * x + c * y;
        const double u = V[3 * k + p], z = V[3 * k + q];
        V[3 * k + p] = c * u - s * z;
        V[3 * k + q] = s * u + c * z;
      }
      for (int k = 0; k < 3; ++k) {  // rows p, q of A: the transposed rotation
        const double x = A[3 * p + k], y = A[3 * q + k];
        A[3 * p + k] = c * x - s * y;
        A[3 * q + k] = s * x + c * y;
      }
    }
  }
  w[0] = A[0];
  w[1] = A[4];
  w[2] = A[8];
}

// a member's slot, or -1 when the id is not a present non-ion particle
__device__ __forceinline__ int rb_slot(const SysParams &P, const MdParams &M, int id) {
  const int s = M.perm_slot[id];
  if (s < 0 || s >= P.ncell * P.cap) return -1;
  if (P.pid[s] != (unsigned long long)id || is_ion_type(P.info[s] & 15)) return -1;
  return s;
}

__device__ __forceinline__ double rb_min_image(double d, double L) { return d - L * rint(d / L); }

__device__ __forceinline__ float rb_wrap(double x, double L, double invL, float Lf) {
  x -= L * floor(x * invL);
  float f = __double2float_rn(x);
  if (f >= Lf) f -= Lf;
  if (f < 0.0f) f = 0.0f;
  return f;
}

__global__ void __launch_bounds__(RB_THREADS) k_body_setup(SysParams P, MdParams M) {
  __shared__ double sh[9 * RB_THREADS];
  __shared__ double R_s[9], sub_s[3];
  __shared__ int bad_s;
  RigidBody *B = M.bodies + blockIdx.x;
  const int t = threadIdx.x, first = B->first, count = B->count, mf = B->mfirst;
  const double L = (double)P.Lf;
  if (t == 0) bad_s = 0;
  __syncthreads();
  const int s0 = rb_slot(P, M, first);
  if (s0 < 0) {
    if (t == 0) B->bad = 1;
    return;
  }
  const float4 p0 = P.pos[s0];
  const double r0[3] = {(double)p0.x, (double)p0.y, (double)p0.z};
  double a[6] = {0, 0, 0, 0, 0, 0};  // offset sums, momentum
  for (int m = t; m < count; m += RB_THREADS) {
    const int s = rb_slot(P, M, first + m);
    if (s < 0) {
      bad_s = 1;
      continue;
    }
    const float4 p = P.pos[s], v = M.vel[s];
    a[0] += rb_min_image((double)p.x - r0[0], L);
    a[1] += rb_min_image((double)p.y - r0[1], L);
    a[2] += rb_min_image((double)p.z - r0[2], L);
    a[3] += (double)v.x;
    a[4] += (double)v.y;
    a[5] += (double)v.z;
  }
  rb_sum<6>(a, sh);
  if (bad_s) {
    if (t == 0) B->bad = 1;
    return;
  }
  const double Mb = (double)count, sub[3] = {a[0] / Mb, a[1] / Mb, a[2] / Mb};
  double b[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // dx dx, dy dy, dz dz, dx dy, dx dz, dy dz; angular momentum
  for (int m = t; m < count; m += RB_THREADS) {
    const int s = rb_slot(P, M, first + m);
    const float4 p = P.pos[s], v = M.vel[s];
    const double d[3] = {rb_min_image((double)p.x - r0[0], L) - sub[0], rb_min_image((double)p.y - r0[1], L) - sub[1],
                         rb_min_image((double)p.z - r0[2], L) - sub[2]};
    const double u[3] = {(double)v.x, (double)v.y, (double)v.z};
    double l[3];
    rb_cross(d, u, l);
    b[0] += d[0] * d[0];
    b[1] += d[1] * d[1];
    b[2] += d[2] * d[2];
    b[3] += d[0] * d[1];
    b[4] += d[0] * d[2];
    b[5] += d[1] * d[2];
    b[6] += l[0];
    b[7] += l[1];
    b[8] += l[2];
  }
  rb_sum<9>(b, sh);
  if (t == 0) {
    double A[9] = {b[1] + b[2], -b[3], -b[4], -b[3], b[0] + b[2], -b[5], -b[4], -b[5], b[0] + b[1]};
    double w[3], V[9];
    rb_eigen(A, w, V);
    int o[3] = {0, 1, 2};  // ascending moments
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j)
        if (w[o[j]] < w[o[i]]) {
          const int x = o[i];
          o[i] = o[j];
          o[j] = x;
        }
    double e[3][3];
    for (int k = 0; k < 2; ++k) {  // the largest component of the first two axes positive
      int big = 0;
      for (int i = 0; i < 3; ++i) {
        e[k][i] = V[3 * i + o[k]];
        if (fabs(e[k][i]) > fabs(e[k][big])) big = i;
      }
      if (e[k][big] < 0.0)
        for (int i = 0; i < 3; ++i) e[k][i] = -e[k][i];
    }
    rb_cross(e[0], e[1], e[2]);
    for (int k = 0; k < 3; ++k) {
      B->I[k] = w[o[k]];
      for (int i = 0; i < 3; ++i) R_s[3 * i + k] = e[k][i];
    }
    for (int i = 0; i < 9; ++i) B->R[i] = R_s[i];
    const double Lm[3] = {b[6], b[7], b[8]};
    rb_tmul(R_s, Lm, B->pi);
    for (int k = 0; k < 3; ++k) {
      B->X[k] = r0[k] + sub[k];
      B->V[k] = a[3 + k] / Mb;
      B->F[k] = 0.0;
      B->T[k] = 0.0;
      sub_s[k] = sub[k];
    }
    B->M = Mb;
    B->bad = (B->I[0] > 1e-9 * (B->I[0] + B->I[1] + B->I[2])) ? 0 : 1;
  }
  __syncthreads();
  for (int m = t; m < count; m += RB_THREADS) {
    const int s = rb_slot(P, M, first + m);
    const float4 p = P.pos[s];
    const double d[3] = {rb_min_image((double)p.x - r0[0], L) - sub_s[0],
                         rb_min_image((double)p.y - r0[1], L) - sub_s[1],
                         rb_min_image((double)p.z - r0[2], L) - sub_s[2]};
    double *db = M.body_d + 3 * (mf + m);
    rb_tmul(R_s, d, db);
    M.body_df[mf + m] = make_float4((float)db[0], (float)db[1], (float)db[2], 0.0f);
  }
}

// the members' rigid velocities V + omega x (R d) (and, with newpos, the
// positions X + R d after a drift, wrapped into the box)
// (the per-member products in FP32: an arm of a few sigma rounds far below the
// FP32 resolution of the positions; the centre and the sums stay FP64)
__device__ __forceinline__ void rb_fmul(const float *R, float4 d, float *o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = R[3 * a] * d.x + R[3 * a + 1] * d.y + R[3 * a + 2] * d.z;
}

// R, omega = R (pi / I) and V of the body in FP32, formed once by thread 0
// (the FP64 pipe is narrow: every thread forming them cost more than the members)
struct RbF32 {
  float R[9], om[3], V[3];
};
__device__ __forceinline__ void rb_f32(const RigidBody &B, RbF32 &F) {
  double w[3], om[3];
  for (int k = 0; k < 3; ++k) w[k] = B.pi[k] / B.I[k];
  rb_mul(B.R, w, om);
  for (int k = 0; k < 9; ++k) F.R[k] = (float)B.R[k];
  for (int k = 0; k < 3; ++k) {
    F.om[k] = (float)om[k];
    F.V[k] = (float)B.V[k];
  }
}

__device__ void rb_members(const SysParams &P, const MdParams &M, const RigidBody &B, bool newpos) {
  __shared__ RbF32 F;
  if (threadIdx.x == 0) rb_f32(B, F);
  __syncthreads();
  float Rf[9], omf[3], Vf[3];
  for (int k = 0; k < 9; ++k) Rf[k] = F.R[k];
  for (int k = 0; k < 3; ++k) {
    omf[k] = F.om[k];
    Vf[k] = F.V[k];
  }
  const double L = (double)P.Lf;
  for (int m = threadIdx.x; m < B.count; m += RB_THREADS) {
    const int s = M.perm_slot[B.first + m];
    float a[3];
    rb_fmul(Rf, M.body_df[B.mfirst + m], a);
    float4 v = M.vel[s];
    v.x = Vf[0] + (omf[1] * a[2] - omf[2] * a[1]);
    v.y = Vf[1] + (omf[2] * a[0] - omf[0] * a[2]);
    v.z = Vf[2] + (omf[0] * a[1] - omf[1] * a[0]);
    M.vel[s] = v;
    if (newpos)
      M.body_newpos[B.mfirst + m] =
          make_float4(rb_wrap(B.X[0] + (double)a[0], L, P.invLd, P.Lf), rb_wrap(B.X[1] + (double)a[1], L, P.invLd, P.Lf),
                      rb_wrap(B.X[2] + (double)a[2], L, P.invLd, P.Lf), 0.0f);
  }
}

__global__ void __launch_bounds__(RB_THREADS) k_body_member_velocities(SysParams P, MdParams M) {
  rb_members(P, M, M.bodies[blockIdx.x], false);
}

// three normals from the Philox block (body, 0, eval, purpose): the Box-Muller
// form of the particles' Langevin noise, in FP32 as theirs
__device__ void rb_normals(uint32_t body, uint32_t eval, uint32_t purpose, uint32_t k0, uint32_t k1, double *g) {
  const uint4 w = philox10(body, 0u, eval, purpose, k0, k1);
  const float u0 = ((float)(w.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u1 = ((float)(w.y >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u2 = ((float)(w.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float u3 = ((float)(w.w >> 8) + 0.5f) * (1.0f / 16777216.0f);
  const float r1 = sqrtf(-2.0f * logf(u0)), r2 = sqrtf(-2.0f * logf(u2));
  float s1, c1, s3, c3;
  sincospif(2.0f * u1, &s1, &c1);
  sincospif(2.0f * u3, &s3, &c3);
  g[0] = (double)(r1 * c1);
  g[1] = (double)(r1 * s1);
  g[2] = (double)(r2 * c3);
}

// force and torque of each body from its members' conservative forces, plus
// the Langevin terms; kick: the closing half kick; then the members' velocities
__global__ void __launch_bounds__(RB_THREADS) k_body_forces(SysParams P, MdParams M, int kick) {
  __shared__ double sh[6 * RB_THREADS];
  __shared__ RigidBody B;
  const int t = threadIdx.x;
  if (t == 0) B = M.bodies[blockIdx.x];
  __syncthreads();
  float Rf[9];
  for (int k = 0; k < 9; ++k) Rf[k] = (float)B.R[k];
  float af[6] = {0, 0, 0, 0, 0, 0};  // this thread's few members, FP32
  for (int m = t; m < B.count; m += RB_THREADS) {
    const int s = M.perm_slot[B.first + m];
    const float4 f = M.fout[s];
    float r[3];
    rb_fmul(Rf, M.body_df[B.mfirst + m], r);
    af[0] += f.x;
    af[1] += f.y;
    af[2] += f.z;
    af[3] += r[1] * f.z - r[2] * f.y;
    af[4] += r[2] * f.x - r[0] * f.z;
    af[5] += r[0] * f.y - r[1] * f.x;
  }
  double a[6];
  for (int k = 0; k < 6; ++k) a[k] = (double)af[k];
  rb_sum<6>(a, sh);
  if (t == 0) {
    double gt[3], gr[3], Lm[3], y[3], S[3];
    rb_normals(blockIdx.x, M.eval, 8u, M.key0, M.key1, gt);
    rb_normals(blockIdx.x, M.eval, 9u, M.key0, M.key1, gr);
    const double gam = M.body_gamma, dt = M.body_dt;
    const double at = sqrt(2.0 * gam * B.M / dt), ar = sqrt(2.0 * gam / dt);
    rb_mul(B.R, B.pi, Lm);
    rb_tmul(B.R, gr, y);
    for (int k = 0; k < 3; ++k) y[k] *= sqrt(B.I[k]);
    rb_mul(B.R, y, S);
    for (int k = 0; k < 3; ++k) {
      B.F[k] = a[k] - gam * B.M * B.V[k] + at * gt[k];
      B.T[k] = a[3 + k] - gam * Lm[k] + ar * S[k];
    }
    if (kick) {
      double tb[3];
      rb_tmul(B.R, B.T, tb);
      for (int k = 0; k < 3; ++k) {
        B.V[k] += 0.5 * dt * B.F[k] / B.M;
        B.pi[k] += 0.5 * dt * tb[k];
      }
    }
    M.bodies[blockIdx.x] = B;
  }
  __syncthreads();
  if (kick) rb_members(P, M, B, false);
}

// exact free rotation about body axis k for a time h
__device__ void rb_rotate(RigidBody &B, int k, double h) {
  const double th = h * B.pi[k] / B.I[k];
  double s, c;
  if (fabs(th) < 1e-2) {  // the Taylor series, truncated below FP64 rounding (|th|^7 / 7! < 2e-18)
    const double t2 = th * th;
    s = th * (1.0 - t2 * (1.0 / 6.0) * (1.0 - t2 * (1.0 / 20.0) * (1.0 - t2 * (1.0 / 42.0))));
    c = 1.0 - t2 * 0.5 * (1.0 - t2 * (1.0 / 12.0) * (1.0 - t2 * (1.0 / 30.0) * (1.0 - t2 * (1.0 / 56.0))));
  } else {
    sincos(th, &s, &c);
  }
  const int i = (k + 1) % 3, j = (k + 2) % 3;
  for (int r = 0; r < 3; ++r) {
    const double x = B.R[3 * r + i], y = B.R[3 * r + j];
    B.R[3 * r + i] = c * x + s * y;
    B.R[3 * r + j] = -s * x + c * y;
  }
  const double pi_i = B.pi[i], pi_j = B.pi[j];
  B.pi[i] = c * pi_i + s * pi_j;
  B.pi[j] = -s * pi_i + c * pi_j;
}

// the opening half kick and the drift of each body, the members' new
// positions into body_newpos and their velocities
__global__ void __launch_bounds__(RB_THREADS) k_body_drift(SysParams P, MdParams M) {
  __shared__ RigidBody B;
  if (threadIdx.x == 0) {
    B = M.bodies[blockIdx.x];
    const double dt = M.body_dt;
    double tb[3];
    rb_tmul(B.R, B.T, tb);
    for (int k = 0; k < 3; ++k) {
      B.V[k] += 0.5 * dt * B.F[k] / B.M;
      B.pi[k] += 0.5 * dt * tb[k];
      B.X[k] += dt * B.V[k];
    }
    rb_rotate(B, 0, 0.5 * dt);
    rb_rotate(B, 1, 0.5 * dt);
    rb_rotate(B, 2, dt);
    rb_rotate(B, 1, 0.5 * dt);
    rb_rotate(B, 0, 0.5 * dt);
    M.bodies[blockIdx.x] = B;
  }
  __syncthreads();
  rb_members(P, M, B, true);
}

// ---------------------------------------------------------------------------
// Ewald reciprocal-space forces, minus the gradient of E_rec: for one half
// space of k with the doubled weights A' (the vectors the CR-MC trials use),
// F_j = 2 q_j sum_k A'_k k Im(S(k)^* exp(i k.r_j)), Im(...) = C sin - D cos,
// S = C + i D of the current positions (k_ewald_sk runs just before).  One
// CTA of 256 threads per particle of the force kernel's list (a particle's
// sum spans thousands of vectors: eight warps keep the SM busy where one warp
// per particle left it waiting on latencies); the axis factors
// exp(i 2 pi n x / L), n <= kmax, from the coordinate's 0.32 fixed-point
// fraction (an exact phase reduction); each thread sums every 256th vector in
// order, the warps by a fixed butterfly, the eight warp sums in warp order;
// the result joins the particle's 2^-24 fixed-point force sums before
// k_md_finish.
// ---------------------------------------------------------------------------
constexpr int EWF_THREADS = 256;
constexpr int EWF_K1 = 33;  // kmax + 1 for kmax <= 32

__device__ __forceinline__ float2 ewf_factor(float x, double invL, int n) {
  const uint32_t U = (uint32_t)(unsigned long long)llrint((double)x * invL * 4294967296.0);
  const uint32_t t = (uint32_t)n * U;
  float sn, cs;
  sincospif((float)t * (2.0f / 4294967296.0f), &sn, &cs);
  return make_float2(cs, sn);
}

__device__ __forceinline__ float2 ewf_get(const float2 *f, int n) {
  const float2 v = f[n < 0 ? -n : n];
  return make_float2(v.x, n < 0 ? -v.y : v.y);
}

__device__ __forceinline__ float2 ewf_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(EWF_THREADS) k_ewald_forces(SysParams P, MdParams M) {
  __shared__ float2 f[3 * EWF_K1];
  __shared__ float part[EWF_THREADS / 32][3];
  const int w = blockIdx.x, t = threadIdx.x, lane = t & 31, wl = t >> 5;
  if (w >= *M.n_particles || w >= M.max_particles) return;  // whole CTA
  const int gi = M.plist[w];
  const float4 p = P.pos[gi];
  if (p.w == 0.0f) return;
  const int ewk = P.ewald_kmax + 1;
  for (int i = t; i < 3 * ewk; i += EWF_THREADS) {
    const int ax = i / ewk, n = i - ax * ewk;
    f[i] = ewf_factor(ax == 0 ? p.x : (ax == 1 ? p.y : p.z), P.invLd, n);
  }
  __syncthreads();
  float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll 4
  for (int i = t; i < P.ewald_nk; i += EWF_THREADS) {
    const int2 v = P.ek_nA[i];
    const float2 hi = P.ek_Shi[i], lo = P.ek_Slo[i];
    const int nx = (int)(signed char)(v.x & 255), ny = (int)(signed char)((v.x >> 8) & 255),
              nz = (int)(signed char)((v.x >> 16) & 255);
    const float C = hi.x + lo.x, D = hi.y + lo.y;
    const float2 e = ewf_mul(ewf_mul(ewf_get(f, nx), ewf_get(f + ewk, ny)), ewf_get(f + 2 * ewk, nz));
    const float g = __int_as_float(v.y) * (C * e.y - D * e.x);
    gx += g * (float)nx;
    gy += g * (float)ny;
    gz += g * (float)nz;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
    gz += __shfl_xor_sync(0xffffffffu, gz, o);
  }
  if (lane == 0) {
    part[wl][0] = gx;
    part[wl][1] = gy;
    part[wl][2] = gz;
  }
  __syncthreads();
  if (t == 0) {
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int k = 0; k < EWF_THREADS / 32; ++k) {
      sx += part[k][0];
      sy += part[k][1];
      sz += part[k][2];
    }
    const float s = 2.0f * p.w * (float)(6.283185307179586 * P.invLd);
    M.fsum[3 * gi] += fix24(s * sx);
    M.fsum[3 * gi + 1] += fix24(s * sy);
    M.fsum[3 * gi + 2] += fix24(s * sz);
  }
}

cudaError_t launch_step_advance(StepDyn *dyn, cudaStream_t s) {
  k_step_advance<<<1, 32, 0, s>>>(dyn);
  return cudaGetLastError();
}

cudaError_t launch_md_forces(const SysParams &P, const MdParams &M, int *plist, int *n_particles, int max_particles,
                             cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(n_particles, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_plist<<<(P.ncell + 255) / 256, 256, 0, s>>>(P, plist, n_particles, max_particles, M.fsum);
  MdParams Q = M;
  Q.plist = plist;
  Q.n_particles = n_particles;
  Q.max_particles = max_particles;
  const unsigned grid = (unsigned)((max_particles + MD_NW - 1) / MD_NW);
  const bool flat = 2.5f * (float)(2 * P.h + 1) * P.af < P.Lf;  // stencil narrower than 0.4 L
  if (Q.fsum) {
    if (flat && P.h == 2 && P.nc >= 5) k_md_forces<5, true, true><<<grid, MD_THREADS, 0, s>>>(P, Q);
    else if (P.h == 2 && P.nc >= 5) k_md_forces<5, true><<<grid, MD_THREADS, 0, s>>>(P, Q);
    else if (P.h == 1 && P.nc >= 3) k_md_forces<3, true><<<grid, MD_THREADS, 0, s>>>(P, Q);
    else k_md_forces<0, true><<<grid, MD_THREADS, 0, s>>>(P, Q);
    if (P.ewald_nk > 0)  // S(k) of these positions is current (launch_ewald_sk before this call)
      k_ewald_forces<<<(unsigned)max_particles, EWF_THREADS, 0, s>>>(P, Q);
    k_md_finish<<<(unsigned)((max_particles + 255) / 256), 256, 0, s>>>(P, Q);
  } else {
    if (P.h == 2 && P.nc >= 5) k_md_forces<5, false><<<grid, MD_THREADS, 0, s>>>(P, Q);
    else if (P.h == 1 && P.nc >= 3) k_md_forces<3, false><<<grid, MD_THREADS, 0, s>>>(P, Q);
    else k_md_forces<0, false><<<grid, MD_THREADS, 0, s>>>(P, Q);
  }
  if (M.n_bodies > 0 && M.mode != 0) k_body_forces<<<M.n_bodies, RB_THREADS, 0, s>>>(P, Q, M.mode == 2 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_kick_drift_rebuild(const SysParams &P, const MdParams &M, const RebuildBufs &B, int *perm_slot,
                                      int n_perm, cudaStream_t s) {
  const int n = P.ncell * P.cap;
  if (M.n_bodies > 0) k_body_drift<<<M.n_bodies, RB_THREADS, 0, s>>>(P, M);
  k_md_kick_drift_scatter<<<(n + 255) / 256, 256, 0, s>>>(P, M, B);
  k_rebuild_sort<<<(P.ncell * 32 + 255) / 256, 256, 0, s>>>(P, B, perm_slot, n_perm);
  return cudaGetLastError();
}

cudaError_t launch_load(const SysParams &P, const LoadBufs &I, const RebuildBufs &B, int *perm_slot, int n_perm,
                        cudaStream_t s) {
  if (I.n > 0) k_load_scatter<<<(I.n + 255) / 256, 256, 0, s>>>(P, I, B);
  k_rebuild_sort<<<(P.ncell * 32 + 255) / 256, 256, 0, s>>>(P, B, perm_slot, n_perm);
  k_load_neutral<<<1, 32, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_load_batch(const SysParams *d_reps, const LoadJob *d_jobs, int n_rep, int max_n, int max_cells,
                              cudaStream_t s) {
  k_load_zero_batch<<<n_rep, 32, 0, s>>>(d_reps);
  if (max_n > 0) k_load_scatter_batch<<<dim3((max_n + 255) / 256, n_rep), 256, 0, s>>>(d_reps, d_jobs);
  k_rebuild_sort_batch<<<dim3((max_cells * 32 + 255) / 256, n_rep), 256, 0, s>>>(d_reps, d_jobs);
  k_load_neutral_batch<<<n_rep, 32, 0, s>>>(d_reps);
  return cudaGetLastError();
}

cudaError_t launch_body_setup(const SysParams &P, const MdParams &M, cudaStream_t s) {
  if (M.n_bodies > 0) k_body_setup<<<M.n_bodies, RB_THREADS, 0, s>>>(P, M);
  return cudaGetLastError();
}

cudaError_t launch_body_member_velocities(const SysParams &P, const MdParams &M, cudaStream_t s) {
  if (M.n_bodies > 0) k_body_member_velocities<<<M.n_bodies, RB_THREADS, 0, s>>>(P, M);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int n,
                          uint4 *out, cudaStream_t s) {
  k_philox<<<(n + 255) / 256, 256, 0, s>>>(c0, c1, c2, c3, k0, k1, n, out);
  return cudaGetLastError();
}

}  // namespace crmc
