// crmc_api.cu -- host side of the C ABI declared in include/crmc.h.
//
// cr_init lays a system out in cell-major device arrays and precomputes the
// chemical constants of Sec. II.C / App. C of the paper in FP64; cr_sweep
// queues the colour phases of the checkerboard schedule; cr_md_step the
// velocity-Verlet/Langevin step that consumes the regulated charges.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "crmc.h"
#include "crmc_common.h"
#include "crmc_kernels.h"

using namespace crmc;

struct cr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  SysParams P{};
  // schedule / launch shape: (threads per CTA, halo registers per thread) of
  // the phase kernel, chosen by timing real sweeps (the chain does not depend
  // on it: the energy sums are exact fixed point)
  int T = 128, R = 4;
  int smem_max = 0;
  int tune_next = 0;     // sweeps timed so far (TUNE_ROUNDS passes over the candidates)
  bool tuning = true;
  float tune_ms[16] = {};
  PhaseShape S{};   // shared-memory capacities for the densest domain
  PhaseShape Sc{};  // compact capacities (most domains; denser ones spill to global memory)
  bool C = false, da_C = false;  // the tuned shapes use Sc
  SysParams *d_reps = nullptr;  // device copy of P (the phase kernel reads it)
  int64_t per_sweep = 0;
  // sizes
  int n_input = 0, n_sites = 0, n_other = 0, n_acid = 0, n_base = 0;
  int64_t capacity = 0;
  // device buffers
  int *d_cnt = nullptr, *d_cnt2 = nullptr, *d_info = nullptr, *d_info2 = nullptr;
  float4 *d_pos = nullptr, *d_pos2 = nullptr, *d_vel = nullptr, *d_vel2 = nullptr, *d_frc = nullptr,
         *d_frc2 = nullptr, *d_fcons = nullptr;
  unsigned long long *d_pid = nullptr, *d_pid2 = nullptr, *d_stats = nullptr;
  long long *d_lnK = nullptr, *d_lntab = nullptr;
  long long *d_counts = nullptr;
  int *d_perm = nullptr, *d_bond_off = nullptr, *d_bond_nbr = nullptr;
  // d_counts holds N_KIND + 2 words: [0, N_KIND) kind counts, [N_KIND] ions found by cr_state
  // (an int), [N_KIND + 1] the error word (an int), read back with one copy
  int *d_err = nullptr, *d_counter = nullptr;
  cr_trial *d_log = nullptr;
  size_t log_cap = 0;
  // dense-domain scratch of the phase kernel and the MD particle list
  float4 *d_gs_pos = nullptr, *d_gs_vel = nullptr;
  unsigned long long *d_gs_id = nullptr;
  long long *d_gs_lnk = nullptr;
  int *d_gs_info = nullptr, *d_gs_rank = nullptr;
  int *d_plist = nullptr, *d_nparts = nullptr;  // MD particle list
  long long *d_fsum = nullptr;                    // MD pair-force sums per slot
  int *d_order = nullptr;                       // launch order of the domains of each colour
  // delayed acceptance: surrogate on the device, records, its own launch-shape tuner
  uint16_t *d_mlp_w = nullptr;
  float *d_mlp_b = nullptr;
  bool has_mlp = false;
  cr_trial_da *d_dlog = nullptr;
  float *d_feat = nullptr;
  size_t dlog_cap = 0, feat_cap = 0;
  int da_T = 128, da_R = 0, da_next = 0;
  bool da_tuning = true;
  float da_ms[8] = {};
  // cr_load inputs (capacity-sized)
  float *d_in_xyz = nullptr, *d_in_vel = nullptr;
  int *d_in_type = nullptr, *d_in_cls = nullptr, *d_site_map = nullptr;
  int8_t *d_in_state = nullptr;
  unsigned long long *d_in_id = nullptr;  // cr_restore inputs (allocated on first use)
  float *d_in_frc = nullptr;
  // cr_state: id ordering on the device and the output arrays in the
  // caller's layouts (capacity-sized), one copy each to the caller
  int *d_present = nullptr;
  int ion_lo_bits = 32;  // the low words of inserted ids stay below 2^ion_lo_bits
  unsigned long long *d_ion_key = nullptr, *d_ion_key2 = nullptr;
  int *d_ion_val = nullptr, *d_ion_val2 = nullptr, *d_ion_rank = nullptr;
  unsigned char *d_sort_tmp = nullptr;
  size_t sort_tmp_bytes = 0;
  float *d_out_xyz = nullptr, *d_out_vel = nullptr, *d_out_frc = nullptr;
  unsigned long long *d_out_id = nullptr;
  int *d_out_type = nullptr, *d_out_cls = nullptr;
  int8_t *d_out_state = nullptr, *d_out_site = nullptr;
  long long *h_small = nullptr;           // pinned: kind counts [N_KIND], ions found, error word
  // chemistry kept for cr_set_pH: reservoir, per-site pK and kind, the
  // current pH and pI_X, and a version that batches compare against
  double pH = 7.0, pIXp = 0.0, pIXm = 0.0;
  bool inv_explicit = false;  // pI values set by cr_set_invocation (kept through pH changes)
  cr_mu_ions mu{};
  std::vector<double> site_pK;
  std::vector<char> site_is_acid;
  std::vector<long long> h_lnK_fx;
  int chem_version = 0;
  // MD
  double fene_K = 30.0, fene_R0 = 1.5;
  uint64_t sweep = 0;
  uint32_t md_eval = 0;
  bool f_valid = false, fcons_valid = false;
  // input encoding kept for cr_load: type of every input particle, site index
  std::vector<int> init_type, init_site;
  int *d_init_type = nullptr;  // init_type on the device (cr_load checks)
  int n_fixed_end = 0;         // one past the last bonded / site particle of cr_init
  // kernel timing (CUDA events on the context stream) and launch counters
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_pairs[2];  // [0] phase kernel, [1] MD force kernel
  size_t ev_next = 0;
  size_t ev_reserved = 0;  // events recorded by a batch's captured cycle (kept out of the pool's reuse)
  double ms[2] = {0.0, 0.0};
  int64_t launches[2] = {0, 0};
  int64_t launches_total = 0;
  // Ewald electrostatics: reciprocal vectors, weights, structure factor
  int2 *d_ek_nA = nullptr;
  float2 *d_ek_Shi = nullptr, *d_ek_Slo = nullptr;
  int *d_ek_list = nullptr, *d_ek_np = nullptr;
  // caller-owned slot arrays (cr_bind_device_buffers) and batch membership
  bool bound = false;
  int batch_refs = 0;
  // rigid bodies (cr_set_rigid_bodies)
  int n_bodies = 0, n_members = 0;
  RigidBody *d_bodies = nullptr;
  int *d_body_member = nullptr;
  double *d_body_d = nullptr;
  float4 *d_body_df = nullptr, *d_body_newpos = nullptr;
};

namespace {

constexpr double LN10 = 2.302585092994045684;
constexpr double RHO0_NA = 0.602214076;  // 1 M in nm^-3

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? CR_OK : (e == cudaErrorMemoryAllocation ? CR_ERR_NOMEM : CR_ERR_CUDA); }

#define CR_CUDA(call)                       \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

template <typename T>
int dalloc(T **p, size_t n) {
  if (n == 0) n = 1;
  return cuda_fail(cudaMalloc((void **)p, n * sizeof(T)));
}

double pIX_of(double pIS, double pH, double pOH) {
  const double m = pH < pOH ? pH : pOH;
  return -std::log10(std::pow(10.0, -pIS) + std::pow(10.0, -m));
}

// value at the 2^-48 fixed-point scale of the Metropolis exponent
long long to_lnfix(double v) { return std::llround(std::ldexp(v, 48)); }

int cell_of_host(float x, float scf, int nc) {
  const float t = x * scf;  // single IEEE multiply
  int c = (int)std::floor(t);
  if (c < 0) c = 0;
  if (c >= nc) c = nc - 1;
  return c;
}

int err_bits_to_code(int bits) {
  if (bits & ERRB_CELL_OVERFLOW) return CR_ERR_CELL_OVERFLOW;
  if (bits & ERRB_CAPACITY) return CR_ERR_CAPACITY;
  if (bits & ERRB_BOND) return CR_ERR_BOND_BROKEN;
  if (bits & ERRB_TIMEOUT) return CR_ERR_TIMEOUT;
  if (bits & ERRB_ARG) return CR_ERR_INVALID_ARG;
  if (bits & ERRB_NOT_NEUTRAL) return CR_ERR_NOT_NEUTRAL;
  return CR_OK;
}

}  // namespace

extern "C" const char *cr_strerror(int code) {
  switch (code) {
    case CR_OK: return "ok";
    case CR_ERR_INVALID_ARG: return "invalid argument or inconsistent system";
    case CR_ERR_NOT_NEUTRAL: return "system is not charge neutral";
    case CR_ERR_CELL_OVERFLOW: return "a cell exceeded its slot capacity";
    case CR_ERR_CAPACITY: return "particle capacity exhausted";
    case CR_ERR_TIMEOUT: return "a bounded device wait gave up";
    case CR_ERR_BOND_BROKEN: return "a FENE bond reached its maximum extension";
    case CR_ERR_CUDA: return "CUDA runtime error";
    case CR_ERR_NOMEM: return "out of memory";
    case CR_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown error";
  }
}

static void free_ctx(cr_ctx *c) {
  if (!c) return;
  if (c->bound) {  // the caller's buffers stay with the caller
    c->d_cnt = nullptr;
    c->d_pos = nullptr;
    c->d_vel = nullptr;
    c->d_pid = nullptr;
    c->d_info = nullptr;
  }
  void *ptrs[] = {c->d_cnt, c->d_cnt2, c->d_info, c->d_info2, c->d_pos, c->d_pos2, c->d_vel, c->d_vel2,
                  c->d_frc, c->d_frc2, c->d_fcons, c->d_pid, c->d_pid2, c->d_stats, c->d_lnK, c->d_lntab,
                  c->d_counts, c->d_perm, c->d_bond_off, c->d_bond_nbr, c->d_log,
                  c->d_in_xyz, c->d_in_vel, c->d_init_type, c->d_in_type, c->d_in_cls, c->d_site_map, c->d_in_state,
                  c->d_in_id, c->d_in_frc, c->d_present, c->d_ion_key, c->d_ion_key2, c->d_ion_val, c->d_ion_val2, c->d_ion_rank, c->d_sort_tmp,
                  c->d_out_xyz, c->d_out_vel, c->d_out_frc, c->d_out_id, c->d_out_type, c->d_out_cls,
                  c->d_out_state, c->d_out_site,
                  c->d_reps, c->d_gs_pos, c->d_gs_vel, c->d_gs_id, c->d_gs_lnk, c->d_gs_info, c->d_gs_rank,
                  c->d_plist, c->d_nparts, c->d_fsum, c->d_mlp_w, c->d_mlp_b, c->d_dlog, c->d_feat, c->d_order,
                  c->d_ek_nA, c->d_ek_Shi, c->d_ek_Slo, c->d_ek_list, c->d_ek_np,
                  c->d_bodies, c->d_body_member, c->d_body_d, c->d_body_df, c->d_body_newpos};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_small) cudaFreeHost(c->h_small);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

// CUDA-event timing of the two main kernels (kind 0: colour phase, 1: MD forces).
// Under stream capture a record is external, so that it becomes an
// event-record node of the graph, read after each of its launches.
static void trecord(cr_ctx *c, cudaEvent_t e) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(e, c->stream);
}
static void tbegin(cr_ctx *c, int kind, int *idx) {
  *idx = -1;
  if (!c->timing) return;
  while (c->ev_pool.size() < c->ev_next + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->ev_pool.push_back(e);
  }
  *idx = (int)c->ev_next;
  c->ev_next += 2;
  trecord(c, c->ev_pool[*idx]);
  (void)kind;
}
static void tend(cr_ctx *c, int kind, int idx) {
  if (idx < 0) return;
  trecord(c, c->ev_pool[idx + 1]);
  c->ev_pairs[kind].push_back({idx, idx + 1});
}
static void tcollect(cr_ctx *c) {
  for (int k = 0; k < 2; ++k) {
    for (auto &pr : c->ev_pairs[k]) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, c->ev_pool[pr.first], c->ev_pool[pr.second]) == cudaSuccess) c->ms[k] += ms;
      c->launches[k]++;
    }
    c->ev_pairs[k].clear();
  }
  c->ev_next = c->ev_reserved;
}

extern "C" void cr_destroy(cr_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

// Lay n particles (input order = id order) into cell-major host arrays.
struct Layout {
  std::vector<int> cnt, perm;
  std::vector<float4> pos, vel;
  std::vector<unsigned long long> pid;
  std::vector<int> info;
  long long kinds[K_OTHER + 1] = {};
  int max_occ = 0;
};

static int layout_particles(const SysParams &P, int n, const float *xyz, const float *vel, const int32_t *type,
                            const int32_t *cls, const int8_t *state, const std::vector<int> &site_of, int cap,
                            int n_perm, Layout &Lo) {
  const int nc = P.nc;
  std::vector<int> cell(n);
  Lo.cnt.assign(P.ncell, 0);
  for (int i = 0; i < n; ++i) {
    const int cx = cell_of_host(xyz[3 * i], P.scf, nc), cy = cell_of_host(xyz[3 * i + 1], P.scf, nc),
              cz = cell_of_host(xyz[3 * i + 2], P.scf, nc);
    cell[i] = cx + nc * (cy + nc * cz);
    Lo.cnt[cell[i]]++;
  }
  Lo.max_occ = n > 0 ? *std::max_element(Lo.cnt.begin(), Lo.cnt.end()) : 0;
  if (cap <= 0) return CR_OK;  // occupancy only
  if (Lo.max_occ > cap) return CR_ERR_CELL_OVERFLOW;
  const size_t nslot = (size_t)P.ncell * cap;
  std::fill(Lo.cnt.begin(), Lo.cnt.end(), 0);
  Lo.pos.assign(nslot, make_float4(0, 0, 0, 0));
  Lo.vel.assign(nslot, make_float4(0, 0, 0, 0));
  Lo.pid.assign(nslot, 0ull);
  Lo.info.assign(nslot, 0);
  Lo.perm.assign(std::max(n_perm, 1), -1);
  for (int i = 0; i < n; ++i) {  // ascending i == ascending id within every cell
    const int cc = cell[i];
    const int g = cc * cap + Lo.cnt[cc]++;
    const int t = type[i];
    const int ion = (t == CR_ACID || t == CR_BASE) && state[i] ? 1 : 0;
    float q = 0.0f;
    int cl = cls[i];
    if (t == CR_ACID) q = ion ? -1.0f : 0.0f;
    else if (t == CR_BASE) q = ion ? 1.0f : 0.0f;
    else if (is_ion_type(t)) { q = (float)ion_sign(t) * P.ion_q; cl = P.ion_cls; }
    Lo.pos[g] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], q);
    if (vel) Lo.vel[g] = make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], 0.0f);
    Lo.pid[g] = (unsigned long long)i;
    const int site = site_of[i] < 0 ? 0 : site_of[i];
    Lo.info[g] = t | (cl << INFO_CLS_SHIFT) | (ion ? INFO_ION_BIT : 0) | (site << INFO_SITE_SHIFT);
    if (i < n_perm) Lo.perm[i] = g;
    int kd = K_OTHER;
    if (t == CR_ACID) kd = ion ? K_A1 : K_A0;
    else if (t == CR_BASE) kd = ion ? K_B1 : K_B0;
    else if (t == CR_XP) kd = K_XP;
    else if (t == CR_XM) kd = K_XM;
    else if (t == CR_SP) kd = K_SP;
    else if (t == CR_SM) kd = K_SM;
    Lo.kinds[kd]++;
  }
  return CR_OK;
}

extern "C" int cr_init(cr_ctx **out, const cr_system *sys, double pH, const double *pK, cr_mu_ions mu, double lB,
                       double rc) {
  if (!out || !sys) return CR_ERR_INVALID_ARG;
  *out = nullptr;
  const int n = sys->n;
  if (n < 0 || sys->capacity < n || !(sys->box_L > 0.0) || !(rc > 0.0) || !(lB >= 0.0) || !(sys->sigma_nm > 0.0))
    return CR_ERR_INVALID_ARG;
  if (n > 0 && (!sys->xyz || !sys->type || !sys->cls || !sys->state || !pK)) return CR_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return CR_ERR_NO_DEVICE;

  cr_ctx *c = new (std::nothrow) cr_ctx();
  if (!c) return CR_ERR_NOMEM;
  cudaGetDevice(&c->device);
  SysParams &P = c->P;

  // ---- geometry (cell side >= rc/h, domains of k^3 cells with k*a >= rc)
  const float Lf = (float)sys->box_L;
  const double L = (double)Lf;
  if (2.0 * rc > L) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  const int h = sys->cells_per_rc > 0 ? sys->cells_per_rc : 2;
  int nc = sys->nc > 0 ? sys->nc : (int)std::floor(h * L / rc);
  if (nc < 1) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  const bool global = sys->schedule == CR_SCHED_GLOBAL;
  int k;
  if (global) {
    k = nc;
    if ((long long)nc * nc * nc > 8192) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  } else {
    k = sys->domain_cells > 0 ? sys->domain_cells : h;
    if (sys->nc <= 0) nc = (nc / (2 * k)) * (2 * k);
    if (nc < 2 * k || nc % (2 * k) != 0) { free_ctx(c); return CR_ERR_INVALID_ARG; }
    if ((double)k * (L / nc) < rc) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  }
  const double a = L / nc;
  if (a * h < rc) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  P.nc = nc;
  P.k = k;
  P.h = h;
  P.nd = global ? 1 : nc / k;
  P.ncol = global ? 1 : 8;
  P.m = sys->trials_per_domain > 0 ? sys->trials_per_domain : 1;
  P.global = global ? 1 : 0;
  P.nr = std::min(k + 2 * h, nc);
  P.ncell = nc * nc * nc;
  P.Lf = Lf;
  P.invL = (float)(1.0 / L);
  P.halfL = (float)(0.5 * L);
  P.Ld = L;
  P.halfLd = 0.5 * L;
  P.scf = (float)((double)nc / L);
  P.a = a;
  P.af = (float)(L / nc);
  c->per_sweep = (int64_t)P.nd * P.nd * P.nd * P.m;

  // ---- energy constants (FP64 -> FP32)
  const double alpha = sys->dsf_alpha;
  const double erc = std::erfc(alpha * rc);
  P.rc2 = (float)(rc * rc);
  P.rcf = (float)rc;
  P.alpha = (float)alpha;
  P.c1 = (float)(erc / rc);
  P.c2 = (float)(erc / (rc * rc) + 2.0 * alpha / std::sqrt(M_PI) * std::exp(-alpha * alpha * rc * rc) / rc);
  P.lBf = (float)lB;
  P.lB_self = sys->dsf_self ? lB * (-(erc / (2.0 * rc) + alpha / std::sqrt(M_PI))) : 0.0;
  // Ewald electrostatics (global schedule only): the real-space term without
  // the DSF shift, the Ewald self term, the reciprocal vectors and weights
  std::vector<int2> ek_nA;
  if (sys->ewald_kmax < 0 || sys->ewald_kmax > 32) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  if (sys->ewald_kmax > 0) {
    if (!global) { free_ctx(c); return CR_ERR_INVALID_ARG; }
    P.c1 = 0.0f;
    P.c2 = 0.0f;
    P.lB_self = lB * (-alpha / std::sqrt(M_PI));
    const int km = sys->ewald_kmax;
    const double V = L * L * L, kf = 2.0 * M_PI / L;
    for (int nz = -km; nz <= km; ++nz)
      for (int ny = -km; ny <= km; ++ny)
        for (int nx = -km; nx <= km; ++nx) {
          const int n2 = nx * nx + ny * ny + nz * nz;
          if (!(n2 > 0 && n2 <= km * km)) continue;
          // one half space: -k contributes the same term (S(-k) = conj S(k))
          if (!(nx > 0 || (nx == 0 && (ny > 0 || (ny == 0 && nz > 0))))) continue;
          const double k2 = kf * kf * n2;
          const float A = (float)(2.0 * 2.0 * M_PI * lB / V * std::exp(-k2 / (4.0 * alpha * alpha)) / k2);
          int Ab;
          std::memcpy(&Ab, &A, sizeof Ab);
          ek_nA.push_back(make_int2((nx & 255) | ((ny & 255) << 8) | ((nz & 255) << 16), Ab));
        }
  }
  P.ewald_kmax = sys->ewald_kmax;
  P.ewald_nk = (int)ek_nA.size();
  P.invLd = 1.0 / L;
  for (int i = 0; i < 4; ++i)  // a pair potential: the class-pair table is symmetric
    for (int j = 0; j < i; ++j)
      if (sys->wca_eps[4 * i + j] != sys->wca_eps[4 * j + i] || sys->wca_sig[4 * i + j] != sys->wca_sig[4 * j + i] ||
          sys->wca_del[4 * i + j] != sys->wca_del[4 * j + i] || (sys->wca_on[4 * i + j] != 0) != (sys->wca_on[4 * j + i] != 0)) {
        free_ctx(c);
        return CR_ERR_INVALID_ARG;
      }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      WcaEntry &w = P.wca[4 * i + j];
      w.eps = (float)sys->wca_eps[4 * i + j];
      w.sig = (float)sys->wca_sig[4 * i + j];
      w.del = (float)sys->wca_del[4 * i + j];
      const double cut = sys->wca_del[4 * i + j] + std::pow(2.0, 1.0 / 6.0) * sys->wca_sig[4 * i + j];
      w.wcut2 = (float)(cut * cut);
      w.eps_d = sys->wca_eps[4 * i + j];
      w.sig_d = sys->wca_sig[4 * i + j];
      w.del_d = sys->wca_del[4 * i + j];
      w.wcut_d = cut;
      w.on = (i != CR_CLS_NONE && j != CR_CLS_NONE && sys->wca_on[4 * i + j]) ? 1 : 0;
    }
  if (sys->ion_cls < 0 || sys->ion_cls > 3) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  P.ion_cls = sys->ion_coupling ? sys->ion_cls : CR_CLS_NONE;
  P.ion_q = sys->ion_coupling ? 1.0f : 0.0f;

  // ---- chemistry (log form), Eq. (pIXgen) and the acceptance rules
  const double pOH = mu.pKw - pH;
  double pIXp, pIXm;
  if (mu.pIX_explicit) { pIXp = mu.pIX_plus; pIXm = mu.pIX_minus; }
  else { pIXp = pIX_of(mu.pI_S_plus, pH, pOH); pIXm = pIX_of(mu.pI_S_minus, pH, pOH); }
  const double D = global ? L : k * a;
  const double ln_z1 = std::log(RHO0_NA * std::pow(D * sys->sigma_nm, 3.0));
  const double ln_salt = -LN10 * (pIXp + pIXm);
  P.lnz1_fx = to_lnfix(ln_z1);
  P.lnsalt_fx = to_lnfix(ln_salt);
  P.lBself_fx = to_lnfix(P.lB_self);
  c->pH = pH;
  c->mu = mu;
  c->pIXp = pIXp;
  c->pIXm = pIXm;

  // ---- particles: validate, classify, sort into cells
  std::vector<int> site_of(n, -1);
  std::vector<double> lnK;
  int nA = 0, nB = 0, qsum = 0;
  for (int i = 0; i < n; ++i) {
    const float X = sys->xyz[3 * i], Y = sys->xyz[3 * i + 1], Z = sys->xyz[3 * i + 2];
    if (!(X >= 0.0f && X < Lf && Y >= 0.0f && Y < Lf && Z >= 0.0f && Z < Lf)) { free_ctx(c); return CR_ERR_INVALID_ARG; }
    const int t = sys->type[i];
    if (t < CR_BEAD || t > CR_SM || sys->cls[i] < 0 || sys->cls[i] > 3) { free_ctx(c); return CR_ERR_INVALID_ARG; }
    if (t == CR_ACID || t == CR_BASE) {
      site_of[i] = (int)lnK.size();
      c->site_pK.push_back(pK[i]);
      c->site_is_acid.push_back(t == CR_ACID ? 1 : 0);
      if (t == CR_ACID) { lnK.push_back(LN10 * ((pH - pK[i]) - pIXp)); nA++; }
      else { lnK.push_back(LN10 * ((pOH - pK[i]) - pIXm)); nB++; }
      const int ion = sys->state[i] ? 1 : 0;
      qsum += ion ? (t == CR_ACID ? -1 : 1) : 0;
    } else if (is_ion_type(t)) qsum += ion_sign(t);
  }
  if ((int)lnK.size() >= MAX_SITES) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  if (qsum != 0) { free_ctx(c); return CR_ERR_NOT_NEUTRAL; }
  P.n_react = 0;
  if (nA > 0) P.react[P.n_react++] = R_ACID;
  if (nB > 0) P.react[P.n_react++] = R_BASE;
  P.react[P.n_react++] = R_SALT;
  P.kxp = K_XP;
  P.kxm = K_XM;
  P.txp = CR_XP;
  P.txm = CR_XM;
  c->n_acid = nA;
  c->n_base = nB;
  c->n_input = n;
  c->n_sites = (int)lnK.size();
  c->capacity = sys->capacity;

  Layout Lo;
  layout_particles(P, n, sys->xyz, sys->vel, sys->type, sys->cls, sys->state, site_of, 0, n, Lo);
  const int max_occ = Lo.max_occ;
  int cap = sys->cell_capacity > 0 ? sys->cell_capacity : std::max(32, ((2 * max_occ + 16) + 7) / 8 * 8);
  if (max_occ > cap) { free_ctx(c); return CR_ERR_CELL_OVERFLOW; }
  P.cap = cap;
  const size_t nslot = (size_t)P.ncell * cap;
  std::vector<int> occ = Lo.cnt;
  layout_particles(P, n, sys->xyz, sys->vel, sys->type, sys->cls, sys->state, site_of, cap, n, Lo);
  std::vector<int> &h_cnt = Lo.cnt, &h_info = Lo.info, &h_perm = Lo.perm;
  std::vector<float4> &h_pos = Lo.pos, &h_vel = Lo.vel;
  std::vector<unsigned long long> &h_pid = Lo.pid;
  long long *kinds = Lo.kinds;
  c->init_type.assign(sys->type, sys->type + n);
  c->init_site = site_of;
  for (int i = 0; i < n; ++i)
    if (!is_ion_type(sys->type[i])) c->n_fixed_end = i + 1;
  c->n_other = (int)kinds[K_OTHER];

  // ---- bonds (CSR by permanent particle)
  const int nb = sys->n_bonds;
  if (nb < 0 || (nb > 0 && !sys->bonds)) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  std::vector<int> deg(n + 1, 0);
  for (int b = 0; b < nb; ++b) {
    const int i = sys->bonds[2 * b], j = sys->bonds[2 * b + 1];
    if (i < 0 || j < 0 || i >= n || j >= n || i == j) { free_ctx(c); return CR_ERR_INVALID_ARG; }
    const int ti = sys->type[i], tj = sys->type[j];
    if (is_ion_type(ti) || is_ion_type(tj)) { free_ctx(c); return CR_ERR_INVALID_ARG; }
    deg[i + 1]++;
    deg[j + 1]++;
  }
  std::partial_sum(deg.begin(), deg.end(), deg.begin());
  std::vector<int> nbr(std::max(2 * nb, 1)), fill(deg.begin(), deg.end() - 1);
  for (int b = 0; b < nb; ++b) {
    const int i = sys->bonds[2 * b], j = sys->bonds[2 * b + 1];
    nbr[fill[i]++] = j;
    nbr[fill[j]++] = i;
  }
  c->fene_K = sys->fene_K;
  c->fene_R0 = sys->fene_R0;
  if (nb > 0 && !(sys->fene_R0 > 0.0)) { free_ctx(c); return CR_ERR_INVALID_ARG; }

  // ---- launch shape: one CTA per active domain; the domain list of the
  // densest domain (plus room for the phase's insertions) sized for shared
  // memory, the halo of the densest region for registers
  P.nact = global ? 1 : (P.nd / 2) * (P.nd / 2) * (P.nd / 2);
  P.dcap_glob = k * k * k * cap + 2 * P.m;
  int maxd = 0, maxh = 0;
  std::vector<int> dsums, hsums;
  {
    const int nr = P.nr;
    auto rc_ = [&](int i, int o) {
      int cc = (i < k + h) ? o + i : o + i - nr;
      cc %= nc;
      if (cc < 0) cc += nc;
      return cc;
    };
    const int norg = global ? 1 : nc;
    for (int oz = 0; oz < norg; ++oz)
      for (int oy = 0; oy < norg; ++oy)
        for (int ox = 0; ox < norg; ++ox) {
          int dsum = 0, hsum = 0;
          for (int iz = 0; iz < nr; ++iz)
            for (int iy = 0; iy < nr; ++iy)
              for (int ix = 0; ix < nr; ++ix) {
                const int cnt = occ[rc_(ix, ox) + nc * (rc_(iy, oy) + nc * rc_(iz, oz))];
                if (ix < k && iy < k && iz < k) dsum += cnt;
                else hsum += cnt;
              }
          maxd = std::max(maxd, dsum);
          maxh = std::max(maxh, hsum);
          dsums.push_back(dsum);
          hsums.push_back(hsum);
        }
  }
  {
    // starting shape before tuning: 128 threads, enough registers for the densest halo
    c->T = 128;
    c->R = 0;  // halo in shared memory until the tuner has timed the shapes
    c->tuning = std::getenv("CRMC_NO_TUNE") == nullptr;
    c->da_tuning = c->tuning;
  }
  P.lnmax = std::max(2 * k * k * k * cap, (int)std::min<long long>((long long)sys->capacity, 1 << 20)) + 2 * P.m + 4;
  std::vector<long long> h_lntab(P.lnmax);
  h_lntab[0] = LLONG_MIN / 4;  // never used: counts in a ratio are >= 1
  for (int i = 1; i < P.lnmax; ++i) h_lntab[i] = to_lnfix(std::log((double)i));
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  PhaseShape &S = c->S;
  S.nr3 = P.nr * P.nr * P.nr;
  S.kc3 = k * k * k;
  S.chunk = std::min(P.m, TRIAL_CHUNK);
  S.ewk = P.ewald_nk > 0 ? P.ewald_kmax + 1 : 0;
  // Shared-memory list and halo capacities: the densest domain of the
  // starting configuration with room for growth, and its densest halo.  The
  // compact set (Sc) is sized for the 90th percentile instead, so that more
  // CTAs fit on an SM; denser domains then keep their list in a global
  // scratch region and read the halo beyond the capacity from global memory.
  // The tuner times shapes with either set.  list_capacity / halo_capacity > 0
  // fix the capacities (both sets).
  S.dcs = sys->list_capacity > 0 ? sys->list_capacity + 2 * P.m : std::max(2 * maxd, maxd + 32) + 2 * P.m;
  S.dcs = std::min(P.dcap_glob, S.dcs);
  S.hcs = sys->halo_capacity > 0 ? sys->halo_capacity : std::min(maxh + maxh / 4 + 32, 4096);
  S.lns = std::min(P.lnmax, S.dcs + 4);
  while (phase_smem_bytes(S, 512, false) > (size_t)smem_max / 2 && S.dcs > 64) {
    S.dcs /= 2;
    S.hcs = std::max(S.hcs / 2, 64);
    S.lns = std::min(P.lnmax, S.dcs + 4);
  }
  if (phase_smem_bytes(S, 512, false) > (size_t)smem_max) { free_ctx(c); return CR_ERR_INVALID_ARG; }
  {
    auto pct90 = [](std::vector<int> v) {
      if (v.empty()) return 0;
      std::sort(v.begin(), v.end());
      return v[(size_t)(0.9 * (double)(v.size() - 1))];
    };
    PhaseShape &Q = c->Sc;
    Q = S;
    if (sys->list_capacity <= 0 && sys->halo_capacity <= 0) {
      const int pd = pct90(dsums), ph = pct90(hsums);
      Q.dcs = std::min(S.dcs, std::max(32, (3 * pd) / 2 + 16) + 2 * P.m);
      Q.hcs = std::min(S.hcs, ph + ph / 4 + 32);
      Q.lns = std::min(P.lnmax, Q.dcs + 4);
    }
  }
  c->smem_max = smem_max;
  P.per_sweep = c->per_sweep;
  P.key_xor = 0u;

  // ---- device buffers
  int rc_ = CR_OK;
#define ALLOC(p, n_)                      \
  if ((rc_ = dalloc(&(p), (n_))) != CR_OK) { \
    free_ctx(c);                          \
    return rc_;                           \
  }
  ALLOC(c->d_cnt, P.ncell);
  ALLOC(c->d_cnt2, P.ncell);
  ALLOC(c->d_pos, nslot);
  ALLOC(c->d_pos2, nslot);
  ALLOC(c->d_vel, nslot);
  ALLOC(c->d_vel2, nslot);
  ALLOC(c->d_frc, nslot);
  ALLOC(c->d_frc2, nslot);
  ALLOC(c->d_fcons, nslot);
  ALLOC(c->d_pid, nslot);
  ALLOC(c->d_pid2, nslot);
  ALLOC(c->d_info, nslot);
  ALLOC(c->d_info2, nslot);
  ALLOC(c->d_stats, 16);
  ALLOC(c->d_lnK, std::max<size_t>(lnK.size(), 1));
  ALLOC(c->d_lntab, P.lnmax);
  ALLOC(c->d_counts, N_KIND + 2);
  ALLOC(c->d_perm, std::max(n, 1));
  ALLOC(c->d_bond_off, n + 1);
  ALLOC(c->d_bond_nbr, std::max(2 * nb, 1));
  ALLOC(c->d_in_xyz, 3 * (size_t)sys->capacity);
  ALLOC(c->d_in_vel, 3 * (size_t)sys->capacity);
  ALLOC(c->d_in_type, (size_t)sys->capacity);
  ALLOC(c->d_in_cls, (size_t)sys->capacity);
  ALLOC(c->d_in_state, (size_t)sys->capacity);
  ALLOC(c->d_site_map, (size_t)std::max(n, 1));
  ALLOC(c->d_init_type, (size_t)std::max(n, 1));
  {
    const size_t cp = (size_t)std::max(sys->capacity, 1);
    ALLOC(c->d_present, (size_t)std::max(n, 1));
    ALLOC(c->d_ion_key, cp);
    ALLOC(c->d_ion_val, cp);
    ALLOC(c->d_ion_rank, cp);
    c->sort_tmp_bytes = state_sort_temp_bytes((int)cp);
    if (c->sort_tmp_bytes > 0) {  // ion lists beyond the tile ranking: device-wide sort
      ALLOC(c->d_ion_key2, cp);
      ALLOC(c->d_ion_val2, cp);
      ALLOC(c->d_sort_tmp, c->sort_tmp_bytes);
    }
    // low word of an inserted id: 2 (domain * trials per domain + trial) + 0/1;
    // ids from cr_load are indices below the capacity
    const unsigned long long lo_max =
        std::max<unsigned long long>(2ull * (unsigned long long)P.nd * P.nd * P.nd * (unsigned long long)P.m,
                                     (unsigned long long)cp);
    c->ion_lo_bits = 1;
    while (c->ion_lo_bits < 32 && (lo_max >> c->ion_lo_bits) != 0) ++c->ion_lo_bits;
    ALLOC(c->d_out_xyz, 3 * cp);
    ALLOC(c->d_out_vel, 3 * cp);
    ALLOC(c->d_out_frc, 3 * cp);
    ALLOC(c->d_out_id, cp);
    ALLOC(c->d_out_type, cp);
    ALLOC(c->d_out_cls, cp);
    ALLOC(c->d_out_state, cp);
    ALLOC(c->d_out_site, (size_t)std::max(c->n_sites, 1));
  }
  {
    // one region per (colour, active domain): a persistent batch sweep may run
    // domains of several colours of one replica at the same time
    const size_t ng = (size_t)P.ncol * P.nact * P.dcap_glob;
    ALLOC(c->d_gs_pos, ng);
    ALLOC(c->d_gs_vel, ng);
    ALLOC(c->d_gs_id, ng);
    ALLOC(c->d_gs_lnk, ng);
    ALLOC(c->d_gs_info, ng);
    ALLOC(c->d_gs_rank, ng);
  }
  ALLOC(c->d_reps, 1);
  ALLOC(c->d_plist, (size_t)std::max(sys->capacity, 1));
  ALLOC(c->d_nparts, 1);
  ALLOC(c->d_fsum, 3 * (size_t)P.ncell * (size_t)P.cap);  // per slot: both ends of each pair add to it
  if (P.ewald_nk > 0) {
    ALLOC(c->d_ek_nA, (size_t)P.ewald_nk);
    ALLOC(c->d_ek_Shi, (size_t)P.ewald_nk);
    ALLOC(c->d_ek_Slo, (size_t)P.ewald_nk);
    ALLOC(c->d_ek_list, (size_t)std::max(sys->capacity, 1));
    ALLOC(c->d_ek_np, 1);
  }
#undef ALLOC
  {
    if (cudaHostAlloc((void **)&c->h_small, 16 * sizeof(long long), 0) != cudaSuccess) {
      free_ctx(c);
      return CR_ERR_NOMEM;
    }
  }
#define COPY(dst, src, n_)                                                                           \
  if ((rc_ = cuda_fail(cudaMemcpy((dst), (src), (n_) * sizeof(*(src)), cudaMemcpyHostToDevice))) != CR_OK) { \
    free_ctx(c);                                                                                     \
    return rc_;                                                                                      \
  }
  COPY(c->d_cnt, h_cnt.data(), (size_t)P.ncell);
  COPY(c->d_pos, h_pos.data(), nslot);
  COPY(c->d_vel, h_vel.data(), nslot);
  COPY(c->d_pid, h_pid.data(), nslot);
  COPY(c->d_info, h_info.data(), nslot);
  std::vector<long long> lnK_fx(lnK.size());
  for (size_t i = 0; i < lnK.size(); ++i) lnK_fx[i] = to_lnfix(lnK[i]);
  if (!lnK.empty()) COPY(c->d_lnK, lnK_fx.data(), lnK_fx.size());
  COPY(c->d_lntab, h_lntab.data(), (size_t)P.lnmax);
  COPY(c->d_perm, h_perm.data(), (size_t)std::max(n, 1));
  COPY(c->d_bond_off, deg.data(), (size_t)n + 1);
  COPY(c->d_bond_nbr, nbr.data(), nbr.size());
  c->d_counter = (int *)(c->d_counts + N_KIND);
  c->d_err = (int *)(c->d_counts + N_KIND + 1);
  cudaMemset(c->d_counts, 0, sizeof(long long) * (N_KIND + 2));
  cudaMemset(c->d_present, 0, sizeof(int) * (size_t)std::max(n, 1));
  COPY(c->d_counts, kinds, (size_t)N_KIND);
  if (n > 0) COPY(c->d_site_map, site_of.data(), (size_t)n);
  if (n > 0) COPY(c->d_init_type, sys->type, (size_t)n);
  if (P.ewald_nk > 0) {
    COPY(c->d_ek_nA, ek_nA.data(), ek_nA.size());
  }
#undef COPY
  cudaMemset(c->d_cnt2, 0, sizeof(int) * P.ncell);
  cudaMemset(c->d_frc, 0, sizeof(float4) * nslot);
  cudaMemset(c->d_fcons, 0, sizeof(float4) * nslot);
  cudaMemset(c->d_stats, 0, sizeof(unsigned long long) * 16);
  P.lnK_fx = c->d_lnK;
  P.lntab_fx = c->d_lntab;
  P.cnt = c->d_cnt;
  P.pos = c->d_pos;
  P.vel = c->d_vel;
  P.pid = c->d_pid;
  P.info = c->d_info;
  P.perm_slot = c->d_perm;
  P.n_perm = n;
  P.stats = c->d_stats;
  P.counts = c->d_counts;
  P.err = c->d_err;
  P.log = nullptr;
  P.gs_pos = c->d_gs_pos;
  P.gs_vel = c->d_gs_vel;
  P.gs_id = c->d_gs_id;
  P.gs_lnk = c->d_gs_lnk;
  P.gs_info = c->d_gs_info;
  P.gs_rank = c->d_gs_rank;
  P.ek_nA = c->d_ek_nA;
  P.ek_Shi = c->d_ek_Shi;
  P.ek_Slo = c->d_ek_Slo;
  P.ek_list = c->d_ek_list;
  P.ek_np = c->d_ek_np;
  P.ek_cap = (int)std::max<int64_t>(sys->capacity, 1);
  P.order = nullptr;
  if (!global && P.nact <= ORDER_MAX_NACT) {
    // densest-first launch order, recomputed every sweep; starts as the identity
    std::vector<int> ident((size_t)P.ncol * P.nact);
    for (size_t i = 0; i < ident.size(); ++i) ident[i] = (int)(i % (size_t)P.nact);
    if (cudaMalloc((void **)&c->d_order, sizeof(int) * ident.size()) != cudaSuccess ||
        cudaMemcpy(c->d_order, ident.data(), sizeof(int) * ident.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_ctx(c);
      return CR_ERR_NOMEM;
    }
    P.order = c->d_order;
  }
  if (cudaMemcpy(c->d_reps, &P, sizeof(SysParams), cudaMemcpyHostToDevice) != cudaSuccess) {
    free_ctx(c);
    return CR_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { free_ctx(c); return CR_ERR_CUDA; }
  *out = c;
  return CR_OK;
}

// the chemistry of the following trials: K_A, K_B per site and K_ion from
// pH and the pI of the exchanged cation and anion, in stream order
static int apply_chem(cr_ctx *ctx, double pH, double pIXp, double pIXm) {
  const double pOH = ctx->mu.pKw - pH;
  const size_t ns = ctx->site_pK.size();
  ctx->h_lnK_fx.resize(ns);
  for (size_t i = 0; i < ns; ++i)
    ctx->h_lnK_fx[i] = to_lnfix(ctx->site_is_acid[i] ? LN10 * ((pH - ctx->site_pK[i]) - pIXp)
                                                     : LN10 * ((pOH - ctx->site_pK[i]) - pIXm));
  // in stream order: the trials queued before this call keep the old constants
  if (ns) CR_CUDA(cudaMemcpyAsync(ctx->d_lnK, ctx->h_lnK_fx.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice,
                                  ctx->stream));
  ctx->P.lnsalt_fx = to_lnfix(-LN10 * (pIXp + pIXm));
  CR_CUDA(cudaMemcpyAsync(ctx->d_reps, &ctx->P, sizeof(SysParams), cudaMemcpyHostToDevice, ctx->stream));
  CR_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->pH = pH;
  ctx->pIXp = pIXp;
  ctx->pIXm = pIXm;
  ctx->chem_version++;
  return CR_OK;
}

extern "C" int cr_set_pH(cr_ctx *ctx, double pH) {
  if (!ctx || !std::isfinite(pH)) return CR_ERR_INVALID_ARG;
  const cr_mu_ions &mu = ctx->mu;
  const double pOH = mu.pKw - pH;
  double pIXp, pIXm;
  if (ctx->inv_explicit) { pIXp = ctx->pIXp; pIXm = ctx->pIXm; }
  else if (mu.pIX_explicit) { pIXp = mu.pIX_plus; pIXm = mu.pIX_minus; }
  else { pIXp = pIX_of(mu.pI_S_plus, pH, pOH); pIXm = pIX_of(mu.pI_S_minus, pH, pOH); }
  return apply_chem(ctx, pH, pIXp, pIXm);
}

extern "C" int cr_set_invocation(cr_ctx *ctx, int32_t cation, int32_t anion, double pI_cation, double pI_anion,
                                 uint32_t reactions) {
  if (!ctx || (cation != CR_XP && cation != CR_SP) || (anion != CR_XM && anion != CR_SM)) return CR_ERR_INVALID_ARG;
  if (!std::isfinite(pI_cation) || !std::isfinite(pI_anion) || reactions == 0 || reactions > 7)
    return CR_ERR_INVALID_ARG;
  SysParams &P = ctx->P;
  int react[3], nr = 0;
  if ((reactions & 1u) && ctx->n_acid > 0) react[nr++] = R_ACID;
  if ((reactions & 2u) && ctx->n_base > 0) react[nr++] = R_BASE;
  if (reactions & 4u) react[nr++] = R_SALT;
  if (nr == 0) return CR_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i) P.react[i] = i < nr ? react[i] : 0;
  P.n_react = nr;
  P.txp = cation;
  P.txm = anion;
  P.kxp = cation == CR_XP ? K_XP : K_SP;
  P.kxm = anion == CR_XM ? K_XM : K_SM;
  ctx->inv_explicit = true;
  return apply_chem(ctx, ctx->pH, pI_cation, pI_anion);
}

extern "C" int cr_ungroup(cr_ctx *ctx, cr_ungrouped *out) {
  if (!ctx || !out) return CR_ERR_INVALID_ARG;
  const double pOH = ctx->mu.pKw - ctx->pH;
  out->p_S_plus = std::pow(10.0, -ctx->mu.pI_S_plus + ctx->pIXp);
  out->p_H = std::pow(10.0, -ctx->pH + ctx->pIXp);
  out->p_S_minus = std::pow(10.0, -ctx->mu.pI_S_minus + ctx->pIXm);
  out->p_OH = std::pow(10.0, -pOH + ctx->pIXm);
  cr_state_view v{};
  const int rc = cr_state(ctx, &v);
  if (rc != CR_OK) return rc;
  out->n_S_plus = out->p_S_plus * (double)v.n_Xp;
  out->n_H = out->p_H * (double)v.n_Xp;
  out->n_S_minus = out->p_S_minus * (double)v.n_Xm;
  out->n_OH = out->p_OH * (double)v.n_Xm;
  return CR_OK;
}

extern "C" int cr_set_stream(cr_ctx *ctx, void *stream) {
  if (!ctx) return CR_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return CR_OK;
}

extern "C" int cr_get_info(const cr_ctx *ctx, cr_info *out) {
  if (!ctx || !out) return CR_ERR_INVALID_ARG;
  const SysParams &P = ctx->P;
  out->nc = P.nc;
  out->k = P.k;
  out->h = P.h;
  out->nd = P.nd;
  out->ncol = P.ncol;
  out->m = P.m;
  out->cap = P.cap;
  out->global = P.global;
  out->trials_per_sweep = ctx->per_sweep;
  out->n_sites = ctx->n_sites;
  out->n_perm = ctx->n_input;
  out->cell_side = P.a;
  out->domain_side = P.global ? (double)P.Lf : P.k * P.a;
  return CR_OK;
}

// whether p is device memory of device dev
static bool device_memory_of(const void *p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

extern "C" int cr_bind_device_buffers(cr_ctx *ctx, const cr_device_buffers *b) {
  if (!ctx || !b || !b->cnt || !b->pos || !b->vel || !b->id || !b->info) return CR_ERR_INVALID_ARG;
  if (ctx->bound || ctx->batch_refs > 0) return CR_ERR_INVALID_ARG;
  const int64_t ncell = ctx->P.ncell, nslot = (int64_t)ctx->P.ncell * ctx->P.cap;
  if (b->n_cells < ncell || b->n_slots < nslot) return CR_ERR_INVALID_ARG;
  const uintptr_t a4 = (uintptr_t)b->cnt | (uintptr_t)b->info, a8 = (uintptr_t)b->id,
                  a16 = (uintptr_t)b->pos | (uintptr_t)b->vel;
  if ((a4 & 3u) || (a8 & 7u) || (a16 & 15u)) return CR_ERR_INVALID_ARG;
  const void *ps[] = {b->cnt, b->pos, b->vel, b->id, b->info};
  for (const void *p : ps)
    if (!device_memory_of(p, ctx->device)) return CR_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  CR_CUDA(cudaMemcpyAsync(b->cnt, ctx->d_cnt, sizeof(int) * (size_t)ncell, cudaMemcpyDeviceToDevice, s));
  CR_CUDA(cudaMemcpyAsync(b->pos, ctx->d_pos, sizeof(float4) * (size_t)nslot, cudaMemcpyDeviceToDevice, s));
  CR_CUDA(cudaMemcpyAsync(b->vel, ctx->d_vel, sizeof(float4) * (size_t)nslot, cudaMemcpyDeviceToDevice, s));
  CR_CUDA(cudaMemcpyAsync(b->id, ctx->d_pid, sizeof(unsigned long long) * (size_t)nslot, cudaMemcpyDeviceToDevice, s));
  CR_CUDA(cudaMemcpyAsync(b->info, ctx->d_info, sizeof(int) * (size_t)nslot, cudaMemcpyDeviceToDevice, s));
  CR_CUDA(cudaStreamSynchronize(s));
  void *old[] = {ctx->d_cnt, ctx->d_pos, ctx->d_vel, ctx->d_pid, ctx->d_info};
  for (void *p : old) cudaFree(p);
  ctx->d_cnt = b->cnt;
  ctx->d_pos = reinterpret_cast<float4 *>(b->pos);
  ctx->d_vel = reinterpret_cast<float4 *>(b->vel);
  ctx->d_pid = reinterpret_cast<unsigned long long *>(b->id);
  ctx->d_info = b->info;
  ctx->bound = true;
  SysParams &P = ctx->P;
  P.cnt = ctx->d_cnt;
  P.pos = ctx->d_pos;
  P.vel = ctx->d_vel;
  P.pid = ctx->d_pid;
  P.info = ctx->d_info;
  CR_CUDA(cudaMemcpyAsync(ctx->d_reps, &P, sizeof(SysParams), cudaMemcpyHostToDevice, s));
  CR_CUDA(cudaStreamSynchronize(s));
  return cr_check(ctx);
}

extern "C" int cr_check(cr_ctx *ctx) {
  if (!ctx) return CR_ERR_INVALID_ARG;
  int *bits = (int *)(ctx->h_small + N_KIND + 1);  // pinned
  CR_CUDA(cudaMemcpyAsync(bits, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CR_CUDA(cudaStreamSynchronize(ctx->stream));
  return err_bits_to_code(*bits);
}

// grow a device record buffer to n entries (records of logged calls only)
template <typename TT>
static int grow(TT **p, size_t *cap, size_t n) {
  if (*cap >= n) return CR_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  CR_CUDA(cudaMalloc((void **)p, sizeof(TT) * n));
  *cap = n;
  return CR_OK;
}

// Online launch-shape tuning (shared by plain and delayed-acceptance sweeps):
// the first sweeps of unlogged calls time each shape of the set (shapes whose
// shared memory does not fit are skipped) in TUNE_ROUNDS round-robin passes,
// and the shape with the shortest of its times is kept: a single pass was
// swayed by one slow sweep and by the state's drift while the chain starts.
// For batches whose persistent mode is left to the tuner (pers != null), the
// candidates are every shape with one launch per colour, then every shape as
// a persistent sweep; *pers receives the chosen mode.  next counts the timed
// sweeps; candidate next % tune_count.
constexpr int TUNE_ROUNDS = 2;

struct TuneRef {
  int &T, &R, &next;
  bool &on;
  float *ms;
  bool &C;  // the chosen shape uses the compact capacities
  bool *pers = nullptr;
};

static int tune_count(const TuneRef &t, bool da) { return phase_shape_count(da) * (t.pers ? 2 : 1); }
static int tune_total(const TuneRef &t, bool da) { return tune_count(t, da) * TUNE_ROUNDS; }
static int tune_cand(const TuneRef &t, bool da) { return t.next % tune_count(t, da); }

static void tune_skip(TuneRef t, const PhaseShape &S, const PhaseShape &Sc, int smem_max, bool da) {
  const int nshape = phase_shape_count(da);
  while (t.on && t.next < tune_total(t, da)) {
    const int c = tune_cand(t, da);
    int t_, r_;
    phase_shape(c % nshape, &t_, &r_, da);
    const PhaseShape &Q = phase_shape_compact(c % nshape, da) ? Sc : S;
    if (phase_shape_smem(Q, t_, r_, da) <= (size_t)smem_max) break;
    t.ms[c] = 1e30f;
    t.next++;
  }
}

static void tune_finish(TuneRef t, float ms, const PhaseShape &S, const PhaseShape &Sc, int smem_max, bool da) {
  const int c = tune_cand(t, da);
  t.ms[c] = t.next < tune_count(t, da) ? ms : std::min(t.ms[c], ms);
  t.next++;
  tune_skip(t, S, Sc, smem_max, da);
  const int nshape = phase_shape_count(da);
  if (t.next == tune_total(t, da)) {
    int best = 0;
    for (int i = 1; i < tune_count(t, da); ++i)
      if (t.ms[i] < t.ms[best]) best = i;
    phase_shape(best % nshape, &t.T, &t.R, da);
    t.C = phase_shape_compact(best % nshape, da);
    if (t.pers) *t.pers = best >= nshape;
    t.on = false;
  }
}

static int sweep_impl(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats, cr_trial *log,
                      bool da = false, cr_trial_da *dlog = nullptr, float *feat = nullptr) {
  if (!ctx) return CR_ERR_INVALID_ARG;
  if (n_trials == 0 || n_trials % (uint64_t)ctx->per_sweep != 0) return CR_ERR_INVALID_ARG;
  if (da && !ctx->has_mlp) return CR_ERR_INVALID_ARG;
  SysParams P = ctx->P;
  cudaStream_t s = ctx->stream;
  if (stats) CR_CUDA(cudaMemsetAsync(ctx->d_stats, 0, sizeof(unsigned long long) * 16, s));
  if (log) {
    int rc = grow(&ctx->d_log, &ctx->log_cap, n_trials);
    if (rc != CR_OK) return rc;
    P.log = ctx->d_log;
    if (da) {
      if ((rc = grow(&ctx->d_dlog, &ctx->dlog_cap, n_trials)) != CR_OK) return rc;
      P.dlog = ctx->d_dlog;
      if (feat) {
        if ((rc = grow(&ctx->d_feat, &ctx->feat_cap, n_trials * MLP_IN)) != CR_OK) return rc;
        P.feat_log = ctx->d_feat;
      }
    }
  }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  // the phase kernel reads the parameters from the device copy; the log
  // pointers are set there only for logged calls
  if (log) CR_CUDA(cudaMemcpyAsync(ctx->d_reps, &P, sizeof(SysParams), cudaMemcpyHostToDevice, s));
  const uint64_t n_sweeps = n_trials / (uint64_t)ctx->per_sweep;
  const uint32_t sweep0 = (uint32_t)ctx->sweep;
  TuneRef tr = da ? TuneRef{ctx->da_T, ctx->da_R, ctx->da_next, ctx->da_tuning, ctx->da_ms, ctx->da_C}
                  : TuneRef{ctx->T, ctx->R, ctx->tune_next, ctx->tuning, ctx->tune_ms, ctx->C};
  for (uint64_t sw = 0; sw < n_sweeps; ++sw) {
    const uint32_t swc = (uint32_t)ctx->sweep++;
    if (!log) tune_skip(tr, ctx->S, ctx->Sc, ctx->smem_max, da);
    const bool tune = tr.on && !log && tr.next < tune_total(tr, da);
    int T = tr.T, R = tr.R;
    const bool compact = tune ? phase_shape_compact(tune_cand(tr, da), da) : tr.C;
    const PhaseShape &SS = compact ? ctx->Sc : ctx->S;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (tune) {
      phase_shape(tune_cand(tr, da), &T, &R, da);
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
    }
    if (P.order) {
      CR_CUDA(launch_domain_order(ctx->d_reps, 1, P.ncol, P.nact, s, swc, k0, k1));
      ctx->launches_total++;
    }
    if (P.ewald_nk > 0) {  // S(k) from scratch at every sweep
      CR_CUDA(launch_ewald_sk(ctx->d_reps, 1, P.ewald_nk, s));
      ctx->launches_total += 2;
    }
    for (int col = 0; col < P.ncol; ++col) {
      int ti;
      tbegin(ctx, 0, &ti);
      CR_CUDA(launch_phase(ctx->d_reps, 1, P.nact, SS, T, R, log != nullptr, da, s, swc, sweep0, col, k0, k1));
      tend(ctx, 0, ti);
      ctx->launches_total++;
    }
    if (tune) {
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      tune_finish(tr, ms, ctx->S, ctx->Sc, ctx->smem_max, da);
    }
  }
  if (log) {
    SysParams Q = ctx->P;
    Q.log = nullptr;
    Q.dlog = nullptr;
    Q.feat_log = nullptr;
    CR_CUDA(cudaMemcpyAsync(ctx->d_reps, &Q, sizeof(SysParams), cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaStreamSynchronize(s));
  }
  ctx->f_valid = false;
  ctx->fcons_valid = false;
  if (log) {
    CR_CUDA(cudaMemcpyAsync(log, ctx->d_log, sizeof(cr_trial) * n_trials, cudaMemcpyDeviceToHost, s));
    if (da && dlog)
      CR_CUDA(cudaMemcpyAsync(dlog, ctx->d_dlog, sizeof(cr_trial_da) * n_trials, cudaMemcpyDeviceToHost, s));
    if (da && feat)
      CR_CUDA(cudaMemcpyAsync(feat, ctx->d_feat, sizeof(float) * MLP_IN * n_trials, cudaMemcpyDeviceToHost, s));
  }
  if (stats) {
    unsigned long long st[16];
    CR_CUDA(cudaMemcpyAsync(st, ctx->d_stats, sizeof(st), cudaMemcpyDeviceToHost, s));
    CR_CUDA(cudaStreamSynchronize(s));
    stats->trials = (int64_t)st[15];
    for (int i = 0; i < 6; ++i) {
      stats->attempts[i] = (int64_t)st[i];
      stats->accepts[i] = (int64_t)st[6 + i];
    }
    stats->no_eligible = (int64_t)st[12];
    stats->edge = (int64_t)st[13];
    stats->overlap = (int64_t)st[14];
  }
  if (log || stats) {
    CR_CUDA(cudaStreamSynchronize(s));
    return cr_check(ctx);
  }
  return CR_OK;
}

extern "C" int cr_sweep(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats) {
  return sweep_impl(ctx, n_trials, seed, stats, nullptr);
}

extern "C" int cr_sweep_log(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats, cr_trial *log) {
  if (!log) return CR_ERR_INVALID_ARG;
  return sweep_impl(ctx, n_trials, seed, stats, log);
}

extern "C" int cr_sweep_da(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats) {
  return sweep_impl(ctx, n_trials, seed, stats, nullptr, true);
}

extern "C" int cr_sweep_da_log(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats, cr_trial *log,
                               cr_trial_da *dlog, float *features) {
  if (!log || !dlog) return CR_ERR_INVALID_ARG;
  return sweep_impl(ctx, n_trials, seed, stats, log, true, dlog, features);
}

extern "C" int cr_set_surrogate(cr_ctx *ctx, const cr_mlp *m) {
  if (!ctx || !m || !m->W1 || !m->b1 || !m->W2 || !m->b2 || !m->W3 || !m->b3 || !m->w4) return CR_ERR_INVALID_ARG;
  if (ctx->P.ewald_nk > 0) return CR_ERR_INVALID_ARG;  // the surrogate's features are local
  const SysParams &P0 = ctx->P;
  // the features use the 5^3 stencil of half-cutoff cells inside the phase's region
  if (P0.global || P0.h != 2 || P0.nc < P0.k + 4 || !std::isfinite(m->b4)) return CR_ERR_INVALID_ARG;
  int smem_ok = 0;
  for (int i = 0; i < phase_shape_count(true); ++i) {
    int t, r;
    phase_shape(i, &t, &r, true);
    smem_ok |= phase_shape_smem(ctx->S, t, r, true) <= (size_t)ctx->smem_max;
  }
  if (!smem_ok) return CR_ERR_INVALID_ARG;
  // transposed BF16 weights (WT[in][out]) and the biases
  std::vector<uint16_t> w(MLPW_N);
  for (int o = 0; o < MLP_H; ++o) {
    for (int k = 0; k < MLP_IN; ++k) w[MLPW_W1 + k * MLP_H + o] = m->W1[o * MLP_IN + k];
    for (int k = 0; k < MLP_H; ++k) {
      w[MLPW_W2 + k * MLP_H + o] = m->W2[o * MLP_H + k];
      w[MLPW_W3 + k * MLP_H + o] = m->W3[o * MLP_H + k];
    }
    w[MLPW_W4 + o] = m->w4[o];
  }
  std::vector<float> b(MLPB_N);
  for (int o = 0; o < MLP_H; ++o) {
    b[o] = m->b1[o];
    b[MLP_H + o] = m->b2[o];
    b[2 * MLP_H + o] = m->b3[o];
  }
  b[3 * MLP_H] = m->b4;
  if (!ctx->d_mlp_w) CR_CUDA(cudaMalloc((void **)&ctx->d_mlp_w, sizeof(uint16_t) * MLPW_N));
  if (!ctx->d_mlp_b) CR_CUDA(cudaMalloc((void **)&ctx->d_mlp_b, sizeof(float) * MLPB_N));
  CR_CUDA(cudaMemcpyAsync(ctx->d_mlp_w, w.data(), sizeof(uint16_t) * MLPW_N, cudaMemcpyHostToDevice, ctx->stream));
  CR_CUDA(cudaMemcpyAsync(ctx->d_mlp_b, b.data(), sizeof(float) * MLPB_N, cudaMemcpyHostToDevice, ctx->stream));
  ctx->P.mlp_w = ctx->d_mlp_w;
  ctx->P.mlp_b = ctx->d_mlp_b;
  CR_CUDA(cudaMemcpyAsync(ctx->d_reps, &ctx->P, sizeof(SysParams), cudaMemcpyHostToDevice, ctx->stream));
  CR_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->has_mlp = true;
  return CR_OK;
}

static MdParams md_params(cr_ctx *ctx, int mode, double dt, double gamma, uint64_t seed) {
  MdParams M{};
  M.dt = (float)dt;
  M.gamma = (float)gamma;
  M.amp = dt > 0.0 ? (float)std::sqrt(2.0 * gamma / dt) : 0.0f;
  M.key0 = (uint32_t)seed;
  M.key1 = (uint32_t)(seed >> 32);
  M.eval = ctx->md_eval;
  M.mode = mode;
  M.vel = ctx->d_vel;
  M.fout = mode == 0 ? ctx->d_fcons : ctx->d_frc;
  M.perm_slot = ctx->d_perm;
  M.bond_off = ctx->d_bond_off;
  M.bond_nbr = ctx->d_bond_nbr;
  M.n_perm = ctx->n_input;
  M.fene_K = (float)ctx->fene_K;
  M.inv_R02 = (float)(1.0 / (ctx->fene_R0 * ctx->fene_R0));
  // the longest pair range (Coulomb cutoff or WCA cutoff), with a margin far
  // above the FP32 rounding of positions and cell boxes
  double reach2 = (double)ctx->P.rc2;
  for (int i = 0; i < 16; ++i)
    if (ctx->P.wca[i].on) reach2 = std::max(reach2, (double)ctx->P.wca[i].wcut2);
  const double reach = std::sqrt(reach2) * 1.001 + 1e-3;
  M.reach2 = (float)(reach * reach);
  M.n_bodies = ctx->n_bodies;
  M.bodies = ctx->d_bodies;
  M.body_member = ctx->d_body_member;
  M.body_d = ctx->d_body_d;
  M.body_df = ctx->d_body_df;
  M.body_newpos = ctx->d_body_newpos;
  M.body_dt = dt;
  M.body_gamma = gamma;
  return M;
}

static void free_bodies(cr_ctx *ctx) {
  void *ptrs[] = {ctx->d_bodies, ctx->d_body_member, ctx->d_body_d, ctx->d_body_df, ctx->d_body_newpos};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  ctx->d_bodies = nullptr;
  ctx->d_body_member = nullptr;
  ctx->d_body_d = nullptr;
  ctx->d_body_df = nullptr;
  ctx->d_body_newpos = nullptr;
  ctx->n_bodies = ctx->n_members = 0;
}

extern "C" int cr_set_rigid_bodies(cr_ctx *ctx, int32_t n_bodies, const int32_t *first, const int32_t *count) {
  if (!ctx || n_bodies < 0 || n_bodies > CR_MAX_BODIES || (n_bodies > 0 && (!first || !count)))
    return CR_ERR_INVALID_ARG;
  if (ctx->batch_refs > 0) return CR_ERR_INVALID_ARG;
  std::vector<int> member((size_t)std::max(ctx->n_input, 1), -1);
  std::vector<RigidBody> hb((size_t)n_bodies);
  int64_t nm = 0;
  for (int b = 0; b < n_bodies; ++b) {
    if (count[b] < 2 || first[b] < 0 || (int64_t)first[b] + count[b] > ctx->n_input) return CR_ERR_INVALID_ARG;
    for (int m = 0; m < count[b]; ++m) {
      if (member[first[b] + m] >= 0) return CR_ERR_INVALID_ARG;  // in two bodies
      member[first[b] + m] = (int)(nm + m);
    }
    hb[b] = RigidBody{};
    hb[b].first = first[b];
    hb[b].count = count[b];
    hb[b].mfirst = (int)nm;
    nm += count[b];
  }
  CR_CUDA(cudaStreamSynchronize(ctx->stream));
  if (n_bodies == 0) {
    free_bodies(ctx);
    ctx->f_valid = false;
    return CR_OK;
  }
  // the new arrays, adopted once every body is valid
  RigidBody *d_b = nullptr;
  int *d_m = nullptr;
  double *d_d = nullptr;
  float4 *d_f = nullptr, *d_n = nullptr;
  auto release = [&]() {
    void *ptrs[] = {d_b, d_m, d_d, d_f, d_n};
    for (void *p : ptrs)
      if (p) cudaFree(p);
  };
  cudaError_t e = cudaMalloc(&d_b, hb.size() * sizeof(RigidBody));
  if (e == cudaSuccess) e = cudaMalloc(&d_m, member.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_d, (size_t)nm * 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_f, (size_t)nm * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&d_n, (size_t)nm * sizeof(float4));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_b, hb.data(), hb.size() * sizeof(RigidBody), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_m, member.data(), member.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  MdParams M = md_params(ctx, 0, 0.0, 0.0, 0);
  M.n_bodies = n_bodies;
  M.bodies = d_b;
  M.body_member = d_m;
  M.body_d = d_d;
  M.body_df = d_f;
  M.body_newpos = d_n;
  if (e == cudaSuccess) e = launch_body_setup(ctx->P, M, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hb.data(), d_b, hb.size() * sizeof(RigidBody), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  bool bad = false;
  for (const RigidBody &b : hb) bad = bad || b.bad != 0;
  if (e == cudaSuccess && !bad) e = launch_body_member_velocities(ctx->P, M, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess || bad) {
    release();
    return e != cudaSuccess ? CR_ERR_CUDA : CR_ERR_INVALID_ARG;
  }
  free_bodies(ctx);
  ctx->n_bodies = n_bodies;
  ctx->n_members = (int)nm;
  ctx->d_bodies = d_b;
  ctx->d_body_member = d_m;
  ctx->d_body_d = d_d;
  ctx->d_body_df = d_f;
  ctx->d_body_newpos = d_n;
  ctx->f_valid = false;  // the next step evaluates the bodies' forces and torques
  ctx->launches_total += 2;
  return CR_OK;
}

extern "C" int cr_rigid_body_state(cr_ctx *ctx, int32_t n_bodies, double *out) {
  if (!ctx || n_bodies != ctx->n_bodies || (n_bodies > 0 && !out)) return CR_ERR_INVALID_ARG;
  if (n_bodies == 0) return CR_OK;
  std::vector<RigidBody> hb((size_t)n_bodies);
  CR_CUDA(cudaMemcpyAsync(hb.data(), ctx->d_bodies, hb.size() * sizeof(RigidBody), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CR_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int b = 0; b < n_bodies; ++b) {
    double *r = out + 22 * (size_t)b;
    std::memcpy(r, hb[b].X, 3 * sizeof(double));
    std::memcpy(r + 3, hb[b].V, 3 * sizeof(double));
    std::memcpy(r + 6, hb[b].R, 9 * sizeof(double));
    std::memcpy(r + 15, hb[b].pi, 3 * sizeof(double));
    std::memcpy(r + 18, hb[b].I, 3 * sizeof(double));
    r[21] = hb[b].M;
  }
  return CR_OK;
}

// one force evaluation
static int md_force_eval(cr_ctx *ctx, const MdParams &M) {
  int ti;
  tbegin(ctx, 1, &ti);
  MdParams Q = M;
  Q.fsum = ctx->d_fsum;
  if (ctx->P.ewald_nk > 0) {  // S(k) of the current positions for the reciprocal forces
    CR_CUDA(launch_ewald_sk(ctx->d_reps, 1, ctx->P.ewald_nk, ctx->stream));
    ctx->launches_total += 3;  // occupied slots, S(k), reciprocal forces
  }
  CR_CUDA(launch_md_forces(ctx->P, Q, ctx->d_plist, ctx->d_nparts, (int)ctx->capacity, ctx->stream));
  tend(ctx, 1, ti);
  ctx->launches_total += 3;  // particle list, pair forces, per-particle finish
  return CR_OK;
}

extern "C" int cr_md_forces(cr_ctx *ctx) {
  if (!ctx) return CR_ERR_INVALID_ARG;
  int rc = md_force_eval(ctx, md_params(ctx, 0, 0.0, 0.0, 0));
  if (rc != CR_OK) return rc;
  ctx->fcons_valid = true;
  return cr_check(ctx);
}

extern "C" int cr_md_step(cr_ctx *ctx, int32_t n_steps, double dt, double gamma, uint64_t seed) {
  if (!ctx || n_steps < 0 || !(dt > 0.0) || !(gamma >= 0.0)) return CR_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  const SysParams &P = ctx->P;
  RebuildBufs B{ctx->d_cnt2, ctx->d_pos2, ctx->d_pid2, ctx->d_info2, ctx->d_vel2, ctx->d_frc2, ctx->d_vel, ctx->d_frc};
  int rc;
  if (!ctx->f_valid) {
    if ((rc = md_force_eval(ctx, md_params(ctx, 1, dt, gamma, seed))) != CR_OK) return rc;
    ctx->md_eval++;
    ctx->f_valid = true;
  }
  for (int st = 0; st < n_steps; ++st) {
    MdParams M = md_params(ctx, 2, dt, gamma, seed);
    CR_CUDA(launch_kick_drift_rebuild(P, M, B, ctx->d_perm, ctx->n_input, s));
    ctx->launches_total += 2;
    if ((rc = md_force_eval(ctx, M)) != CR_OK) return rc;
    ctx->md_eval++;
  }
  ctx->fcons_valid = false;
  return CR_OK;
}

extern "C" int cr_md_begin(cr_ctx *ctx, double dt, double gamma, uint64_t seed) {
  if (!ctx || !(dt > 0.0) || !(gamma >= 0.0)) return CR_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  const SysParams &P = ctx->P;
  RebuildBufs B{ctx->d_cnt2, ctx->d_pos2, ctx->d_pid2, ctx->d_info2, ctx->d_vel2, ctx->d_frc2, ctx->d_vel, ctx->d_frc};
  int rc;
  if (!ctx->f_valid) {
    if ((rc = md_force_eval(ctx, md_params(ctx, 1, dt, gamma, seed))) != CR_OK) return rc;
    ctx->md_eval++;
  }
  MdParams M = md_params(ctx, 2, dt, gamma, seed);
  CR_CUDA(launch_kick_drift_rebuild(P, M, B, ctx->d_perm, ctx->n_input, s));
  ctx->launches_total += 2;
  ctx->f_valid = false;  // positions moved: the closing kick needs new forces
  ctx->fcons_valid = false;
  return CR_OK;
}

// cr_md_end's force evaluation; in a captured cycle (dyn) the key and the
// evaluation counter come from the step parameters in device memory
static int md_end_impl(cr_ctx *ctx, double dt, double gamma, uint64_t seed, const StepDyn *dyn, unsigned rep,
                       int eval_off = 0) {
  MdParams M = md_params(ctx, 2, dt, gamma, seed);
  M.dyn = dyn;
  M.rep = rep;
  M.eval_off = eval_off;
  return md_force_eval(ctx, M);
}

// the force evaluation that opens a captured step whose forces are stale (as
// cr_md_begin does it call by call: Langevin terms, no kick), counters from dyn
static int md_first_impl(cr_ctx *ctx, double dt, double gamma, const StepDyn *dyn, unsigned rep) {
  MdParams M = md_params(ctx, 1, dt, gamma, 0);
  M.dyn = dyn;
  M.rep = rep;
  const int rc = md_force_eval(ctx, M);
  if (rc == CR_OK) ctx->f_valid = true;  // the captured md_begin then only kicks and drifts
  return rc;
}

extern "C" int cr_md_end(cr_ctx *ctx, double dt, double gamma, uint64_t seed) {
  if (!ctx || !(dt > 0.0) || !(gamma >= 0.0)) return CR_ERR_INVALID_ARG;
  int rc;
  if ((rc = md_end_impl(ctx, dt, gamma, seed, nullptr, 0)) != CR_OK) return rc;
  ctx->md_eval++;
  ctx->f_valid = true;
  ctx->fcons_valid = false;
  return CR_OK;
}

// the sort bits of a context's ion keys: inserted ids are (phase + 1) << 32 |
// low word with phase < sweeps * colours, the keys put the high word above the
// low word's ion_lo_bits bits; one spare bit keeps the sort's padding last
static int ion_end_bit(const cr_ctx *ctx) {
  const uint64_t hi_max = ctx->sweep * (uint64_t)ctx->P.ncol + 1;
  int end_bit = ctx->ion_lo_bits + 1;
  while (end_bit < 64 && (hi_max >> (end_bit - ctx->ion_lo_bits - 1)) != 0) ++end_bit;
  return end_bit;
}

// A state read in two halves around one synchronisation of the stream:
// state_begin queues the id marks (when arrays are wanted) and the copies of
// the counts and the error word; state_arrays, with those on the host, fills
// the counts of the view and queues the ordering and one copy per array.
static int state_begin(cr_ctx *ctx, const cr_state_view *out, cudaStream_t s, StateBufs &B, bool &want,
                       bool integrator_forces = false) {
  long long *hs = ctx->h_small;  // pinned: [0, N_KIND) kind counts, [N_KIND] ions found, [N_KIND + 1] error word
  want = out->xyz || out->vel || out->force || out->id || out->type || out->state || out->site_state || out->cls;
  B = StateBufs{};
  B.n_input = ctx->n_input;
  B.cap = (int)ctx->capacity;
  B.lo_bits = ctx->ion_lo_bits;
  B.present = ctx->d_present;
  B.n_ions = ctx->d_counter;
  B.ion_key = ctx->d_ion_key;
  B.ion_key_alt = ctx->d_ion_key2;
  B.ion_val = ctx->d_ion_val;
  B.ion_val_alt = ctx->d_ion_val2;
  B.ion_rank = ctx->d_ion_rank;
  B.sort_tmp = ctx->d_sort_tmp;
  B.sort_tmp_bytes = ctx->sort_tmp_bytes;
  B.vel_src = ctx->d_vel;
  if (integrator_forces) B.frc_src = ctx->f_valid ? ctx->d_frc : nullptr;  // a checkpoint: the next half kick's forces
  else B.frc_src = ctx->fcons_valid ? ctx->d_fcons : nullptr;
  B.xyz = out->xyz ? ctx->d_out_xyz : nullptr;
  B.vel = out->vel ? ctx->d_out_vel : nullptr;
  B.frc = out->force ? ctx->d_out_frc : nullptr;
  B.id = out->id ? ctx->d_out_id : nullptr;
  B.type = out->type ? ctx->d_out_type : nullptr;
  B.cls = out->cls ? ctx->d_out_cls : nullptr;
  B.state = out->state ? ctx->d_out_state : nullptr;
  B.site = out->site_state ? ctx->d_out_site : nullptr;
  if (want) {
    CR_CUDA(launch_state_mark(ctx->P, B, s));
    ctx->launches_total++;
  }
  // kind counts, ions found and the error word: adjacent, one copy
  CR_CUDA(cudaMemcpyAsync(hs, ctx->d_counts, (N_KIND + 2) * sizeof(long long), cudaMemcpyDeviceToHost, s));
  return CR_OK;
}

static int state_arrays(cr_ctx *ctx, cr_state_view *out, cudaStream_t s, const StateBufs &B, bool want) {
  const long long *hs = ctx->h_small;
  const int n_ions = *(const int *)(hs + N_KIND), bits = *(const int *)(hs + N_KIND + 1);
  out->n_A = hs[K_A0] + hs[K_A1];
  out->n_Am = hs[K_A1];
  out->n_B = hs[K_B0] + hs[K_B1];
  out->n_Bp = hs[K_B1];
  out->n_Xp = hs[K_XP];
  out->n_Xm = hs[K_XM];
  out->n_Sp = hs[K_SP];
  out->n_Sm = hs[K_SM];
  out->n = out->n_A + out->n_B + out->n_Xp + out->n_Xm + out->n_Sp + out->n_Sm + ctx->n_other;
  out->net_charge = out->n_Xp + out->n_Sp - out->n_Xm - out->n_Sm - out->n_Am + out->n_Bp;
  out->alpha = out->n_A > 0 ? (double)out->n_Am / (double)out->n_A : 0.0;
  const int err0 = err_bits_to_code(bits);
  if (!want) return err0;
  const int64_t n = out->n;
  const int64_t n_present = n - n_ions;
  int rc = err0;
  if (rc == CR_OK && n > ctx->capacity) rc = CR_ERR_CAPACITY;
  if (rc == CR_OK && (n_ions < 0 || n_ions > ctx->capacity || n_present < 0 || n_present > ctx->n_input))
    rc = CR_ERR_CUDA;
  if (rc != CR_OK) {  // clear the marks for the next read
    CR_CUDA(cudaMemsetAsync(ctx->d_present, 0, sizeof(int) * (size_t)std::max(ctx->n_input, 1), s));
    CR_CUDA(cudaMemsetAsync(ctx->d_counter, 0, sizeof(int), s));
    return rc;
  }
  const int end_bit = ion_end_bit(ctx);
  int nl = 0;
  CR_CUDA(launch_state_order(ctx->P, B, (int)n_present, n_ions, end_bit, s, &nl));
  ctx->launches_total += nl;
  const size_t nn = (size_t)n;
  if (out->xyz) CR_CUDA(cudaMemcpyAsync(out->xyz, B.xyz, sizeof(float) * 3 * nn, cudaMemcpyDeviceToHost, s));
  if (out->vel) CR_CUDA(cudaMemcpyAsync(out->vel, B.vel, sizeof(float) * 3 * nn, cudaMemcpyDeviceToHost, s));
  if (out->force) CR_CUDA(cudaMemcpyAsync(out->force, B.frc, sizeof(float) * 3 * nn, cudaMemcpyDeviceToHost, s));
  if (out->id) CR_CUDA(cudaMemcpyAsync(out->id, B.id, sizeof(uint64_t) * nn, cudaMemcpyDeviceToHost, s));
  if (out->type) CR_CUDA(cudaMemcpyAsync(out->type, B.type, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, s));
  if (out->cls) CR_CUDA(cudaMemcpyAsync(out->cls, B.cls, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, s));
  if (out->state) CR_CUDA(cudaMemcpyAsync(out->state, B.state, nn, cudaMemcpyDeviceToHost, s));
  if (out->site_state && ctx->n_sites > 0)
    CR_CUDA(cudaMemcpyAsync(out->site_state, B.site, (size_t)ctx->n_sites, cudaMemcpyDeviceToHost, s));
  return CR_OK;
}

extern "C" int cr_state(cr_ctx *ctx, cr_state_view *out) {
  if (!ctx || !out) return CR_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  StateBufs B;
  bool want = false;
  int rc = state_begin(ctx, out, s, B, want);
  if (rc != CR_OK) return rc;
  CR_CUDA(cudaStreamSynchronize(s));
  rc = state_arrays(ctx, out, s, B, want);
  if (rc != CR_OK || !want) return rc;
  CR_CUDA(cudaStreamSynchronize(s));
  return CR_OK;
}

extern "C" int cr_checkpoint(cr_ctx *ctx, cr_state_view *out, cr_counters *counters) {
  if (!ctx || !out || !counters) return CR_ERR_INVALID_ARG;
  cudaStream_t s = ctx->stream;
  StateBufs B;
  bool want = false;
  int rc = state_begin(ctx, out, s, B, want, true);
  if (rc != CR_OK) return rc;
  CR_CUDA(cudaStreamSynchronize(s));
  rc = state_arrays(ctx, out, s, B, want);
  if (rc != CR_OK) return rc;
  if (want) CR_CUDA(cudaStreamSynchronize(s));
  counters->sweep = ctx->sweep;
  counters->md_eval = ctx->md_eval;
  counters->forces_valid = ctx->f_valid ? 1 : 0;
  return CR_OK;
}

extern "C" int cr_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int32_t n,
                         uint32_t *out) {
  if (n < 0 || (n > 0 && !out)) return CR_ERR_INVALID_ARG;
  if (n == 0) return CR_OK;
  uint4 *d = nullptr;
  CR_CUDA(cudaMalloc((void **)&d, sizeof(uint4) * n));
  cudaError_t e = launch_philox(c0, c1, c2, c3, k0, k1, n, d, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, d, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return cuda_fail(e);
}

extern "C" int cr_load(cr_ctx *ctx, int32_t n, const float *xyz, const float *vel, const int32_t *type,
                       const int32_t *cls, const int8_t *state) {
  if (!ctx || n < 0 || n > ctx->capacity || ctx->n_bodies > 0) return CR_ERR_INVALID_ARG;
  if (n > 0 && (!xyz || !type || !cls || !state)) return CR_ERR_INVALID_ARG;
  // every bonded / site particle of cr_init must be there (at its index; the
  // load kernels check each particle and the neutrality on the device)
  if (n < ctx->n_fixed_end) return CR_ERR_INVALID_ARG;
  const SysParams &P = ctx->P;
  cudaStream_t s = ctx->stream;
  if (n > 0) {
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_xyz, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    if (vel) CR_CUDA(cudaMemcpyAsync(ctx->d_in_vel, vel, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_type, type, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_cls, cls, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_state, state, sizeof(int8_t) * n, cudaMemcpyHostToDevice, s));
  }
  CR_CUDA(cudaMemsetAsync(ctx->d_counts, 0, sizeof(long long) * N_KIND, s));
  LoadBufs I{ctx->d_in_xyz, vel ? ctx->d_in_vel : nullptr, ctx->d_in_type, ctx->d_in_cls, ctx->d_site_map,
             ctx->d_in_state, n, ctx->n_input, ctx->d_init_type};
  RebuildBufs B{ctx->d_cnt2, ctx->d_pos2, ctx->d_pid2, ctx->d_info2, ctx->d_vel2, ctx->d_frc2, ctx->d_vel, ctx->d_frc};
  CR_CUDA(launch_load(P, I, B, ctx->d_perm, ctx->n_input, s));
  ctx->launches_total += 3;
  ctx->f_valid = false;
  ctx->fcons_valid = false;
  return CR_OK;
}

extern "C" int cr_restore(cr_ctx *ctx, int32_t n, const float *xyz, const float *vel, const float *force,
                          const uint64_t *id, const int32_t *type, const int32_t *cls, const int8_t *state,
                          const cr_counters *counters) {
  if (!ctx || !counters || n < 0 || n > ctx->capacity || ctx->n_bodies > 0) return CR_ERR_INVALID_ARG;
  if (n > 0 && (!xyz || !type || !cls || !state || !id)) return CR_ERR_INVALID_ARG;
  if (counters->forces_valid && n > 0 && !force) return CR_ERR_INVALID_ARG;
  if (counters->sweep > (uint64_t)UINT32_MAX / (uint64_t)std::max(ctx->P.ncol, 1)) return CR_ERR_INVALID_ARG;
  // ids: unique; every bonded / site particle of cr_init present; the others
  // input ions (below the input count) or inserted ions (at least 2^32)
  {
    std::vector<char> seen((size_t)std::max(ctx->n_input, 1), 0);
    std::vector<uint64_t> ions;
    for (int32_t i = 0; i < n; ++i) {
      const uint64_t d = id[i];
      if (d < (uint64_t)ctx->n_input) {
        if (seen[d]) return CR_ERR_INVALID_ARG;
        seen[d] = 1;
      } else if (d >> 32) {
        ions.push_back(d);
      } else {
        return CR_ERR_INVALID_ARG;
      }
    }
    for (int i = 0; i < ctx->n_input; ++i)
      if (!seen[i] && !is_ion_type(ctx->init_type[i])) return CR_ERR_INVALID_ARG;
    std::sort(ions.begin(), ions.end());
    if (std::adjacent_find(ions.begin(), ions.end()) != ions.end()) return CR_ERR_INVALID_ARG;
  }
  if (!ctx->d_in_id) CR_CUDA(cudaMalloc((void **)&ctx->d_in_id, sizeof(unsigned long long) * (size_t)ctx->capacity));
  if (!ctx->d_in_frc) CR_CUDA(cudaMalloc((void **)&ctx->d_in_frc, sizeof(float) * 3 * (size_t)ctx->capacity));
  const SysParams &P = ctx->P;
  cudaStream_t s = ctx->stream;
  const bool with_f = counters->forces_valid != 0;
  if (n > 0) {
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_xyz, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    if (vel) CR_CUDA(cudaMemcpyAsync(ctx->d_in_vel, vel, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    if (with_f) CR_CUDA(cudaMemcpyAsync(ctx->d_in_frc, force, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_id, id, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_type, type, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_cls, cls, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CR_CUDA(cudaMemcpyAsync(ctx->d_in_state, state, sizeof(int8_t) * n, cudaMemcpyHostToDevice, s));
  }
  CR_CUDA(cudaMemsetAsync(ctx->d_counts, 0, sizeof(long long) * N_KIND, s));
  LoadBufs I{ctx->d_in_xyz, vel ? ctx->d_in_vel : nullptr, ctx->d_in_type, ctx->d_in_cls, ctx->d_site_map,
             ctx->d_in_state, n, ctx->n_input, ctx->d_init_type, ctx->d_in_id, with_f ? ctx->d_in_frc : nullptr};
  RebuildBufs B{ctx->d_cnt2, ctx->d_pos2, ctx->d_pid2, ctx->d_info2, ctx->d_vel2, ctx->d_frc2, ctx->d_vel, ctx->d_frc};
  CR_CUDA(launch_load(P, I, B, ctx->d_perm, ctx->n_input, s));
  ctx->launches_total += 3;
  ctx->sweep = counters->sweep;
  ctx->md_eval = counters->md_eval;
  ctx->f_valid = with_f;
  ctx->fcons_valid = false;
  return CR_OK;
}

extern "C" int cr_set_timing(cr_ctx *ctx, int32_t enable) {
  if (!ctx) return CR_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  return CR_OK;
}

extern "C" int cr_get_timing(cr_ctx *ctx, double *ms, int64_t *launches, int64_t *launches_total, int32_t reset) {
  if (!ctx) return CR_ERR_INVALID_ARG;
  CR_CUDA(cudaStreamSynchronize(ctx->stream));
  tcollect(ctx);
  for (int k = 0; k < 2; ++k) {
    if (ms) ms[k] = ctx->ms[k];
    if (launches) launches[k] = ctx->launches[k];
  }
  if (launches_total) *launches_total = ctx->launches_total;
  if (reset) {
    ctx->ms[0] = ctx->ms[1] = 0.0;
    ctx->launches[0] = ctx->launches[1] = 0;
    ctx->launches_total = 0;
  }
  return CR_OK;
}

extern "C" int cr_set_launch_shape(cr_ctx *ctx, int32_t threads, int32_t regs) {
  if (!ctx) return CR_ERR_INVALID_ARG;
  if (threads == 0) {  // re-enable tuning
    ctx->tuning = true;
    ctx->tune_next = 0;
    ctx->da_tuning = true;
    ctx->da_next = 0;
    return CR_OK;
  }
  bool found = false;
  for (int i = 0; i < phase_shape_count(false); ++i) {
    int t, r;
    phase_shape(i, &t, &r, false);
    if (t == threads && r == regs) {
      ctx->T = t;
      ctx->R = r;
      ctx->C = false;
      ctx->tuning = false;
      found = true;
    }
  }
  for (int i = 0; i < phase_shape_count(true); ++i) {  // delayed-acceptance sweeps, where supported
    int t, r;
    phase_shape(i, &t, &r, true);
    if (t == threads && r == regs) {
      ctx->da_T = t;
      ctx->da_R = r;
      ctx->da_C = false;
      ctx->da_tuning = false;
      found = true;
    }
  }
  return found ? CR_OK : CR_ERR_INVALID_ARG;
}

extern "C" int cr_get_launch_shape(const cr_ctx *ctx, int32_t *threads, int32_t *regs) {
  if (!ctx || !threads || !regs) return CR_ERR_INVALID_ARG;
  *threads = ctx->T;
  *regs = ctx->R;
  return CR_OK;
}

// ---------------------------------------------------------------------------
// batches of replicas: one phase launch per colour for all replicas
// ---------------------------------------------------------------------------
struct cr_batch {
  std::vector<cr_ctx *> ctx;
  std::vector<int> chem_seen;  // each context's chemistry version in d_reps
  // persistent sweeps (k_cr_sweep): on by default; the replicas' prefix of
  // active domains per colour and the launch's device words (task counter,
  // abort flag, per-(replica, colour) completion counters), zeroed per launch
  int pmode = -1;              // persistent mode: -1 chosen by the tuner, 0 off, 1 per-domain, 2 per-colour
  bool persistent = true;      // the mode in use (auto: the tuner's choice once it finished)
  bool da_persistent = true;
  bool fine = false;           // per-domain dependencies (every replica's halo within its neighbouring domains)
  bool fine_ok = false;        // the geometry allows them
  int ctas_per_sm = 0;         // resident CTAs per SM of a persistent sweep (0: as many as fit)
  int *d_rep_first = nullptr;  // [n + 1] active domains per colour, then [n + 1] domains (prefix sums)
  unsigned *d_words = nullptr;
  size_t words = 0, flag_words = 0;
  int tasks_per_colour = 0;
  int sms = 0;
  // captured MD/CR-MC cycle (cr_batch_cycle): the step parameters in device
  // memory, the instantiated graph and what it was captured with
  StepDyn *d_dyn = nullptr;
  cudaStream_t cstream = nullptr;  // capture stream
  cudaGraphExec_t graph = nullptr;
  double g_dt = 0.0, g_gamma = 0.0;
  int g_T = 0, g_R = 0, g_da = -1;
  bool g_C = false, g_pers = false, g_fine = false, g_timing = false;
  bool g_ff = false;  // the graph's step evaluates the forces first (a step after a load)
  int64_t g_kernels = 0;                      // kernels per graph launch
  std::vector<std::pair<int, int>> g_pairs;  // phase-kernel event pairs recorded by the graph (timing)
  SysParams *d_reps = nullptr;  // one entry per replica (key_xor = replica index)
  PhaseShape S{}, Sc{};
  bool C = false, da_C = false;
  int grid_x = 0, ncol = 8;
  int T = 128, R = 4;
  int smem_max = 0;
  bool tuning = true;
  int tune_next = 0;
  float tune_ms[32] = {};
  int da_T = 128, da_R = 0, da_next = 0;
  bool da_tuning = true;
  float da_ms[16] = {};
  std::vector<SysParams> reps;  // host copy of d_reps
  cudaStream_t stream = nullptr;  // the contexts' shared stream (destroy does not touch the contexts)
  int order_nc = 0, order_nact = 0;  // largest box and colour among replicas with a launch order (0: none)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaEvent_t fork = nullptr;
  // packed reads and loads: per-replica descriptors (pinned host + device),
  // the replicas' counts and error words, staging arrays of stride entries
  // per replica
  StateBufs *h_sbufs = nullptr, *d_sbufs = nullptr;
  LoadJob *h_jobs = nullptr, *d_jobs = nullptr;
  long long *h_nout = nullptr, *d_nout = nullptr;  // h_nout[n] also holds the error words (as ints)
  int *d_errout = nullptr;
  int64_t pk_stride = 0;
  float *d_pk_xyz = nullptr, *d_pk_vel = nullptr;
  unsigned long long *d_pk_id = nullptr;
  int *d_pk_type = nullptr, *d_pk_cls = nullptr;
  int8_t *d_pk_state = nullptr;
  bool holds_refs = false;  // the contexts' batch_refs count this batch
  int ewald_nk_max = 0;     // largest number of Ewald reciprocal vectors over the replicas
};

// The device address of caller memory the GPU can access directly (device
// memory, or pinned host memory: on GB300 host writes and reads go over
// NVLink-C2C), else null (pageable memory goes through the staging arrays).
template <typename TT>
static TT *device_view(TT *p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<TT *>(a.devicePointer);
  return nullptr;
}

static void free_packed_staging(cr_batch *b) {
  void *p[] = {b->d_pk_xyz, b->d_pk_vel, b->d_pk_id, b->d_pk_type, b->d_pk_cls, b->d_pk_state};
  for (void *x : p)
    if (x) cudaFree(x);
  b->d_pk_xyz = b->d_pk_vel = nullptr;
  b->d_pk_id = nullptr;
  b->d_pk_type = b->d_pk_cls = nullptr;
  b->d_pk_state = nullptr;
  b->pk_stride = 0;
}

// device staging of stride entries per replica for the packed calls, and the
// per-replica descriptors; allocated on first use, grown with the stride
static int ensure_packed(cr_batch *b, int64_t stride) {
  const size_t n = b->ctx.size();
  if (!b->h_sbufs) {
    if (cudaHostAlloc((void **)&b->h_sbufs, n * sizeof(StateBufs), 0) != cudaSuccess ||
        cudaHostAlloc((void **)&b->h_jobs, n * sizeof(LoadJob), 0) != cudaSuccess ||
        cudaHostAlloc((void **)&b->h_nout, 2 * n * sizeof(long long), 0) != cudaSuccess)
      return CR_ERR_NOMEM;
    if (cudaMalloc((void **)&b->d_sbufs, n * sizeof(StateBufs)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_jobs, n * sizeof(LoadJob)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_nout, n * sizeof(long long)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_errout, n * sizeof(int)) != cudaSuccess)
      return CR_ERR_NOMEM;
  }
  if (stride <= b->pk_stride) return CR_OK;
  free_packed_staging(b);
  const size_t m = n * (size_t)stride;
  if (cudaMalloc((void **)&b->d_pk_xyz, 3 * m * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_pk_vel, 3 * m * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_pk_id, m * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_pk_type, m * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_pk_cls, m * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_pk_state, m) != cudaSuccess) {
    free_packed_staging(b);
    return CR_ERR_NOMEM;
  }
  b->pk_stride = stride;
  return CR_OK;
}

extern "C" int cr_batch_create(cr_batch **out, cr_ctx *const *ctxs, int32_t n) {
  if (!out || !ctxs || n <= 0) return CR_ERR_INVALID_ARG;
  *out = nullptr;
  cr_batch *b = new (std::nothrow) cr_batch();
  if (!b) return CR_ERR_NOMEM;
  b->ctx.assign(ctxs, ctxs + n);
  for (int r = 0; r < n; ++r) b->chem_seen.push_back(ctxs[r] ? ctxs[r]->chem_version : 0);
  std::vector<SysParams> reps(n);
  int maxR = 1;
  for (int r = 0; r < n; ++r) {
    cr_ctx *c = ctxs[r];
    if (!c || c->P.ncol != ctxs[0]->P.ncol || c->sweep != ctxs[0]->sweep || c->stream != ctxs[0]->stream ||
        c->n_bodies > 0) {
      delete b;
      return CR_ERR_INVALID_ARG;
    }
    reps[r] = c->P;
    reps[r].key_xor = (uint32_t)r;
    reps[r].log = nullptr;
    b->S.dcs = std::max(b->S.dcs, c->S.dcs);
    b->S.hcs = std::max(b->S.hcs, c->S.hcs);
    b->S.lns = std::max(b->S.lns, c->S.lns);
    b->S.nr3 = std::max(b->S.nr3, c->S.nr3);
    b->S.kc3 = std::max(b->S.kc3, c->S.kc3);
    b->S.chunk = std::max(b->S.chunk, c->S.chunk);
    b->S.ewk = std::max(b->S.ewk, c->S.ewk);
    b->ewald_nk_max = std::max(b->ewald_nk_max, c->P.ewald_nk);
    b->Sc.dcs = std::max(b->Sc.dcs, c->Sc.dcs);
    b->Sc.hcs = std::max(b->Sc.hcs, c->Sc.hcs);
    b->Sc.lns = std::max(b->Sc.lns, c->Sc.lns);
    b->Sc.nr3 = std::max(b->Sc.nr3, c->Sc.nr3);
    b->Sc.kc3 = std::max(b->Sc.kc3, c->Sc.kc3);
    b->Sc.chunk = std::max(b->Sc.chunk, c->Sc.chunk);
    b->Sc.ewk = std::max(b->Sc.ewk, c->Sc.ewk);
    b->grid_x = std::max(b->grid_x, c->P.nact);
    maxR = std::max(maxR, c->R);
  }
  b->ncol = ctxs[0]->P.ncol;
  b->stream = ctxs[0]->stream;
  b->R = 0;
  (void)maxR;
  b->tuning = std::getenv("CRMC_NO_TUNE") == nullptr;
  b->da_tuning = b->tuning;
  b->reps = reps;
  for (int r = 0; r < n; ++r)
    if (reps[r].order) {
      b->order_nc = std::max(b->order_nc, reps[r].nc);
      b->order_nact = std::max(b->order_nact, reps[r].nact);
    }
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctxs[0]->device);
  if (phase_smem_bytes(b->S, 512, false) > (size_t)smem_max) { delete b; return CR_ERR_INVALID_ARG; }
  b->smem_max = smem_max;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, ctxs[0]->device);
  if (cudaMalloc((void **)&b->d_reps, sizeof(SysParams) * n) != cudaSuccess) { delete b; return CR_ERR_NOMEM; }
  if (cudaMemcpy(b->d_reps, reps.data(), sizeof(SysParams) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(b->d_reps);
    delete b;
    return CR_ERR_CUDA;
  }
  b->streams.resize(n);
  b->events.resize(n);
  for (int r = 0; r < n; ++r) {
    cudaStreamCreateWithFlags(&b->streams[r], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&b->events[r], cudaEventDisableTiming);
  }
  cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  {  // persistent-sweep schedule: per-domain dependencies when every
     // replica's region (its domain and h cells around it) lies within the
     // 3^3 block of domains around it (h <= k) and the schedule is coloured
    std::vector<int> first(2 * (n + 1), 0);
    bool fine = true;
    for (int r = 0; r < n; ++r) {
      first[r + 1] = first[r] + reps[r].nact;
      first[n + 1 + r + 1] = first[n + 1 + r] + reps[r].nd * reps[r].nd * reps[r].nd;
      fine = fine && !reps[r].global && reps[r].h <= reps[r].k && reps[r].nd >= 2;
    }
    b->fine = b->fine_ok = fine;
    b->tasks_per_colour = first[n];
    b->flag_words = (size_t)first[2 * n + 1];
    b->words = 2 + (size_t)n * b->ncol + b->flag_words;
    if (cudaMalloc((void **)&b->d_rep_first, sizeof(int) * 2 * (n + 1)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_words, sizeof(unsigned) * b->words) != cudaSuccess ||
        cudaMemcpy(b->d_rep_first, first.data(), sizeof(int) * 2 * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
      cr_batch_destroy(b);
      return CR_ERR_NOMEM;
    }
  }
  for (cr_ctx *c : b->ctx) c->batch_refs++;  // (contexts in a batch cannot be bound)
  b->holds_refs = true;
  *out = b;
  return CR_OK;
}

extern "C" void cr_batch_destroy(cr_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->holds_refs)
    for (cr_ctx *c : b->ctx)
      if (c) c->batch_refs--;
  for (size_t r = 0; r < b->streams.size(); ++r) {
    cudaStreamSynchronize(b->streams[r]);
    cudaStreamDestroy(b->streams[r]);
    cudaEventDestroy(b->events[r]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_reps) cudaFree(b->d_reps);
  if (b->d_rep_first) cudaFree(b->d_rep_first);
  if (b->d_words) cudaFree(b->d_words);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->ctx[0]->ev_reserved = 0;
  }
  if (b->d_dyn) cudaFree(b->d_dyn);
  if (b->cstream) cudaStreamDestroy(b->cstream);
  free_packed_staging(b);
  void *dp[] = {b->d_sbufs, b->d_jobs, b->d_nout, b->d_errout};
  for (void *x : dp)
    if (x) cudaFree(x);
  void *hp[] = {b->h_sbufs, b->h_jobs, b->h_nout};
  for (void *x : hp)
    if (x) cudaFreeHost(x);
  delete b;
}

static int batch_refresh_chem(cr_batch *b);

// one persistent sweep launch of every replica (words zeroed first)
static int batch_launch_persistent(cr_batch *b, const PhaseShape &SS, int T, int R, bool da, uint32_t swc,
                                   uint32_t sweep0, uint32_t k0, uint32_t k1, int withhold = -1,
                                   unsigned long long wait_ns = 2000000000ull, const StepDyn *dyn = nullptr) {
  cr_ctx *c0 = b->ctx[0];
  cudaStream_t s = c0->stream;
  CR_CUDA(cudaMemsetAsync(b->d_words, 0, sizeof(unsigned) * b->words, s));
  SweepSched Q{};
  Q.n_rep = (int)b->ctx.size();
  Q.ncol = b->ncol;
  Q.tasks_total = b->tasks_per_colour * b->ncol;
  Q.fine = b->fine ? 1 : 0;
  Q.rep_first = b->d_rep_first;
  Q.dom_first = b->d_rep_first + b->ctx.size() + 1;
  Q.next = b->d_words;
  Q.abort = (int *)(b->d_words + 1);
  Q.done = b->d_words + 2;
  Q.flags = Q.done + b->ctx.size() * b->ncol;
  Q.wait_ns = wait_ns;
  Q.withhold_rep = withhold;
  int ti;
  tbegin(c0, 0, &ti);
  const int sms = b->sms > 0 ? b->sms : 1;
  CR_CUDA(launch_sweep(b->d_reps, SS, T, R, da, s, swc, sweep0, k0, k1, Q, b->ctas_per_sm * sms, dyn));
  tend(c0, 0, ti);
  c0->launches_total++;
  return CR_OK;
}

static int batch_sweep_impl(cr_batch *b, uint64_t n_sweeps, uint64_t seed, bool da) {
  if (!b || n_sweeps == 0) return CR_ERR_INVALID_ARG;
  cr_ctx *c0 = b->ctx[0];
  cudaStream_t s = c0->stream;
  const int n = (int)b->ctx.size();
  if (da) {  // every replica needs its surrogate; refresh the device copies of the parameters
    bool changed = false;
    for (int r = 0; r < n; ++r) {
      cr_ctx *c = b->ctx[r];
      if (!c->has_mlp) return CR_ERR_INVALID_ARG;
      if (b->reps[r].mlp_w != c->P.mlp_w || b->reps[r].mlp_b != c->P.mlp_b) {
        b->reps[r].mlp_w = c->P.mlp_w;
        b->reps[r].mlp_b = c->P.mlp_b;
        changed = true;
      }
    }
    if (changed)
      CR_CUDA(cudaMemcpyAsync(b->d_reps, b->reps.data(), sizeof(SysParams) * n, cudaMemcpyHostToDevice, s));
  }
  {  // a context's chemistry changed: its copy in the batch follows
    const int rc = batch_refresh_chem(b);
    if (rc != CR_OK) return rc;
  }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint32_t sweep0 = (uint32_t)c0->sweep;
  bool &pers_choice = da ? b->da_persistent : b->persistent;
  TuneRef tr = da ? TuneRef{b->da_T, b->da_R, b->da_next, b->da_tuning, b->da_ms, b->da_C}
                  : TuneRef{b->T, b->R, b->tune_next, b->tuning, b->tune_ms, b->C};
  if (b->pmode < 0) tr.pers = &pers_choice;
  else pers_choice = b->pmode != 0;
  const int nshape = phase_shape_count(da);
  for (uint64_t sw = 0; sw < n_sweeps; ++sw) {
    const uint32_t swc = (uint32_t)c0->sweep;
    for (cr_ctx *c : b->ctx) {
      c->sweep++;
      c->f_valid = false;
      c->fcons_valid = false;
    }
    tune_skip(tr, b->S, b->Sc, b->smem_max, da);
    const bool tune = tr.on && tr.next < tune_total(tr, da);
    int T = tr.T, R = tr.R;
    bool persistent = pers_choice;
    const int cand = tune ? tune_cand(tr, da) : 0;
    const bool compact = tune ? phase_shape_compact(cand % nshape, da) : tr.C;
    const PhaseShape &SS = compact ? b->Sc : b->S;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (tune) {
      phase_shape(cand % nshape, &T, &R, da);
      if (tr.pers) persistent = cand >= nshape;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
    }
    if (b->order_nc > 0) {
      CR_CUDA(launch_domain_order(b->d_reps, n, b->ncol, b->order_nact, s, swc, k0, k1));
      c0->launches_total++;
    }
    if (b->ewald_nk_max > 0) {  // S(k) of every replica from scratch at every sweep
      CR_CUDA(launch_ewald_sk(b->d_reps, n, b->ewald_nk_max, s));
      c0->launches_total += 2;
    }
    if (persistent) {
      const int rc = batch_launch_persistent(b, SS, T, R, da, swc, sweep0, k0, k1);
      if (rc != CR_OK) return rc;
    } else {
      for (int col = 0; col < b->ncol; ++col) {
        int ti;
        tbegin(c0, 0, &ti);
        CR_CUDA(launch_phase(b->d_reps, n, b->grid_x, SS, T, R, false, da, s, swc, sweep0, col, k0, k1));
        tend(c0, 0, ti);
        c0->launches_total++;
      }
    }
    if (tune) {
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      tune_finish(tr, ms, b->S, b->Sc, b->smem_max, da);
    }
  }
  return CR_OK;
}

extern "C" int cr_batch_sweep(cr_batch *b, uint64_t n_sweeps, uint64_t seed) {
  return batch_sweep_impl(b, n_sweeps, seed, false);
}

extern "C" int cr_batch_set_persistent(cr_batch *b, int32_t mode, int32_t ctas_per_sm) {
  if (!b || mode < -1 || mode > 2 || ctas_per_sm < 0) return CR_ERR_INVALID_ARG;
  b->pmode = mode;
  b->persistent = b->da_persistent = mode != 0;
  b->fine = mode != 2 && b->fine_ok;
  b->ctas_per_sm = ctas_per_sm;
  return CR_OK;
}

extern "C" int cr_batch_selftest_wait_timeout(cr_batch *b, int32_t replica, double timeout_ms) {
  if (!b || replica < 0 || replica >= (int)b->ctx.size() || !(timeout_ms > 0.0) || timeout_ms > 10000.0)
    return CR_ERR_INVALID_ARG;
  cr_ctx *c0 = b->ctx[0];
  const uint32_t swc = (uint32_t)c0->sweep;
  for (cr_ctx *c : b->ctx) {
    c->sweep++;
    c->f_valid = false;
    c->fcons_valid = false;
  }
  int T = b->T, R = b->R;
  const PhaseShape &SS = b->C ? b->Sc : b->S;
  if (b->tuning) {  // a shape every context supports
    T = 128;
    R = 0;
  }
  if (b->order_nc > 0) {
    CR_CUDA(launch_domain_order(b->d_reps, (int)b->ctx.size(), b->ncol, b->order_nact, c0->stream, swc, 1u, 0u));
    c0->launches_total++;
  }
  const int rc = batch_launch_persistent(b, b->tuning ? b->S : SS, T, R, false, swc, swc, 1u, 0u, replica,
                                         (unsigned long long)(timeout_ms * 1e6));
  if (rc != CR_OK) return rc;
  CR_CUDA(cudaStreamSynchronize(c0->stream));
  int worst = CR_OK;
  for (cr_ctx *c : b->ctx) {
    const int e = cr_check(c);
    if (e != CR_OK && worst == CR_OK) worst = e;
  }
  return worst;
}

extern "C" int cr_batch_sweep_da(cr_batch *b, uint64_t n_sweeps, uint64_t seed) {
  return batch_sweep_impl(b, n_sweeps, seed, true);
}

// run an MD call on every replica of a batch, concurrently on per-replica streams
template <typename Fn>
static int batch_md(cr_batch *b, Fn fn) {
  if (!b) return CR_ERR_INVALID_ARG;
  cudaStream_t s = b->ctx[0]->stream;
  CR_CUDA(cudaEventRecord(b->fork, s));
  int rc = CR_OK;
  for (size_t r = 0; r < b->ctx.size(); ++r) {
    cr_ctx *c = b->ctx[r];
    CR_CUDA(cudaStreamWaitEvent(b->streams[r], b->fork, 0));
    c->stream = b->streams[r];
    const bool timing = c->timing;
    c->timing = false;
    const int e = fn(c, (uint64_t)r);
    c->timing = timing;
    c->stream = s;
    if (e != CR_OK && rc == CR_OK) rc = e;
    CR_CUDA(cudaEventRecord(b->events[r], b->streams[r]));
    CR_CUDA(cudaStreamWaitEvent(s, b->events[r], 0));
    b->ctx[0]->launches_total += (r > 0) ? c->launches_total : 0;
    if (r > 0) c->launches_total = 0;
  }
  return rc;
}

extern "C" int cr_batch_md_step(cr_batch *b, int32_t n_steps, double dt, double gamma, uint64_t seed) {
  return batch_md(b, [&](cr_ctx *c, uint64_t r) { return cr_md_step(c, n_steps, dt, gamma, seed ^ (r << 32)); });
}

extern "C" int cr_batch_md_begin(cr_batch *b, double dt, double gamma, uint64_t seed) {
  return batch_md(b, [&](cr_ctx *c, uint64_t r) { return cr_md_begin(c, dt, gamma, seed ^ (r << 32)); });
}

extern "C" int cr_batch_md_end(cr_batch *b, double dt, double gamma, uint64_t seed) {
  return batch_md(b, [&](cr_ctx *c, uint64_t r) { return cr_md_end(c, dt, gamma, seed ^ (r << 32)); });
}

// a context's chemistry changed (cr_set_pH, cr_set_invocation): its copy in
// the batch follows (the per-site constants are the context's own array)
static int batch_refresh_chem(cr_batch *b) {
  bool changed = false;
  const int n = (int)b->ctx.size();
  for (int r = 0; r < n; ++r)
    if (b->chem_seen[r] != b->ctx[r]->chem_version) {
      const SysParams &Pc = b->ctx[r]->P;
      SysParams &Pb = b->reps[r];
      Pb.lnsalt_fx = Pc.lnsalt_fx;
      Pb.n_react = Pc.n_react;
      for (int i = 0; i < 3; ++i) Pb.react[i] = Pc.react[i];
      Pb.kxp = Pc.kxp;
      Pb.kxm = Pc.kxm;
      Pb.txp = Pc.txp;
      Pb.txm = Pc.txm;
      b->chem_seen[r] = b->ctx[r]->chem_version;
      changed = true;
    }
  if (changed)
    CR_CUDA(cudaMemcpyAsync(b->d_reps, b->reps.data(), sizeof(SysParams) * n, cudaMemcpyHostToDevice,
                            b->ctx[0]->stream));
  return CR_OK;
}

// Capture one cycle of every replica -- MD begin (kick, drift, cell
// rebuild), one sweep with the tuned launch form, MD end (forces with the
// new charges, closing kick), step advance -- as a CUDA graph whose kernels
// read the step's seeds and counters from b->d_dyn.  ff: the step opens with
// a force evaluation (forces stale, e.g. after a load), as cr_md_begin does
// call by call; its closing evaluation then counts one further.  The
// contexts' host-side counters are left as they were (the caller advances
// them per launch).
static int batch_capture_cycle(cr_batch *b, double dt, double gamma, bool da, bool ff) {
  cr_ctx *c0 = b->ctx[0];
  const int n = (int)b->ctx.size();
  // captured on the batch's own stream (the caller's may be the legacy
  // default stream, which cannot be captured); launched on the caller's
  if (!b->cstream && cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking) != cudaSuccess) return CR_ERR_CUDA;
  const cudaStream_t user = c0->stream;
  for (cr_ctx *c : b->ctx) c->stream = b->cstream;
  cudaStream_t s = b->cstream;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  c0->ev_reserved = 0;
  if (!c0->ev_pairs[0].empty() || !c0->ev_pairs[1].empty()) tcollect(c0);
  std::vector<uint64_t> sweeps(n);
  std::vector<uint32_t> evals(n);
  std::vector<int64_t> launches(n);
  std::vector<char> fvalid(n);
  for (int r = 0; r < n; ++r) {
    sweeps[r] = b->ctx[r]->sweep;
    evals[r] = b->ctx[r]->md_eval;
    launches[r] = b->ctx[r]->launches_total;
    fvalid[r] = b->ctx[r]->f_valid ? 1 : 0;
  }
  const int T = da ? b->da_T : b->T, R = da ? b->da_R : b->R;
  const bool C = da ? b->da_C : b->C, pers = da ? b->da_persistent : b->persistent;
  const PhaseShape &SS = C ? b->Sc : b->S;
  const StepDyn *dyn = b->d_dyn;
  int rc = CR_OK;
  while (c0->ev_pool.size() < c0->ev_next + 2 * (size_t)(b->ncol + 2)) {  // no event creation while capturing
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (cr_ctx *c : b->ctx) c->stream = user;
      return CR_ERR_CUDA;
    }
    c0->ev_pool.push_back(e);
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    for (cr_ctx *c : b->ctx) c->stream = user;
    return CR_ERR_CUDA;
  }
  {
    if (ff) rc = batch_md(b, [&](cr_ctx *c, uint64_t r) { return md_first_impl(c, dt, gamma, dyn, (unsigned)r); });
    if (rc == CR_OK) rc = batch_md(b, [&](cr_ctx *c, uint64_t) { return cr_md_begin(c, dt, gamma, 0); });
    if (rc == CR_OK && b->order_nc > 0) {
      if (launch_domain_order(b->d_reps, n, b->ncol, b->order_nact, s, 0, 0, 0, dyn) != cudaSuccess) rc = CR_ERR_CUDA;
      c0->launches_total++;
    }
    if (rc == CR_OK) {
      if (pers) {
        rc = batch_launch_persistent(b, SS, T, R, da, 0, 0, 0, 0, -1, 2000000000ull, dyn);
      } else {
        for (int col = 0; col < b->ncol && rc == CR_OK; ++col) {
          int ti;
          tbegin(c0, 0, &ti);
          if (launch_phase(b->d_reps, n, b->grid_x, SS, T, R, false, da, s, 0, 0, col, 0, 0, dyn) != cudaSuccess)
            rc = CR_ERR_CUDA;
          tend(c0, 0, ti);
          c0->launches_total++;
        }
      }
    }
    if (rc == CR_OK)
      rc = batch_md(b, [&](cr_ctx *c, uint64_t r) {
        return md_end_impl(c, dt, gamma, 0, dyn, (unsigned)r, ff ? 1 : 0);
      });
    if (rc == CR_OK && launch_step_advance(b->d_dyn, s) != cudaSuccess) rc = CR_ERR_CUDA;
    c0->launches_total++;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s, &g);
  if (rc == CR_OK && ec != cudaSuccess) rc = CR_ERR_CUDA;
  if (rc == CR_OK && cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
    b->graph = nullptr;
    rc = CR_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  // the phase-kernel events the graph records, and the kernels it launches
  b->g_pairs = c0->ev_pairs[0];
  c0->ev_pairs[0].clear();
  c0->ev_pairs[1].clear();
  c0->ev_reserved = c0->ev_next;
  int64_t kernels = 0;
  for (int r = 0; r < n; ++r) {
    kernels += b->ctx[r]->launches_total - launches[r];
    b->ctx[r]->launches_total = launches[r];
    b->ctx[r]->sweep = sweeps[r];
    b->ctx[r]->md_eval = evals[r];
    b->ctx[r]->f_valid = fvalid[r] != 0;
    b->ctx[r]->fcons_valid = false;
  }
  for (cr_ctx *c : b->ctx) c->stream = user;
  b->g_ff = ff;
  b->g_kernels = kernels;
  b->g_dt = dt;
  b->g_gamma = gamma;
  b->g_T = T;
  b->g_R = R;
  b->g_C = C;
  b->g_pers = pers;
  b->g_fine = b->fine;
  b->g_da = da ? 1 : 0;
  b->g_timing = c0->timing;
  return rc;
}

extern "C" int cr_batch_cycle(cr_batch *b, int32_t n_steps, double dt, double gamma, uint64_t sweep_seed0,
                              uint64_t md_seed0, int32_t da) {
  if (!b || n_steps < 0 || !(dt > 0.0) || !(gamma >= 0.0)) return CR_ERR_INVALID_ARG;
  for (cr_ctx *c : b->ctx)
    if (c->P.ewald_nk > 0) return CR_ERR_INVALID_ARG;  // the captured cycle has no S(k) nodes
  cr_ctx *c0 = b->ctx[0];
  cudaStream_t s = c0->stream;
  if (da)
    for (cr_ctx *c : b->ctx)
      if (!c->has_mlp) return CR_ERR_INVALID_ARG;
  // a step runs from the graph once the tuner has finished and the replicas'
  // counters agree: the step's own graph when every replica holds the forces
  // of a completed step, the graph that evaluates them first when none does
  // (a step after a load); otherwise steps run call by call
  auto graphable = [&](bool forces) {
    if (da ? b->da_tuning : b->tuning) return false;
    for (cr_ctx *c : b->ctx)
      if (c->f_valid != forces || c->md_eval != c0->md_eval || c->sweep != c0->sweep || c->stream != s) return false;
    return true;
  };
  int step = 0;
  int rc = CR_OK;
  const bool ff = graphable(false);
  if (!ff) {
    for (; step < n_steps && !graphable(true); ++step) {
      if ((rc = cr_batch_md_begin(b, dt, gamma, md_seed0 + (uint64_t)step)) != CR_OK) return rc;
      if ((rc = batch_sweep_impl(b, 1, sweep_seed0 + (uint64_t)step, da != 0)) != CR_OK) return rc;
      if ((rc = cr_batch_md_end(b, dt, gamma, md_seed0 + (uint64_t)step)) != CR_OK) return rc;
    }
  }
  if (step == n_steps) return CR_OK;
  if ((rc = batch_refresh_chem(b)) != CR_OK) return rc;
  if (da) {  // the surrogates' device copies
    bool changed = false;
    for (size_t r = 0; r < b->ctx.size(); ++r)
      if (b->reps[r].mlp_w != b->ctx[r]->P.mlp_w || b->reps[r].mlp_b != b->ctx[r]->P.mlp_b) {
        b->reps[r].mlp_w = b->ctx[r]->P.mlp_w;
        b->reps[r].mlp_b = b->ctx[r]->P.mlp_b;
        changed = true;
      }
    if (changed)
      CR_CUDA(cudaMemcpyAsync(b->d_reps, b->reps.data(), sizeof(SysParams) * b->ctx.size(), cudaMemcpyHostToDevice, s));
  }
  if (!b->d_dyn) CR_CUDA(cudaMalloc((void **)&b->d_dyn, sizeof(StepDyn)));
  const int T = da ? b->da_T : b->T, R = da ? b->da_R : b->R;
  const bool C = da ? b->da_C : b->C, pers = da ? b->da_persistent : b->persistent;
  while (step < n_steps) {
    const bool first = ff && step == 0;  // only a call's first step can have stale forces
    if (!b->graph || b->g_dt != dt || b->g_gamma != gamma || b->g_T != T || b->g_R != R || b->g_C != C ||
        b->g_pers != pers || b->g_fine != b->fine || b->g_da != (da ? 1 : 0) || b->g_timing != c0->timing ||
        b->g_ff != first) {
      if ((rc = batch_capture_cycle(b, dt, gamma, da != 0, first)) != CR_OK) return rc;
    }
    // this call's seeds and counters (a pageable source: staged before the call returns)
    StepDyn d{};
    d.step = 0;
    d.sweep_seed0 = sweep_seed0 + (uint64_t)step;
    d.md_seed0 = md_seed0 + (uint64_t)step;
    d.sweep0 = (uint32_t)c0->sweep;
    d.eval0 = c0->md_eval;
    CR_CUDA(cudaMemcpyAsync(b->d_dyn, &d, sizeof(StepDyn), cudaMemcpyHostToDevice, s));
    for (; step < n_steps; ++step) {
      CR_CUDA(cudaGraphLaunch(b->graph, s));
      for (cr_ctx *c : b->ctx) {
        c->sweep++;
        c->md_eval += first ? 2 : 1;
        c->f_valid = true;
        c->fcons_valid = false;
      }
      c0->launches_total += b->g_kernels;
      if (c0->timing) {  // the phase kernels' event pairs of this launch
        CR_CUDA(cudaStreamSynchronize(s));
        for (auto &pr : b->g_pairs) {
          float ms = 0.0f;
          if (cudaEventElapsedTime(&ms, c0->ev_pool[pr.first], c0->ev_pool[pr.second]) == cudaSuccess) c0->ms[0] += ms;
          c0->launches[0]++;
        }
      }
      if (first) {  // the following steps use the step's own graph
        ++step;
        break;
      }
    }
  }
  return CR_OK;
}

extern "C" int cr_batch_load(cr_batch *b, const cr_load_args *args) {
  if (!b || !args) return CR_ERR_INVALID_ARG;
  return batch_md(b, [&](cr_ctx *c, uint64_t r) {
    const cr_load_args &a = args[r];
    return cr_load(c, a.n, a.xyz, a.vel, a.type, a.cls, a.state);
  });
}

// cr_state of every replica: the halves of all replicas run on the
// replicas' streams, two synchronisations in all
extern "C" int cr_batch_state(cr_batch *b, cr_state_view *views) {
  if (!b || !views) return CR_ERR_INVALID_ARG;
  const size_t n = b->ctx.size();
  cudaStream_t s = b->ctx[0]->stream;
  CR_CUDA(cudaEventRecord(b->fork, s));
  std::vector<StateBufs> B(n);
  std::vector<char> want(n, 0);
  int rc = CR_OK;
  for (size_t r = 0; r < n; ++r) {
    CR_CUDA(cudaStreamWaitEvent(b->streams[r], b->fork, 0));
    bool w = false;
    const int e = state_begin(b->ctx[r], &views[r], b->streams[r], B[r], w);
    want[r] = w;
    if (e != CR_OK) return e;
  }
  for (size_t r = 0; r < n; ++r) CR_CUDA(cudaStreamSynchronize(b->streams[r]));
  for (size_t r = 0; r < n; ++r) {
    const int e = state_arrays(b->ctx[r], &views[r], b->streams[r], B[r], want[r] != 0);
    if (e != CR_OK && rc == CR_OK) rc = e;
  }
  for (size_t r = 0; r < n; ++r) CR_CUDA(cudaStreamSynchronize(b->streams[r]));
  return rc;
}

extern "C" int cr_batch_state_packed(cr_batch *b, cr_batch_packed *p) {
  if (!b || !p || !p->n) return CR_ERR_INVALID_ARG;
  const size_t R = b->ctx.size();
  int64_t capmax = 0;
  int max_slots = 0;
  for (cr_ctx *c : b->ctx) {
    capmax = std::max<int64_t>(capmax, c->capacity);
    max_slots = std::max(max_slots, c->P.ncell * c->P.cap);
  }
  if (p->stride < capmax) return CR_ERR_INVALID_ARG;
  const int64_t S = p->stride;
  // the view of replica r in the packed arrays (the per-context read of a
  // replica whose ion list is beyond the batched ranking)
  auto view_of = [&](size_t r) {
    cr_state_view v{};
    v.xyz = p->xyz ? p->xyz + 3 * r * S : nullptr;
    v.vel = p->vel ? p->vel + 3 * r * S : nullptr;
    v.id = p->id ? p->id + r * S : nullptr;
    v.type = p->type ? p->type + r * S : nullptr;
    v.state = p->state ? p->state + r * S : nullptr;
    v.cls = p->cls ? p->cls + r * S : nullptr;
    return v;
  };
  int rc = ensure_packed(b, S);
  if (rc != CR_OK) return rc;
  cudaStream_t s = b->ctx[0]->stream;
  // host arrays the GPU can address (pinned memory) are written in place by
  // the ordering kernel, whose threads write consecutive entries; the others
  // go through the device staging and one bulk copy per array
  float *zx = device_view(p->xyz), *zv = device_view(p->vel);
  uint64_t *zi = device_view(p->id);
  int32_t *zt = device_view(p->type), *zc = device_view(p->cls);
  int8_t *zs = device_view(p->state);
  for (size_t r = 0; r < R; ++r) {
    cr_ctx *c = b->ctx[r];
    StateBufs &B = b->h_sbufs[r];
    B = StateBufs{};
    B.n_input = c->n_input;
    B.cap = (int)c->capacity;
    B.lo_bits = c->ion_lo_bits;
    B.present = c->d_present;
    B.n_ions = c->d_counter;
    B.ion_key = c->d_ion_key;
    B.ion_val = c->d_ion_val;
    B.ion_rank = c->d_ion_rank;
    B.vel_src = c->d_vel;
    B.counts = c->d_counts;
    B.n_other = c->n_other;
    B.end_bit = ion_end_bit(c);
    B.xyz = p->xyz ? (zx ? zx : b->d_pk_xyz) + 3 * r * S : nullptr;
    B.vel = p->vel ? (zv ? zv : b->d_pk_vel) + 3 * r * S : nullptr;
    B.id = p->id ? (zi ? (unsigned long long *)zi : b->d_pk_id) + r * S : nullptr;
    B.type = p->type ? (zt ? zt : b->d_pk_type) + r * S : nullptr;
    B.cls = p->cls ? (zc ? zc : b->d_pk_cls) + r * S : nullptr;
    B.state = p->state ? (zs ? zs : b->d_pk_state) + r * S : nullptr;
  }
  CR_CUDA(cudaMemcpyAsync(b->d_sbufs, b->h_sbufs, R * sizeof(StateBufs), cudaMemcpyHostToDevice, s));
  CR_CUDA(launch_state_batch(b->d_reps, b->d_sbufs, (int)R, max_slots, (int)capmax, b->d_nout, b->d_errout, s));
  b->ctx[0]->launches_total += 3;
  CR_CUDA(cudaMemcpyAsync(b->h_nout, b->d_nout, R * sizeof(long long), cudaMemcpyDeviceToHost, s));
  int *herr = (int *)(b->h_nout + R);
  CR_CUDA(cudaMemcpyAsync(herr, b->d_errout, R * sizeof(int), cudaMemcpyDeviceToHost, s));
  const size_t m = R * (size_t)S;
  if (p->xyz && !zx) CR_CUDA(cudaMemcpyAsync(p->xyz, b->d_pk_xyz, 3 * m * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (p->vel && !zv) CR_CUDA(cudaMemcpyAsync(p->vel, b->d_pk_vel, 3 * m * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (p->id && !zi) CR_CUDA(cudaMemcpyAsync(p->id, b->d_pk_id, m * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  if (p->type && !zt) CR_CUDA(cudaMemcpyAsync(p->type, b->d_pk_type, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (p->cls && !zc) CR_CUDA(cudaMemcpyAsync(p->cls, b->d_pk_cls, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (p->state && !zs) CR_CUDA(cudaMemcpyAsync(p->state, b->d_pk_state, m, cudaMemcpyDeviceToHost, s));
  CR_CUDA(cudaStreamSynchronize(s));
  rc = CR_OK;
  for (size_t r = 0; r < R; ++r) {
    p->n[r] = b->h_nout[r];
    const int e = err_bits_to_code(herr[r]);
    if (rc == CR_OK && e != CR_OK) rc = e;
    if (rc == CR_OK && b->h_nout[r] < 0) {  // more ions than the batched ranking takes: read it by itself
      cr_state_view v = view_of(r);
      rc = cr_state(b->ctx[r], &v);
      p->n[r] = v.n;
    }
  }
  return rc;
}

extern "C" int cr_batch_load_packed(cr_batch *b, const cr_batch_packed *p) {
  if (!b || !p || !p->n || !p->xyz || !p->type || !p->cls || !p->state) return CR_ERR_INVALID_ARG;
  const size_t R = b->ctx.size();
  int64_t capmax = 0, max_n = 0;
  int max_cells = 0;
  for (size_t r = 0; r < R; ++r) {
    cr_ctx *c = b->ctx[r];
    if (p->n[r] < c->n_fixed_end || p->n[r] > c->capacity) return CR_ERR_INVALID_ARG;
    capmax = std::max<int64_t>(capmax, c->capacity);
    max_n = std::max<int64_t>(max_n, p->n[r]);
    max_cells = std::max(max_cells, c->P.ncell);
  }
  if (p->stride < capmax) return CR_ERR_INVALID_ARG;
  const int64_t S = p->stride;
  int rc = ensure_packed(b, S);
  if (rc != CR_OK) return rc;
  cudaStream_t s = b->ctx[0]->stream;
  const size_t m = R * (size_t)S;
  // arrays the GPU can address are read in place; the others are staged
  const float *zx = device_view(p->xyz), *zv = device_view(p->vel);
  const int32_t *zt = device_view(p->type), *zc = device_view(p->cls);
  const int8_t *zs = device_view(p->state);
  if (!zx) CR_CUDA(cudaMemcpyAsync(b->d_pk_xyz, p->xyz, 3 * m * sizeof(float), cudaMemcpyHostToDevice, s));
  if (p->vel && !zv) CR_CUDA(cudaMemcpyAsync(b->d_pk_vel, p->vel, 3 * m * sizeof(float), cudaMemcpyHostToDevice, s));
  if (!zt) CR_CUDA(cudaMemcpyAsync(b->d_pk_type, p->type, m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (!zc) CR_CUDA(cudaMemcpyAsync(b->d_pk_cls, p->cls, m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (!zs) CR_CUDA(cudaMemcpyAsync(b->d_pk_state, p->state, m, cudaMemcpyHostToDevice, s));
  const float *ix = zx ? zx : b->d_pk_xyz, *iv = p->vel ? (zv ? zv : b->d_pk_vel) : nullptr;
  const int32_t *it = zt ? zt : b->d_pk_type, *ic = zc ? zc : b->d_pk_cls;
  const int8_t *is = zs ? zs : b->d_pk_state;
  for (size_t r = 0; r < R; ++r) {
    cr_ctx *c = b->ctx[r];
    LoadJob &J = b->h_jobs[r];
    J.I = LoadBufs{ix + 3 * r * S, iv ? iv + 3 * r * S : nullptr, it + r * S, ic + r * S, c->d_site_map,
                   is + r * S, (int)p->n[r], c->n_input, c->d_init_type};
    J.B = RebuildBufs{c->d_cnt2, c->d_pos2, c->d_pid2, c->d_info2, c->d_vel2, c->d_frc2, c->d_vel, c->d_frc};
    J.perm_slot = c->d_perm;
    J.n_perm = c->n_input;
    c->f_valid = false;
    c->fcons_valid = false;
  }
  CR_CUDA(cudaMemcpyAsync(b->d_jobs, b->h_jobs, R * sizeof(LoadJob), cudaMemcpyHostToDevice, s));
  CR_CUDA(launch_load_batch(b->d_reps, b->d_jobs, (int)R, (int)max_n, max_cells, s));
  b->ctx[0]->launches_total += 4;
  return CR_OK;
}

extern "C" int cr_batch_set_launch_shape(cr_batch *b, int32_t threads, int32_t regs) {
  if (!b) return CR_ERR_INVALID_ARG;
  if (threads == 0) {  // re-enable tuning
    b->tuning = b->da_tuning = true;
    b->tune_next = b->da_next = 0;
    return CR_OK;
  }
  if (b->pmode < 0) b->persistent = b->da_persistent = false;  // a fixed shape without a fixed mode: per colour
  bool found = false;
  for (int da = 0; da < 2; ++da)
    for (int i = 0; i < phase_shape_count(da != 0); ++i) {
      int t, r;
      phase_shape(i, &t, &r, da != 0);
      if (t != threads || r != regs || phase_shape_smem(b->S, t, r, da != 0) > (size_t)b->smem_max) continue;
      if (da) {
        b->da_T = t;
        b->da_R = r;
        b->da_C = false;
        b->da_tuning = false;
      } else {
        b->T = t;
        b->R = r;
        b->C = false;
        b->tuning = false;
      }
      found = true;
    }
  return found ? CR_OK : CR_ERR_INVALID_ARG;
}

extern "C" int cr_batch_get_launch_shape(const cr_batch *b, int32_t *threads, int32_t *regs) {
  if (!b || !threads || !regs) return CR_ERR_INVALID_ARG;
  *threads = b->T;
  *regs = b->R;
  return CR_OK;
}

// ---------------------------------------------------------------------------
// context access for the allocation-free force entry point (crmc_noalloc.cu):
// the force evaluation of cr_md_forces with the particle-list scratch and the
// slot-indexed force output supplied by the caller; the context's own force
// buffers and its validity flags are left alone.
// ---------------------------------------------------------------------------
namespace crmc {

int ctx_md_forces_into(cr_ctx *ctx, float4 *fout, int *plist, int *n_particles, int max_particles) {
  if (ctx->P.ewald_nk > 0) return CR_ERR_INVALID_ARG;  // no S(k) scratch here: DSF forces only
  MdParams M = md_params(ctx, 0, 0.0, 0.0, 0);
  M.fout = fout;
  CR_CUDA(launch_md_forces(ctx->P, M, plist, n_particles, max_particles, ctx->stream));
  ctx->launches_total += 2;
  return CR_OK;
}

const SysParams &ctx_params(const cr_ctx *ctx) { return ctx->P; }
cudaStream_t ctx_stream(const cr_ctx *ctx) { return ctx->stream; }
int64_t ctx_capacity(const cr_ctx *ctx) { return ctx->capacity; }
int ctx_device(const cr_ctx *ctx) { return ctx->device; }
void ctx_count_launch(cr_ctx *ctx) { ctx->launches_total++; }

}  // namespace crmc
