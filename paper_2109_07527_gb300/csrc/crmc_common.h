// crmc_common.h -- data layout and kernel parameter records shared by the
// host side (crmc_api.cu) and the kernels (crmc_kernels.cu) of libcrmc.so.
//
// Device layout of one system (cell-major, "slots"):
//   cnt[ncell]                 used slots of each cell (particles sorted by id)
//   pos[ncell * cap]  float4   x, y, z, effective charge
//   pid[ncell * cap]  u64      particle id (input index; inserted ions >= 2^32)
//   info[ncell * cap] i32      type | cls << 4 | ionised << 6 | site index << 8
//   vel, frc[ncell * cap]      MD velocity and total force (float4)
// A cell's particles occupy slots [c*cap, c*cap + cnt[c]) in ascending id.
#pragma once
#include <cstdint>

#include "crmc.h"

namespace crmc {

// kinds of slots: site states, the grouped ions X+- and the salt ions S+-
// kept apart from them (grand-reaction invocations); K_OTHER is never counted
enum Kind { K_A0 = 0, K_A1 = 1, K_B0 = 2, K_B1 = 3, K_XP = 4, K_XM = 5, K_SP = 6, K_SM = 7, K_OTHER = 8 };
constexpr int N_KIND = 8;  // counted kinds
// per-CTA counters of a phase: [0] list size, [1 + kind] kind counts (kinds
// 0..K_OTHER), [MISC_INIT + kind] the counted kinds' values at the start
constexpr int MISC_INIT = 10, MISC_N = 20;
enum Reaction { R_ACID = 0, R_BASE = 1, R_SALT = 2 };
// free monovalent ions: the grouped X+- and the salt ions S+- (same interactions)
__host__ __device__ inline bool is_ion_type(int t) { return t == CR_XP || t == CR_XM || t == CR_SP || t == CR_SM; }
__host__ __device__ inline int ion_sign(int t) { return (t == CR_XP || t == CR_SP) ? 1 : -1; }

constexpr int INFO_TYPE_MASK = 15;
constexpr int INFO_CLS_SHIFT = 4;
constexpr int INFO_ION_BIT = 1 << 6;
constexpr int INFO_SITE_SHIFT = 8;
constexpr int MAX_SITES = 1 << 23;
constexpr int TRIAL_CHUNK = 32;   // trials whose random numbers are drawn at once
constexpr int MAX_REGION_CELLS = 512;
constexpr float BIG_TERM = 1048576.0f;  // 2^20 kT: larger pair changes count as overlaps
constexpr float FIX_SCALE = 4294967296.0f;  // fixed-point scale 2^32 of the energy sums
constexpr double FIX_INV = 1.0 / 4294967296.0;
// The Metropolis exponent lnA is summed in 64-bit fixed point with scale 2^48
// (integer adds, no FP64 on the trial's critical path).  |dE| is clamped at
// 2^14 kT, where the decision no longer depends on it (ln u >= -37).
constexpr double LNFIX = 281474976710656.0;  // 2^48
constexpr long long DE_CLAMP32 = 1ll << 46;  // 2^14 kT at scale 2^32
// an FP32 ln u decides directly when it is farther than this from lnA
// (1e-4 at scale 2^48); inside the band ln u is recomputed in FP64
constexpr long long LNU_BAND = 28147497671ll;

struct WcaEntry {
  float eps, sig, del, wcut2;  // FP32 (MD forces, range pre-check)
  int on;
  double eps_d, sig_d, del_d, wcut_d;  // FP64 (WCA changes of inserted / deleted ions)
};

// Everything a phase (or MD) kernel needs about one system (one replica).
// The phase kernel reads it from a device array (one entry per replica);
// the MD kernels take it by value.
struct SysParams {
  // geometry
  int nc, k, h, nd, ncol, m, cap, global, nr, ncell;
  int nact;             // active domains per colour phase
  float Lf, invL, scf, halfL;  // box, 1/box, cells per unit length (FP32, decides cells), L/2
  double Ld, halfLd;
  double a;             // cell side in FP64
  float af;             // cell side in FP32 (insertion coordinates)
  // energy, FP32 pair constants
  float rc2, rcf, alpha, c1, c2, lBf;
  double lB_self;       // lB * DSF self coefficient (0 when off)
  WcaEntry wca[16];
  int ion_cls;          // class of inserted ions (CR_CLS_NONE for ghosts)
  float ion_q;          // |effective charge| of inserted ions (0 for ghosts)
  // chemistry (log form, fixed point 2^-48)
  long long lnz1_fx, lnsalt_fx, lBself_fx;
  int n_react;
  int react[3];
  // the invocation: kinds and types of the cation and anion that the
  // reactions exchange with the reservoir (K_XP / CR_XP or K_SP / CR_SP, and
  // K_XM / CR_XM or K_SM / CR_SM)
  int kxp, kxm, txp, txm;
  const long long *lnK_fx;    // per site
  const long long *lntab_fx;  // ln(i) for 0 < i < lnmax
  int lnmax;
  uint32_t key_xor;     // XOR-ed into the high Philox key word (replica index)
  // state
  int *cnt;
  float4 *pos, *vel;
  unsigned long long *pid;
  int *info;
  int *perm_slot;  // slot of each permanent particle (bonded partners)
  int n_perm;
  // domain lists that do not fit in shared memory (one region per CTA of a phase)
  float4 *gs_pos, *gs_vel;
  unsigned long long *gs_id;
  long long *gs_lnk;
  int *gs_info, *gs_rank;
  int dcap_glob;        // entries per CTA region (k^3 * cap + 2 m)
  // bookkeeping
  unsigned long long *stats;  // [16]: attempts[6], accepts[6], no-elig, edge, overlap, trials
  long long *counts;          // [N_KIND] global counts per kind K_A0..K_SM
  int *err;                   // error bits
  cr_trial *log;              // trial records (device) or null
  long long per_sweep;        // trials per sweep (log indexing)
  // delayed acceptance: surrogate weights (BF16, transposed: W1T [48][128],
  // W2T, W3T [128][128], w4 [128]), biases (b1, b2, b3, b4), records
  const uint16_t *mlp_w;
  const float *mlp_b;
  cr_trial_da *dlog;          // DA records (device) or null
  float *feat_log;            // 48 features per trial (device) or null
  // launch order of each colour's domains, largest region first (ncol x nact),
  // or null for the natural order
  int *order;
  // Ewald electrostatics (ewald_nk > 0, global schedule): the reciprocal
  // vectors n of one half space (three signed bytes each; S(-k) is the
  // conjugate of S(k), so -k adds the same term) with their weights
  // 2 A_k = 2 (2 pi lB / V) exp(-k^2 / (4 alpha^2)) / k^2 (FP32), and S(k) of
  // the state as an unevaluated sum hi + lo of two FP32 complex numbers
  // (about 48 bits; the trials read hi)
  int ewald_nk, ewald_kmax;
  const int2 *ek_nA;  // (n code, weight bits) of each reciprocal vector
  float2 *ek_Shi, *ek_Slo;
  double invLd;  // 1 / L in FP64
  int *ek_list, *ek_np;  // occupied slots (the structure-factor kernel's particle list) and their number
  int ek_cap;            // entries of ek_list (the capacity in particles)
};

// domains are launched densest first for colours of at most this many domains
constexpr int ORDER_MAX_NACT = 4096;

// surrogate MLP sizes and the offsets of its parts in mlp_w / mlp_b
constexpr int MLP_IN = 48;
constexpr int MLP_H = 128;
constexpr int MLPW_W1 = 0;
constexpr int MLPW_W2 = MLP_IN * MLP_H;
constexpr int MLPW_W3 = MLPW_W2 + MLP_H * MLP_H;
constexpr int MLPW_W4 = MLPW_W3 + MLP_H * MLP_H;
constexpr int MLPW_N = MLPW_W4 + MLP_H;
constexpr int MLPB_N = 3 * MLP_H + 1;

// Launch-wide shared-memory shape of a phase launch (the same for every CTA;
// the maximum over the replicas of a batch).
struct PhaseShape {
  int dcs;     // domain-list entries held in shared memory
  int hcs;     // halo particles held in shared memory (shapes without halo registers)
  int lns;     // log-table entries held in shared memory
  int nr3;     // region cells
  int kc3;     // domain cells
  int chunk;   // trials whose random numbers are drawn at once (min(m, TRIAL_CHUNK))
  int ewk;     // Ewald: kmax + 1 phase factors per axis and changed particle (0 without Ewald)
};

// error bits in *err
constexpr int ERRB_CELL_OVERFLOW = 1;
constexpr int ERRB_CAPACITY = 2;
constexpr int ERRB_BOND = 4;
constexpr int ERRB_TIMEOUT = 8;
constexpr int ERRB_ARG = 16;
constexpr int ERRB_NOT_NEUTRAL = 32;

}  // namespace crmc
