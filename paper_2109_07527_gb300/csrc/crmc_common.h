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

enum Kind { K_A0 = 0, K_A1 = 1, K_B0 = 2, K_B1 = 3, K_XP = 4, K_XM = 5, K_OTHER = 6 };
enum Reaction { R_ACID = 0, R_BASE = 1, R_SALT = 2 };

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

struct WcaEntry {
  float eps, sig, del, wcut2;  // FP32 (MD forces, range pre-check)
  int on;
  double eps_d, sig_d, del_d, wcut_d;  // FP64 (WCA changes of inserted / deleted ions)
};

// Everything a phase (or MD) kernel needs, passed by value.
struct SysParams {
  // geometry
  int nc, k, h, nd, ncol, m, cap, global, nr, ncell;
  float Lf, invL, scf, halfL;  // box, 1/box, cells per unit length (FP32, decides cells), L/2
  double Ld, halfLd;
  double a;             // cell side in FP64 (insertion coordinates)
  // energy, FP32 pair constants
  float rc2, rcf, alpha, c1, c2, lBf;
  double lB_self;       // lB * DSF self coefficient (0 when off)
  WcaEntry wca[16];
  int ion_cls;          // class of inserted ions (CR_CLS_NONE for ghosts)
  float ion_q;          // |effective charge| of inserted ions (0 for ghosts)
  // chemistry (log form, FP64)
  double ln_z1, ln_salt;
  int n_react;
  int react[3];
  const double *lnK;    // per site
  const double *lntab;  // ln(i) for 0 < i < lnmax
  int lnmax;
  // state
  int *cnt;
  float4 *pos, *vel;
  unsigned long long *pid;
  int *info;
  int *perm_slot;  // slot of each permanent particle (bonded partners)
  int n_perm;
  // bookkeeping
  unsigned long long *stats;  // [16]: attempts[6], accepts[6], no-elig, edge, overlap, trials
  long long *counts;          // [6] global counts per kind K_A0..K_XM
  int *err;                   // error bits
  cr_trial *log;              // trial records (device) or null
  long long log_base;
  int dcap;                   // capacity of the domain list in shared memory
};

// error bits in *err
constexpr int ERRB_CELL_OVERFLOW = 1;
constexpr int ERRB_CAPACITY = 2;
constexpr int ERRB_BOND = 4;
constexpr int ERRB_TIMEOUT = 8;
constexpr int ERRB_ARG = 16;

}  // namespace crmc
