/*
 * crmc_oracle.c -- plain, slow, FP64 CPU oracle for the charge-regulation
 * Monte Carlo (CR-MC) stage of the hybrid MD/CR-MC method of Curk, Yuan and
 * Luijten (arXiv:2109.07527), plus the MD forces and the Langevin
 * velocity-Verlet step that consume the regulated charges.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or constant generator with the CUDA path; it is compiled separately
 * with plain gcc (-O2 -ffp-contract=off, no fast-math).
 *
 * What it follows (sections / equations of the paper):
 *   - Sec. II.B, Eqs. (acid_new)-(salt_new): three generalised reactions
 *     A <-> A- + X+,  B <-> B+ + X-,  0 <-> X+ + X-.
 *   - Sec. II.C: six moves (forward/reverse of each reaction) proposed with
 *     equal probability; participants drawn uniformly among the eligible
 *     particles; no eligible particle -> automatic rejection.
 *   - Sec. II.C, Eq. (QQ) and the acceptance rules Eqs. (acidacc), (MCmetro),
 *     the base pair, (MCsaltf), (MCmetro2), written in log form.
 *   - App. C, Eq. (pIXgen): 10^-pI_X = 10^-pI_S + 10^-min(pH, pOH).
 *   - Eq. (LJe)/(LJ): WCA with an optional expanded distance Delta.
 *   - Sec. III.A: velocity Verlet with a Langevin thermostat; Sec. IV.B: the
 *     nanoparticles carry their sites rigidly (rigid bodies, see
 *     or_set_bodies).
 * Readings where the paper is silent:
 *   - The energy model is a damped-shifted-force (DSF) Coulomb cutoff sum plus
 *     WCA (the paper uses PPPM), with the DSF self term; or, under the global
 *     schedule, the Ewald sum that PPPM evaluates on a mesh (real-space erfc
 *     within rc, reciprocal vectors 0 < |n| <= kmax, self term), S(k)
 *     recomputed at every sweep and carried by the accepted trials within it;
 *     the MD forces are minus the gradient of the same energy.
 *   - Rigid bodies: unit mass per member, the principal frame, the symmetric
 *     rotation splitting of Dullweber, Leimkuhler and McLachlan, and the
 *     Langevin thermostat acting on each body as a whole.
 *   - Moves are domain-local under an 8-colour checkerboard schedule: the
 *     paired ion is inserted in / deleted from the trial's domain, and the
 *     acceptance uses that domain's volume and counts.  The "global" schedule
 *     (one domain = the whole box) is the paper's rule verbatim.
 *   - pKw = 14 unless given; rho0 = 1 M; rho0*N_A = 0.602214076 nm^-3.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with the counter
 *     layout documented at or_trial().
 *
 * Parity pins for every function are in tests/test_oracle_*.py (closed forms,
 * exact enumeration, flux symmetry, known-answer vectors, invariants).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NEUTRAL (-2)
#define OR_ERR_CAPACITY (-4)
#define OR_ERR_BOND (-6)
#define OR_ERR_NOMEM (-8)

/* Particle types.  T_XP / T_XM are the grouped monovalent ions X+ / X- of
 * Sec. II.B; T_SP / T_SM are salt ions kept apart from them (S+ / S-) when
 * the scheme is applied separately to dissociated and salt ions, the
 * grand-reaction ensemble of Sec. II.B and App. B.  All four interact alike
 * (charge +-1, the ions' short-range class); only the reactions tell them
 * apart. */
enum { T_BEAD = 0, T_ACID = 1, T_BASE = 2, T_XP = 3, T_XM = 4, T_CORE = 5, T_SP = 6, T_SM = 7 };
static int is_ion(int t) { return t == T_XP || t == T_XM || t == T_SP || t == T_SM; }
/* kinds of particles for the eligibility lists and counts */
enum { K_A0 = 0, K_A1 = 1, K_B0 = 2, K_B1 = 3, K_XP = 4, K_XM = 5, K_SP = 6, K_SM = 7, K_OTHER = 8, N_KIND = 9 };
enum { R_ACID = 0, R_BASE = 1, R_SALT = 2 };
enum { F_ACC = 1, F_NOELIG = 2, F_EDGE = 4, F_OVERLAP = 8 };
#define CLS_NONE 3
#define BIG_TERM 1048576.0 /* 2^20 kT: larger pair changes count as overlaps */

/* Planted mistakes, used only by the tests that show the pins catch them. */
enum { PLANT_NONE = 0, PLANT_DROP_ION_COUNT = 1, PLANT_DE_SIGN = 2,
       PLANT_DROP_SELF = 3, PLANT_DROP_PAIR_CC = 4, PLANT_WRONG_VOLUME = 5,
       PLANT_DA_ONE_SIDED = 6, PLANT_DA_STAGE2_FULL = 7, PLANT_SPECIES_COUNT = 8,
       PLANT_EWALD_HALF_RECIP = 9, PLANT_RIGID_TORQUE_SIGN = 10, PLANT_RIGID_NO_ROT_NOISE = 11,
       PLANT_EWALD_FORCE_SIGN = 12 };

/* ----------------------------------------------------------------------- */
/* Philox4x32-10: 10 rounds of the Philox S-box on a 128-bit counter with a
 * 64-bit key bumped by the Weyl constants between rounds (Salmon et al.,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11). */
static void philox(const uint32_t c_in[4], const uint32_t k_in[2], uint32_t out[4]) {
  uint32_t c0 = c_in[0], c1 = c_in[1], c2 = c_in[2], c3 = c_in[3];
  uint32_t k0 = k_in[0], k1 = k_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) { philox(ctr, key, out); }

/* integer in [0, n) from one 32-bit word: floor(w * n / 2^32) */
static int64_t pick(uint32_t w, int64_t n) { return (int64_t)(((uint64_t)w * (uint64_t)n) >> 32); }

/* uniform in (0,1) with 53 random bits from two words */
static double unif53(uint32_t whi, uint32_t wlo) {
  double a = (double)(whi >> 5), b = (double)(wlo >> 6);
  return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0);
}

/* ----------------------------------------------------------------------- */
typedef struct {
  int32_t n, capacity;
  double box_L, sigma_nm;
  double lB, rc, alpha;
  int32_t dsf_self, ion_coupling, ion_cls;
  double pH, pKw, pIS_plus, pIS_minus;
  int32_t pIX_explicit;
  double pIX_plus, pIX_minus;
  int32_t nc, domain_cells, trials_per_domain, schedule, cells_per_rc;
  double wca_eps[16], wca_sig[16], wca_del[16];
  int32_t wca_on[16];
  double fene_K, fene_R0;
  int32_t n_bonds;
  int32_t ewald_kmax; /* 0: DSF cutoff energy; > 0: Ewald sum with reciprocal vectors 0 < |n|^2 <= kmax^2 */
} or_params;

typedef struct {
  int32_t move, flags;
  uint64_t id_a, id_b;
  double dE, S, lnA, lnu;
} or_trial;

/* A rigid body (Sec. IV.B: the nanoparticles' sites are rigidly attached to
 * the shell; the body's mass is the sum of its members', one unit each): the
 * permanent particles with ids [first, first + count).  State: centre of mass
 * X (not wrapped) and its velocity V, orientation R (row-major; lab = R body,
 * the body axes the principal axes, in ascending order of the moments I),
 * angular momentum pi in the body frame; F and T are the force and the torque
 * (lab frame, Langevin terms included) of the last force evaluation; d the
 * members' offsets from X in the body frame. */
typedef struct {
  int first, count;
  double M, I[3];
  double X[3], V[3], R[9], pi[3];
  double F[3], T[3];
  double *d;
} or_body;

typedef struct {
  /* box, cells and schedule */
  double L, a;
  float Lf, scf;
  int nc, k, nd, ncol, m, global;
  /* energy model */
  double lB, rc, alpha, phi_c1, phi_c2, self_coef;
  int dsf_self, ion_coupling, ion_cls;
  double eps[4][4], sig[4][4], del[4][4], wcut[4][4];
  int on[4][4];
  /* chemistry (log form) */
  double pH, pOH, pIXp, pIXm, ln_z1, ln_salt;
  double pKw, pIS_plus, pIS_minus;
  int pIX_explicit;
  int n_sites;
  double *lnK; /* per site: ln10*(pH-pKa-pI_X+) for acids, ln10*(pOH-pKb-pI_X-) for bases */
  double *pK;  /* per site: pKa or pKb as given */
  int *site_type; /* per site: T_ACID or T_BASE */
  int react[3], n_react;
  /* the invocation: kinds (and types) of the cation and anion that the acid,
   * base and salt reactions exchange with the reservoir */
  int kxp, kxm, txp, txm;
  /* particles */
  int n, cap;
  float *x, *y, *z;
  int *type, *cls, *site, *st; /* st: 1 = ionised site */
  uint64_t *id;
  double *vx, *vy, *vz, *fx, *fy, *fz;
  int f_valid;
  /* bonds (by particle id, which is the input index for permanent particles) */
  int nb;
  int *bi, *bj;
  double K, R0;
  /* counters */
  uint64_t sweep, md_evals;
  int64_t stats[16];
  int plant;
  /* learned delayed acceptance: surrogate weights (BF16 values held as
   * floats), on when has_mlp and da are set */
  int has_mlp, da;
  float *W1, *b1, *W2, *b2, *W3, *b3, *w4, b4;
  /* Ewald electrostatics (ewald_kmax > 0): reciprocal vectors k = 2 pi n / L
   * (kn: n, 3 ints each), their weights kA = (2 pi lB / V) exp(-k^2/(4 alpha^2)) / k^2,
   * the structure factor S(k) = sum_j q_j exp(i k.r_j) of the current state and
   * the change dS of the last evaluated trial */
  int ewald_kmax, nk;
  int *kn;
  double *kA, *Sre, *Sim, *dSre, *dSim;
  /* rigid bodies (or_set_bodies); body_of: body of each permanent id, -1 none */
  int n_input, nbody;
  or_body *body;
  int *body_of;
} Oracle;

static int g_plant = PLANT_NONE;
void or_plant(int kind) { g_plant = kind; }

static const double LN10 = 2.302585092994045684;
static const double RHO0_NA = 0.602214076; /* 1 M in nm^-3 */

/* DSF pair potential (Fennell & Gezelter 2006): phi(rc) = 0 and phi'(rc) = 0. */
static double dsf_phi(const Oracle *o, double r) {
  return erfc(o->alpha * r) / r - o->phi_c1 + o->phi_c2 * (r - o->rc);
}
/* -d phi / dr */
static double dsf_force(const Oracle *o, double r) {
  double ar = o->alpha * r;
  return erfc(ar) / (r * r) + 2.0 * o->alpha / sqrt(M_PI) * exp(-ar * ar) / r - o->phi_c2;
}

/* WCA / expanded WCA, Eq. (LJe) with C = 1/4: s = r - Delta */
static double wca_u(double eps, double sig, double s) {
  double sr6 = pow(sig / s, 6.0);
  return 4.0 * eps * (sr6 * sr6 - sr6) + eps;
}
static double wca_f(double eps, double sig, double s) { /* -dU/ds */
  double sr6 = pow(sig / s, 6.0);
  return 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / s;
}

double or_dsf_phi(double alpha, double rc, double r) {
  Oracle o; memset(&o, 0, sizeof o);
  o.alpha = alpha; o.rc = rc;
  o.phi_c1 = erfc(alpha * rc) / rc;
  o.phi_c2 = erfc(alpha * rc) / (rc * rc) + 2.0 * alpha / sqrt(M_PI) * exp(-alpha * alpha * rc * rc) / rc;
  return dsf_phi(&o, r);
}
double or_dsf_force(double alpha, double rc, double r) {
  Oracle o; memset(&o, 0, sizeof o);
  o.alpha = alpha; o.rc = rc;
  o.phi_c2 = erfc(alpha * rc) / (rc * rc) + 2.0 * alpha / sqrt(M_PI) * exp(-alpha * alpha * rc * rc) / rc;
  return dsf_force(&o, r);
}
double or_wca_u(double eps, double sig, double del, double r) {
  double s = r - del;
  if (s >= pow(2.0, 1.0 / 6.0) * sig) return 0.0;
  return wca_u(eps, sig, s);
}

static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* charge that enters the energy */
static double qeff(const Oracle *o, int t, int ionised) {
  switch (t) {
    case T_ACID: return ionised ? -1.0 : 0.0;
    case T_BASE: return ionised ? 1.0 : 0.0;
    case T_XP: case T_SP: return o->ion_coupling ? 1.0 : 0.0;
    case T_XM: case T_SM: return o->ion_coupling ? -1.0 : 0.0;
    default: return 0.0;
  }
}
static int qnom(int t, int ionised) {
  switch (t) {
    case T_ACID: return ionised ? -1 : 0;
    case T_BASE: return ionised ? 1 : 0;
    case T_XP: case T_SP: return 1;
    case T_XM: case T_SM: return -1;
    default: return 0;
  }
}

/* cell of a coordinate: floor(fl32(x * (nc/L))) clamped; taken in FP32 on
 * both sides because it decides an integer (which domain owns a particle). */
static int cell_of(const Oracle *o, float x) {
  float t = x * o->scf;
  int c = (int)floorf(t);
  if (c < 0) c = 0;
  if (c >= o->nc) c = o->nc - 1;
  return c;
}

/* domain index and canonical in-domain cell rank of a position, for offset off */
static void domain_of(const Oracle *o, const int off[3], float x, float y, float z, int *dom, int *rank) {
  int c[3] = {cell_of(o, x), cell_of(o, y), cell_of(o, z)};
  int dd[3], ll[3];
  for (int i = 0; i < 3; ++i) {
    int s = ((c[i] - off[i]) % o->nc + o->nc) % o->nc;
    dd[i] = s / o->k;
    ll[i] = s % o->k;
  }
  *dom = dd[0] + o->nd * (dd[1] + o->nd * dd[2]);
  *rank = ll[0] + o->k * (ll[1] + o->k * ll[2]);
}

/* ----------------------------------------------------------------------- */
void or_destroy(Oracle *o) {
  if (!o) return;
  free(o->x); free(o->y); free(o->z); free(o->type); free(o->cls); free(o->site); free(o->st);
  free(o->id); free(o->vx); free(o->vy); free(o->vz); free(o->fx); free(o->fy); free(o->fz);
  free(o->lnK); free(o->pK); free(o->site_type); free(o->bi); free(o->bj);
  free(o->W1); free(o->b1); free(o->W2); free(o->b2); free(o->W3); free(o->b3); free(o->w4);
  free(o->kn); free(o->kA); free(o->Sre); free(o->Sim); free(o->dSre); free(o->dSim);
  for (int b = 0; b < o->nbody; ++b) free(o->body[b].d);
  free(o->body); free(o->body_of);
  free(o);
}

/* pI of the grouped ion from the salt pI and the reservoir pH, Eq. (pIXgen) */
/* ---- Ewald sum (standard form; e.g. Frenkel & Smit, Understanding Molecular
 * Simulation, ch. 12): E = E_real + E_rec + E_self with
 *   E_real = lB sum_{i<j, r < rc} q_i q_j erfc(alpha r) / r   (minimum image),
 *   E_rec  = (2 pi lB / V) sum_{k != 0} exp(-k^2 / (4 alpha^2)) / k^2 |S(k)|^2,
 *   E_self = -lB alpha / sqrt(pi) sum_i q_i^2,
 * tin-foil boundary (no surface term; every state here is neutral).  The
 * paper's energy model is PPPM (Sec. III.A), a mesh evaluation of this sum. */
static double ewald_phase(const Oracle *o, int i, double x, double y, double z) {
  const double kf = 2.0 * M_PI / o->L;
  return kf * ((double)o->kn[3 * i] * x + (double)o->kn[3 * i + 1] * y + (double)o->kn[3 * i + 2] * z);
}
/* S(k) of the current state, from scratch */
static void ewald_structure(const Oracle *o, double *re, double *im) {
  for (int i = 0; i < o->nk; ++i) {
    re[i] = 0.0;
    im[i] = 0.0;
  }
  for (int j = 0; j < o->n; ++j) {
    const double q = qeff(o, o->type[j], o->st[j]);
    if (q == 0.0) continue;
    for (int i = 0; i < o->nk; ++i) {
      const double ph = ewald_phase(o, i, o->x[j], o->y[j], o->z[j]);
      re[i] += q * cos(ph);
      im[i] += q * sin(ph);
    }
  }
}
static double ewald_recip_energy(const Oracle *o, const double *re, const double *im) {
  double E = 0.0;
  for (int i = 0; i < o->nk; ++i) E += o->kA[i] * (re[i] * re[i] + im[i] * im[i]);
  if (g_plant == PLANT_EWALD_HALF_RECIP) E *= 0.5;
  return E;
}

static double pIX_of(double pIS, double pH, double pOH) {
  double m = pH < pOH ? pH : pOH;
  return -log10(pow(10.0, -pIS) + pow(10.0, -m));
}

Oracle *or_create(const or_params *p, const float *xyz, const int32_t *type, const int32_t *cls,
                  const int8_t *state, const double *pK, const int32_t *bonds, const float *vel,
                  int32_t *err) {
  *err = OR_ERR_ARG;
  if (p->n < 0 || p->capacity < p->n || p->box_L <= 0 || p->rc <= 0) return NULL;
  Oracle *o = (Oracle *)calloc(1, sizeof(Oracle));
  if (!o) { *err = OR_ERR_NOMEM; return NULL; }
  o->Lf = (float)p->box_L;
  o->L = (double)o->Lf;
  o->lB = p->lB; o->rc = p->rc; o->alpha = p->alpha;
  o->dsf_self = p->dsf_self; o->ion_coupling = p->ion_coupling; o->ion_cls = p->ion_cls;
  if (2.0 * o->rc > o->L) { free(o); return NULL; }
  o->phi_c1 = erfc(o->alpha * o->rc) / o->rc;
  o->phi_c2 = erfc(o->alpha * o->rc) / (o->rc * o->rc) +
              2.0 * o->alpha / sqrt(M_PI) * exp(-o->alpha * o->alpha * o->rc * o->rc) / o->rc;
  o->self_coef = -(erfc(o->alpha * o->rc) / (2.0 * o->rc) + o->alpha / sqrt(M_PI));
  o->ewald_kmax = p->ewald_kmax;
  if (o->ewald_kmax < 0 || o->ewald_kmax > 64) { free(o); return NULL; }
  if (o->ewald_kmax > 0) {
    /* Ewald: the real-space term lB q_i q_j erfc(alpha r) / r within rc (DSF
     * without its shift), the self term -lB alpha / sqrt(pi) q^2 and the
     * reciprocal sum.  Only the global schedule (one trial at a time, the
     * paper's own rule): trials of different domains would interact through
     * S(k), so concurrent domain-local trials would not be independent. */
    if (p->schedule != 1) { free(o); return NULL; }
    o->phi_c1 = 0.0;
    o->phi_c2 = 0.0;
    o->self_coef = -o->alpha / sqrt(M_PI);
    o->dsf_self = 1;
    const int km = o->ewald_kmax;
    const double V = o->L * o->L * o->L, kf = 2.0 * M_PI / o->L;
    int nk = 0;
    for (int nz = -km; nz <= km; ++nz)
      for (int ny = -km; ny <= km; ++ny)
        for (int nx = -km; nx <= km; ++nx) {
          const int n2 = nx * nx + ny * ny + nz * nz;
          if (n2 > 0 && n2 <= km * km) nk++;
        }
    o->nk = nk;
    o->kn = malloc((size_t)3 * nk * sizeof(int));
    o->kA = malloc((size_t)nk * sizeof(double));
    o->Sre = calloc((size_t)nk, sizeof(double)); o->Sim = calloc((size_t)nk, sizeof(double));
    o->dSre = calloc((size_t)nk, sizeof(double)); o->dSim = calloc((size_t)nk, sizeof(double));
    nk = 0;
    for (int nz = -km; nz <= km; ++nz)
      for (int ny = -km; ny <= km; ++ny)
        for (int nx = -km; nx <= km; ++nx) {
          const int n2 = nx * nx + ny * ny + nz * nz;
          if (!(n2 > 0 && n2 <= km * km)) continue;
          const double k2 = kf * kf * n2;
          o->kn[3 * nk] = nx; o->kn[3 * nk + 1] = ny; o->kn[3 * nk + 2] = nz;
          o->kA[nk] = 2.0 * M_PI * o->lB / V * exp(-k2 / (4.0 * o->alpha * o->alpha)) / k2;
          nk++;
        }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      o->eps[i][j] = p->wca_eps[4 * i + j];
      o->sig[i][j] = p->wca_sig[4 * i + j];
      o->del[i][j] = p->wca_del[4 * i + j];
      o->on[i][j] = (i != CLS_NONE && j != CLS_NONE) ? p->wca_on[4 * i + j] : 0;
      o->wcut[i][j] = o->del[i][j] + pow(2.0, 1.0 / 6.0) * o->sig[i][j];
    }
  /* cells and domains: cell side a >= rc/h; a domain is k^3 cells with
   * k*a >= rc, so same-colour domains are at least rc apart.  Domain-local
   * moves conserve each domain's net charge, so k >= 2 is what lets charge
   * cross cell boundaries when the per-sweep offset re-partitions the box. */
  int h = p->cells_per_rc > 0 ? p->cells_per_rc : 2;
  int nc = p->nc > 0 ? p->nc : (int)floor(h * o->L / o->rc);
  o->global = p->schedule == 1;
  if (nc < 1) { free(o); return NULL; }
  if (o->global) {
    o->nc = nc; o->k = nc; o->nd = 1; o->ncol = 1;
  } else {
    int k = p->domain_cells > 0 ? p->domain_cells : h;
    if (p->nc <= 0) nc = (nc / (2 * k)) * (2 * k);
    if (nc < 2 * k || nc % (2 * k) != 0) { free(o); return NULL; }
    o->nc = nc; o->k = k; o->nd = nc / k; o->ncol = 8;
    if ((double)k * (o->L / nc) < o->rc) { free(o); return NULL; }
  }
  o->a = o->L / o->nc;
  if (o->a * h < o->rc) { free(o); return NULL; }
  o->scf = (float)((double)o->nc / o->L);
  o->m = p->trials_per_domain > 0 ? p->trials_per_domain : 1;
  /* chemistry */
  o->pH = p->pH;
  o->pKw = p->pKw;
  o->pIS_plus = p->pIS_plus;
  o->pIS_minus = p->pIS_minus;
  o->pIX_explicit = p->pIX_explicit;
  o->pOH = p->pKw - p->pH;
  if (p->pIX_explicit) { o->pIXp = p->pIX_plus; o->pIXm = p->pIX_minus; }
  else { o->pIXp = pIX_of(p->pIS_plus, o->pH, o->pOH); o->pIXm = pIX_of(p->pIS_minus, o->pH, o->pOH); }
  double D = o->global ? o->L : o->k * o->a;
  double v_nm3 = pow(D * p->sigma_nm, 3.0);
  o->ln_z1 = log(RHO0_NA * v_nm3);
  o->ln_salt = -LN10 * (o->pIXp + o->pIXm);
  /* particles */
  o->n = p->n; o->cap = p->capacity; o->n_input = p->n;
  size_t C = (size_t)(o->cap > 0 ? o->cap : 1);
  o->x = malloc(C * sizeof(float)); o->y = malloc(C * sizeof(float)); o->z = malloc(C * sizeof(float));
  o->type = malloc(C * sizeof(int)); o->cls = malloc(C * sizeof(int)); o->site = malloc(C * sizeof(int));
  o->st = malloc(C * sizeof(int)); o->id = malloc(C * sizeof(uint64_t));
  o->vx = calloc(C, sizeof(double)); o->vy = calloc(C, sizeof(double)); o->vz = calloc(C, sizeof(double));
  o->fx = calloc(C, sizeof(double)); o->fy = calloc(C, sizeof(double)); o->fz = calloc(C, sizeof(double));
  int ns = 0, nA = 0, nB = 0;
  for (int i = 0; i < p->n; ++i) if (type[i] == T_ACID || type[i] == T_BASE) ns++;
  o->lnK = malloc((size_t)(ns > 0 ? ns : 1) * sizeof(double));
  o->pK = malloc((size_t)(ns > 0 ? ns : 1) * sizeof(double));
  o->site_type = malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int));
  int qsum = 0;
  ns = 0;
  for (int i = 0; i < p->n; ++i) {
    float X = xyz[3 * i], Y = xyz[3 * i + 1], Z = xyz[3 * i + 2];
    if (!(X >= 0.0f && X < o->Lf && Y >= 0.0f && Y < o->Lf && Z >= 0.0f && Z < o->Lf)) { or_destroy(o); return NULL; }
    if (type[i] < 0 || type[i] > T_SM || cls[i] < 0 || cls[i] > 3) { or_destroy(o); return NULL; }
    o->x[i] = X; o->y[i] = Y; o->z[i] = Z;
    o->type[i] = type[i];
    o->cls[i] = is_ion(type[i]) ? (o->ion_coupling ? o->ion_cls : CLS_NONE) : cls[i];
    o->id[i] = (uint64_t)i;
    o->site[i] = -1;
    o->st[i] = 0;
    if (type[i] == T_ACID || type[i] == T_BASE) {
      o->site[i] = ns;
      o->st[i] = state[i] ? 1 : 0;
      o->pK[ns] = pK[i];
      o->site_type[ns] = type[i];
      if (type[i] == T_ACID) { o->lnK[ns] = LN10 * ((o->pH - pK[i]) - o->pIXp); nA++; }
      else { o->lnK[ns] = LN10 * ((o->pOH - pK[i]) - o->pIXm); nB++; }
      ns++;
    }
    qsum += qnom(type[i], o->st[i]);
    if (vel) { o->vx[i] = vel[3 * i]; o->vy[i] = vel[3 * i + 1]; o->vz[i] = vel[3 * i + 2]; }
  }
  o->n_sites = ns;
  if (qsum != 0) { or_destroy(o); *err = OR_ERR_NEUTRAL; return NULL; }
  if (o->ewald_kmax > 0) ewald_structure(o, o->Sre, o->Sim);
  o->n_react = 0;
  if (nA > 0) o->react[o->n_react++] = R_ACID;
  if (nB > 0) o->react[o->n_react++] = R_BASE;
  o->react[o->n_react++] = R_SALT;
  o->kxp = K_XP; o->kxm = K_XM; o->txp = T_XP; o->txm = T_XM;
  /* bonds */
  o->nb = p->n_bonds; o->K = p->fene_K; o->R0 = p->fene_R0;
  o->bi = malloc((size_t)(o->nb > 0 ? o->nb : 1) * sizeof(int));
  o->bj = malloc((size_t)(o->nb > 0 ? o->nb : 1) * sizeof(int));
  for (int b = 0; b < o->nb; ++b) {
    int i = bonds[2 * b], j = bonds[2 * b + 1];
    if (i < 0 || j < 0 || i >= p->n || j >= p->n || is_ion(type[i]) || is_ion(type[j])) { or_destroy(o); return NULL; }
    o->bi[b] = i; o->bj[b] = j;
  }
  o->plant = g_plant;
  *err = OR_OK;
  return o;
}

/* ----------------------------------------------------------------------- */
/* Energy of one pair in a given state.  qi, qj are effective charges. */
static double pair_u(const Oracle *o, double qi, int ci, double qj, int cj, double r, int *overlap,
                     int check_hard) {
  double u = 0.0;
  if (r < o->rc && qi != 0.0 && qj != 0.0) u += o->lB * qi * qj * dsf_phi(o, r);
  if (o->on[ci][cj] && r < o->wcut[ci][cj]) {
    double s = r - o->del[ci][cj];
    if (check_hard && s < 0.5 * o->sig[ci][cj]) { *overlap = 1; return 0.0; }
    u += wca_u(o->eps[ci][cj], o->sig[ci][cj], s);
  }
  return u;
}

/* Gross magnitude of one pair's energy in a given state: the sum of the
 * absolute values of the components that FP32 evaluation rounds, used as the
 * scale of the FP32-vs-FP64 tolerance (the pair energies themselves cancel
 * internally near the cutoffs). */
static double gross_coul(const Oracle *o, double qi, double qj, double r) {
  if (!(r < o->rc) || qi == 0.0 || qj == 0.0) return 0.0;
  return fabs(o->lB * qi * qj) * (erfc(o->alpha * r) / r + o->phi_c1 + o->phi_c2 * fabs(r - o->rc));
}
static double gross_wca(const Oracle *o, int ci, int cj, double r) {
  if (!o->on[ci][cj] || !(r < o->wcut[ci][cj])) return 0.0;
  double s = r - o->del[ci][cj];
  double sr6 = pow(o->sig[ci][cj] / s, 6.0);
  return o->eps[ci][cj] * (4.0 * sr6 * sr6 + 4.0 * sr6 + 1.0);
}

typedef struct {
  int idx;              /* index of an existing particle, -1 for an inserted one */
  float x, y, z;
  int cls;
  double q_old, q_new;  /* effective charges in the old / new state */
  int pres_old, pres_new;
} change_t;

static double dist(const Oracle *o, float ax, float ay, float az, float bx, float by, float bz) {
  double dx = min_image((double)ax - (double)bx, o->L);
  double dy = min_image((double)ay - (double)by, o->L);
  double dz = min_image((double)az - (double)bz, o->L);
  return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Delta E = E_new - E_old, summed pair by pair over every pair that contains a
 * changed particle, plus the DSF self-energy change.  S = the gross
 * magnitude of the summed terms (gross_coul / gross_wca of the states that
 * differ, plus |self change|), the scale of the FP32 tolerance. */
static double delta_E(Oracle *o, const change_t *c, int nc, int *overlap, double *S_out) {
  double dE = 0.0, S = 0.0;
  *overlap = 0;
  for (int a = 0; a < nc; ++a) {
    for (int j = 0; j < o->n; ++j) {
      int skip = 0;
      for (int b = 0; b < nc; ++b) if (c[b].idx == j) skip = 1;
      if (skip) continue;
      double qj = qeff(o, o->type[j], o->st[j]);
      double r = dist(o, c[a].x, c[a].y, c[a].z, o->x[j], o->y[j], o->z[j]);
      int ov = 0;
      double un = c[a].pres_new ? pair_u(o, c[a].q_new, c[a].cls, qj, o->cls[j], r, &ov, !c[a].pres_old) : 0.0;
      double uo = c[a].pres_old ? pair_u(o, c[a].q_old, c[a].cls, qj, o->cls[j], r, &ov, 0) : 0.0;
      double du = un - uo;
      if (ov || !(fabs(du) < BIG_TERM)) { *overlap = 1; continue; }
      dE += du;
      S += (c[a].pres_new ? gross_coul(o, c[a].q_new, qj, r) : 0.0) +
           (c[a].pres_old ? gross_coul(o, c[a].q_old, qj, r) : 0.0);
      if (c[a].pres_new != c[a].pres_old) S += gross_wca(o, c[a].cls, o->cls[j], r);
    }
  }
  /* pairs among the changed particles themselves */
  if (g_plant != PLANT_DROP_PAIR_CC) {
    for (int a = 0; a < nc; ++a)
      for (int b = a + 1; b < nc; ++b) {
        double r = dist(o, c[a].x, c[a].y, c[a].z, c[b].x, c[b].y, c[b].z);
        int ov = 0;
        int hard = (c[a].pres_new && !c[a].pres_old) || (c[b].pres_new && !c[b].pres_old);
        double un = (c[a].pres_new && c[b].pres_new) ? pair_u(o, c[a].q_new, c[a].cls, c[b].q_new, c[b].cls, r, &ov, hard) : 0.0;
        double uo = (c[a].pres_old && c[b].pres_old) ? pair_u(o, c[a].q_old, c[a].cls, c[b].q_old, c[b].cls, r, &ov, 0) : 0.0;
        double du = un - uo;
        if (ov || !(fabs(du) < BIG_TERM)) { *overlap = 1; continue; }
        dE += du;
        int pn = c[a].pres_new && c[b].pres_new, po = c[a].pres_old && c[b].pres_old;
        S += (pn ? gross_coul(o, c[a].q_new, c[b].q_new, r) : 0.0) + (po ? gross_coul(o, c[a].q_old, c[b].q_old, r) : 0.0);
        if (pn != po) S += gross_wca(o, c[a].cls, c[b].cls, r);
      }
  }
  if (o->dsf_self && g_plant != PLANT_DROP_SELF) {
    for (int a = 0; a < nc; ++a) {
      double ds = o->lB * o->self_coef *
                  ((c[a].pres_new ? c[a].q_new * c[a].q_new : 0.0) - (c[a].pres_old ? c[a].q_old * c[a].q_old : 0.0));
      dE += ds;
      S += fabs(ds);
    }
  }
  if (o->ewald_kmax > 0) {
    /* reciprocal part: the change of sum_k A_k |S(k)|^2 when the changed
     * particles' charges dq = q_new - q_old (0 where absent) enter S(k); the
     * change of S is kept for the commit */
    double dEr = 0.0, Sr = 0.0;
    for (int i = 0; i < o->nk; ++i) {
      double dre = 0.0, dim = 0.0;
      for (int a = 0; a < nc; ++a) {
        const double dq = (c[a].pres_new ? c[a].q_new : 0.0) - (c[a].pres_old ? c[a].q_old : 0.0);
        if (dq == 0.0) continue;
        const double ph = ewald_phase(o, i, c[a].x, c[a].y, c[a].z);
        dre += dq * cos(ph);
        dim += dq * sin(ph);
      }
      o->dSre[i] = dre;
      o->dSim[i] = dim;
      const double nre = o->Sre[i] + dre, nim = o->Sim[i] + dim;
      const double term =
          o->kA[i] * ((nre * nre + nim * nim) - (o->Sre[i] * o->Sre[i] + o->Sim[i] * o->Sim[i]));
      dEr += term;
      Sr += fabs(term);
    }
    if (g_plant == PLANT_EWALD_HALF_RECIP) {
      dEr *= 0.5;
      Sr *= 0.5;
    }
    dE += dEr;
    S += Sr;
  }
  *S_out = S;
  return dE;
}

/* kind of a particle for the eligibility lists */
static int kind_of(const Oracle *o, int j) {
  switch (o->type[j]) {
    case T_ACID: return o->st[j] ? K_A1 : K_A0;
    case T_BASE: return o->st[j] ? K_B1 : K_B0;
    case T_XP: return K_XP;
    case T_XM: return K_XM;
    case T_SP: return K_SP;
    case T_SM: return K_SM;
    default: return K_OTHER;
  }
}

typedef struct { int rank; uint64_t id; int idx; } elig_t;
static int elig_cmp(const void *pa, const void *pb) {
  const elig_t *a = pa, *b = pb;
  if (a->rank != b->rank) return a->rank < b->rank ? -1 : 1;
  if (a->id != b->id) return a->id < b->id ? -1 : 1;
  return 0;
}

/* index of the k-th particle of a kind in domain d, in canonical order:
 * in-domain cells in (z, y, x) order, then ascending id within a cell */
static int kth_eligible(const Oracle *o, const int off[3], int d, int kind, int64_t kth, elig_t *buf) {
  int cnt = 0;
  for (int j = 0; j < o->n; ++j) {
    if (kind_of(o, j) != kind) continue;
    int dom, rank;
    domain_of(o, off, o->x[j], o->y[j], o->z[j], &dom, &rank);
    if (dom != d) continue;
    buf[cnt].rank = rank; buf[cnt].id = o->id[j]; buf[cnt].idx = j; cnt++;
  }
  qsort(buf, (size_t)cnt, sizeof(elig_t), elig_cmp);
  if (kth < 0 || kth >= cnt) return -1;
  return buf[kth].idx;
}

static void domain_counts(const Oracle *o, const int off[3], int d, int64_t cnt[N_KIND]) {
  for (int i = 0; i < N_KIND; ++i) cnt[i] = 0;
  for (int j = 0; j < o->n; ++j) {
    int dom, rank;
    domain_of(o, off, o->x[j], o->y[j], o->z[j], &dom, &rank);
    if (dom == d) cnt[kind_of(o, j)]++;
  }
}

/* insertion coordinate: the ion is placed uniformly in the trial's domain
 * (Sec. II.C: an ion is taken from the reservoir and placed into the
 * system).  The discretisation is in FP32: f = top 24 bits of w times 2^-24,
 * u = fl32(c0 + k f) wrapped into [0, nc), x = fl32(u * fl32(L/nc)), wrapped
 * into [0, L).  A point that rounds out of the domain is rejected. */
static float insert_coord(const Oracle *o, int c0, uint32_t w) {
  float f = (float)(w >> 8) * (1.0f / 16777216.0f);
  float kf = (float)o->k * f;
  float u = (float)c0 + kf;
  if (u >= (float)o->nc) u -= (float)o->nc;
  float af = (float)(o->L / o->nc);
  float xf = u * af;
  if (xf >= o->Lf) xf -= o->Lf;
  return xf;
}

static void remove_particle(Oracle *o, int j) {
  int last = o->n - 1;
  if (j != last) {
    o->x[j] = o->x[last]; o->y[j] = o->y[last]; o->z[j] = o->z[last];
    o->type[j] = o->type[last]; o->cls[j] = o->cls[last]; o->site[j] = o->site[last];
    o->st[j] = o->st[last]; o->id[j] = o->id[last];
    o->vx[j] = o->vx[last]; o->vy[j] = o->vy[last]; o->vz[j] = o->vz[last];
    o->fx[j] = o->fx[last]; o->fy[j] = o->fy[last]; o->fz[j] = o->fz[last];
  }
  o->n--;
}

/* Maxwell-Boltzmann velocity of an inserted ion (unit mass, kT = 1): three
 * normal deviates by the Box-Muller transform of the four 24-bit uniforms of
 * the Philox block (k, d, phase, purpose), purpose 6 for the first inserted
 * ion of a trial and 7 for the second. */
static void ion_velocity(const uint32_t key[2], int k, int d, uint32_t phi, uint32_t purpose, double v[3]) {
  uint32_t c[4] = {(uint32_t)k, (uint32_t)d, phi, purpose}, w[4];
  philox(c, key, w);
  double u[4];
  for (int i = 0; i < 4; ++i) u[i] = (double)(((float)(w[i] >> 8) + 0.5f) * (1.0f / 16777216.0f));
  double r1 = sqrt(-2.0 * log(u[0])), r2 = sqrt(-2.0 * log(u[2]));
  v[0] = r1 * cos(2.0 * M_PI * u[1]);
  v[1] = r1 * sin(2.0 * M_PI * u[1]);
  v[2] = r2 * cos(2.0 * M_PI * u[3]);
}

static int add_ion(Oracle *o, int t, float x, float y, float z, uint64_t id, const double v[3]) {
  if (o->n >= o->cap) return OR_ERR_CAPACITY;
  int j = o->n++;
  o->x[j] = x; o->y[j] = y; o->z[j] = z;
  o->type[j] = t; o->cls[j] = o->ion_coupling ? o->ion_cls : CLS_NONE;
  o->site[j] = -1; o->st[j] = 0; o->id[j] = id;
  o->vx[j] = v[0]; o->vy[j] = v[1]; o->vz[j] = v[2];
  o->fx[j] = o->fy[j] = o->fz[j] = 0.0;
  return OR_OK;
}

static int net_charge(const Oracle *o) {
  int q = 0;
  for (int j = 0; j < o->n; ++j) q += qnom(o->type[j], o->st[j]);
  return q;
}

/* One trial (phase phi, domain d, trial k in the domain).
 * Philox key = (seed_lo, seed_hi); counters (k, d, phi, purpose):
 *   purpose 0 -> w0 move, w1 site choice, w2 first ion choice, w3 second ion choice
 *   purpose 1 -> w0..w2 position of ion A, w3 x of ion B
 *   purpose 2 -> w0, w1 y, z of ion B; w2, w3 the Metropolis uniform
 * New ion ids: (phi+1) << 32 | 2*(d*m + k) + b, b = 0 (ion A / X+) or 1 (X-). */
/* ----------------------------------------------------------------------- */
/* Learned delayed acceptance (Christen & Fox, J. Comput. Graph. Stat. 14,
 * 795 (2005)) in front of the exact Metropolis test of Sec. II.C.  The paper
 * itself evaluates every trial exactly; this stage is the surrogate fast path.
 *   stage 1: accept with min(1, R exp(-(dE_self + dE~))), R the combinatorial
 *            and chemical factor of the move, dE_self the exact DSF self-term
 *            change and dE~ the surrogate estimate of the pair-energy change;
 *            a stage-1 rejection ends the trial without the exact pair sum;
 *   stage 2: accept with min(1, exp(-(dE_pair - dE~))).
 * The two-stage acceptance satisfies detailed balance with respect to
 * Eq. (QQ) when dE~(y -> x) = -dE~(x -> y): the features change sign under
 * move reversal (the particles other than the two changed ones are the same
 * in x and y) and the surrogate is antisymmetrised, dE~ = (mlp(F) - mlp(-F))/2.
 *
 * Features (48 integers) of a change of particles a (site, or cation of a
 * salt move) and b (ion, or anion), over the cells of the 5^3 stencil of
 * half-cutoff cells around each changed particle's cell, grouped into 8
 * shells by the squared integer cell offset {0},{1},{2},{3},{4},{5},{6},{8,9,12}:
 *   F[24 s +  0 + shell] += dq_s * (charge of each ion in those cells)
 *   F[24 s +  8 + shell] += dq_s * (charge of each site in those cells)
 *   F[24 s + 16 + shell] += eta_s  (for each particle in those cells)
 * dq_s = change of s's effective charge, eta_s = +1 inserted, -1 deleted,
 * 0 otherwise; every particle other than a and b counts.  The a-b pair adds
 *   F[shell(b relative to a)] += q_a' q_b' - q_a q_b  (primes: after the move).
 * MLP 48 -> 128 -> 128 -> 128 -> 1 with ReLU, BF16 weights and FP32 biases,
 * evaluated in FP32: each output is its bias plus one fused multiply-add per
 * weight in input order. */
#define MLP_IN 48
#define MLP_H 128

static float bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, sizeof f);
  return f;
}

static float *bf16_array(const uint16_t *w, int n) {
  float *f = malloc((size_t)n * sizeof(float));
  for (int i = 0; i < n; ++i) f[i] = bf16_value(w[i]);
  return f;
}

static float *f32_array(const float *w, int n) {
  float *f = malloc((size_t)n * sizeof(float));
  memcpy(f, w, (size_t)n * sizeof(float));
  return f;
}

/* W1 [128][48], W2 and W3 [128][128] (out x in), w4 [128]: BF16 bit patterns */
int32_t or_set_surrogate(Oracle *o, const uint16_t *W1, const float *b1, const uint16_t *W2, const float *b2,
                         const uint16_t *W3, const float *b3, const uint16_t *w4, float b4) {
  free(o->W1); free(o->b1); free(o->W2); free(o->b2); free(o->W3); free(o->b3); free(o->w4);
  o->W1 = bf16_array(W1, MLP_H * MLP_IN); o->b1 = f32_array(b1, MLP_H);
  o->W2 = bf16_array(W2, MLP_H * MLP_H); o->b2 = f32_array(b2, MLP_H);
  o->W3 = bf16_array(W3, MLP_H * MLP_H); o->b3 = f32_array(b3, MLP_H);
  o->w4 = bf16_array(w4, MLP_H); o->b4 = b4;
  o->has_mlp = 1;
  return OR_OK;
}

/* delayed acceptance on (1) or off (0); needs a surrogate */
int32_t or_set_da(Oracle *o, int32_t on) {
  if (on && o->ewald_kmax > 0) return OR_ERR_ARG;
  if (on && !o->has_mlp) return OR_ERR_ARG;
  o->da = on ? 1 : 0;
  return OR_OK;
}

static void dense_relu(const float *W, const float *b, const float *x, int n_in, float *y) {
  for (int i = 0; i < MLP_H; ++i) {
    float a = b[i];
    for (int k = 0; k < n_in; ++k) a = fmaf(W[i * n_in + k], x[k], a);
    y[i] = a > 0.0f ? a : 0.0f;
  }
}

static float mlp_forward(const Oracle *o, const float *F) {
  float h1[MLP_H], h2[MLP_H], h3[MLP_H];
  dense_relu(o->W1, o->b1, F, MLP_IN, h1);
  dense_relu(o->W2, o->b2, h1, MLP_H, h2);
  dense_relu(o->W3, o->b3, h2, MLP_H, h3);
  float y = o->b4;
  for (int k = 0; k < MLP_H; ++k) y = fmaf(o->w4[k], h3[k], y);
  return y;
}

float or_mlp(const Oracle *o, const float *F) { return o->has_mlp ? mlp_forward(o, F) : NAN; }

static float surrogate_dE(const Oracle *o, const float *F) {
  float G[MLP_IN];
  for (int k = 0; k < MLP_IN; ++k) G[k] = -F[k];
  const float yp = mlp_forward(o, F);
  if (g_plant == PLANT_DA_ONE_SIDED) return yp;
  const float ym = mlp_forward(o, G);
  return 0.5f * (yp - ym);
}

float or_surrogate(const Oracle *o, const float *F) { return o->has_mlp ? surrogate_dE(o, F) : NAN; }

/* shell of a squared integer cell offset; -1 cannot occur in a 5^3 stencil */
static const int SHELL_OF_N2[13] = {0, 1, 2, 3, 4, 5, 6, -1, 7, 7, -1, -1, 7};

static int cell_delta(const Oracle *o, int cb, int ca) {
  int d = ((cb - ca) % o->nc + o->nc) % o->nc;
  if (d > o->nc / 2) d -= o->nc;
  return d;
}

/* shell of the cell of b relative to the cell of a, -1 outside the stencil */
static int shell_between(const Oracle *o, float ax, float ay, float az, float bx, float by, float bz) {
  const int dx = cell_delta(o, cell_of(o, bx), cell_of(o, ax));
  const int dy = cell_delta(o, cell_of(o, by), cell_of(o, ay));
  const int dz = cell_delta(o, cell_of(o, bz), cell_of(o, az));
  if (abs(dx) > 2 || abs(dy) > 2 || abs(dz) > 2) return -1;
  return SHELL_OF_N2[dx * dx + dy * dy + dz * dz];
}

static int iround(double v) { return (int)lround(v); }

static void da_features(const Oracle *o, const change_t *ch, float *F) {
  int acc[MLP_IN];
  memset(acc, 0, sizeof acc);
  for (int s = 0; s < 2; ++s) {
    const change_t *c = &ch[s];
    const int dq = iround((c->pres_new ? c->q_new : 0.0) - (c->pres_old ? c->q_old : 0.0));
    const int eta = c->pres_new - c->pres_old;
    for (int j = 0; j < o->n; ++j) {
      if (j == ch[0].idx || j == ch[1].idx) continue;
      const int sh = shell_between(o, c->x, c->y, c->z, o->x[j], o->y[j], o->z[j]);
      if (sh < 0) continue;
      const int t = o->type[j];
      const int q = iround(qeff(o, t, o->st[j]));
      if (is_ion(t)) acc[24 * s + sh] += dq * q;
      else if (t == T_ACID || t == T_BASE) acc[24 * s + 8 + sh] += dq * q;
      acc[24 * s + 16 + sh] += eta;
    }
  }
  const int sh = shell_between(o, ch[0].x, ch[0].y, ch[0].z, ch[1].x, ch[1].y, ch[1].z);
  if (sh >= 0) {
    const int qn = (ch[0].pres_new && ch[1].pres_new) ? iround(ch[0].q_new) * iround(ch[1].q_new) : 0;
    const int qo = (ch[0].pres_old && ch[1].pres_old) ? iround(ch[0].q_old) * iround(ch[1].q_old) : 0;
    acc[sh] += qn - qo;
  }
  for (int k = 0; k < MLP_IN; ++k) F[k] = (float)acc[k];
}

/* exact DSF self-term change of a set of changed particles (part of dE) */
static double self_change(const Oracle *o, const change_t *c, int nc) {
  if (!o->dsf_self || g_plant == PLANT_DROP_SELF) return 0.0;
  double ds = 0.0;
  for (int a = 0; a < nc; ++a)
    ds += o->lB * o->self_coef *
          ((c[a].pres_new ? c[a].q_new * c[a].q_new : 0.0) - (c[a].pres_old ? c[a].q_old * c[a].q_old : 0.0));
  return ds;
}

/* extra per-trial record of the delayed-acceptance stages */
typedef struct {
  float dE_sur;    /* surrogate pair-energy change */
  int32_t stage;   /* 0 no surrogate evaluated, 1 rejected at stage 1, 2 passed stage 1 */
  double lnA2;     /* dE~ - dE_pair (NaN on overlap) */
  double lnu2;     /* log of the stage-2 uniform */
} or_trial_da;

static int or_trial_one(Oracle *o, const uint32_t key[2], const int off[3], uint32_t phi, int d, int k,
                        or_trial *rec, int forced, elig_t *buf, int64_t *hist, int hist_n,
                        int64_t *trans, or_trial_da *drec, float *feat, double *dEpair) {
  uint32_t c0[4] = {(uint32_t)k, (uint32_t)d, phi, 0u}, c1[4] = {(uint32_t)k, (uint32_t)d, phi, 1u},
           c2[4] = {(uint32_t)k, (uint32_t)d, phi, 2u};
  uint32_t P0[4], P1[4], P2[4];
  philox(c0, key, P0); philox(c1, key, P1); philox(c2, key, P2);
  int mv = (int)pick(P0[0], 2 * o->n_react);
  int r = o->react[mv >> 1];
  int fwd = (mv & 1) == 0;
  or_trial t;
  t.move = 2 * r + (fwd ? 0 : 1);
  t.flags = 0; t.id_a = UINT64_MAX; t.id_b = UINT64_MAX;
  t.dE = 0.0; t.S = 0.0; t.lnA = -INFINITY;
  t.lnu = log(unif53(P2[2], P2[3]));
  o->stats[t.move]++;

  int64_t cnt[N_KIND];
  domain_counts(o, off, d, cnt);
  int64_t cnt_acc[N_KIND]; /* the counts the acceptance rules use */
  memcpy(cnt_acc, cnt, sizeof cnt);
  if (g_plant == PLANT_SPECIES_COUNT) {
    cnt_acc[o->kxp] = cnt[K_XP] + cnt[K_SP];
    cnt_acc[o->kxm] = cnt[K_XM] + cnt[K_SM];
  }
  /* origin cell of the domain and the two candidate insertion points */
  int dd[3] = {d % o->nd, (d / o->nd) % o->nd, d / (o->nd * o->nd)};
  int org[3];
  for (int i = 0; i < 3; ++i) org[i] = (off[i] + dd[i] * o->k) % o->nc;
  float pa[3] = {insert_coord(o, org[0], P1[0]), insert_coord(o, org[1], P1[1]), insert_coord(o, org[2], P1[2])};
  float pb[3] = {insert_coord(o, org[0], P1[3]), insert_coord(o, org[1], P2[0]), insert_coord(o, org[2], P2[1])};
  uint64_t base = ((uint64_t)(phi + 1u) << 32);
  uint64_t idA = base | (uint64_t)(uint32_t)(2u * ((uint32_t)d * (uint32_t)o->m + (uint32_t)k));
  uint64_t idB = idA + 1u;

  change_t ch[2];
  int nch = 0;
  int site = -1, ionA = -1, ionB = -1;
  double ln_ratio = 0.0; /* log of the combinatorial / chemical factor */
  int noelig = 0, edge = 0;
  double lnz = o->ln_z1;
  if (g_plant == PLANT_WRONG_VOLUME) lnz += 1.0;
  if (r == R_ACID || r == R_BASE) {
    int k0 = r == R_ACID ? K_A0 : K_B0, k1 = r == R_ACID ? K_A1 : K_B1;
    int kx = r == R_ACID ? o->kxp : o->kxm;
    double qs = r == R_ACID ? -1.0 : 1.0;
    if (fwd) {
      if (cnt[k0] == 0) noelig = 1;
      else {
        site = kth_eligible(o, off, d, k0, pick(P0[1], cnt[k0]), buf);
        int dom, rank;
        domain_of(o, off, pa[0], pa[1], pa[2], &dom, &rank);
        if (dom != d) edge = 1;
        t.id_a = o->id[site]; t.id_b = idA;
        ch[0] = (change_t){site, o->x[site], o->y[site], o->z[site], o->cls[site], 0.0, qs, 1, 1};
        ch[1] = (change_t){-1, pa[0], pa[1], pa[2], o->ion_coupling ? o->ion_cls : CLS_NONE, 0.0,
                           o->ion_coupling ? -qs : 0.0, 0, 1};
        nch = 2;
        ln_ratio = log((double)cnt[k0]) + lnz - log((double)(cnt[k1] + 1));
        if (g_plant != PLANT_DROP_ION_COUNT) ln_ratio -= log((double)(cnt_acc[kx] + 1));
        ln_ratio += o->lnK[o->site[site]];
      }
    } else {
      if (cnt[k1] == 0 || cnt[kx] == 0) noelig = 1;
      else {
        site = kth_eligible(o, off, d, k1, pick(P0[1], cnt[k1]), buf);
        ionA = kth_eligible(o, off, d, kx, pick(P0[2], cnt[kx]), buf);
        t.id_a = o->id[site]; t.id_b = o->id[ionA];
        ch[0] = (change_t){site, o->x[site], o->y[site], o->z[site], o->cls[site], qs, 0.0, 1, 1};
        ch[1] = (change_t){ionA, o->x[ionA], o->y[ionA], o->z[ionA], o->cls[ionA],
                           qeff(o, o->type[ionA], 0), 0.0, 1, 0};
        nch = 2;
        ln_ratio = log((double)cnt[k1]) - log((double)(cnt[k0] + 1)) - lnz;
        if (g_plant != PLANT_DROP_ION_COUNT) ln_ratio += log((double)cnt_acc[kx]);
        ln_ratio -= o->lnK[o->site[site]];
      }
    }
  } else { /* salt */
    if (fwd) {
      int dom, rank;
      domain_of(o, off, pa[0], pa[1], pa[2], &dom, &rank);
      if (dom != d) edge = 1;
      domain_of(o, off, pb[0], pb[1], pb[2], &dom, &rank);
      if (dom != d) edge = 1;
      t.id_a = idA; t.id_b = idB;
      int icls = o->ion_coupling ? o->ion_cls : CLS_NONE;
      ch[0] = (change_t){-1, pa[0], pa[1], pa[2], icls, 0.0, o->ion_coupling ? 1.0 : 0.0, 0, 1};
      ch[1] = (change_t){-1, pb[0], pb[1], pb[2], icls, 0.0, o->ion_coupling ? -1.0 : 0.0, 0, 1};
      nch = 2;
      ln_ratio = 2.0 * lnz + o->ln_salt;
      if (g_plant != PLANT_DROP_ION_COUNT) ln_ratio -= log((double)(cnt_acc[o->kxp] + 1)) + log((double)(cnt_acc[o->kxm] + 1));
    } else {
      if (cnt[o->kxp] == 0 || cnt[o->kxm] == 0) noelig = 1;
      else {
        ionA = kth_eligible(o, off, d, o->kxp, pick(P0[2], cnt[o->kxp]), buf);
        ionB = kth_eligible(o, off, d, o->kxm, pick(P0[3], cnt[o->kxm]), buf);
        t.id_a = o->id[ionA]; t.id_b = o->id[ionB];
        ch[0] = (change_t){ionA, o->x[ionA], o->y[ionA], o->z[ionA], o->cls[ionA], qeff(o, o->txp, 0), 0.0, 1, 0};
        ch[1] = (change_t){ionB, o->x[ionB], o->y[ionB], o->z[ionB], o->cls[ionB], qeff(o, o->txm, 0), 0.0, 1, 0};
        nch = 2;
        ln_ratio = -2.0 * lnz - o->ln_salt;
        if (g_plant != PLANT_DROP_ION_COUNT) ln_ratio += log((double)cnt_acc[o->kxp]) + log((double)cnt_acc[o->kxm]);
      }
    }
  }
  int accept = 0;
  or_trial_da td = {0.0f, 0, NAN, NAN};
  if (feat) for (int q = 0; q < MLP_IN; ++q) feat[q] = 0.0f;
  if (dEpair) *dEpair = NAN;
  if (noelig) t.flags |= F_NOELIG;
  else if (edge) t.flags |= F_EDGE;
  else if (o->da) {
    /* delayed acceptance; forced: bit 1 forces stage 1 to bit 0, bit 3
     * forces stage 2 to bit 2 (tie protocol of the parity tests) */
    float F[MLP_IN];
    da_features(o, ch, F);
    const float sur = surrogate_dE(o, F);
    const double dself = self_change(o, ch, nch);
    int ov = 0;
    double S = 0.0;
    const double dE = delta_E(o, ch, nch, &ov, &S); /* recorded always, decisive only after stage 1 */
    t.S = S;
    t.lnA = ln_ratio - dself - (double)sur;
    int s1 = t.lnu < t.lnA;
    if (forced >= 0 && (forced & 2)) s1 = forced & 1;
    uint32_t c3[4] = {(uint32_t)k, (uint32_t)d, phi, 3u}, P3[4];
    philox(c3, key, P3);
    td.dE_sur = sur;
    td.stage = s1 ? 2 : 1;
    td.lnu2 = log(unif53(P3[0], P3[1]));
    if (feat) memcpy(feat, F, sizeof F);
    if (ov) {
      t.dE = INFINITY;
      if (s1) t.flags |= F_OVERLAP;
    } else {
      t.dE = dE;
      td.lnA2 = (double)sur - (dE - dself);
      if (g_plant == PLANT_DA_STAGE2_FULL) td.lnA2 = ln_ratio - dE;
      if (dEpair) *dEpair = dE - dself;
      if (s1) {
        accept = td.lnu2 < td.lnA2;
        if (forced >= 0 && (forced & 8)) accept = (forced >> 2) & 1;
      }
    }
  } else {
    int ov = 0;
    double S = 0.0;
    if (feat) da_features(o, ch, feat);
    double dE = delta_E(o, ch, nch, &ov, &S);
    if (g_plant == PLANT_DE_SIGN) dE = -dE;
    t.S = S;
    if (ov) { t.flags |= F_OVERLAP; t.dE = INFINITY; }
    else {
      t.dE = dE;
      t.lnA = ln_ratio - dE;
      accept = t.lnu < t.lnA;
      if (dEpair) *dEpair = dE - self_change(o, ch, nch);
    }
    if (forced >= 0 && !(t.flags & (F_NOELIG | F_EDGE | F_OVERLAP))) accept = forced;
  }
  if (drec) *drec = td;
  if (accept) {
    t.flags |= F_ACC;
    o->stats[6 + t.move]++;
    if (o->ewald_kmax > 0)
      for (int i = 0; i < o->nk; ++i) {
        o->Sre[i] += o->dSre[i];
        o->Sim[i] += o->dSim[i];
      }
    int s_before = 0;
    if (hist_n > 0) for (int j = 0; j < o->n; ++j) if (o->site[j] >= 0 && o->site[j] < hist_n && o->st[j]) s_before |= 1 << o->site[j];
    double va[3], vb[3];
    ion_velocity(key, k, d, phi, 6u, va);
    ion_velocity(key, k, d, phi, 7u, vb);
    if (r == R_ACID || r == R_BASE) {
      if (fwd) {
        o->st[site] = 1;
        if (add_ion(o, r == R_ACID ? o->txp : o->txm, pa[0], pa[1], pa[2], idA, va)) return OR_ERR_CAPACITY;
      } else {
        o->st[site] = 0;
        remove_particle(o, ionA);
      }
    } else {
      if (fwd) {
        if (add_ion(o, o->txp, pa[0], pa[1], pa[2], idA, va)) return OR_ERR_CAPACITY;
        if (add_ion(o, o->txm, pb[0], pb[1], pb[2], idB, vb)) return OR_ERR_CAPACITY;
      } else {
        int hi = ionA > ionB ? ionA : ionB, lo = ionA > ionB ? ionB : ionA;
        remove_particle(o, hi);
        remove_particle(o, lo);
      }
    }
    if (trans && (r == R_ACID || r == R_BASE) && o->site[site] < hist_n) {
      int s_after = s_before ^ (1 << o->site[site]);
      trans[(int64_t)s_before * hist_n + o->site[site]]++;
      (void)s_after;
    }
  }
  if (hist && hist_n > 0) {
    int s = 0;
    for (int j = 0; j < o->n; ++j) if (o->site[j] >= 0 && o->site[j] < hist_n && o->st[j]) s |= 1 << o->site[j];
    hist[s]++;
  }
  if (rec) *rec = t;
  if (net_charge(o) != 0) return OR_ERR_NEUTRAL;
  return OR_OK;
}

int64_t or_trials_per_sweep(const Oracle *o) {
  return (int64_t)o->nd * o->nd * o->nd * o->m;
}

/* Run n_trials (a multiple of the trials per sweep).  Sweeps continue the
 * context's sweep counter.  log: one record per trial in schedule order
 * (colour phases in order, domains ascending, trials in the domain).
 * forced: optional per-trial decision override (-1 = none) used only to step
 * over a tie at the acceptance threshold.  hist/trans: optional state
 * histogram over the first hist_n sites and site-flip transition counts.
 * dlog / feat / dEpair: optional per-trial delayed-acceptance records, the
 * 48 surrogate features and the exact pair-energy change (dE minus the self
 * term; NaN when not evaluated or on overlap). */
int32_t or_sweep(Oracle *o, int64_t n_trials, uint64_t seed, or_trial *log, const int8_t *forced,
                 int64_t *hist, int32_t hist_n, int64_t *trans, or_trial_da *dlog, float *feat, double *dEpair) {
  int64_t per = or_trials_per_sweep(o);
  if (n_trials < 0 || n_trials % per != 0) return OR_ERR_ARG;
  if (hist_n < 0 || hist_n > 20) return OR_ERR_ARG;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  elig_t *buf = malloc((size_t)(o->cap > 0 ? o->cap : 1) * sizeof(elig_t));
  int64_t t = 0;
  o->f_valid = 0; /* the MD step re-evaluates forces after every CR-MC call */
  int rc = OR_OK;
  for (int64_t sw = 0; sw < n_trials / per && rc == OR_OK; ++sw) {
    uint64_t s = o->sweep++;
    if (o->ewald_kmax > 0) ewald_structure(o, o->Sre, o->Sim);  /* from scratch at every sweep */
    int off[3] = {0, 0, 0};
    if (!o->global) {
      uint32_t c[4] = {0u, 0u, (uint32_t)s, 4u}, w[4];
      philox(c, key, w);
      for (int i = 0; i < 3; ++i) off[i] = (int)pick(w[i], o->nc);
    }
    for (int col = 0; col < o->ncol && rc == OR_OK; ++col) {
      uint32_t phi = (uint32_t)(s * (uint64_t)o->ncol + (uint64_t)col);
      int ndom = o->nd * o->nd * o->nd;
      for (int d = 0; d < ndom && rc == OR_OK; ++d) {
        int dx = d % o->nd, dy = (d / o->nd) % o->nd, dz = d / (o->nd * o->nd);
        int colour = o->global ? 0 : ((dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2));
        if (colour != col) continue;
        for (int k = 0; k < o->m && rc == OR_OK; ++k, ++t) {
          int f = forced ? forced[t] : -1;
          rc = or_trial_one(o, key, off, phi, d, k, log ? &log[t] : NULL, f, buf, hist, hist_n, trans,
                            dlog ? &dlog[t] : NULL, feat ? feat + (size_t)t * MLP_IN : NULL,
                            dEpair ? &dEpair[t] : NULL);
        }
      }
    }
  }
  free(buf);
  return rc;
}

/* counts: [n_A, n_A-, n_B, n_B+, n_X+, n_X-, n, net charge, n_S+, n_S-] */
void or_counts(const Oracle *o, int64_t *out) {
  int64_t c[10] = {0};
  for (int j = 0; j < o->n; ++j) {
    switch (o->type[j]) {
      case T_ACID: c[0]++; if (o->st[j]) c[1]++; break;
      case T_BASE: c[2]++; if (o->st[j]) c[3]++; break;
      case T_XP: c[4]++; break;
      case T_XM: c[5]++; break;
      case T_SP: c[8]++; break;
      case T_SM: c[9]++; break;
      default: break;
    }
  }
  c[6] = o->n;
  c[7] = net_charge(o);
  memcpy(out, c, sizeof c);
}

void or_stats(const Oracle *o, int64_t *out) { memcpy(out, o->stats, sizeof o->stats); }

int32_t or_n(const Oracle *o) { return o->n; }
int32_t or_geometry(const Oracle *o, int32_t *out) {
  out[0] = o->nc; out[1] = o->k; out[2] = o->nd; out[3] = o->ncol; out[4] = o->m; out[5] = o->global;
  return OR_OK;
}
/* A new reservoir pH between sweeps (the paper's implementation accepts a
 * time-dependent pH, App. B): pOH = pKw - pH, the grouped pI_X of Eq.
 * (pIXgen) unless given explicitly, and the equilibrium constants
 * K_A = 10^(pH - pKa - pI_X+), K_B = 10^(pOH - pKb - pI_X-) and
 * K_ion = 10^(-pI_X+ - pI_X-) of every site, recomputed as at creation. */
void or_set_pH(Oracle *o, double pH) {
  o->pH = pH;
  o->pOH = o->pKw - pH;
  if (!o->pIX_explicit) {
    o->pIXp = pIX_of(o->pIS_plus, o->pH, o->pOH);
    o->pIXm = pIX_of(o->pIS_minus, o->pH, o->pOH);
  }
  o->ln_salt = -LN10 * (o->pIXp + o->pIXm);
  for (int s = 0; s < o->n_sites; ++s)
    o->lnK[s] = o->site_type[s] == T_ACID ? LN10 * ((o->pH - o->pK[s]) - o->pIXp)
                                          : LN10 * ((o->pOH - o->pK[s]) - o->pIXm);
}

/* One invocation of the scheme (App. B: the method can be invoked repeatedly
 * with different types of ions, which realises the grand-reaction ensemble;
 * Sec. II.B: applied separately to dissociated and salt ions).  The acid,
 * base and salt reactions of Eqs. (acid_new)-(salt_new) of the following
 * sweeps exchange a cation of type `cation` (T_XP or T_SP) and an anion of
 * type `anion` (T_XM or T_SM) with the reservoir, at chemical potentials
 * pI_cation and pI_anion in place of pI_X+ and pI_X-:
 *   K_A = 10^(pH - pKa - pI_cation), K_B = 10^(pOH - pKb - pI_anion),
 *   K_ion = 10^(-pI_cation - pI_anion);
 * the count n_X+- in the acceptance rules is the count of the invocation's
 * own type (each species has its own ideal term in Eq. (QQ)).  `reactions`
 * selects acid (1), base (2) and salt (4) moves, kept only where the system
 * has such sites.  The pI values stay fixed through a later pH change. */
int32_t or_set_invocation(Oracle *o, int32_t cation, int32_t anion, double pI_cation, double pI_anion,
                          int32_t reactions) {
  if ((cation != T_XP && cation != T_SP) || (anion != T_XM && anion != T_SM)) return OR_ERR_ARG;
  if (!isfinite(pI_cation) || !isfinite(pI_anion) || reactions <= 0 || reactions > 7) return OR_ERR_ARG;
  int nA = 0, nB = 0;
  for (int s = 0; s < o->n_sites; ++s) { if (o->site_type[s] == T_ACID) nA++; else nB++; }
  int react[3], nr = 0;
  if ((reactions & 1) && nA > 0) react[nr++] = R_ACID;
  if ((reactions & 2) && nB > 0) react[nr++] = R_BASE;
  if (reactions & 4) react[nr++] = R_SALT;
  if (nr == 0) return OR_ERR_ARG;
  memcpy(o->react, react, sizeof react);
  o->n_react = nr;
  o->txp = cation; o->txm = anion;
  o->kxp = cation == T_XP ? K_XP : K_SP;
  o->kxm = anion == T_XM ? K_XM : K_SM;
  o->pIX_explicit = 1;
  o->pIXp = pI_cation;
  o->pIXm = pI_anion;
  or_set_pH(o, o->pH);
  return OR_OK;
}

/* Ungrouping of the combined ions (Sec. II.D, last paragraph): a grouped
 * ion belongs to subspecies i with probability p_i = 10^(-pI_i + pI_X).
 * out[0] = p of S+ in X+, out[1] = p of H+ in X+, out[2] = p of S- in X-,
 * out[3] = p of OH- in X-; the rest of each group (1 - the two) is the
 * counter-ion of the acid or base that sets a non-neutral pH (App. C). */
void or_ungroup(const Oracle *o, double *out) {
  out[0] = pow(10.0, -o->pIS_plus + o->pIXp);
  out[1] = pow(10.0, -o->pH + o->pIXp);
  out[2] = pow(10.0, -o->pIS_minus + o->pIXm);
  out[3] = pow(10.0, -o->pOH + o->pIXm);
}

void or_chem(const Oracle *o, double *out) {
  out[0] = o->pIXp; out[1] = o->pIXm; out[2] = o->ln_z1; out[3] = o->ln_salt; out[4] = o->a;
  out[5] = o->self_coef; out[6] = o->pOH;
}

/* particle dump in internal order (callers sort by id) */
void or_particles(const Oracle *o, float *xyz, uint64_t *id, int32_t *type, int8_t *state, double *vel) {
  for (int j = 0; j < o->n; ++j) {
    if (xyz) { xyz[3 * j] = o->x[j]; xyz[3 * j + 1] = o->y[j]; xyz[3 * j + 2] = o->z[j]; }
    if (id) id[j] = o->id[j];
    if (type) type[j] = o->type[j];
    if (state) state[j] = (int8_t)o->st[j];
    if (vel) { vel[3 * j] = o->vx[j]; vel[3 * j + 1] = o->vy[j]; vel[3 * j + 2] = o->vz[j]; }
  }
}

/* site states by site index */
void or_site_states(const Oracle *o, int8_t *out) {
  for (int j = 0; j < o->n; ++j) if (o->site[j] >= 0) out[o->site[j]] = (int8_t)o->st[j];
}

/* Total energy of the current configuration (all pairs, brute force). */
double or_energy(const Oracle *o) {
  double E = 0.0;
  for (int i = 0; i < o->n; ++i) {
    double qi = qeff(o, o->type[i], o->st[i]);
    for (int j = i + 1; j < o->n; ++j) {
      int ov = 0;
      double r = dist(o, o->x[i], o->y[i], o->z[i], o->x[j], o->y[j], o->z[j]);
      E += pair_u(o, qi, o->cls[i], qeff(o, o->type[j], o->st[j]), o->cls[j], r, &ov, 0);
    }
    if (o->dsf_self && !(o->ewald_kmax > 0 && g_plant == PLANT_DROP_SELF)) E += o->lB * o->self_coef * qi * qi;
  }
  if (o->ewald_kmax > 0) {
    double *re = malloc((size_t)o->nk * sizeof(double)), *im = malloc((size_t)o->nk * sizeof(double));
    ewald_structure(o, re, im);
    E += ewald_recip_energy(o, re, im);
    free(re);
    free(im);
  }
  return E;
}

/* Ewald parts of the energy: out = {real (pairs within rc, Coulomb only),
 * reciprocal, self}; zeros without Ewald */
void or_ewald_parts(const Oracle *o, double *out) {
  out[0] = out[1] = out[2] = 0.0;
  if (o->ewald_kmax <= 0) return;
  for (int i = 0; i < o->n; ++i) {
    const double qi = qeff(o, o->type[i], o->st[i]);
    for (int j = i + 1; j < o->n; ++j) {
      const double qj = qeff(o, o->type[j], o->st[j]);
      const double r = dist(o, o->x[i], o->y[i], o->z[i], o->x[j], o->y[j], o->z[j]);
      if (r < o->rc && qi != 0.0 && qj != 0.0) out[0] += o->lB * qi * qj * erfc(o->alpha * r) / r;
    }
    out[2] += o->lB * o->self_coef * qi * qi;
  }
  double *re = malloc((size_t)o->nk * sizeof(double)), *im = malloc((size_t)o->nk * sizeof(double));
  ewald_structure(o, re, im);
  out[1] = ewald_recip_energy(o, re, im);
  free(re);
  free(im);
}
int32_t or_ewald_nk(const Oracle *o) { return o->nk; }

/* FENE bond energy, U = -K R0^2/2 ln(1 - (r/R0)^2) summed over bonds (the
 * CR-MC moves never change it; the MD tests use it for -grad E). */
double or_bond_energy(const Oracle *o) {
  double E = 0.0;
  int *where = malloc((size_t)(o->cap > 0 ? o->cap : 1) * sizeof(int));
  for (int j = 0; j < o->cap; ++j) where[j] = -1;
  for (int j = 0; j < o->n; ++j) if (o->id[j] < (uint64_t)o->cap) where[o->id[j]] = j;
  for (int b = 0; b < o->nb; ++b) {
    int i = where[o->bi[b]], j = where[o->bj[b]];
    double r = dist(o, o->x[i], o->y[i], o->z[i], o->x[j], o->y[j], o->z[j]);
    double x2 = (r / o->R0) * (r / o->R0);
    E += x2 < 1.0 ? -0.5 * o->K * o->R0 * o->R0 * log(1.0 - x2) : INFINITY;
  }
  free(where);
  return E;
}

/* ----------------------------------------------------------------------- */
/* Reciprocal-space Ewald forces, minus the gradient of E_rec over r_j:
 * F_j = 2 q_j sum_k A_k k Im(S(k)^* exp(i k.r_j)), Im(...) = C sin - D cos
 * with S = C + i D of the current positions (every k of the sphere).  fs
 * gets the per-component sums of the terms' magnitudes. */
static void ewald_recip_forces(const Oracle *o, double *F, double *fs) {
  double *re = malloc((size_t)o->nk * sizeof(double)), *im = malloc((size_t)o->nk * sizeof(double));
  ewald_structure(o, re, im);
  const double kf = 2.0 * M_PI / o->L;
  for (int j = 0; j < o->n; ++j) {
    const double q = qeff(o, o->type[j], o->st[j]);
    if (q == 0.0) continue;
    for (int i = 0; i < o->nk; ++i) {
      const double ph = ewald_phase(o, i, o->x[j], o->y[j], o->z[j]);
      double t = 2.0 * q * o->kA[i] * (re[i] * sin(ph) - im[i] * cos(ph));
      if (g_plant == PLANT_EWALD_FORCE_SIGN) t = -t;
      for (int c = 0; c < 3; ++c) {
        const double fc = t * kf * (double)o->kn[3 * i + c];
        F[3 * j + c] += fc;
        if (fs) fs[3 * j + c] += fabs(fc);
      }
    }
  }
  free(re);
  free(im);
}

/* ----------------------------------------------------------------------- */
/* MD: conservative forces (DSF Coulomb + WCA over all pairs within the
 * cutoffs, brute force with the minimum image, plus FENE bonds
 * U = -K R0^2/2 ln(1 - (r/R0)^2)); with Ewald electrostatics the real-space
 * erfc pair forces plus the reciprocal-space forces.  fs: per component sum
 * of |pair force|. */
static int forces_cons(const Oracle *o, double *F, double *fs) {
  memset(F, 0, (size_t)o->n * 3 * sizeof(double));
  if (fs) memset(fs, 0, (size_t)o->n * 3 * sizeof(double));
  for (int i = 0; i < o->n; ++i) {
    double qi = qeff(o, o->type[i], o->st[i]);
    for (int j = i + 1; j < o->n; ++j) {
      double qj = qeff(o, o->type[j], o->st[j]);
      double d[3] = {min_image((double)o->x[i] - o->x[j], o->L), min_image((double)o->y[i] - o->y[j], o->L),
                     min_image((double)o->z[i] - o->z[j], o->L)};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double f = 0.0, g = 0.0; /* along (r_i - r_j)/r, positive = repulsive; g: gross magnitude */
      if (r < o->rc && qi != 0.0 && qj != 0.0) {
        double ar = o->alpha * r;
        f += o->lB * qi * qj * dsf_force(o, r);
        g += fabs(o->lB * qi * qj) * (erfc(ar) / (r * r) + 2.0 * o->alpha / sqrt(M_PI) * exp(-ar * ar) / r + o->phi_c2);
      }
      int ci = o->cls[i], cj = o->cls[j];
      if (o->on[ci][cj] && r < o->wcut[ci][cj]) {
        double s = r - o->del[ci][cj], sr6 = pow(o->sig[ci][cj] / s, 6.0);
        f += wca_f(o->eps[ci][cj], o->sig[ci][cj], s);
        g += 24.0 * o->eps[ci][cj] * (2.0 * sr6 * sr6 + sr6) / s;
      }
      if (f == 0.0) continue;
      for (int c = 0; c < 3; ++c) {
        double fc = f * d[c] / r;
        F[3 * i + c] += fc;
        F[3 * j + c] -= fc;
        if (fs) { fs[3 * i + c] += g * fabs(d[c]) / r; fs[3 * j + c] += g * fabs(d[c]) / r; }
      }
    }
  }
  if (o->ewald_kmax > 0) ewald_recip_forces(o, F, fs);
  if (o->nb > 0) {
    /* permanent particles keep their input index as id; map id -> index */
    int *where = malloc((size_t)o->cap * sizeof(int));
    for (int j = 0; j < o->cap; ++j) where[j] = -1;
    for (int j = 0; j < o->n; ++j) if (o->id[j] < (uint64_t)o->cap) where[o->id[j]] = j;
    for (int b = 0; b < o->nb; ++b) {
      int i = where[o->bi[b]], j = where[o->bj[b]];
      double d[3] = {min_image((double)o->x[i] - o->x[j], o->L), min_image((double)o->y[i] - o->y[j], o->L),
                     min_image((double)o->z[i] - o->z[j], o->L)};
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      double x2 = r2 / (o->R0 * o->R0);
      if (x2 >= 1.0) { free(where); return OR_ERR_BOND; }
      double g = -o->K / (1.0 - x2); /* F_i = g * (r_i - r_j) */
      for (int c = 0; c < 3; ++c) {
        F[3 * i + c] += g * d[c];
        F[3 * j + c] -= g * d[c];
        if (fs) { fs[3 * i + c] += fabs(g * d[c]); fs[3 * j + c] += fabs(g * d[c]); }
      }
    }
    free(where);
  }
  return OR_OK;
}

int32_t or_forces(const Oracle *o, double *F, double *fs) {
  return forces_cons(o, F, fs);
}

/* Langevin part of the force, drawn per particle id and force evaluation:
 * -gamma v + sqrt(2 gamma T / dt) xi, xi ~ N(0,1) from Box-Muller on Philox
 * (key = seed, counter = (id_lo, id_hi, eval, 5)), uniforms ((w >> 8) + 0.5) 2^-24. */
static int is_member(const Oracle *o, int j);
static void langevin(const Oracle *o, double *F, double gamma, double T, double dt, uint64_t seed, uint64_t ev) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  double amp = sqrt(2.0 * gamma * T / dt);
  for (int j = 0; j < o->n; ++j) {
    if (is_member(o, j)) continue; /* a rigid body's thermostat acts on the body */
    uint32_t c[4] = {(uint32_t)o->id[j], (uint32_t)(o->id[j] >> 32), (uint32_t)ev, 5u}, w[4];
    philox(c, key, w);
    double u[4];
    for (int i = 0; i < 4; ++i) u[i] = (double)(((float)(w[i] >> 8) + 0.5f) * (1.0f / 16777216.0f));
    double r1 = sqrt(-2.0 * log(u[0])), r2 = sqrt(-2.0 * log(u[2]));
    double g[3] = {r1 * cos(2.0 * M_PI * u[1]), r1 * sin(2.0 * M_PI * u[1]), r2 * cos(2.0 * M_PI * u[3])};
    F[3 * j] += -gamma * o->vx[j] + amp * g[0];
    F[3 * j + 1] += -gamma * o->vy[j] + amp * g[1];
    F[3 * j + 2] += -gamma * o->vz[j] + amp * g[2];
  }
}

static float wrapf(const Oracle *o, double x) {
  x -= o->L * floor(x / o->L);
  float f = (float)x;
  if (f >= o->Lf) f -= o->Lf;
  if (f < 0.0f) f = 0.0f;
  return f;
}

/* ----------------------------------------------------------------------- */
/* Rigid bodies.  Newton-Euler equations for each body, with the Langevin
 * thermostat acting on the body as a whole (the reading of Sec. IV.B's
 * Langevin-thermostatted nanoparticles): the force on the centre of mass gets
 * -gamma M V + sqrt(2 gamma M / dt) xi, the torque (lab frame)
 * -gamma L + sqrt(2 gamma / dt) I_lab^(1/2) xi' with L = R pi the angular
 * momentum and I_lab^(1/2) = R diag(sqrt(I)) R^T, so that every translational
 * and rotational degree of freedom relaxes at the rate gamma towards kT = 1.
 * xi, xi': Box-Muller normals of the Philox blocks (body, 0, eval, 8) and
 * (body, 0, eval, 9) under the MD key.  Members get no thermostat of their
 * own; their pair forces act on the body.
 * Velocity Verlet: half kicks V += dt/2 F/M, pi += dt/2 R^T T; the drift
 * X += dt V and the free rotation by the symmetric splitting of Dullweber,
 * Leimkuhler and McLachlan (J. Chem. Phys. 107, 5840 (1997)): exact rotations
 * about the body axes 1, 2, 3, 2, 1 for dt/2, dt/2, dt, dt/2, dt/2.  A member
 * then sits at wrap(X + R d) with the velocity V + omega x (R d),
 * omega = R (pi / I). */

static int is_member(const Oracle *o, int j) {
  return o->nbody > 0 && o->id[j] < (uint64_t)o->n_input && o->body_of[o->id[j]] >= 0;
}

/* index of every permanent id (-1 absent) */
static int *permanent_index(const Oracle *o) {
  int *where = malloc((size_t)(o->n_input > 0 ? o->n_input : 1) * sizeof(int));
  for (int j = 0; j < o->n_input; ++j) where[j] = -1;
  for (int j = 0; j < o->n; ++j) if (o->id[j] < (uint64_t)o->n_input) where[o->id[j]] = j;
  return where;
}

static void rb_mul(const double R[9], const double v[3], double out[3]) {
  for (int a = 0; a < 3; ++a) out[a] = R[3 * a] * v[0] + R[3 * a + 1] * v[1] + R[3 * a + 2] * v[2];
}
static void rb_tmul(const double R[9], const double v[3], double out[3]) {
  for (int a = 0; a < 3; ++a) out[a] = R[a] * v[0] + R[3 + a] * v[1] + R[6 + a] * v[2];
}
static void rb_cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Eigenvalues w and eigenvectors (the columns of V) of a symmetric 3x3 matrix
 * by cyclic Jacobi rotations (Golub & Van Loan, Matrix Computations, Sec. 8.5). */
static void jacobi3(const double A_in[9], double w[3], double V[9]) {
  double A[9];
  memcpy(A, A_in, sizeof(A));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double diag = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-32 * diag || off == 0.0) break;
    static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int r = 0; r < 3; ++r) {
      int p = PQ[r][0], q = PQ[r][1];
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      double tau = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      for (int k = 0; k < 3; ++k) { /* A <- A J, V <- V J */
        double akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - s * akq;
        A[3 * k + q] = s * akp + c * akq;
        double vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - s * vkq;
        V[3 * k + q] = s * vkp + c * vkq;
      }
      for (int k = 0; k < 3; ++k) { /* A <- J^T A */
        double apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - s * aqk;
        A[3 * q + k] = s * apk + c * aqk;
      }
    }
  }
  for (int k = 0; k < 3; ++k) w[k] = A[4 * k];
}

/* exact free rotation about body axis k for a time t: R <- R Rot_k(theta),
 * pi <- Rot_k(theta)^T pi, theta = t pi_k / I_k */
static void rb_rotate(or_body *b, int k, double t) {
  double th = t * b->pi[k] / b->I[k], c = cos(th), s = sin(th);
  int i = (k + 1) % 3, j = (k + 2) % 3;
  for (int a = 0; a < 3; ++a) {
    double ri = b->R[3 * a + i], rj = b->R[3 * a + j];
    b->R[3 * a + i] = c * ri + s * rj;
    b->R[3 * a + j] = -s * ri + c * rj;
  }
  double pi_i = b->pi[i], pi_j = b->pi[j];
  b->pi[i] = c * pi_i + s * pi_j;
  b->pi[j] = -s * pi_i + c * pi_j;
}

/* members' velocities (and, with pos, positions) from the body's state */
static void rb_place(Oracle *o, const or_body *b, const int *where, int pos) {
  double om[3], w[3];
  for (int k = 0; k < 3; ++k) w[k] = b->pi[k] / b->I[k];
  rb_mul(b->R, w, om);
  for (int m = 0; m < b->count; ++m) {
    int j = where[b->first + m];
    double a[3], u[3];
    rb_mul(b->R, b->d + 3 * m, a);
    rb_cross(om, a, u);
    o->vx[j] = b->V[0] + u[0]; o->vy[j] = b->V[1] + u[1]; o->vz[j] = b->V[2] + u[2];
    if (pos) {
      o->x[j] = wrapf(o, b->X[0] + a[0]);
      o->y[j] = wrapf(o, b->X[1] + a[1]);
      o->z[j] = wrapf(o, b->X[2] + a[2]);
    }
  }
}

/* three normal deviates from the Philox block (c0, 0, eval, purpose), the
 * Box-Muller form of the particles' Langevin noise */
static void rb_normals(const uint32_t key[2], uint32_t c0, uint32_t ev, uint32_t purpose, double g[3]) {
  uint32_t c[4] = {c0, 0u, ev, purpose}, w[4];
  philox(c, key, w);
  double u[4];
  for (int i = 0; i < 4; ++i) u[i] = (double)(((float)(w[i] >> 8) + 0.5f) * (1.0f / 16777216.0f));
  double r1 = sqrt(-2.0 * log(u[0])), r2 = sqrt(-2.0 * log(u[2]));
  g[0] = r1 * cos(2.0 * M_PI * u[1]);
  g[1] = r1 * sin(2.0 * M_PI * u[1]);
  g[2] = r2 * cos(2.0 * M_PI * u[3]);
}

/* force and torque of every body from its members' forces F, plus the
 * Langevin terms; kick: the half kick that closes a step */
static void rb_forces(Oracle *o, const double *F, double gamma, double dt, uint64_t seed, uint64_t ev, int kick) {
  if (o->nbody == 0) return;
  int *where = permanent_index(o);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int bi = 0; bi < o->nbody; ++bi) {
    or_body *b = &o->body[bi];
    double Fb[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    for (int m = 0; m < b->count; ++m) {
      int j = where[b->first + m];
      double a[3], t[3];
      rb_mul(b->R, b->d + 3 * m, a);
      if (g_plant == PLANT_RIGID_TORQUE_SIGN) rb_cross(F + 3 * j, a, t);
      else rb_cross(a, F + 3 * j, t);
      for (int k = 0; k < 3; ++k) { Fb[k] += F[3 * j + k]; T[k] += t[k]; }
    }
    double gt[3], gr[3], L[3], sg[3], S[3];
    rb_normals(key, (uint32_t)bi, (uint32_t)ev, 8u, gt);
    rb_normals(key, (uint32_t)bi, (uint32_t)ev, 9u, gr);
    double at = sqrt(2.0 * gamma * b->M / dt), ar = sqrt(2.0 * gamma / dt);
    rb_mul(b->R, b->pi, L);
    rb_tmul(b->R, gr, sg); /* I_lab^(1/2) xi' = R diag(sqrt I) R^T xi' */
    for (int k = 0; k < 3; ++k) sg[k] *= sqrt(b->I[k]);
    rb_mul(b->R, sg, S);
    for (int k = 0; k < 3; ++k) {
      Fb[k] += -gamma * b->M * b->V[k] + at * gt[k];
      T[k] += -gamma * L[k] + (g_plant == PLANT_RIGID_NO_ROT_NOISE ? 0.0 : ar * S[k]);
      b->F[k] = Fb[k];
      b->T[k] = T[k];
    }
    if (kick) {
      double tb[3];
      rb_tmul(b->R, b->T, tb);
      for (int k = 0; k < 3; ++k) { b->V[k] += 0.5 * dt * b->F[k] / b->M; b->pi[k] += 0.5 * dt * tb[k]; }
      rb_place(o, b, where, 0);
    }
  }
  free(where);
}

/* the opening half kick and the drift of every body; members follow */
static void rb_kick_drift(Oracle *o, double dt) {
  if (o->nbody == 0) return;
  int *where = permanent_index(o);
  for (int bi = 0; bi < o->nbody; ++bi) {
    or_body *b = &o->body[bi];
    double tb[3];
    rb_tmul(b->R, b->T, tb);
    for (int k = 0; k < 3; ++k) { b->V[k] += 0.5 * dt * b->F[k] / b->M; b->pi[k] += 0.5 * dt * tb[k]; }
    for (int k = 0; k < 3; ++k) b->X[k] += dt * b->V[k];
    rb_rotate(b, 0, 0.5 * dt);
    rb_rotate(b, 1, 0.5 * dt);
    rb_rotate(b, 2, dt);
    rb_rotate(b, 1, 0.5 * dt);
    rb_rotate(b, 0, 0.5 * dt);
    rb_place(o, b, where, 1);
  }
  free(where);
}

/* Declare rigid bodies: body b is the permanent particles with ids
 * [first[b], first[b] + count[b]) (at least two, none of them an ion, no id
 * in two bodies).  The centre of mass and the inertia tensor come from the
 * current positions (minimum-image offsets from the first member), V from
 * the members' total momentum, the angular momentum from their velocities
 * about the centre; the body axes are the principal axes, in ascending order
 * of the moments, each of the first two with its largest component positive,
 * the third their cross product.  A body whose smallest moment is below
 * 1e-9 of the trace (collinear members) is refused.  The members' velocities
 * become the rigid ones.  n = 0 removes every body. */
int32_t or_set_bodies(Oracle *o, int32_t nb, const int32_t *first, const int32_t *count) {
  if (nb < 0 || (nb > 0 && (!first || !count))) return OR_ERR_ARG;
  int *mark = calloc((size_t)(o->n_input > 0 ? o->n_input : 1), sizeof(int));
  int *where = permanent_index(o);
  int rc = OR_OK;
  for (int b = 0; b < nb && rc == OR_OK; ++b) {
    if (count[b] < 2 || first[b] < 0 || (int64_t)first[b] + count[b] > o->n_input) { rc = OR_ERR_ARG; break; }
    for (int m = 0; m < count[b]; ++m) {
      int id = first[b] + m;
      if (mark[id] || where[id] < 0 || is_ion(o->type[where[id]])) { rc = OR_ERR_ARG; break; }
      mark[id] = 1;
    }
  }
  free(mark);
  or_body *nbody = NULL;
  if (rc == OR_OK && nb > 0) {
    nbody = calloc((size_t)nb, sizeof(or_body));
    for (int bi = 0; bi < nb && rc == OR_OK; ++bi) {
      or_body *b = &nbody[bi];
      b->first = first[bi];
      b->count = count[bi];
      b->M = (double)b->count;
      b->d = malloc((size_t)b->count * 3 * sizeof(double));
      int j0 = where[b->first];
      double r0[3] = {o->x[j0], o->y[j0], o->z[j0]}, s[3] = {0, 0, 0}, P[3] = {0, 0, 0};
      for (int m = 0; m < b->count; ++m) {
        int j = where[b->first + m];
        double r[3] = {o->x[j], o->y[j], o->z[j]}, v[3] = {o->vx[j], o->vy[j], o->vz[j]};
        for (int k = 0; k < 3; ++k) {
          b->d[3 * m + k] = min_image(r[k] - r0[k], o->L);
          s[k] += b->d[3 * m + k];
          P[k] += v[k];
        }
      }
      double I[9] = {0}, L[3] = {0, 0, 0};
      for (int k = 0; k < 3; ++k) { b->X[k] = r0[k] + s[k] / b->M; b->V[k] = P[k] / b->M; }
      for (int m = 0; m < b->count; ++m) {
        int j = where[b->first + m];
        double *d = b->d + 3 * m, v[3] = {o->vx[j], o->vy[j], o->vz[j]}, l[3];
        for (int k = 0; k < 3; ++k) d[k] -= s[k] / b->M;
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) I[3 * a + c] += (a == c ? d2 : 0.0) - d[a] * d[c];
        rb_cross(d, v, l);
        for (int k = 0; k < 3; ++k) L[k] += l[k];
      }
      double w[3], V[9];
      jacobi3(I, w, V);
      int ord[3] = {0, 1, 2}; /* ascending moments */
      for (int a = 0; a < 3; ++a)
        for (int c = a + 1; c < 3; ++c)
          if (w[ord[c]] < w[ord[a]]) { int t = ord[a]; ord[a] = ord[c]; ord[c] = t; }
      double e[3][3];
      for (int k = 0; k < 2; ++k) {
        int big = 0;
        for (int a = 0; a < 3; ++a) {
          e[k][a] = V[3 * a + ord[k]];
          if (fabs(e[k][a]) > fabs(e[k][big])) big = a;
        }
        if (e[k][big] < 0.0) for (int a = 0; a < 3; ++a) e[k][a] = -e[k][a];
      }
      rb_cross(e[0], e[1], e[2]);
      for (int k = 0; k < 3; ++k) {
        b->I[k] = w[ord[k]];
        for (int a = 0; a < 3; ++a) b->R[3 * a + k] = e[k][a];
      }
      if (!(b->I[0] > 1e-9 * (b->I[0] + b->I[1] + b->I[2]))) { rc = OR_ERR_ARG; break; }
      rb_tmul(b->R, L, b->pi);
      for (int m = 0; m < b->count; ++m) {
        double dl[3] = {b->d[3 * m], b->d[3 * m + 1], b->d[3 * m + 2]};
        rb_tmul(b->R, dl, b->d + 3 * m);
      }
    }
  }
  if (rc != OR_OK) {
    if (nbody) for (int b = 0; b < nb; ++b) free(nbody[b].d);
    free(nbody);
    free(where);
    return rc;
  }
  for (int b = 0; b < o->nbody; ++b) free(o->body[b].d);
  free(o->body);
  free(o->body_of);
  o->body = nbody;
  o->nbody = nb;
  o->body_of = malloc((size_t)(o->n_input > 0 ? o->n_input : 1) * sizeof(int));
  for (int j = 0; j < o->n_input; ++j) o->body_of[j] = -1;
  for (int b = 0; b < nb; ++b)
    for (int m = 0; m < o->body[b].count; ++m) o->body_of[o->body[b].first + m] = b;
  for (int b = 0; b < nb; ++b) rb_place(o, &o->body[b], where, 0);
  free(where);
  o->f_valid = 0;
  return OR_OK;
}

/* per body 22 values: X[3], V[3], R[9] (row-major), pi[3], I[3], M */
int32_t or_body_state(const Oracle *o, double *out) {
  for (int b = 0; b < o->nbody; ++b) {
    const or_body *B = &o->body[b];
    double *r = out + 22 * b;
    memcpy(r, B->X, 3 * sizeof(double));
    memcpy(r + 3, B->V, 3 * sizeof(double));
    memcpy(r + 6, B->R, 9 * sizeof(double));
    memcpy(r + 15, B->pi, 3 * sizeof(double));
    memcpy(r + 18, B->I, 3 * sizeof(double));
    r[21] = B->M;
  }
  return o->nbody;
}

/* overwrite X, V, R and pi of every body (records as or_body_state writes
 * them; I and M are kept) to re-synchronise with another run */
int32_t or_set_body_state(Oracle *o, const double *in, int32_t nb) {
  if (nb != o->nbody) return OR_ERR_ARG;
  for (int b = 0; b < nb; ++b) {
    or_body *B = &o->body[b];
    const double *r = in + 22 * b;
    memcpy(B->X, r, 3 * sizeof(double));
    memcpy(B->V, r + 3, 3 * sizeof(double));
    memcpy(B->R, r + 6, 9 * sizeof(double));
    memcpy(B->pi, r + 15, 3 * sizeof(double));
  }
  return OR_OK;
}

/* Velocity Verlet with Langevin friction/noise added at each force
 * evaluation (unit mass, kT = 1).  Forces are re-evaluated first when the
 * CR-MC stage changed the system since the last evaluation. */
int32_t or_md_step(Oracle *o, int32_t n_steps, double dt, double gamma, uint64_t seed) {
  double *F = malloc((size_t)(o->n > 0 ? o->n : 1) * 3 * sizeof(double));
  int rc = OR_OK;
  if (!o->f_valid) {
    rc = forces_cons(o, F, NULL);
    if (rc) { free(F); return rc; }
    rb_forces(o, F, gamma, dt, seed, o->md_evals, 0);
    langevin(o, F, gamma, 1.0, dt, seed, o->md_evals++);
    for (int j = 0; j < o->n; ++j) { o->fx[j] = F[3 * j]; o->fy[j] = F[3 * j + 1]; o->fz[j] = F[3 * j + 2]; }
    o->f_valid = 1;
  }
  for (int s = 0; s < n_steps; ++s) {
    for (int j = 0; j < o->n; ++j) {
      if (is_member(o, j)) continue;
      o->vx[j] += 0.5 * dt * o->fx[j]; o->vy[j] += 0.5 * dt * o->fy[j]; o->vz[j] += 0.5 * dt * o->fz[j];
      o->x[j] = wrapf(o, (double)o->x[j] + dt * o->vx[j]);
      o->y[j] = wrapf(o, (double)o->y[j] + dt * o->vy[j]);
      o->z[j] = wrapf(o, (double)o->z[j] + dt * o->vz[j]);
    }
    rb_kick_drift(o, dt);
    rc = forces_cons(o, F, NULL);
    if (rc) break;
    rb_forces(o, F, gamma, dt, seed, o->md_evals, 1);
    langevin(o, F, gamma, 1.0, dt, seed, o->md_evals++);
    for (int j = 0; j < o->n; ++j) {
      o->fx[j] = F[3 * j]; o->fy[j] = F[3 * j + 1]; o->fz[j] = F[3 * j + 2];
      if (is_member(o, j)) continue;
      o->vx[j] += 0.5 * dt * o->fx[j]; o->vy[j] += 0.5 * dt * o->fy[j]; o->vz[j] += 0.5 * dt * o->fz[j];
    }
  }
  free(F);
  return rc;
}

/* overwrite positions / velocities from id-sorted arrays (used to re-sync the
 * oracle to a state before a parity window) */
/* The MD step split around a CR-MC call: or_md_begin evaluates the forces
 * if a CR-MC call changed the system since the last evaluation, then does
 * the first half kick and the drift; or_md_end evaluates the forces (with the
 * charges after any CR-MC trials run in between) and does the closing half
 * kick.  begin + end with nothing in between is or_md_step with one step. */
int32_t or_md_begin(Oracle *o, double dt, double gamma, uint64_t seed) {
  double *F = malloc((size_t)(o->n > 0 ? o->n : 1) * 3 * sizeof(double));
  int rc = OR_OK;
  if (!o->f_valid) {
    rc = forces_cons(o, F, NULL);
    if (rc) { free(F); return rc; }
    rb_forces(o, F, gamma, dt, seed, o->md_evals, 0);
    langevin(o, F, gamma, 1.0, dt, seed, o->md_evals++);
    for (int j = 0; j < o->n; ++j) { o->fx[j] = F[3 * j]; o->fy[j] = F[3 * j + 1]; o->fz[j] = F[3 * j + 2]; }
  }
  for (int j = 0; j < o->n; ++j) {
    if (is_member(o, j)) continue;
    o->vx[j] += 0.5 * dt * o->fx[j]; o->vy[j] += 0.5 * dt * o->fy[j]; o->vz[j] += 0.5 * dt * o->fz[j];
    o->x[j] = wrapf(o, (double)o->x[j] + dt * o->vx[j]);
    o->y[j] = wrapf(o, (double)o->y[j] + dt * o->vy[j]);
    o->z[j] = wrapf(o, (double)o->z[j] + dt * o->vz[j]);
  }
  rb_kick_drift(o, dt);
  o->f_valid = 0;
  free(F);
  return rc;
}

int32_t or_md_end(Oracle *o, double dt, double gamma, uint64_t seed) {
  double *F = malloc((size_t)(o->n > 0 ? o->n : 1) * 3 * sizeof(double));
  int rc = forces_cons(o, F, NULL);
  if (!rc) {
    rb_forces(o, F, gamma, dt, seed, o->md_evals, 1);
    langevin(o, F, gamma, 1.0, dt, seed, o->md_evals++);
    for (int j = 0; j < o->n; ++j) {
      o->fx[j] = F[3 * j]; o->fy[j] = F[3 * j + 1]; o->fz[j] = F[3 * j + 2];
      if (is_member(o, j)) continue;
      o->vx[j] += 0.5 * dt * o->fx[j]; o->vy[j] += 0.5 * dt * o->fy[j]; o->vz[j] += 0.5 * dt * o->fz[j];
    }
    o->f_valid = 1;
  }
  free(F);
  return rc;
}

int32_t or_set_positions(Oracle *o, const uint64_t *ids, const float *xyz, const float *vel, int32_t n) {
  if (n != o->n) return OR_ERR_ARG;
  for (int j = 0; j < o->n; ++j) {
    int lo = 0, hi = n - 1, at = -1;
    while (lo <= hi) {
      int mid = (lo + hi) / 2;
      if (ids[mid] == o->id[j]) { at = mid; break; }
      if (ids[mid] < o->id[j]) lo = mid + 1; else hi = mid - 1;
    }
    if (at < 0) return OR_ERR_ARG;
    o->x[j] = xyz[3 * at]; o->y[j] = xyz[3 * at + 1]; o->z[j] = xyz[3 * at + 2];
    if (vel) { o->vx[j] = vel[3 * at]; o->vy[j] = vel[3 * at + 1]; o->vz[j] = vel[3 * at + 2]; }
  }
  o->f_valid = 0;
  return OR_OK;
}
