/*
 * crmc.h -- C ABI of libcrmc.so: the charge-regulation Monte Carlo (CR-MC)
 * stage of the hybrid MD/CR-MC method (Curk, Yuan & Luijten, arXiv:2109.07527)
 * on one GB300 GPU, with the MD force/integration step that consumes the
 * regulated charges.
 *
 * Conventions for every entry point:
 *   - Return value: CR_OK (0) on success, a negative CR_ERR_* code otherwise.
 *     No C++ exception crosses this boundary.  cr_strerror() names the codes.
 *   - Host pointers are owned by the caller and only read or written during
 *     the call.  The library owns all device memory of a context; it is
 *     released by cr_destroy().
 *   - Work is queued on the context's CUDA stream (cr_set_stream); calls that
 *     return host data (cr_state, cr_sweep with stats or log, cr_md_forces
 *     with output) synchronise that stream.
 *   - Units: lengths in sigma, energies in kT (beta = 1), charges in e.
 *
 * The method (paper references):
 *   Reactions (Sec. II.B, Eqs. acid_new, base_new, salt_new):
 *       A <-> A- + X+,   B <-> B+ + X-,   0 <-> X+ + X-
 *   with all monovalent cations grouped into X+ and anions into X-
 *   (Eqs. mux1, mux2; App. A).  Six moves, forward/reverse with equal
 *   probability, participants drawn uniformly from the eligible particles,
 *   automatic rejection when none exists (Sec. II.C).  Acceptance
 *   (Sec. II.C, Eqs. acidacc, MCmetro, the base pair, MCsaltf, MCmetro2):
 *     acid fwd : min[1, (nA - nA-) rho0 NA v / ((nA- + 1)(nX+ + 1)) 10^(pH - pKa - pIX+) e^-dE]
 *     acid rev : min[1, nA- nX+ / ((nA - nA- + 1) rho0 NA v) 10^(-pH + pKa + pIX+) e^-dE]
 *     base     : the same with pOH, pKb, pIX-, nX-
 *     salt ins : min[1, (rho0 NA v)^2 / ((nX+ + 1)(nX- + 1)) 10^(-pIX+ - pIX-) e^-dE]
 *     salt del : min[1, nX+ nX- / (rho0 NA v)^2 10^(pIX+ + pIX-) e^-dE]
 *   with rho0 = 1 M and 10^-pIX = 10^-pIS + 10^-min(pH, pOH) (App. C, Eq. pIXgen).
 *   This library evaluates the moves domain-locally: v is the volume of the
 *   trial's domain, the counts are that domain's counts, and the paired ion
 *   is inserted in / deleted from that domain; same-colour domains of an
 *   8-colour checkerboard are at least r_c apart and run concurrently.
 *   CR_SCHED_GLOBAL (one domain = the box) gives the paper's rule verbatim.
 *   Energy: damped-shifted-force Coulomb (cutoff r_c, damping alpha, with its
 *   self term) + WCA / expanded WCA (Eq. LJe); the paper itself uses PPPM.
 */
#ifndef CRMC_H
#define CRMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CR_OK 0
#define CR_ERR_INVALID_ARG (-1)   /* bad argument or inconsistent system */
#define CR_ERR_NOT_NEUTRAL (-2)   /* initial system is not charge neutral */
#define CR_ERR_CELL_OVERFLOW (-3) /* a cell exceeded its slot capacity */
#define CR_ERR_CAPACITY (-4)      /* particle capacity exhausted */
#define CR_ERR_TIMEOUT (-5)       /* a bounded device wait gave up */
#define CR_ERR_BOND_BROKEN (-6)   /* a FENE bond reached R0 */
#define CR_ERR_CUDA (-7)          /* a CUDA runtime call failed */
#define CR_ERR_NOMEM (-8)         /* device or host allocation failed */
#define CR_ERR_NO_DEVICE (-9)     /* no CUDA device is visible */

/* ---- particle types (input encoding) ---- */
#define CR_BEAD 0 /* neutral monomer / bead */
#define CR_ACID 1 /* acid site: neutral A or ionised A- (charge -1) */
#define CR_BASE 2 /* base site: neutral B or ionised B+ (charge +1) */
#define CR_XP 3   /* grouped monovalent cation X+ */
#define CR_XM 4   /* grouped monovalent anion X- */
#define CR_CORE 5 /* neutral nanoparticle core (expanded WCA) */
/* Salt ions kept apart from X+- (Sec. II.B: the scheme applied separately to
 * dissociated and salt ions, the grand-reaction ensemble; App. B: the method
 * invoked repeatedly with different types of ions).  They interact exactly as
 * X+- (charge +-1, the ions' class); only cr_set_invocation tells them apart.
 * Without invocations, X+ and X- play the roles of H+ and OH-. */
#define CR_SP 6   /* salt cation S+ */
#define CR_SM 7   /* salt anion S- */

/* short-range class 3 never interacts by WCA */
#define CR_CLS_NONE 3

#define CR_SCHED_COLOURED 0 /* 8-colour checkerboard of domains */
#define CR_SCHED_GLOBAL 1   /* one domain = the whole box (paper's rule) */

/* trial-record flags */
#define CR_TRIAL_ACCEPTED 1
#define CR_TRIAL_NO_ELIGIBLE 2 /* automatic rejection: no eligible particle */
#define CR_TRIAL_EDGE 4        /* insertion point rounded out of the domain */
#define CR_TRIAL_OVERLAP 8     /* hard overlap of an inserted ion: dE = +inf */

typedef struct cr_ctx cr_ctx; /* opaque, library-owned */

/* System description, read by cr_init (the arrays are copied). */
typedef struct {
  int32_t n;            /* particles at start (>= 0) */
  int32_t capacity;     /* maximum particles over the run (>= n) */
  double box_L;         /* side of the cubic periodic box; rounded to FP32 */
  double sigma_nm;      /* sigma in nm, converts v to nm^3 for rho0 N_A v */
  const float *xyz;     /* [3n] positions in [0, box_L) */
  const int32_t *type;  /* [n] CR_BEAD .. CR_CORE */
  const int32_t *cls;   /* [n] short-range class 0..3 (ions take ion_cls) */
  const int8_t *state;  /* [n] sites: 1 = ionised; ignored for others */
  const float *vel;     /* [3n] velocities, or NULL for zero */
  int32_t n_bonds;      /* FENE bonds */
  const int32_t *bonds; /* [2 n_bonds] particle indices; no ions */
  double fene_K, fene_R0;
  double wca_eps[16], wca_sig[16], wca_del[16]; /* class-pair table [4*ci + cj], symmetric */
  int32_t wca_on[16];
  double dsf_alpha;        /* DSF damping (1/sigma) */
  int32_t dsf_self;        /* 1: include the DSF self energy of each charge */
  int32_t ion_coupling;    /* 1: ions charged and WCA-interacting; 0: ghost ions */
  int32_t ion_cls;         /* short-range class of X+/X- */
  int32_t cells_per_rc;    /* h: cell side >= r_c / h (default 2) */
  int32_t domain_cells;    /* k: a domain is k^3 cells, k * cell >= r_c (default h) */
  int32_t trials_per_domain; /* m: sequential trials per domain per colour phase */
  int32_t schedule;        /* CR_SCHED_COLOURED or CR_SCHED_GLOBAL */
  int32_t nc;              /* cells per dimension; 0 = automatic */
  int32_t cell_capacity;   /* slots per cell; 0 = automatic */
  int32_t list_capacity;   /* domain particles held in shared memory per CTA; 0 = automatic */
  int32_t halo_capacity;   /* halo particles held on chip per CTA; 0 = automatic */
  int32_t ewald_kmax;      /* 0: DSF energy; > 0: Ewald electrostatics (global schedule only), below */
} cr_system;

/* Ewald electrostatics (ewald_kmax > 0).  The paper's energy model is PPPM
 * (Sec. III.A), a mesh evaluation of the Ewald sum; here the sum is taken
 * directly: E = E_real + E_rec + E_self with E_real = lB sum_{i<j, r < rc}
 * q_i q_j erfc(alpha r) / r (alpha = dsf_alpha), E_rec = (2 pi lB / V) sum_k
 * exp(-k^2 / (4 alpha^2)) / k^2 |S(k)|^2 over k = 2 pi n / L with
 * 0 < |n|^2 <= ewald_kmax^2, S(k) = sum_j q_j exp(i k.r_j), and E_self = -lB
 * alpha / sqrt(pi) sum_j q_j^2 (tin-foil boundary; every state is neutral).
 * A trial's Delta E is the real-space pair sum of its changed particles, the
 * self change and the change of E_rec, with S(k) recomputed at every sweep and
 * carried by the accepted trials within it.  Only with CR_SCHED_GLOBAL, the
 * paper's one-trial-at-a-time rule: trials of different domains would
 * interact through S(k), so concurrent domain-local trials would not be
 * independent.  MD forces are minus the gradient of the same energy: the
 * real-space erfc pair forces plus F_j = 2 q_j sum_k A_k k Im(S(k)^*
 * exp(i k.r_j)) (A_k the weights above), S(k) recomputed from the positions
 * at every force evaluation (cr_md_forces, cr_md_step, cr_md_begin /
 * cr_md_end).  Not available with Ewald (INVALID_ARG): delayed acceptance,
 * the captured batch cycle (cr_batch_cycle) and cr_md_forces_noalloc.
 * ewald_kmax <= 32. */

/* Reservoir ions: pI_S of the symmetric salt per sign and pKw; with
 * pIX_explicit = 1 the grouped pI_X+- are taken as given (e.g. pIX+ = pH,
 * pIX- = pOH for the conventional reaction ensemble). */
typedef struct {
  double pI_S_plus, pI_S_minus, pKw;
  int32_t pIX_explicit;
  double pIX_plus, pIX_minus;
} cr_mu_ions;

/* Per-call statistics (attempts and accepts per move: 2*reaction + reverse,
 * reaction 0 acid, 1 base, 2 salt). */
typedef struct {
  int64_t trials;
  int64_t attempts[6], accepts[6];
  int64_t no_eligible, edge, overlap;
} cr_sweep_stats;

/* One trial record (schedule order: colour phases, domains ascending,
 * trials within a domain).  ids: UINT64_MAX when unused. */
typedef struct {
  int32_t move;  /* 2*reaction + (0 forward, 1 reverse) */
  int32_t flags; /* CR_TRIAL_* */
  uint64_t id_a; /* site (acid/base) or first ion (salt) */
  uint64_t id_b; /* ion paired with the site, or second ion */
  double dE;     /* energy change (kT); +inf on overlap */
  double S;      /* gross magnitude of the summed pair terms (tolerance scale) */
  double lnA;    /* log acceptance ratio */
  double lnu;    /* log of the Metropolis uniform */
} cr_trial;

/* ---- learned delayed acceptance (DA) ----
 * A surrogate stage in front of the exact Metropolis test (Christen & Fox,
 * 2005; the paper evaluates every trial exactly):
 *   stage 1: accept with min(1, R exp(-(dE_self + dE~))), R the combinatorial
 *            and chemical factor of the move (Sec. II.C), dE_self the exact
 *            DSF self-term change, dE~ the surrogate pair-energy change; a
 *            stage-1 rejection ends the trial without the exact pair sum;
 *   stage 2: accept with min(1, exp(-(dE_pair - dE~))).
 * The chain keeps the stationary distribution of Eq. (QQ) because dE~ is
 * antisymmetric under move reversal: dE~ = (mlp(F) - mlp(-F)) / 2 with
 * features F that change sign when the move is reversed.  Features (48): for
 * each changed particle s (a = the site, or the cation of a salt move; b =
 * the ion, or the anion) over the 5^3 half-cutoff cells around its cell,
 * binned into 8 shells by the squared integer cell offset
 * {0},{1},{2},{3},{4},{5},{6},{8,9,12}: dq_s x (ion charge), dq_s x (site
 * charge) and eta_s x (particle count), every particle other than a and b
 * counted (dq_s: charge change of s; eta_s: +1 inserted, -1 deleted, else 0);
 * plus q_a' q_b' - q_a q_b added at the shell of b relative to a.
 * MLP 48 -> 128 -> 128 -> 128 -> 1, ReLU, BF16 weights, FP32 biases and FP32
 * arithmetic (one fused multiply-add per weight in input order).
 * Needs the coloured schedule, cells_per_rc = 2 and nc >= domain_cells + 4. */
typedef struct {
  const uint16_t *W1;  /* [128][48] BF16 bit patterns (row = output) */
  const float *b1;     /* [128] */
  const uint16_t *W2;  /* [128][128] */
  const float *b2;     /* [128] */
  const uint16_t *W3;  /* [128][128] */
  const float *b3;     /* [128] */
  const uint16_t *w4;  /* [128] */
  float b4;
} cr_mlp;

/* Per-trial record of the DA stages (alongside cr_trial, whose lnA is then
 * the stage-1 log ratio). */
typedef struct {
  float dE_sur;  /* surrogate dE~ */
  int32_t stage; /* 0 no surrogate evaluated, 1 rejected at stage 1, 2 passed stage 1 */
  double lnA2;   /* dE~ - dE_pair (NaN on overlap) */
  double lnu2;   /* log of the stage-2 uniform (Philox purpose 3) */
} cr_trial_da;

/* State view: counts always; arrays when non-NULL (sizes >= n, n_sites). */
typedef struct {
  int64_t n, n_A, n_Am, n_B, n_Bp, n_Xp, n_Xm, net_charge;
  double alpha;          /* n_A- / n_A (0 when there are no acids) */
  int64_t n_Sp, n_Sm;    /* salt ions kept apart (CR_SP, CR_SM; 0 without invocations) */
  float *xyz;            /* [3n] */
  float *vel;            /* [3n] */
  float *force;          /* [3n] forces of the last cr_md_forces (zero once a sweep or step ran) */
  uint64_t *id;          /* [n] particle ids (input index; inserted ions >= 2^32) */
  int32_t *type;         /* [n] */
  int8_t *state;         /* [n] 1 = ionised site */
  int8_t *site_state;    /* [n_sites] by site index (input order of the sites) */
  int32_t *cls;          /* [n] interaction class (0..3), as cr_load takes it */
} cr_state_view;

typedef struct {
  int32_t nc, k, h, nd, ncol, m, cap, global;
  int64_t trials_per_sweep;
  int32_t n_sites, n_perm;
  double cell_side, domain_side;
} cr_info;

/* Create a context: copies the system to the device, precomputes the
 * chemical constants (pH, per-particle pK [n] of sites, reservoir ions,
 * Bjerrum length lB, cutoff rc).  Errors: INVALID_ARG (geometry, ranges,
 * rc > L/2, a WCA class-pair table that is not symmetric), NOT_NEUTRAL,
 * NO_DEVICE, NOMEM, CUDA. */
int cr_init(cr_ctx **out, const cr_system *sys, double pH, const double *pK, cr_mu_ions mu, double lB,
            double rc);

/* Run n_trials CR-MC trials (a positive multiple of trials_per_sweep) with
 * Philox key `seed`; sweeps continue the context's sweep counter.  stats
 * (nullable) receives this call's counts and synchronises the stream. */
int cr_sweep(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats);

/* As cr_sweep, and writes one cr_trial per trial to the host array `log`
 * (n_trials entries).  Slower: used by the parity tests. */
int cr_sweep_log(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats, cr_trial *log);

/* Load the DA surrogate (host arrays, copied).  Errors: INVALID_ARG when the
 * context's geometry does not support DA (see above). */
int cr_set_surrogate(cr_ctx *ctx, const cr_mlp *mlp);

/* As cr_sweep with delayed acceptance (needs cr_set_surrogate). */
int cr_sweep_da(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats);

/* As cr_sweep_da with per-trial records on the host: log [n_trials],
 * dlog [n_trials] and, when non-NULL, features [48 n_trials] (the surrogate
 * input of each trial, zeros when none was evaluated).  The exact pair sum
 * is evaluated for every trial here (recorded in log.dE) but decides only
 * after stage 1, as in cr_sweep_da.  Feature/energy pairs recorded here are
 * the training data of the surrogate (dE_pair = dE~ - lnA2). */
int cr_sweep_da_log(cr_ctx *ctx, uint64_t n_trials, uint64_t seed, cr_sweep_stats *stats, cr_trial *log,
                    cr_trial_da *dlog, float *features);

/* Evaluate the conservative MD forces (DSF Coulomb + WCA + FENE) with the
 * current charges; they become readable through cr_state().force.  The paper
 * couples CR-MC to MD whose every step needs a full force evaluation with the
 * regulated charges (Sec. II.D); the pair forces are -dU/dr of the same DSF
 * and WCA / expanded-WCA (Eqs. LJ, LJe) energies the trials use, the bonds
 * FENE, U = -K R0^2/2 ln(1 - (r/R0)^2) (the paper's own chain model, Eq.
 * bond, is harmonic).  FP32 pair terms summed in exact 2^-24 fixed point. */
int cr_md_forces(cr_ctx *ctx);

/* n_steps of velocity Verlet with Langevin friction gamma and noise at kT = 1
 * (unit mass), time step dt, noise key seed: the integrator and thermostat of
 * the paper's MD (Sec. III.A: velocity Verlet, Langevin damping time tau,
 * dt = 0.005 tau), CR-MC trials running between MD steps (Sec. II.D).  The
 * noise is applied at each force evaluation (BBK form), Box-Muller normals
 * from Philox purpose 5 counted by particle id and force evaluation.  Forces are re-evaluated first
 * when CR-MC changed the system since the last evaluation.  Errors:
 * BOND_BROKEN, CELL_OVERFLOW. */
int cr_md_step(cr_ctx *ctx, int32_t n_steps, double dt, double gamma, uint64_t seed);

/* One MD step split around CR-MC calls (Sec. III.A's velocity Verlet and
 * Langevin thermostat, with the MC trials of Sec. II.C inside the step; the
 * paper interleaves n_MC trials with n_MD steps, Sec. II.D), so that a cycle
 * of trials and one MD step needs a single force evaluation: cr_md_begin evaluates the forces if
 * CR-MC changed the system since the last evaluation, then does the first
 * half kick and the drift (and rebuilds the cells); CR-MC calls may follow;
 * cr_md_end evaluates the forces with the current charges (Langevin terms
 * included) and does the closing half kick.  begin + end with nothing in
 * between equals cr_md_step with one step.  Inserted ions carry
 * Maxwell-Boltzmann velocities (unit mass, kT = 1). */
int cr_md_begin(cr_ctx *ctx, double dt, double gamma, uint64_t seed);
int cr_md_end(cr_ctx *ctx, double dt, double gamma, uint64_t seed);

/* ---- rigid bodies (mobile nanoparticles) ----
 * Sec. IV.B's nanoparticles carry their acid / base groups rigidly attached
 * to the shell, the body's mass the sum of its members' (257 m for a core and
 * 256 groups), under a Langevin thermostat.  cr_set_rigid_bodies declares
 * n_bodies bodies: body b is the permanent particles with ids
 * [first[b], first[b] + count[b]) (input indices of cr_init; at least two
 * members, none of them an ion, no id in two bodies; n_bodies <=
 * CR_MAX_BODIES).  From the current configuration (on the device): the
 * centre of mass X (minimum-image offsets from the first member, unit mass
 * per member), V from the members' momentum, the principal axes of the
 * inertia tensor in ascending order of the moments I (the first two with
 * their largest component positive, the third their cross product) as the
 * body frame R (lab = R body), the angular momentum from the members'
 * velocities about X; the members' velocities become the rigid ones.  From
 * then on cr_md_step / cr_md_begin / cr_md_end move each body as a whole:
 * the members' pair forces give the body's force and torque, the thermostat
 * acts on the body (centre of mass: -gamma M V + sqrt(2 gamma M / dt) xi;
 * rotation, lab frame: -gamma L + sqrt(2 gamma / dt) R diag(sqrt I) R^T xi',
 * Box-Muller normals of the Philox blocks (b, 0, evaluation, 8) and
 * (b, 0, evaluation, 9) under the MD seed), velocity Verlet kicks V and the
 * body-frame angular momentum pi, the drift moves X and rotates the body by
 * the symmetric splitting of Dullweber, Leimkuhler and McLachlan (J. Chem.
 * Phys. 107, 5840 (1997): exact rotations about the body axes 1, 2, 3, 2, 1
 * for dt/2, dt/2, dt, dt/2, dt/2); members sit at X + R d, wrapped, with the
 * velocity V + omega x (R d).  Body arithmetic in FP64.  CR-MC trials change
 * the members' charge states as before.  n_bodies = 0 removes the bodies.
 * Errors: INVALID_ARG (a range or member as above, collinear members, a
 * context in a batch); nothing changes then.  While bodies
 * are declared, cr_load and cr_restore are refused (declare them again after
 * a load into a fresh context) and the context cannot join a batch.
 * cr_rigid_body_state writes 22 doubles per body: X[3], V[3], R[9]
 * (row-major), pi[3], I[3], M; n_bodies must be the number declared. */
#define CR_MAX_BODIES (1 << 20)
int cr_set_rigid_bodies(cr_ctx *ctx, int32_t n_bodies, const int32_t *first, const int32_t *count);
int cr_rigid_body_state(cr_ctx *ctx, int32_t n_bodies, double *out);

/* The force evaluation of cr_md_forces, allocating nothing, with the results
 * written to caller-owned device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library allocate device
 * memory while they run, e.g. an MD engine that owns every device buffer
 * through its own pool, or a time-critical loop in which a device allocation
 * (which may synchronise the whole device) is not acceptable.
 *
 * force: device array of 4 * n_slots floats (16-byte aligned); slot g gets
 *        (fx, fy, fz, 0) of the particle held in it, empty slots (0, 0, 0, 0).
 * id:    device array of n_slots particle ids; UINT64_MAX marks an empty slot.
 * n_slots must be at least nc^3 * cap (cr_get_info); slots beyond that are
 * not written.  Both arrays stay owned by the caller.  The context's own
 * force buffers (cr_state().force) are not touched.
 *
 * Scratch: the particle list lives in one fixed device array of the library,
 * sized for CR_NOALLOC_MAX_PARTICLES particles and shared by every context
 * on a device.  A context created with a capacity above that maximum gets
 * CR_ERR_CAPACITY before anything is launched.  The call clears the scratch
 * counter itself.  Calls whose work overlaps on the GPU (different streams or
 * contexts without ordering between them) race on that scratch: order them
 * on one stream or with events.  Every call looks the scratch's device
 * address up (cudaGetSymbolAddress) with the context's device current.  The
 * forces equal cr_md_forces' bit for bit; this entry finishes each particle
 * on one lane of its warp (cr_md_forces hands the sums to a per-particle
 * kernel through a context buffer), so it is slower on large systems.
 * Synchronises the context's stream.  Errors: INVALID_ARG (NULL or
 * misaligned pointer, n_slots too small, context device not current),
 * CAPACITY, CELL_OVERFLOW, CUDA. */
#define CR_NOALLOC_MAX_PARTICLES 262144
int cr_md_forces_noalloc(cr_ctx *ctx, float *force, uint64_t *id, int64_t n_slots);

/* Fill the view (counts always; arrays when non-NULL) and synchronise.  The
 * counts are the particle numbers of Eq. (QQ) (n_A-, n_B+, n_X+, n_X-); alpha
 * is the instantaneous degree of dissociation n_A- / n_A whose average is the
 * paper's observable alpha = <n_A-> / n_A (Sec. II.D).
 * Arrays are ordered by particle id (the ordering runs on the device: input
 * ids by a prefix count, inserted ions by their rank among the ion ids, or a
 * device-wide radix sort past 16,384 ions), one device-to-host copy per
 * array; pinned host arrays make those copies asynchronous DMA. */
int cr_state(cr_ctx *ctx, cr_state_view *out);

/* Replace the configuration with n particles from host arrays (xyz [3n],
 * vel [3n] or NULL, type [n], cls [n], state [n]; pinned memory gives
 * asynchronous copies).  Particle ids become the indices.  Bonded and site
 * particles must be those given to cr_init, at the same indices (the state
 * arrays returned by cr_state qualify); ions may differ.  The arrays are
 * checked and the cells rebuilt on the device, asynchronously: INVALID_ARG
 * for NULL arrays or n out of range at once; a particle of unknown type or
 * class, outside [0, L), or a bonded / site particle missing or moved
 * (INVALID_ARG), a configuration that is not neutral (NOT_NEUTRAL) and a full
 * cell (CELL_OVERFLOW) at the next synchronising call (cr_check, cr_state);
 * the context is then unusable. */
int cr_load(cr_ctx *ctx, int32_t n, const float *xyz, const float *vel, const int32_t *type, const int32_t *cls,
            const int8_t *state);

/* ---- checkpoint / resume ----
 * A run split into a checkpoint and a restore into a fresh context (created
 * by cr_init from the same system, pH and parameters) continues the unsplit
 * chain bit for bit: the trials' random numbers are Philox counters of the
 * sweep number (Sec. II.C's moves drawn per phase), the Langevin noise of the
 * force-evaluation number, and the cells stay ordered by particle id.
 * cr_counters carries those counters and whether the integrator holds the
 * forces of the next half kick (after cr_md_end / cr_md_step, not after
 * cr_md_begin or a sweep). */
typedef struct {
  uint64_t sweep;       /* sweeps run so far */
  uint32_t md_eval;     /* force evaluations so far */
  int32_t forces_valid; /* 1: the checkpoint's forces feed the next half kick */
} cr_counters;
/* cr_state (same arrays, ordered by id), except that out->force receives the
 * integrator's forces (Langevin terms included) when they are valid, zeros
 * otherwise; and the counters.  Synchronises. */
int cr_checkpoint(cr_ctx *ctx, cr_state_view *out, cr_counters *counters);
/* cr_load with the particle ids (input ids below 2^32 as given to cr_init,
 * inserted ions at or above 2^32), the integrator forces (read when
 * counters->forces_valid; may be NULL otherwise) and the counters of a
 * checkpoint.  The ids are checked on the host (unique; every bonded and
 * site particle of cr_init present; INVALID_ARG otherwise), the particles
 * on the device as by cr_load. */
int cr_restore(cr_ctx *ctx, int32_t n, const float *xyz, const float *vel, const float *force, const uint64_t *id,
               const int32_t *type, const int32_t *cls, const int8_t *state, const cr_counters *counters);

/* Launch shape of the colour-phase kernel: threads per domain and halo
 * particles held in registers per thread.  Supported pairs: (32|64|128|256|512,
 * 0) halo in shared memory; (128, 4), (256, 2), (512, 1) halo in registers.
 * By default the first unlogged sweeps time every supported shape (with full
 * and with compact shared-memory capacities) in two passes, one shape per
 * sweep, and keep the shape with the shortest time; the
 * trial outcomes never depend on the shape (the energy sums are exact fixed
 * point).  cr_set_launch_shape(ctx, 0, 0) restarts the tuning; an unsupported
 * pair gives CR_ERR_INVALID_ARG. */
int cr_set_launch_shape(cr_ctx *ctx, int32_t threads, int32_t regs);
int cr_get_launch_shape(const cr_ctx *ctx, int32_t *threads, int32_t *regs);

/* Record CUDA events around every colour-phase and MD-force launch. */
int cr_set_timing(cr_ctx *ctx, int32_t enable);

/* Synchronise and report: ms[2] summed device time and launches[2] of the
 * colour-phase kernel (0) and the MD force kernel (1) since the last reset,
 * and the number of kernels this context launched.  reset != 0 zeroes them. */
int cr_get_timing(cr_ctx *ctx, double *ms, int64_t *launches, int64_t *launches_total, int32_t reset);

/* A new reservoir pH from the next trial on: the paper's implementation
 * accepts a variable (time-dependent) pH, e.g. to follow a system's response
 * to a pH increase (App. B).  Recomputes pOH = pKw - pH, the grouped pI_X+-
 * of Eq. (pIXgen) (unless they were given explicitly) and the equilibrium
 * constants K_A = 10^(pH - pKa - pI_X+), K_B = 10^(pOH - pKb - pI_X-) and
 * K_ion = 10^(-pI_X+ - pI_X-) (Sec. II.D) exactly as cr_init does, in stream
 * order (trials queued before the call keep the old pH).  Batches holding the
 * context pick the change up at their next sweep.  Synchronises. */
int cr_set_pH(cr_ctx *ctx, double pH);

/* One invocation of the scheme for the following sweeps (App. B: the method
 * can be invoked repeatedly to perform reactions with different types of
 * ions, which realises the grand-reaction ensemble; Sec. II.B).  The acid,
 * base and salt reactions of Eqs. (acid_new)-(salt_new) then exchange a
 * cation of type `cation` (CR_XP or CR_SP) and an anion of type `anion`
 * (CR_XM or CR_SM) with the reservoir at chemical potentials pI_cation and
 * pI_anion in place of pI_X+ and pI_X-:
 *   K_A = 10^(pH - pKa - pI_cation), K_B = 10^(pOH - pKb - pI_anion),
 *   K_ion = 10^(-pI_cation - pI_anion);
 * the ion counts in the acceptance rules (Eqs. (MCmetro)-(MCmetro2)) are the
 * counts of those two types (each species has its own ideal term in Eq.
 * (QQ)); ions of the other two types are bystanders that only interact.
 * `reactions` is a bit mask: 1 acid, 2 base, 4 salt moves, kept where the
 * system has such sites (the move is drawn uniformly among those kept).
 * Examples: RxMC is (CR_XP, CR_XM, pH, pOH, 7); the grand-reaction ensemble
 * alternates (CR_XP, CR_XM, pH, pOH, 5), (CR_SP, CR_SM, pI_S+, pI_S-, 5),
 * (CR_XP, CR_SM, pH, pI_S-, 4), (CR_SP, CR_XM, pI_S+, pOH, 4).  The pI values
 * stay as given through a later cr_set_pH (which recomputes K_A and K_B from
 * them).  In stream order, like cr_set_pH; batches holding the context pick
 * it up at their next sweep.  INVALID_ARG for other types, a non-finite pI or
 * no reaction left.  Synchronises. */
int cr_set_invocation(cr_ctx *ctx, int32_t cation, int32_t anion, double pI_cation, double pI_anion,
                      uint32_t reactions);

/* Ungrouping of the combined ions (Sec. II.D, last paragraph): a grouped ion
 * belongs to subspecies i with probability p_i = 10^(-pI_i + pI_X), exact in
 * equilibrium.  p_S_plus, p_H: salt cation and H+ in X+; p_S_minus, p_OH:
 * salt anion and OH- in X-; the remainder of each group (1 - the two) is the
 * counter-ion of the acid or base that sets a non-neutral pH (App. C).  n_*:
 * those fractions of the current n_X+ / n_X- (reads the counts;
 * synchronises). */
typedef struct {
  double p_S_plus, p_H, p_S_minus, p_OH;
  double n_S_plus, n_H, n_S_minus, n_OH;
} cr_ungrouped;
int cr_ungroup(cr_ctx *ctx, cr_ungrouped *out);

/* Geometry and schedule of the context. */
int cr_get_info(const cr_ctx *ctx, cr_info *out);

/* Use a caller CUDA stream (a cudaStream_t passed as void*; NULL = default). */
int cr_set_stream(cr_ctx *ctx, void *stream);

/* ---- device memory owned by the caller ----
 * The paper has no counterpart: this is the boundary's memory rule, under
 * which the caller's allocator (e.g. PyTorch tensors) may own the device
 * memory of the configuration and read it in place.  The buffers are the
 * slot arrays of the cell list in the layout cr_get_info describes: n_cells
 * = nc^3 cells of cap slots, slot g = cell * cap + i for i < cnt[cell], the
 * particles of a cell in ascending id:
 *   cnt  [n_cells]    int32   particles per cell                (4-byte aligned)
 *   pos  [4 n_slots]  float   x, y, z, effective charge        (16-byte aligned)
 *   vel  [4 n_slots]  float   vx, vy, vz, 0                     (16-byte aligned)
 *   id   [n_slots]    uint64  particle id (input index; inserted ions >= 2^32)
 *   info [n_slots]    int32   type | cls << 4 | ionised << 6 | site index << 8
 * The context copies its configuration into them, frees its own copies of
 * these arrays and works in the caller's buffers from then on (sweeps, MD,
 * cr_state, cr_load, checkpoints); the caller keeps them allocated and does
 * not write them until cr_destroy, which does not free them.  Contents are
 * current after any synchronising call (cr_check, cr_state).  One bind per
 * context, before the context joins a batch.  Errors: INVALID_ARG (NULL or
 * misaligned pointer, a size below the layout's, memory that is not device
 * memory of the context's device, a second bind, a context in a batch), CUDA.
 * Synchronises. */
typedef struct {
  int32_t *cnt;
  float *pos, *vel;
  uint64_t *id;
  int32_t *info;
  int64_t n_cells, n_slots;
} cr_device_buffers;
int cr_bind_device_buffers(cr_ctx *ctx, const cr_device_buffers *buf);

/* Check the device error word (synchronises): CR_OK or the first error. */
int cr_check(cr_ctx *ctx);

void cr_destroy(cr_ctx *ctx);
const char *cr_strerror(int code);

/* ---- batches of independent replicas (e.g. the points of a pH sweep) ----
 * A batch advances n contexts together: one colour-phase launch per colour
 * covers every domain of every replica.  Replica r uses the Philox key
 * (seed_lo, seed_hi ^ r), so its chain equals cr_sweep on that context alone
 * with seed ^ (r << 32).  The contexts stay owned by the caller, must outlive
 * the batch, share one stream and sweep counter (e.g. freshly created) and
 * the same schedule kind; their counts, states and errors are read per
 * context (cr_state, cr_check). */
typedef struct cr_batch cr_batch;
int cr_batch_create(cr_batch **out, cr_ctx *const *ctxs, int32_t n);
/* n_sweeps sweeps on every replica (each replica runs its own trials per sweep). */
int cr_batch_sweep(cr_batch *b, uint64_t n_sweeps, uint64_t seed);
/* The same with delayed acceptance (every context needs a surrogate). */
int cr_batch_sweep_da(cr_batch *b, uint64_t n_sweeps, uint64_t seed);
/* cr_md_step on every replica, concurrently (replica r uses seed ^ (r << 32)). */
int cr_batch_md_step(cr_batch *b, int32_t n_steps, double dt, double gamma, uint64_t seed);
/* cr_md_begin / cr_md_end on every replica (replica r uses seed ^ (r << 32)). */
int cr_batch_md_begin(cr_batch *b, double dt, double gamma, uint64_t seed);
int cr_batch_md_end(cr_batch *b, double dt, double gamma, uint64_t seed);
/* n_steps MD/CR-MC cycles of every replica: step s is cr_batch_md_begin,
 * one sweep (cr_batch_sweep, or cr_batch_sweep_da when da != 0) and
 * cr_batch_md_end, with seeds sweep_seed0 + s and md_seed0 + s -- the
 * hybrid scheme of the paper with the trials of Sec. II.C between the drift
 * and the force evaluation of a velocity-Verlet/Langevin step (Sec. III.A).
 * Once the launch-shape tuner has finished and every replica holds the
 * forces of a completed step, each step is one launch of a CUDA graph
 * captured from those calls (captured again when dt, gamma, the launch form
 * or timing change); its kernels read the step's seeds and counters from
 * device memory.  When no replica holds valid forces (e.g. every replica was
 * just loaded), the call's first step is one launch of a graph that opens
 * with the force evaluation cr_md_begin would make (one graph is kept: a
 * change between the two forms captures again).  Other steps run call by
 * call.  The chain is the same as the calls made one by one. */
int cr_batch_cycle(cr_batch *b, int32_t n_steps, double dt, double gamma, uint64_t sweep_seed0, uint64_t md_seed0,
                   int32_t da);
/* cr_load of every replica of the batch: args[0 .. n-1], one per context in
 * the order given to cr_batch_create; the uploads and load kernels of the
 * replicas run concurrently on the batch's streams.  Errors as cr_load's;
 * returns the first. */
typedef struct {
  int32_t n;
  const float *xyz, *vel;
  const int32_t *type, *cls;
  const int8_t *state;
} cr_load_args;
int cr_batch_load(cr_batch *b, const cr_load_args *args);
/* Packed batch I/O: one host array per quantity for all replicas, replica
 * r's entries starting at r * stride (stride >= the largest capacity; xyz and
 * vel hold 3 floats per entry).  cr_batch_state_packed fills the arrays that
 * are not NULL and n[r] (the particles of replica r, ordered by id as
 * cr_state; entries past n[r] in a replica's block are unspecified) with two
 * kernel launches, one copy per array and one synchronisation for the whole
 * batch (contexts above 16,384 particles of capacity take the per-context
 * path).  cr_batch_load_packed is cr_load of every replica from such arrays
 * (n[r] in; vel may be NULL), checked on the device like cr_load; its
 * per-particle errors come at the next synchronising call.  A load reads
 * arrays the GPU can address (device memory, pinned host memory) in place,
 * others through device staging with one copy each; it reads them
 * asynchronously, so they must not change before the stream has passed the
 * load.  A read writes through device staging and one copy per array. */
typedef struct {
  int64_t stride;
  float *xyz, *vel;
  uint64_t *id;
  int32_t *type, *cls;
  int8_t *state;
  int64_t *n;
} cr_batch_packed;
int cr_batch_state_packed(cr_batch *b, cr_batch_packed *p);
int cr_batch_load_packed(cr_batch *b, const cr_batch_packed *p);
/* cr_state of every replica of the batch into views[0 .. n-1] (one view per
 * context, in the order given to cr_batch_create); the replicas' reads run
 * concurrently on the batch's streams with two synchronisations in all.
 * Returns the first error of a replica. */
int cr_batch_state(cr_batch *b, cr_state_view *views);
/* Persistent sweeps (mode 1): a batch sweep is one launch in
 * which CTAs claim (colour, replica, domain) tasks in that order and a domain
 * of colour c > 0 starts once its neighbouring domains of lower colours have
 * finished (a domain's phase reads only its own and its neighbours' cells,
 * Sec. II.C's moves being local to it) -- so colours overlap within and
 * across replicas and no colour phase waits for the slowest domain of the
 * batch.  Mode 2: a domain waits for its replica's whole previous colour
 * (also what mode 1 does when a replica's halo reaches past its neighbouring
 * domains).  Mode 0: one launch per colour.  Mode -1 (the default): the
 * launch-shape tuner times every shape in both forms (mode 1 and mode 0), in
 * two passes, and keeps the fastest; fixing a shape with cr_batch_set_launch_shape then
 * selects mode 0 unless a mode was set.  ctas_per_sm > 0 caps the
 * resident CTAs per SM of a persistent launch (0: as many as fit).  Every
 * wait is bounded in time; one that runs out sets CR_ERR_TIMEOUT on its
 * replica and the rest of the sweep is skipped.  The chain is the same in
 * every mode. */
int cr_batch_set_persistent(cr_batch *b, int32_t mode, int32_t ctas_per_sm);
/* Failure-detection self-test of those waits (no counterpart in the paper):
 * one persistent sweep in which `replica` never reports that it finished
 * colour 0, so the tasks of its colour 1 wait until timeout_ms (at most
 * 10 s) runs out; the wait then records the timeout and the launch skips
 * its remaining tasks and ends.  Returns CR_ERR_TIMEOUT when that path
 * worked.  The replicas' chains are then incomplete (their contexts keep the
 * error); the device stays usable.  Synchronises. */
int cr_batch_selftest_wait_timeout(cr_batch *b, int32_t replica, double timeout_ms);
/* Fix the batch's launch shape (as cr_set_launch_shape; 0, 0 restarts the tuning). */
int cr_batch_set_launch_shape(cr_batch *b, int32_t threads, int32_t regs);
int cr_batch_get_launch_shape(const cr_batch *b, int32_t *threads, int32_t *regs);
void cr_batch_destroy(cr_batch *b);

/* ---- training of the DA surrogate (MSE on feature / pair-energy pairs, Adam) ----
 * Every matrix product runs on the tensor cores (tcgen05.mma, BF16 operands,
 * FP32 accumulation in tensor memory); masters, gradients and Adam moments are
 * FP32, activations BF16.  X must be 16-byte aligned.  Parameter vector order (FP32, N = 39425):
 * W1 [128][48], b1 [128], W2 [128][128], b2, W3 [128][128], b3, w4 [128], b4. */
typedef struct cr_trainer cr_trainer;
typedef struct {
  int32_t max_batch;  /* largest batch (a multiple of 128) */
  double lr, beta1, beta2, eps;  /* Adam */
  double target_clip; /* targets are clipped to [-clip, clip] (kT); <= 0: no clip */
  int32_t unfused;    /* 0: the fused step (one kernel per SM runs each 128-row tile's forward,
                         loss, backward and weight-gradient products on the tensor cores with
                         every operand in shared memory); 1: one product per launch */
} cr_train_cfg;
#define CR_TRAIN_N_PARAMS 39425
int cr_train_create(cr_trainer **out, const cr_mlp *init, const cr_train_cfg *cfg);
int cr_train_set_stream(cr_trainer *t, void *stream);
/* One Adam step on `batch` rows (a multiple of 128, <= max_batch): X device
 * [batch][48] FP32 features, target device [batch] FP32 pair-energy changes.
 * loss (host, nullable): the batch's MSE before the step (synchronises). */
int cr_train_step(cr_trainer *t, const float *X, const float *target, int32_t batch, float *loss);
/* Loss and gradients (host [CR_TRAIN_N_PARAMS], nullable) without an update. */
int cr_train_gradients(cr_trainer *t, const float *X, const float *target, int32_t batch, float *grads, float *loss);
/* One Adam step (Kingma & Ba, 2015: bias-corrected first and second moments;
 * the hyperparameters of cr_train_cfg applied in FP32) with caller-supplied
 * gradients instead of a batch's: host grads [CR_TRAIN_N_PARAMS] in the
 * parameter vector order above.  The update of cr_train_step alone (it counts
 * as a step of the trainer).  Synchronises. */
int cr_train_apply(cr_trainer *t, const float *grads);
/* Adam's first and second moments (host [CR_TRAIN_N_PARAMS] each, nullable),
 * in the parameter vector order.  Synchronises. */
int cr_train_moments(cr_trainer *t, float *m, float *v);
/* Current parameters: FP32 masters (params, nullable) and the cr_mlp layout
 * (BF16 of the masters; each pointer nullable). */
int cr_train_get(cr_trainer *t, float *params, uint16_t *W1, float *b1, uint16_t *W2, float *b2, uint16_t *W3,
                 float *b3, uint16_t *w4, float *b4);
int cr_train_stats(const cr_trainer *t, int64_t *steps, int64_t *launches);
void cr_train_destroy(cr_trainer *t);

/* The tensor-core product used by the trainer, exposed for parity tests:
 * D [M][N] (FP32, device) = A [M][K] B [N][K]^T (BF16 bit patterns, device,
 * row-major, K a multiple of 8, N = 48 or 128); accumulate != 0 adds into D
 * (split over K), else overwrites.  Synchronises the stream. */
int cr_mma_bf16(const uint16_t *A, const uint16_t *B, float *D, int32_t M, int32_t N, int32_t K, int32_t accumulate,
                void *stream);

/* Failure-detection self-test of the tensor-core product's bounded waits (no
 * counterpart in the paper): one 128 x 128 x 64 product of cr_mma_bf16's kind
 * whose only operand copy is withheld, so that the MMA issuer's wait for it,
 * and every thread's wait for the accumulator, run out after `polls` polls;
 * the CTA then records the timeout, frees its tensor memory and returns
 * without touching D.  Returns CR_ERR_TIMEOUT when that path worked (the
 * device stays usable; nothing faults or hangs), CR_OK if the wait did not
 * run out.  A [128][64], B [128][64] BF16 and D [128][128] FP32: device
 * buffers as for cr_mma_bf16.  Synchronises the stream. */
int cr_selftest_mma_timeout(const uint16_t *A, const uint16_t *B, float *D, uint32_t polls, void *stream);

/* Philox4x32-10 on the device for n consecutive counters (c0 + i, c1, c2, c3),
 * key (k0, k1); out: host array of 4n words.  Exposed for parity tests. */
int cr_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int32_t n,
              uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif /* CRMC_H */
