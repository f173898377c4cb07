// crmc_kernels.h -- launch interface between the C-ABI host code and the
// kernels of libcrmc.so.
#pragma once
#include <cuda_runtime.h>

#include "crmc_common.h"

namespace crmc {

// Per-step values of a captured MD/CR-MC cycle (cr_batch_cycle), read by the
// kernels from device memory so that one CUDA graph serves every step: step s
// of a call uses the seeds seed0 + s, the sweep counter sweep0 + s and the
// force-evaluation counter eval0 + s; the graph's last node advances step.
struct StepDyn {
  unsigned long long step;
  unsigned long long sweep_seed0, md_seed0;
  unsigned int sweep0, eval0;
};

// A rigid body (a nanoparticle and its sites): the permanent particles with
// ids [first, first + count), members mfirst .. mfirst + count - 1 of the
// body arrays.  X (not wrapped) and V: centre of mass and its velocity; R
// (row-major, lab = R body): orientation, the body axes the principal axes in
// ascending order of the moments I; pi: angular momentum in the body frame;
// M: mass (one unit per member); F, T: force and torque (lab frame, Langevin
// terms included) of the last force evaluation.  bad: set by the setup when
// a member is missing or an ion, or the moments are degenerate.
struct RigidBody {
  double X[3], V[3], R[9], pi[3], I[3], M;
  double F[3], T[3];
  int first, count, mfirst, bad;
};

struct MdParams {
  float dt, gamma, amp;   // time step, friction, sqrt(2 gamma kT / dt)
  uint32_t key0, key1, eval;
  int mode;               // 0 conservative, 1 + Langevin, 2 + Langevin + half kick
  float4 *vel, *fout;     // slot arrays
  const int *perm_slot, *bond_off, *bond_nbr;
  int n_perm;
  float fene_K, inv_R02;
  const int *plist;        // occupied slots (filled by the launcher)
  const int *n_particles;  // entries of plist
  int max_particles;       // capacity of plist
  float reach2;            // squared interaction reach with a margin (cells beyond it are skipped)
  long long *fsum;         // [3 slots] pair-force sums (2^-24 fixed point) by slot, each pair evaluated once
                           // and added to both ends, handed to the per-particle finish kernel;
                           // null: every pair from both ends, the force kernel finishes itself
  const StepDyn *dyn;      // non-null in a captured cycle: key = (md_seed0 + step) ^ (rep << 32),
                           // eval = eval0 + step + eval_off
  unsigned int rep;
  int eval_off;            // 1 for the closing evaluation of a captured step that evaluated the forces first
  // rigid bodies (n_bodies > 0): body_member[id] = member index of permanent
  // id, -1 for a free particle; body_d: [3 members] offsets in the body frame;
  // body_newpos: [members] member positions after the drift
  int n_bodies;
  RigidBody *bodies;
  const int *body_member;
  double *body_d;
  float4 *body_df;     // [members] the same offsets in FP32 (the per-member products)
  float4 *body_newpos;
  double body_dt, body_gamma;  // the step and the friction in FP64 for the bodies
};

struct RebuildBufs {
  int *cnt;
  float4 *pos;
  unsigned long long *pid;
  int *info;
  float4 *vel, *frc;          // scratch copies
  float4 *vel_src, *frc_src;  // primary velocity / force arrays
};

// the configuration read back in id order (crmc_state.cu); output arrays
// that are null are not written
constexpr int STATE_BLOCK_SORT_MAX = 16384;  // ions ranked by tile counting; more: device-wide sort
struct StateBufs {
  int n_input, cap;               // input ids are 0..n_input-1; ion list capacity
  int lo_bits;                    // the low words of ion ids stay below 2^lo_bits
  int *present;                   // [n_input] slot + 1 of each input id, 0 absent
  int *n_ions;                    // number of inserted ions found
  unsigned long long *ion_key, *ion_key_alt;  // [cap] ion sort keys (the alternates for the device-wide sort)
  int *ion_val, *ion_val_alt;                 // [cap] their slots
  int *ion_rank;                              // [cap] rank of each ion among the ion ids
  void *sort_tmp;                 // device-wide sort scratch (capacities above STATE_BLOCK_SORT_MAX)
  size_t sort_tmp_bytes;
  const float4 *vel_src, *frc_src;  // velocities; forces (null: zeros)
  const long long *counts;          // the context's kind counts (batch reads take n from them)
  int n_other, end_bit;             // particles of no kind; sort bits (batch reads)
  float *xyz, *vel, *frc;           // [3n]
  unsigned long long *id;           // [n]
  int *type, *cls;                  // [n]
  int8_t *state;                    // [n]
  int8_t *site;                     // [n_sites] by site index
};

struct LoadBufs {
  const float *xyz, *vel;
  const int *type, *cls, *site;  // site: site index of input particle i (-1 none)
  const int8_t *state;
  int n, n_site_map;
  const int *init_type;  // [n_site_map] types given to cr_init (bonded and site particles stay at their index)
  const unsigned long long *id;  // [n] particle ids (a restore), or null: the ids are the indices
  const float *frc;              // [3n] integrator forces (a restore), or null: zero
};

// one replica's load in a batched load
struct LoadJob {
  LoadBufs I;
  RebuildBufs B;
  int *perm_slot;
  int n_perm;
};

// phase kernel shapes (threads, halo registers); da: the delayed-acceptance set
size_t phase_smem_bytes(const PhaseShape &S, int threads, bool da);
int phase_shape_count(bool da);
size_t phase_shape_smem(const PhaseShape &S, int threads, int regs, bool da);
void phase_shape(int i, int *threads, int *regs, bool da);
bool phase_shape_compact(int i, bool da);  // shape i uses the compact list and halo capacities
cudaError_t launch_phase(const SysParams *d_reps, int n_rep, int grid_x, const PhaseShape &S, int threads, int R,
                         bool log, bool da, cudaStream_t s, uint32_t sweep, uint32_t sweep0, int colour,
                         uint32_t k0, uint32_t k1, const StepDyn *dyn = nullptr);
// Schedule of a persistent sweep (k_cr_sweep): tasks (colour, replica, rank)
// claimed in that order; next, done and abort are device words zeroed before
// every launch.
struct SweepSched {
  int n_rep, ncol, tasks_total;
  int fine;               // 1: per-domain dependencies (flags); 0: per-(replica, colour) counters (done)
  const int *rep_first;   // [n_rep + 1] prefix sums of the replicas' active domains per colour
  const int *dom_first;   // [n_rep + 1] prefix sums of the replicas' domain counts (flags)
  unsigned *next;         // task counter
  unsigned *done;         // [n_rep * ncol] finished tasks of each (replica, colour)
  unsigned *flags;        // [dom_first[n_rep]] finished domains
  int *abort;             // set when a wait ran out: the remaining tasks are skipped
  unsigned long long wait_ns;  // limit of one dependency wait (ns)
  int withhold_rep;       // self-test of the waits: this replica never reports colour 0 (-1: none)
};
// one sweep of every replica in one persistent launch; max_ctas > 0 caps the grid
cudaError_t launch_sweep(const SysParams *d_reps, const PhaseShape &S, int threads, int R, bool da, cudaStream_t s,
                         uint32_t sweep, uint32_t sweep0, uint32_t k0, uint32_t k1, const SweepSched &Q,
                         int max_ctas, const StepDyn *dyn = nullptr);
// the step counter of a captured cycle (the graph's last node)
cudaError_t launch_step_advance(StepDyn *dyn, cudaStream_t s);
// launch order of every colour's domains for one sweep (densest region first);
// does nothing for colours beyond the ordering limit
cudaError_t launch_domain_order(const SysParams *d_reps, int n_rep, int ncol, int nact, cudaStream_t s, uint32_t sweep,
                                uint32_t k0, uint32_t k1, const StepDyn *dyn = nullptr);
// particle list (plist, n_particles: device scratch of max_particles + 1
// ints), then the force kernel (one warp per particle)
cudaError_t launch_md_forces(const SysParams &P, const MdParams &M, int *plist, int *n_particles, int max_particles,
                             cudaStream_t s);
// half kick, drift and wrap fused with the scatter into the new cells, then
// the per-cell id sort back into the primary arrays
cudaError_t launch_kick_drift_rebuild(const SysParams &P, const MdParams &M, const RebuildBufs &B, int *perm_slot,
                                      int n_perm, cudaStream_t s);
cudaError_t launch_load(const SysParams &P, const LoadBufs &I, const RebuildBufs &B, int *perm_slot, int n_perm,
                        cudaStream_t s);
// loads of every replica of a batch (counts zeroed, scatter, cell sort,
// neutrality), four launches
cudaError_t launch_load_batch(const SysParams *d_reps, const LoadJob *d_jobs, int n_rep, int max_n, int max_cells,
                              cudaStream_t s);
// state read-back: mark the slots (ion count into *B.n_ions), then, with the
// counts known, place the input ids, sort the ions (bits [0, end_bit) of their
// keys), write the arrays and clear the marks (adds the kernels it launched to
// *launches); the device-wide sort needs state_sort_temp_bytes(cap) of scratch
// (0 when every ion list fits the one-CTA sort)
cudaError_t launch_state_mark(const SysParams &P, const StateBufs &B, cudaStream_t s);
cudaError_t launch_state_order(const SysParams &P, const StateBufs &B, int n_present, int n_ions, int end_bit,
                               cudaStream_t s, int *launches);
size_t state_sort_temp_bytes(int cap);
// every replica of a batch in two launches (marks, ordering), the counts read
// on the device; n_out[r] = particles of replica r, -1 when its read needs the
// per-context path; err_out[r] its error word
cudaError_t launch_state_batch(const SysParams *d_reps, const StateBufs *d_bufs, int n_rep, int max_slots,
                               int max_cap, long long *d_n_out, int *d_err_out, cudaStream_t s);
// Ewald: S(k) of every replica of a batch from scratch (the occupied slots
// listed, then one thread per reciprocal vector); max_nk: the largest
// number of reciprocal vectors over the replicas
cudaError_t launch_ewald_sk(const SysParams *d_reps, int n_rep, int max_nk, cudaStream_t s);
// rigid bodies: centre, principal frame, body-frame offsets and momenta from
// the current configuration (bodies[] carries first, count and mfirst);
// then, once every body is valid, the members' rigid velocities
cudaError_t launch_body_setup(const SysParams &P, const MdParams &M, cudaStream_t s);
cudaError_t launch_body_member_velocities(const SysParams &P, const MdParams &M, cudaStream_t s);
cudaError_t launch_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int n,
                          uint4 *out, cudaStream_t s);

}  // namespace crmc
