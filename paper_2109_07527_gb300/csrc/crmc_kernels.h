// crmc_kernels.h -- launch interface between the C-ABI host code and the
// kernels of libcrmc.so.
#pragma once
#include <cuda_runtime.h>

#include "crmc_common.h"

namespace crmc {

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
};

struct RebuildBufs {
  int *cnt;
  float4 *pos;
  unsigned long long *pid;
  int *info;
  float4 *vel, *frc;          // scratch copies
  float4 *vel_src, *frc_src;  // primary velocity / force arrays
};

struct DumpBufs {
  int *counter;
  int cap;
  float4 *pos, *vel, *frc;
  unsigned long long *pid;
  int *info;
  const float4 *vel_src, *frc_src;
};

struct LoadBufs {
  const float *xyz, *vel;
  const int *type, *cls, *site;  // site: site index of input particle i (-1 none)
  const int8_t *state;
  int n, n_site_map;
};

// phase kernel shapes (threads, halo registers); da: the delayed-acceptance set
size_t phase_smem_bytes(const PhaseShape &S, int threads, bool da);
int phase_shape_count(bool da);
size_t phase_shape_smem(const PhaseShape &S, int threads, int regs, bool da);
void phase_shape(int i, int *threads, int *regs, bool da);
bool phase_shape_compact(int i, bool da);  // shape i uses the compact list and halo capacities
cudaError_t launch_phase(const SysParams *d_reps, int n_rep, int grid_x, const PhaseShape &S, int threads, int R,
                         bool log, bool da, cudaStream_t s, uint32_t sweep, uint32_t sweep0, int colour,
                         uint32_t k0, uint32_t k1);
// launch order of every colour's domains for one sweep (densest region first);
// does nothing for colours beyond the ordering limit
cudaError_t launch_domain_order(const SysParams *d_reps, int n_rep, int ncol, int nact, cudaStream_t s, uint32_t sweep,
                                uint32_t k0, uint32_t k1);
// particle list (plist, n_particles: device scratch of max_particles + 1
// ints), then the force kernel (one warp per particle)
cudaError_t launch_md_forces(const SysParams &P, const MdParams &M, int *plist, int *n_particles, int max_particles,
                             cudaStream_t s);
cudaError_t launch_kick_drift(const SysParams &P, const MdParams &M, cudaStream_t s);
cudaError_t launch_rebuild(const SysParams &P, const RebuildBufs &B, int *perm_slot, int n_perm, cudaStream_t s);
cudaError_t launch_load(const SysParams &P, const LoadBufs &I, const RebuildBufs &B, int *perm_slot, int n_perm,
                        cudaStream_t s);
cudaError_t launch_perm_slots(const SysParams &P, int *perm_slot, int n_perm, cudaStream_t s);
cudaError_t launch_dump(const SysParams &P, const DumpBufs &D, cudaStream_t s);
cudaError_t launch_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, int n,
                          uint4 *out, cudaStream_t s);

}  // namespace crmc
