// crmc_noalloc.cu -- cr_md_forces_noalloc: the MD force evaluation with its
// scratch in a fixed device array of the library, for callers that cannot let
// a library allocate device memory while they run (an MD engine that owns
// every device buffer through its own pool; a time-critical loop in which a
// device allocation, which may synchronise the whole device, is not
// acceptable).  The paper has no counterpart.  The forces are those of
// cr_md_forces bit for bit: the same pair terms summed in the same exact
// 2^-24 fixed point.  This entry runs the force kernel's variant that
// finishes each particle on lane 0 of its warp (no per-particle sum buffer,
// no flat-frame distances), which is slower than the split form
// cr_md_forces uses but needs no scratch beyond the particle list; the
// flat-frame differences equal the minimum-image ones exactly, so the two
// variants agree to the bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "crmc.h"
#include "crmc_common.h"
#include "crmc_kernels.h"

namespace crmc {
// context access (crmc_api.cu)
int ctx_md_forces_into(cr_ctx *ctx, float4 *fout, int *plist, int *n_particles, int max_particles);
const SysParams &ctx_params(const cr_ctx *ctx);
cudaStream_t ctx_stream(const cr_ctx *ctx);
int64_t ctx_capacity(const cr_ctx *ctx);
int ctx_device(const cr_ctx *ctx);
void ctx_count_launch(cr_ctx *ctx);
}  // namespace crmc

using namespace crmc;

// Scratch of the particle list: word 0 is the list's length (cleared by the
// launcher before every evaluation), the list of occupied slots starts at word
// 64 (256-byte aligned).  About 1 MiB per device.
#define CR_NOALLOC_SCRATCH_HEAD 64
static __device__ __align__(256) int g_md_scratch[CR_NOALLOC_SCRATCH_HEAD + CR_NOALLOC_MAX_PARTICLES];

namespace {

constexpr int SCRATCH_HEAD = CR_NOALLOC_SCRATCH_HEAD;

// Address of the scratch on the current device.  Host code sees the array's
// name only as a host-side stand-in, so the device address is looked up on
// every call (cheap next to the call's synchronisation); a cached address
// would go stale after a device reset.
int scratch_on_device(int **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_md_scratch);
  if (e != cudaSuccess || !p) return e == cudaErrorMemoryAllocation ? CR_ERR_NOMEM : CR_ERR_CUDA;
  *out = static_cast<int *>(p);
  return CR_OK;
}

// Slot ids for the caller; empty slots get UINT64_MAX and a zero force (the
// force kernel writes the occupied slots).
__global__ void k_slot_ids(SysParams P, float4 *force, unsigned long long *id) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= P.ncell * P.cap) return;
  const int c = g / P.cap;
  if (g - c * P.cap < P.cnt[c]) {
    id[g] = P.pid[g];
  } else {
    id[g] = ~0ull;
    force[g] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

}  // namespace

extern "C" int cr_md_forces_noalloc(cr_ctx *ctx, float *force, uint64_t *id, int64_t n_slots) {
  if (!ctx || !force || !id) return CR_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(force) & 15u) != 0 || (reinterpret_cast<uintptr_t>(id) & 7u) != 0)
    return CR_ERR_INVALID_ARG;
  const SysParams &P = ctx_params(ctx);
  const int64_t slots = (int64_t)P.ncell * P.cap;
  if (n_slots < slots) return CR_ERR_INVALID_ARG;
  if (ctx_capacity(ctx) > CR_NOALLOC_MAX_PARTICLES) return CR_ERR_CAPACITY;
  int current = -1;
  if (cudaGetDevice(&current) != cudaSuccess) return CR_ERR_CUDA;
  if (current != ctx_device(ctx)) return CR_ERR_INVALID_ARG;  // the context's device must be current
  int *scratch = nullptr;
  int rc = scratch_on_device(&scratch);
  if (rc != CR_OK) return rc;
  float4 *f4 = reinterpret_cast<float4 *>(force);
  rc = ctx_md_forces_into(ctx, f4, scratch + SCRATCH_HEAD, scratch, (int)ctx_capacity(ctx));
  if (rc != CR_OK) return rc;
  if (slots > 0) {
    k_slot_ids<<<(unsigned)((slots + 255) / 256), 256, 0, ctx_stream(ctx)>>>(
        P, f4, reinterpret_cast<unsigned long long *>(id));
    if (cudaGetLastError() != cudaSuccess) return CR_ERR_CUDA;
    ctx_count_launch(ctx);
  }
  return cr_check(ctx);
}
