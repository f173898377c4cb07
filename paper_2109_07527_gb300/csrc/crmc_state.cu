// crmc_state.cu -- the configuration read back in particle-id order, on the
// device (sm_103a): the occupied cell slots are mapped to ids, input particles
// (ids below n_input, dense) are placed by a prefix count over the ids present,
// inserted ions (ids >= 2^32) by a radix sort of their ids, and every requested
// array is written in the caller's layout, ready for one copy each.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>

#include <cstdint>

#include "crmc_device.cuh"
#include "crmc_kernels.h"

namespace crmc {

namespace {

// every occupied slot: input ids mark their slot (slot + 1), inserted ions
// append (id, slot) to the ion list (one atomic per warp)
__global__ void k_state_mark(SysParams P, StateBufs B) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
  const int c = g / P.cap;
  const bool have = g < P.ncell * P.cap && g - c * P.cap < P.cnt[c];
  unsigned long long id = 0;
  if (have) id = P.pid[g];
  const bool ion = have && id >= (unsigned long long)B.n_input;
  if (have && !ion) B.present[id] = g + 1;
  const unsigned m = __ballot_sync(0xffffffffu, ion);
  if (m == 0u) return;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(B.n_ions, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!ion) return;
  const int o = base + __popc(m & ((1u << lane) - 1u));
  if (o >= B.cap) return;  // more ions than slots: the host sees the count and reports it
  B.ion_key[o] = id;
  B.ion_val[o] = g;
}

// exclusive prefix count of the input ids present (one CTA; each thread scans
// a contiguous range)
constexpr int SCAN_THREADS = 1024;
__global__ void __launch_bounds__(SCAN_THREADS) k_state_scan(StateBufs B) {
  __shared__ int part[SCAN_THREADS / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int n = B.n_input;
  const int per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += B.present[i] != 0;
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) part[w] = x;
  __syncthreads();
  if (w == 0) {
    int v = part[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    part[lane] = v;
  }
  __syncthreads();
  int run = x - s + (w > 0 ? part[w - 1] : 0);
  for (int i = lo; i < hi; ++i) {
    B.pre[i] = run;
    run += B.present[i] != 0;
  }
}

// one thread per output entry: input ids first (their prefix count), then
// the sorted ions; each requested array in the caller's layout
__global__ void k_state_emit(SysParams P, StateBufs B, int n_present, int n_ions, const int *ion_slot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int o, g;
  if (i < B.n_input) {
    g = B.present[i] - 1;
    if (g < 0) return;
    o = B.pre[i];
  } else {
    const int r = i - B.n_input;
    if (r >= n_ions) return;
    g = ion_slot[r];
    o = n_present + r;
  }
  const float4 p = P.pos[g];
  const int info = P.info[g];
  const int t = info & INFO_TYPE_MASK;
  const int ionised = (info & INFO_ION_BIT) ? 1 : 0;
  if (B.xyz) { B.xyz[3 * o] = p.x; B.xyz[3 * o + 1] = p.y; B.xyz[3 * o + 2] = p.z; }
  if (B.vel) {
    const float4 v = B.vel_src[g];
    B.vel[3 * o] = v.x; B.vel[3 * o + 1] = v.y; B.vel[3 * o + 2] = v.z;
  }
  if (B.frc) {
    const float4 f = B.frc_src ? B.frc_src[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    B.frc[3 * o] = f.x; B.frc[3 * o + 1] = f.y; B.frc[3 * o + 2] = f.z;
  }
  if (B.id) B.id[o] = P.pid[g];
  if (B.type) B.type[o] = t;
  if (B.state) B.state[o] = (int8_t)ionised;
  if (B.cls) B.cls[o] = (info >> INFO_CLS_SHIFT) & 3;
  if (B.site && (t == CR_ACID || t == CR_BASE)) B.site[info >> INFO_SITE_SHIFT] = (int8_t)ionised;
}

}  // namespace

cudaError_t launch_state_mark(const SysParams &P, const StateBufs &B, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(B.n_ions, 0, sizeof(int), s);
  if (e == cudaSuccess && B.n_input > 0) e = cudaMemsetAsync(B.present, 0, sizeof(int) * (size_t)B.n_input, s);
  if (e != cudaSuccess) return e;
  const int n = P.ncell * P.cap;
  k_state_mark<<<(n + 255) / 256, 256, 0, s>>>(P, B);
  return cudaGetLastError();
}

size_t state_sort_temp_bytes(int cap) {
  size_t bytes = 0;
  cub::DoubleBuffer<unsigned long long> k(nullptr, nullptr);
  cub::DoubleBuffer<int> v(nullptr, nullptr);
  if (cub::DeviceRadixSort::SortPairs(nullptr, bytes, k, v, cap) != cudaSuccess) return 0;
  return bytes;
}

cudaError_t launch_state_emit(const SysParams &P, const StateBufs &B, int n_present, int n_ions, int end_bit,
                              cudaStream_t s, int *launches) {
  int n_launch = 0;
  if (B.n_input > 0) {
    k_state_scan<<<1, SCAN_THREADS, 0, s>>>(B);
    ++n_launch;
  }
  const int *slot = B.ion_val;
  if (n_ions > 1) {  // ions by id: LSD radix sort of the bits that can vary
    cub::DoubleBuffer<unsigned long long> k(B.ion_key, B.ion_key_alt);
    cub::DoubleBuffer<int> v(B.ion_val, B.ion_val_alt);
    size_t bytes = B.sort_tmp_bytes;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(B.sort_tmp, bytes, k, v, n_ions, 0, end_bit, s);
    if (e != cudaSuccess) return e;
    slot = v.Current();
    n_launch += (end_bit + 7) / 8 + 2;  // histogram, scan and one pass per 8 bits
  }
  const int n = B.n_input + n_ions;
  if (n > 0) {
    k_state_emit<<<(n + 255) / 256, 256, 0, s>>>(P, B, n_present, n_ions, slot);
    ++n_launch;
  }
  if (launches) *launches += n_launch;
  return cudaGetLastError();
}

}  // namespace crmc
