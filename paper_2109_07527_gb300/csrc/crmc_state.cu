// crmc_state.cu -- the configuration read back in particle-id order, on the
// device (sm_103a): the occupied cell slots are mapped to ids, input particles
// (ids below n_input, dense) are placed by a prefix count over the ids present,
// inserted ions (ids >= 2^32) by a radix sort of their ids, and every requested
// array is written in the caller's layout, ready for one copy each.
//
// Between two reads the id marks (present[]) and the ion counter are zero:
// the ordering kernel clears what the mark kernel set.
#include <cuda_runtime.h>

#include <cub/block/block_radix_sort.cuh>
#include <cub/device/device_radix_sort.cuh>

#include <cstdint>

#include "crmc_device.cuh"
#include "crmc_kernels.h"

namespace crmc {

namespace {

constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_ITEMS = 16;  // ions sorted inside one CTA: up to 16,384
using IonSort = cub::BlockRadixSort<unsigned long long, ORDER_THREADS, ORDER_ITEMS, int>;

// every occupied slot: input ids mark their slot (slot + 1), inserted ions
// append (key, slot) to the ion list (one atomic per warp); the key keeps the
// order of the ids: (id >> 32) << lo_bits | (id & 0xffffffff), as the low
// word of an inserted id stays below 2^lo_bits
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
  B.ion_key[o] = ((id >> 32) << B.lo_bits) | (id & 0xffffffffull);
  B.ion_val[o] = g;
}

__device__ __forceinline__ void emit(const SysParams &P, const StateBufs &B, int g, int o) {
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

// CTA 0: the input ids present, by an exclusive prefix count (each thread a
// contiguous range), written and unmarked.  CTA 1: the ions after them, in
// id order -- sorted here (block radix sort of the keys) or, for more than
// one CTA holds, already sorted by the device-wide sort (sorted_slot).
__global__ void __launch_bounds__(ORDER_THREADS) k_state_order(SysParams P, StateBufs B, int n_present, int n_ions,
                                                               int end_bit, const int *sorted_slot) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int t = threadIdx.x;
  if (blockIdx.x == 0) {
    int *part = (int *)smem;
    const int lane = t & 31, w = t >> 5;
    const int n = B.n_input;
    const int per = (n + ORDER_THREADS - 1) / ORDER_THREADS;
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
      const int g = B.present[i] - 1;
      if (g >= 0) {
        emit(P, B, g, run++);
        B.present[i] = 0;
      }
    }
    return;
  }
  if (t == 0) *B.n_ions = 0;  // the count came to the host as n_ions
  if (sorted_slot) {
    for (int r = t; r < n_ions; r += ORDER_THREADS) emit(P, B, sorted_slot[r], n_present + r);
    return;
  }
  if (n_ions == 0) return;
  unsigned long long key[ORDER_ITEMS];
  int val[ORDER_ITEMS];
#pragma unroll
  for (int i = 0; i < ORDER_ITEMS; ++i) {  // blocked arrangement, padded with the largest key
    const int r = t * ORDER_ITEMS + i;
    key[i] = r < n_ions ? B.ion_key[r] : ~0ull;
    val[i] = r < n_ions ? B.ion_val[r] : -1;
  }
  IonSort(*(typename IonSort::TempStorage *)smem).Sort(key, val, 0, end_bit);
#pragma unroll
  for (int i = 0; i < ORDER_ITEMS; ++i) {
    const int r = t * ORDER_ITEMS + i;
    if (r < n_ions) emit(P, B, val[i], n_present + r);
  }
}

}  // namespace

cudaError_t launch_state_mark(const SysParams &P, const StateBufs &B, cudaStream_t s) {
  const int n = P.ncell * P.cap;
  k_state_mark<<<(n + 255) / 256, 256, 0, s>>>(P, B);
  return cudaGetLastError();
}

size_t state_sort_temp_bytes(int cap) {
  if (cap <= STATE_BLOCK_SORT_MAX) return 0;
  size_t bytes = 0;
  cub::DoubleBuffer<unsigned long long> k(nullptr, nullptr);
  cub::DoubleBuffer<int> v(nullptr, nullptr);
  if (cub::DeviceRadixSort::SortPairs(nullptr, bytes, k, v, cap) != cudaSuccess) return 0;
  return bytes;
}

cudaError_t launch_state_order(const SysParams &P, const StateBufs &B, int n_present, int n_ions, int end_bit,
                               cudaStream_t s, int *launches) {
  static_assert(ORDER_THREADS * ORDER_ITEMS == STATE_BLOCK_SORT_MAX, "block sort capacity");
  const size_t smem = sizeof(typename IonSort::TempStorage) > sizeof(int) * 32 ? sizeof(typename IonSort::TempStorage)
                                                                               : sizeof(int) * 32;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_state_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int n_launch = 1;
  const int *sorted = nullptr;
  if (n_ions > STATE_BLOCK_SORT_MAX) {  // beyond one CTA: device-wide radix sort first
    if (!B.sort_tmp || !B.ion_key_alt || !B.ion_val_alt) return cudaErrorInvalidValue;
    cub::DoubleBuffer<unsigned long long> k(B.ion_key, B.ion_key_alt);
    cub::DoubleBuffer<int> v(B.ion_val, B.ion_val_alt);
    size_t bytes = B.sort_tmp_bytes;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(B.sort_tmp, bytes, k, v, n_ions, 0, end_bit, s);
    if (e != cudaSuccess) return e;
    sorted = v.Current();
    n_launch += (end_bit + 7) / 8 + 2;  // histogram, scan and one pass per 8 bits
  }
  k_state_order<<<2, ORDER_THREADS, smem, s>>>(P, B, n_present, n_ions, end_bit, sorted);
  if (launches) *launches += n_launch;
  return cudaGetLastError();
}

}  // namespace crmc
