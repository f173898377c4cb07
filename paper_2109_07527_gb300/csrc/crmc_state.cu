// crmc_state.cu -- the configuration read back in particle-id order, on the
// device (sm_103a): the occupied cell slots are mapped to ids, input particles
// (ids below n_input, dense) are placed by a prefix count over the ids present,
// inserted ions (ids >= 2^32) by their rank among the ion ids (counted in
// 1024 x 1024 tiles over many CTAs; a device-wide radix sort past 16,384
// ions), and every requested array is written in the caller's layout.
//
// Between two reads the id marks (present[]) and the ion counter are zero:
// the ordering kernel clears what the mark kernel set.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>

#include <cstdint>

#include "crmc_device.cuh"
#include "crmc_kernels.h"

namespace crmc {

namespace {

constexpr int ORDER_THREADS = 1024;
constexpr int RANK_TILE = 1024;  // ion keys per rank-counting tile

// every occupied slot: input ids mark their slot (slot + 1), inserted ions
// append (key, slot) to the ion list (one atomic per warp); the key keeps the
// order of the ids: (id >> 32) << lo_bits | (id & 0xffffffff), as the low
// word of an inserted id stays below 2^lo_bits
__device__ __forceinline__ void mark_slot(const SysParams &P, const StateBufs &B, int g) {
  const int lane = threadIdx.x & 31;
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
  B.ion_rank[o] = 0;
}

// rank of every ion key among the n ion keys (the keys are distinct): CTA
// (x, y) adds, for the keys of tile x, how many keys of tile y are smaller
__device__ __forceinline__ void rank_tile(const StateBufs &B, int n) {
  __shared__ unsigned long long ks[RANK_TILE];
  const int t = threadIdx.x;
  const int i = blockIdx.x * RANK_TILE + t, j0 = blockIdx.y * RANK_TILE;
  if (j0 >= n || (int)blockIdx.x * RANK_TILE >= n) return;  // the whole CTA
  ks[t] = j0 + t < n ? B.ion_key[j0 + t] : ~0ull;
  __syncthreads();
  if (i >= n) return;
  const unsigned long long k = B.ion_key[i];
  const int m = min(RANK_TILE, n - j0);
  int c = 0;
#pragma unroll 8
  for (int j = 0; j < m; ++j) c += ks[j] < k ? 1 : 0;
  if (c) atomicAdd(&B.ion_rank[i], c);
}

__global__ void __launch_bounds__(RANK_TILE) k_ion_rank(StateBufs B, int n) { rank_tile(B, n); }
__global__ void __launch_bounds__(RANK_TILE) k_ion_rank_batch(const StateBufs *__restrict__ bufs) {
  const StateBufs &B = bufs[blockIdx.z];
  rank_tile(B, min(*B.n_ions, STATE_BLOCK_SORT_MAX));
}

__global__ void k_state_mark(SysParams P, StateBufs B) { mark_slot(P, B, blockIdx.x * blockDim.x + threadIdx.x); }

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

// The input ids present, in id order, written and unmarked (one CTA): the
// ids are taken 1024 at a time, each thread one id, and a present id's place
// is the number of present ids before it (ballots and a scan of the warps'
// counts), so that consecutive threads write consecutive entries.
__device__ __forceinline__ void order_inputs(const SysParams &P, const StateBufs &B, int *part) {
  __shared__ int base_s;
  const int t = threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  const int n = B.n_input;
  if (t == 0) base_s = 0;
  for (int c0 = 0; c0 < n; c0 += ORDER_THREADS) {
    const int i = c0 + t;
    const int g = i < n ? B.present[i] - 1 : -1;
    const unsigned bal = __ballot_sync(0xffffffffu, g >= 0);
    if (lane == 0) part[w] = __popc(bal);
    __syncthreads();
    if (w == 0) {  // inclusive scan of the warps' counts
      int v = part[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      part[lane] = v;
    }
    __syncthreads();
    if (g >= 0) {
      emit(P, B, g, base_s + (w > 0 ? part[w - 1] : 0) + __popc(bal & ((1u << lane) - 1u)));
      B.present[i] = 0;
    }
    __syncthreads();
    if (t == 0) base_s += part[ORDER_THREADS / 32 - 1];
  }
}

// The ions after the input ids, in id order: in the order of the device-wide
// sort (sorted_slot), or by their ranks, which are first turned into the slot
// of each rank (the ranked keys' array takes it) so that the entries are
// written in order.
__device__ __forceinline__ void order_ions(const SysParams &P, const StateBufs &B, int n_present, int n_ions,
                                           const int *sorted_slot) {
  if (sorted_slot) {
    for (int r = threadIdx.x; r < n_ions; r += ORDER_THREADS) emit(P, B, sorted_slot[r], n_present + r);
    return;
  }
  unsigned long long *slot_of_rank = B.ion_key;  // the keys were consumed by the ranking
  for (int i = threadIdx.x; i < n_ions; i += ORDER_THREADS)
    slot_of_rank[B.ion_rank[i]] = (unsigned long long)B.ion_val[i];
  __syncthreads();
  for (int r = threadIdx.x; r < n_ions; r += ORDER_THREADS) emit(P, B, (int)slot_of_rank[r], n_present + r);
}

// CTA 0 the input ids, CTA 1 the ions (counts from the host)
__global__ void __launch_bounds__(ORDER_THREADS) k_state_order(SysParams P, StateBufs B, int n_present, int n_ions,
                                                               const int *sorted_slot) {
  __shared__ int part[ORDER_THREADS / 32];
  if (blockIdx.x == 0) {
    order_inputs(P, B, part);
    return;
  }
  if (threadIdx.x == 0) *B.n_ions = 0;  // the count came to the host as n_ions
  order_ions(P, B, n_present, n_ions, sorted_slot);
}

// Every replica of a batch (blockIdx.y) at once, the counts read on the
// device: n from the kind counts, n_ions from the mark kernel.  A replica
// whose ions exceed the tile ranking (or whose counts are inconsistent) gets
// n_out = -1 and only its marks cleared.  n_out and err_out receive each
// replica's particle count and error word.
__global__ void k_state_mark_batch(const SysParams *__restrict__ reps, const StateBufs *__restrict__ bufs) {
  mark_slot(reps[blockIdx.y], bufs[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(ORDER_THREADS) k_state_order_batch(const SysParams *__restrict__ reps,
                                                                     const StateBufs *__restrict__ bufs,
                                                                     long long *n_out, int *err_out) {
  __shared__ int part[ORDER_THREADS / 32];
  const int r = blockIdx.y;
  const SysParams &P = reps[r];
  const StateBufs &B = bufs[r];
  const long long *cn = B.counts;
  const long long n = cn[K_A0] + cn[K_A1] + cn[K_B0] + cn[K_B1] + cn[K_XP] + cn[K_XM] + cn[K_SP] + cn[K_SM] + B.n_other;
  const int n_ions = *B.n_ions;
  const long long n_present = n - n_ions;
  const bool ok = n_ions >= 0 && n_ions <= STATE_BLOCK_SORT_MAX && n <= B.cap && n_present >= 0 &&
                  n_present <= B.n_input && *P.err == 0;
  __syncthreads();  // every thread has read the ion count
  if (blockIdx.x == 0) {
    if (ok) {
      order_inputs(P, B, part);
    } else {
      for (int i = threadIdx.x; i < B.n_input; i += ORDER_THREADS) B.present[i] = 0;
    }
    if (threadIdx.x == 0) {
      n_out[r] = ok ? n : -1;
      err_out[r] = *P.err;
    }
    return;
  }
  if (threadIdx.x == 0) *B.n_ions = 0;
  if (ok) order_ions(P, B, (int)n_present, n_ions, nullptr);
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
  int n_launch = 1;
  const int *sorted = nullptr;
  if (n_ions > STATE_BLOCK_SORT_MAX) {  // many ions: device-wide radix sort
    if (!B.sort_tmp || !B.ion_key_alt || !B.ion_val_alt) return cudaErrorInvalidValue;
    cub::DoubleBuffer<unsigned long long> k(B.ion_key, B.ion_key_alt);
    cub::DoubleBuffer<int> v(B.ion_val, B.ion_val_alt);
    size_t bytes = B.sort_tmp_bytes;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(B.sort_tmp, bytes, k, v, n_ions, 0, end_bit, s);
    if (e != cudaSuccess) return e;
    sorted = v.Current();
    n_launch += (end_bit + 7) / 8 + 2;  // histogram, scan and one pass per 8 bits
  } else if (n_ions > 1) {
    const unsigned nt = (unsigned)((n_ions + RANK_TILE - 1) / RANK_TILE);
    k_ion_rank<<<dim3(nt, nt), RANK_TILE, 0, s>>>(B, n_ions);
    ++n_launch;
  }
  k_state_order<<<2, ORDER_THREADS, 0, s>>>(P, B, n_present, n_ions, sorted);
  if (launches) *launches += n_launch;
  return cudaGetLastError();
}

cudaError_t launch_state_batch(const SysParams *d_reps, const StateBufs *d_bufs, int n_rep, int max_slots,
                               int max_cap, long long *d_n_out, int *d_err_out, cudaStream_t s) {
  if (max_slots > 0) k_state_mark_batch<<<dim3((max_slots + 255) / 256, n_rep), 256, 0, s>>>(d_reps, d_bufs);
  const unsigned nt = (unsigned)((min(max_cap, STATE_BLOCK_SORT_MAX) + RANK_TILE - 1) / RANK_TILE);
  if (nt > 0) k_ion_rank_batch<<<dim3(nt, nt, n_rep), RANK_TILE, 0, s>>>(d_bufs);
  k_state_order_batch<<<dim3(2, n_rep), ORDER_THREADS, 0, s>>>(d_reps, d_bufs, d_n_out, d_err_out);
  return cudaGetLastError();
}

}  // namespace crmc
