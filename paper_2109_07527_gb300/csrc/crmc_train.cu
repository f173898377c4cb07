// crmc_train.cu -- training of the delayed-acceptance surrogate (MLP
// 48 -> 128 -> 128 -> 128 -> 1, ReLU) by mean squared error with Adam, on the
// fifth-generation tensor cores of sm_103a.
//
// The training step runs as one kernel, k_train_fused (below): each SM's CTA
// takes its share of the batch's 128-row tiles through every product of the
// step on the tensor cores with the weights resident in shared memory, and
// k_sum_adam sums the CTAs' partial gradients in order and applies Adam.
// The unfused form (cr_train_cfg.unfused) and the exposed product
// cr_mma_bf16 use k_mma, one launch per product:
// D[M x N] = A[M x K] B[N x K]^T with BF16 operands that TMA stages
// into 128-byte-swizzled shared memory (a 4-deep ring of 64-wide K slices),
// tcgen05.mma (cta_group::1, M = 128) accumulating FP32 in tensor memory,
// and an epilogue that reads the accumulator with tcgen05.ld and applies
// bias + ReLU, the ReLU mask of the backward pass, the output layer and loss
// (fused into the last forward product), or, for the weight gradients, one
// slice per split of K (the batch) that a second kernel sums in split order
// (deterministic; only the exposed product cr_mma_bf16 accumulates with
// atomics).  One warp issues the TMA copies, one thread the MMAs;
// every wait on an mbarrier has an iteration limit after which the CTA
// records an error, lets its copies and MMAs in flight finish (again with a
// limit), frees its tensor memory and returns.
//
// Training step on a batch of B rows (B a multiple of 128), masters in FP32:
//   H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), H3 = relu(H2 W3^T + b3)
//   y = H3 w4 + b4, L = sum (y - t)^2 / (2B), dy = (y - t) / B
//   G3 = dy w4^T * [H3 > 0]; gW3 = G3^T H2; G2 = (G3 W3) * [H2 > 0]; gW2 = G2^T H1
//   G1 = (G2 W2) * [H1 > 0]; gW1 = G1^T X; gb = column sums; gw4 = H3^T dy
//   Adam on every parameter; BF16 copies (and transposes) of the weights.
// Activations and back-propagated errors are stored as BF16 between the
// products (row-major and transposed, so that every operand is K-major).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "crmc.h"
#include "crmc_common.h"

namespace crmc {
namespace {

constexpr int GM = 128;          // tile rows (MMA M)
constexpr int GK = 64;           // K per pipeline stage: one 128-byte swizzle row of BF16
constexpr int GSTAGES = 4;
constexpr uint32_t SPIN_LIMIT = 1u << 22;

// epilogues: bias + ReLU; backward ReLU mask with column sums; atomic add (split-K
// into one output); output layer + loss; plain store; plain store of one split's
// partial result (split-K into per-split slices, summed afterwards in split order)
enum Epi { EPI_RELU = 0, EPI_MASK = 1, EPI_ATOMIC = 2, EPI_HEAD = 3, EPI_STORE = 4, EPI_PARTIAL = 5 };

struct GemmEpi {
  const float *bias;        // [N] (RELU, HEAD)
  const uint16_t *mask;     // BF16 [M][ldm]: keep where > 0 (MASK)
  int ldm;
  uint16_t *out;            // BF16 [M][ldo] (RELU, MASK, HEAD)
  int ldo;
  uint16_t *outT;           // BF16 [N][ldt] (RELU, MASK, HEAD)
  int ldt;
  float *colsum;            // [N] column sums of the stored FP32 values (MASK)
  float *outF;              // FP32 [M][ldf] (ATOMIC: += ; STORE: =)
  int ldf;
  // output layer and loss (HEAD): y = h3 . w4 + b4 per row
  const uint16_t *w4;       // BF16 [128]
  const float *b4;
  const float *target;      // [M]
  float inv_batch;
  uint16_t *g3;             // BF16 [M][128] and [128][ldt3]: dy w4 [h3 > 0]
  uint16_t *g3T;
  int ldt3;
  float *gb3, *gw4, *gb4, *loss;
  int *err;
  uint32_t spin;      // polls of every bounded mbarrier wait (0: SPIN_LIMIT)
  int withhold_first; // self-test only: the producer issues no copy for the first K slice
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on a phase of an mbarrier: false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap *map, uint64_t *bar, void *dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzle layout: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                             // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                   // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                             // descriptor version
  d |= (uint64_t)2 << 61;                             // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's row (TMEM lane)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 accumulator columns of this thread's row, one wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint16_t to_bf16(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float from_bf16(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// Column sums of a warp's 32 x 16 chunk (row = lane) through the warp's
// shared-memory tile tb (32 x 17 floats, conflict-free): every lane stores its
// 16 values, lanes l and l + 16 add rows 0-15 and 16-31 of column l & 15, one
// shuffle joins the halves.  The sums are valid in lanes 0-15.
__device__ __forceinline__ float chunk_colsum(float *tb, const float (&x)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 16; ++j) tb[lane * 17 + j] = x[j];
  __syncwarp();
  const int col = lane & 15, r0 = (lane >> 4) * 16;
  float sum = 0.0f;
#pragma unroll
  for (int r = 0; r < 16; ++r) sum += tb[(r0 + r) * 17 + col];
  sum += __shfl_down_sync(0xffffffffu, sum, 16);
  __syncwarp();  // the tile is reused by the next chunk
  return sum;
}

// Transposed BF16 store of a warp's 32 x 16 chunk (row = lane): out^T rows
// n .. n + 15, columns row0 .. row0 + 31, through the warp's shared-memory tile
// tb (16 x 40 halves): two 16-byte stores per lane instead of 16 two-byte
// stores.  A warp with rows past M stores element by element.
__device__ __forceinline__ void store_chunk_T(uint16_t *tb, const uint16_t (&h)[16], uint16_t *outT, int ldt, int n,
                                              int row0, int M) {
  const int lane = threadIdx.x & 31;
  if (row0 + 32 > M) {
    const int row = row0 + lane;
    if (row < M)
#pragma unroll
      for (int j = 0; j < 16; ++j) outT[(size_t)(n + j) * ldt + row] = h[j];
    return;
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) tb[j * 40 + lane] = h[j];
  __syncwarp();
  const int j = lane >> 1, half = lane & 1;
  const uint4 *src = (const uint4 *)(tb + j * 40 + half * 16);
  uint4 *dst = (uint4 *)(outT + (size_t)(n + j) * ldt + row0 + half * 16);
  dst[0] = src[0];
  dst[1] = src[1];
  __syncwarp();  // the tile is reused by the next chunk
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int BN>
__host__ __device__ constexpr int tmem_cols() {
  return BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
}

template <int BN>
constexpr size_t mma_smem_bytes() {  // alignment slack, operand ring, barriers, column accumulators
  return 1024 + (size_t)GSTAGES * (GM * 128 + BN * 128) + 256 + 2 * BN * sizeof(float);
}

// ---------------------------------------------------------------------------
// D = A B^T on one 128 x BN tile (blockIdx.x, blockIdx.y) and one K range
// (blockIdx.z) of k_split columns (a multiple of GK)
// ---------------------------------------------------------------------------
template <int BN, int EPI>
__global__ void __launch_bounds__(128, 1)
    k_mma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
          int k_split, GemmEpi E) {
  extern __shared__ uint8_t smem_raw[];
  // aligned by an offset from the shared array itself, so that the compiler
  // keeps shared-memory (not generic) accesses
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *sA = smem;
  uint8_t *sB = smem + GSTAGES * GM * 128;
  uint64_t *full = (uint64_t *)(sB + GSTAGES * BN * 128);
  uint64_t *empty = full + GSTAGES;
  uint64_t *done = empty + GSTAGES;
  uint32_t *tmem_slot = (uint32_t *)(done + 1);
  float *colacc = (float *)(sB + GSTAGES * BN * 128 + 256);  // per-CTA column sums [2][BN]
  constexpr uint32_t TCOLS = tmem_cols<BN>();
  constexpr uint32_t IDESC = idesc_bf16(GM, BN);
  constexpr uint32_t STAGE_BYTES = (GM + BN) * 128;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * GM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * k_split;
  const int kend = min(K, kbeg + k_split);
  const int nk = kend > kbeg ? (kend - kbeg + GK - 1) / GK : 0;

  for (int i = threadIdx.x; i < 2 * BN; i += blockDim.x) colacc[i] = 0.0f;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // the whole warp allocates the accumulator columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const uint32_t lim = E.spin ? E.spin : SPIN_LIMIT;
  int fail = 0;
  int issued = 0;  // producer: stages whose copies were issued
  // the self-test withholds the first slice (its MMA issuer's wait runs out;
  // nothing of that slice is in flight, so the drain below skips it)
  const int first_issued = E.withhold_first ? 1 : 0;
  if (nk > 0 && warp == 0 && lane == 0) {  // TMA producer
    for (int kb = first_issued; kb < nk; ++kb) {
      const int s = kb % GSTAGES;
      if (kb >= GSTAGES && !mbar_wait(&empty[s], ((kb / GSTAGES) - 1) & 1, lim)) {
        fail = 1;
        break;
      }
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_2d(&mapA, &full[s], sA + s * GM * 128, kbeg + kb * GK, m0);
      tma_load_2d(&mapB, &full[s], sB + s * BN * 128, kbeg + kb * GK, n0);
      issued = kb + 1;
    }
  } else if (nk > 0 && warp == 1 && lane == 0) {  // MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % GSTAGES;
      if (!mbar_wait(&full[s], (kb / GSTAGES) & 1, lim)) {
        fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * GM * 128), b0 = smem_u32(sB + s * BN * 128);
#pragma unroll
      for (int kk = 0; kk < GK / 16; ++kk)
        umma_bf16(tmem, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), IDESC, (kb | kk) != 0 ? 1u : 0u);
      umma_commit(&empty[s]);  // frees the stage once these MMAs have read it
    }
    umma_commit(done);  // completes when every MMA issued above has finished
  }
  // everyone: wait for the accumulator (bounded), agree on failure
  bool ok = nk == 0 || mbar_wait(done, 0, lim);
  fail = __syncthreads_or(fail || !ok);
  tc_fence_after();

  const int row = m0 + warp * 32 + lane;
  const bool rv = row < M;
  // the epilogue's column-sum tile of this warp: in the operand ring, whose
  // copies and MMAs have all completed once the accumulator is ready
  float *tbuf = (float *)sA + warp * 32 * 17;
  uint16_t *tb16 = (uint16_t *)((float *)sA + 4 * 32 * 17) + warp * 16 * 40;
  __syncwarp();
  if (!fail && nk > 0) {
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
    if constexpr (EPI == EPI_HEAD) {
      // pass 1: h3 = relu(z3 + b3) (BF16, stored), y = h3 . w4 + b4
      float y = 0.0f;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(tbase + c0, v);
        uint16_t hb[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          const float h = fmaxf(v[j] + E.bias[n], 0.0f);
          hb[j] = to_bf16(h);
          y = fmaf(from_bf16(hb[j]), from_bf16(E.w4[n]), y);
        }
        if (rv) {
          uint4 *o = (uint4 *)(E.out + (size_t)row * E.ldo + n0 + c0);
          o[0] = make_uint4(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16), hb[4] | (hb[5] << 16), hb[6] | (hb[7] << 16));
          o[1] = make_uint4(hb[8] | (hb[9] << 16), hb[10] | (hb[11] << 16), hb[12] | (hb[13] << 16),
                            hb[14] | (hb[15] << 16));
        }
      }
      y += *E.b4;
      const float diff = rv ? y - E.target[row] : 0.0f;
      const float dy = diff * E.inv_batch;
      const float l = warp_sum_f(0.5f * diff * diff * E.inv_batch);
      if (lane == 0) atomicAdd(E.loss, l);
      const float gb4 = warp_sum_f(dy);
      if (lane == 0) atomicAdd(E.gb4, gb4);
      // pass 2: g3 = dy w4 [h3 > 0]; column sums gb3 (of g3) and gw4 (of dy h3)
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint4 raw[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        if (rv) {
          const uint4 *src = (const uint4 *)(E.out + (size_t)row * E.ldo + n0 + c0);
          raw[0] = src[0];
          raw[1] = src[1];
        }
        const uint16_t *hb = (const uint16_t *)raw;
        uint16_t gb[16];
        float gv[16], wv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          const float h = from_bf16(hb[j]);
          const float g = h > 0.0f ? dy * from_bf16(E.w4[n]) : 0.0f;
          gb[j] = to_bf16(g);
          gv[j] = g;
          wv[j] = dy * h;
        }
        store_chunk_T(tb16, gb, E.g3T, E.ldt3, n0 + c0, m0 + warp * 32, M);
        {  // column sums of g3 (gb3) and of dy h3 (gw4)
          const float sg = chunk_colsum(tbuf, gv), sw = chunk_colsum(tbuf, wv);
          if (lane < 16) {
            atomicAdd(&colacc[c0 + lane], sg);
            atomicAdd(&colacc[BN + c0 + lane], sw);
          }
        }
        if (rv) {
          uint4 *o = (uint4 *)(E.g3 + (size_t)row * 128 + n0 + c0);
          o[0] = make_uint4(gb[0] | (gb[1] << 16), gb[2] | (gb[3] << 16), gb[4] | (gb[5] << 16), gb[6] | (gb[7] << 16));
          o[1] = make_uint4(gb[8] | (gb[9] << 16), gb[10] | (gb[11] << 16), gb[12] | (gb[13] << 16),
                            gb[14] | (gb[15] << 16));
        }
      }
    } else {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tmem_ld16(tbase + c0, v);
        if constexpr (EPI == EPI_PARTIAL) {
          if (rv && n0 + c0 + 16 <= N) {  // slice blockIdx.z of [splits][M][ldf], 16-byte stores
            float4 *o = (float4 *)(E.outF + ((size_t)blockIdx.z * M + row) * E.ldf + n0 + c0);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
            o[2] = make_float4(v[8], v[9], v[10], v[11]);
            o[3] = make_float4(v[12], v[13], v[14], v[15]);
          }
        } else if constexpr (EPI == EPI_ATOMIC || EPI == EPI_STORE) {
          if (rv) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = n0 + c0 + j;
              if (n < N) {
                if (EPI == EPI_ATOMIC) atomicAdd(&E.outF[(size_t)row * E.ldf + n], v[j]);
                else E.outF[(size_t)row * E.ldf + n] = v[j];
              }
            }
          }
        } else {
        uint16_t hb[16];
        uint16_t mrow[16];  // the mask row's 16 BF16 values (two 16-byte loads)
        if (EPI == EPI_MASK) {
          uint4 mr[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
          if (rv) {
            const uint4 *src = (const uint4 *)(E.mask + (size_t)row * E.ldm + n0 + c0);
            mr[0] = src[0];
            mr[1] = src[1];
          }
          memcpy(mrow, mr, sizeof(mrow));
        }
        float xs[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          float x;
          if (EPI == EPI_RELU) {
            x = fmaxf(v[j] + E.bias[n], 0.0f);
          } else {  // EPI_MASK
            const float mk = rv ? from_bf16(mrow[j]) : 0.0f;
            x = mk > 0.0f ? v[j] : 0.0f;
          }
          xs[j] = rv ? x : 0.0f;
          hb[j] = to_bf16(x);
        }
        if (E.outT) store_chunk_T(tb16, hb, E.outT, E.ldt, n0 + c0, m0 + warp * 32, M);
        if (EPI == EPI_MASK) {  // column sums of the masked values
          const float cs = chunk_colsum(tbuf, xs);
          if (lane < 16) atomicAdd(&colacc[c0 + lane], cs);
        }
        if (rv && E.out) {
          uint4 *o = (uint4 *)(E.out + (size_t)row * E.ldo + n0 + c0);
          o[0] = make_uint4(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16), hb[4] | (hb[5] << 16), hb[6] | (hb[7] << 16));
          o[1] = make_uint4(hb[8] | (hb[9] << 16), hb[10] | (hb[11] << 16), hb[12] | (hb[13] << 16),
                            hb[14] | (hb[15] << 16));
        }
        }
      }
    }
  }
  if (fail) {
    // let this CTA's copies in flight land before its shared memory goes away
    if (warp == 0 && lane == 0)
      for (int kb = max(first_issued, issued - GSTAGES); kb < issued; ++kb)
        mbar_wait(&full[kb % GSTAGES], (kb / GSTAGES) & 1, lim);
    if (threadIdx.x == 0) atomicOr(E.err, ERRB_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (!fail && nk > 0) {  // one global add per column and CTA
    if (EPI == EPI_MASK)
      for (int i = threadIdx.x; i < BN && n0 + i < N; i += blockDim.x) atomicAdd(&E.colsum[n0 + i], colacc[i]);
    if (EPI == EPI_HEAD)
      for (int i = threadIdx.x; i < BN && n0 + i < N; i += blockDim.x) {
        atomicAdd(&E.gb3[n0 + i], colacc[i]);
        atomicAdd(&E.gw4[n0 + i], colacc[BN + i]);
      }
  }
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
}

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
// X (FP32 [B][48]) -> BF16 Xb [B][64] (zero padded) and XbT [48][B]; targets clipped
__global__ void k_prep(const float *X, const float *t, int B, float clip, uint16_t *Xb, uint16_t *XbT, float *tc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * 64) return;
  const int r = i / 64, c = i % 64;
  const uint16_t v = c < MLP_IN ? to_bf16(X[(size_t)r * MLP_IN + c]) : (uint16_t)0;
  Xb[(size_t)r * 64 + c] = v;
  if (c < MLP_IN) XbT[(size_t)c * B + r] = v;
  if (c == 0) tc[r] = fminf(fmaxf(t[r], -clip), clip);
}

// parameter layout of the masters, gradients and Adam moments
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H, OFF_B2 = OFF_W2 + MLP_H * MLP_H,
              OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H * MLP_H, OFF_W4 = OFF_B3 + MLP_H,
              OFF_B4 = OFF_W4 + MLP_H, N_PARAMS = OFF_B4 + 1;

struct Bf16Copies {
  uint16_t *W1p;  // [128][64] (K padded)
  uint16_t *W2, *W2T, *W3, *W3T, *w4;
};

// BF16 copies of the masters (and transposes), as the products take them
__global__ void k_weights_bf16(const float *P, Bf16Copies C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_H * 64) {
    const int o = i / 64, k = i % 64;
    C.W1p[i] = k < MLP_IN ? to_bf16(P[OFF_W1 + o * MLP_IN + k]) : (uint16_t)0;
  }
  if (i < MLP_H * MLP_H) {
    const int o = i / MLP_H, k = i % MLP_H;
    const uint16_t a = to_bf16(P[OFF_W2 + i]), b = to_bf16(P[OFF_W3 + i]);
    C.W2[i] = a;
    C.W3[i] = b;
    C.W2T[k * MLP_H + o] = a;
    C.W3T[k * MLP_H + o] = b;
  }
  if (i < MLP_H) C.w4[i] = to_bf16(P[OFF_W4 + i]);
}

// sum of the split-K slices [splits][count] in split order (deterministic)
__global__ void k_sum_splits(const float *__restrict__ part, int splits, int count, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float acc = 0.0f;
  for (int z = 0; z < splits; ++z) acc += part[(size_t)z * count + i];
  out[i] = acc;
}

// Adam (bias-corrected) on every master parameter
__global__ void k_adam(float *P, const float *G, float *Mm, float *Vv, int n, float lr, float beta1, float beta2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = beta1 * Mm[i] + (1.0f - beta1) * g;
  const float v = beta2 * Vv[i] + (1.0f - beta2) * g * g;
  Mm[i] = m;
  Vv[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// ---------------------------------------------------------------------------
// The fused training step (k_train_fused): each CTA (one per SM, 128 threads,
// thread = row of a 128-row tile) runs, tile after tile, the three forward
// products, the output layer and loss, the two backward data products and the
// three weight-gradient products.  Operands never leave the SM: the threads
// write X, h1, h2 and the back-propagated errors G3, G2, G1 as BF16 into
// 128-byte-swizzled K-major tiles in shared memory (the layout TMA gives the
// products of k_mma), the weights stay resident there, the products
// accumulate in tensor memory -- the weight gradients across all of the CTA's
// tiles -- and each CTA writes its partial gradients once.  The weight-
// gradient products (K = the tile's rows) and the backward data products
// (B = W, K = W's output index) read the same stored tiles as MN-major
// operands (transpose bits of the instruction descriptor; LBO = the 64-column
// slice stride, SBO = 8 rows), so no transposed copy is written.  The bias
// and output-layer gradients are column sums in shared memory, the loss a
// block sum.  A second kernel sums the CTAs' partials in CTA order
// (deterministic).  Every mbarrier wait is bounded.
// ---------------------------------------------------------------------------
constexpr int FT_THREADS = 256;  // two warps per tensor-memory lane quarter: columns 0-63 and 64-127
constexpr uint32_t FT_TILE = 16384;         // one 128-row x 64-column BF16 slice
constexpr uint32_t FT_G3 = 0;               // G3, then G1 [128 x 128] (read as MN-major operands)
constexpr uint32_t FT_H2 = 2 * FT_TILE;     // h2, then G2 [128 x 128]
constexpr uint32_t FT_H1 = 4 * FT_TILE;     // h1 [128 x 128]
constexpr uint32_t FT_X = 6 * FT_TILE;      // X [128 x 64]: 48 features, zero padding
constexpr uint32_t FT_W1 = 7 * FT_TILE;     // W1 [128 out x 64 in]
constexpr uint32_t FT_W2 = 8 * FT_TILE;     // W2 [128 x 128]
constexpr uint32_t FT_W3 = 10 * FT_TILE;    // W3 [128 x 128]
constexpr uint32_t FT_MISC = 12 * FT_TILE;  // column-sum tiles, accumulators, barrier, tensor-memory slot
constexpr uint32_t FT_ACC = FT_MISC + 8 * 32 * 17 * 4;     // [4][128] gb1, gb2, gb3, gw4; [4] gb4, loss
constexpr uint32_t FT_BIAS = FT_ACC + (4 * 128 + 4) * 4;  // [4][128] b1, b2, b3 and w4 (FP32), staged once
constexpr uint32_t FT_YP = FT_BIAS + 4 * 128 * 4;          // [2][128] the output layer's two half sums
constexpr uint32_t FT_BAR = FT_YP + 2 * 128 * 4;
constexpr uint32_t FT_ONES = (FT_BAR + 64 + 1023) / 1024 * 1024;  // [16 x 64] BF16 ones (a K-major B operand)
constexpr size_t FT_SMEM = 1024 + FT_ONES + 2048;
// tensor-memory columns: the products' accumulator, the weight gradients and
// the bias gradients (G^T 1: 16 equal columns each)
constexpr uint32_t TM_Z = 0, TM_GW3 = 128, TM_GW2 = 256, TM_GW1 = 384, TM_GB3 = 432, TM_GB2 = 448, TM_GB1 = 464;
// per-CTA partials: the parameters' gradients and the loss, padded to 16 bytes
constexpr int PART_STRIDE = (N_PARAMS + 1 + 3) / 4 * 4;

// byte offset of 16-byte chunk j (of 8) of row r in a K-major 128-byte-swizzled slice
__device__ __forceinline__ uint32_t sw128(int r, int j) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}
// 16 BF16 values of row r, columns c .. c + 15 (c a multiple of 16), into / from a tile of slices
__device__ __forceinline__ void st_row16(uint8_t *tile, int r, int c, const uint16_t (&h)[16]) {
  uint8_t *sl = tile + (uint32_t)(c >> 6) * FT_TILE;
  const int j = (c & 63) >> 3;
  *(uint4 *)(sl + sw128(r, j)) =
      make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
  *(uint4 *)(sl + sw128(r, j + 1)) =
      make_uint4(h[8] | (h[9] << 16), h[10] | (h[11] << 16), h[12] | (h[13] << 16), h[14] | (h[15] << 16));
}
__device__ __forceinline__ void ld_row16(const uint8_t *tile, int r, int c, uint16_t (&h)[16]) {
  const uint8_t *sl = tile + (uint32_t)(c >> 6) * FT_TILE;
  const int j = (c & 63) >> 3;
  const uint4 a = *(const uint4 *)(sl + sw128(r, j)), b = *(const uint4 *)(sl + sw128(r, j + 1));
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    h[2 * i] = (uint16_t)(w[i] & 0xFFFFu);
    h[2 * i + 1] = (uint16_t)(w[i] >> 16);
  }
}

// Shared-memory descriptor of an MN-major operand read from K-major-stored
// 128-byte-swizzled slices: the 64-element blocks along M (or N) are the
// slices (LBO = slice stride), the 8-deep groups along K are 8 stored rows
// (SBO = 1024 bytes).
__device__ __forceinline__ uint64_t sdesc_mn128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(FT_TILE >> 4) << 16;  // leading byte offset
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
constexpr uint32_t IDESC_TA = 1u << 15, IDESC_TB = 1u << 16;  // A / B MN-major

// A descriptor moved on by a byte offset (the start-address field holds
// address >> 4 and stays below its 14-bit limit inside shared memory), so
// that the unrolled issue loops below add constants to two base descriptors
// instead of building each descriptor anew.
__device__ __forceinline__ uint64_t dmove(uint64_t d, uint32_t bytes) { return d + (uint64_t)(bytes >> 4); }
// byte offset of K step kk (16 elements) in a K-major tile of 64-column slices
__host__ __device__ constexpr uint32_t kstep(int kk) { return (uint32_t)(kk >> 2) * FT_TILE + (uint32_t)(kk & 3) * 32; }

// D = A B^T with both K-major (K = 64 * KS), by thread 0
template <int KS>
__device__ __forceinline__ void ft_mma_kk(uint32_t d, uint32_t a, uint32_t b, uint32_t idesc) {
  const uint64_t da = sdesc_sw128(a), db = sdesc_sw128(b);
#pragma unroll
  for (int kk = 0; kk < 4 * KS; ++kk) umma_bf16(d, dmove(da, kstep(kk)), dmove(db, kstep(kk)), idesc, kk ? 1u : 0u);
}
// D (+)= A^T B over the tile's 128 rows (K = stored rows; A and B MN-major views)
__device__ __forceinline__ void ft_mma_mn(uint32_t d, uint32_t a, uint32_t b, uint32_t idesc, bool acc) {
  const uint64_t da = sdesc_mn128(a), db = sdesc_mn128(b);
  const uint32_t acc0 = acc ? 1u : 0u;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) umma_bf16(d, dmove(da, kk * 2048), dmove(db, kk * 2048), idesc, kk ? 1u : acc0);
}
// D = A W with A K-major (K = W's stored rows) and W read as an MN-major operand
__device__ __forceinline__ void ft_mma_kmn(uint32_t d, uint32_t a, uint32_t w, uint32_t idesc) {
  const uint64_t da = sdesc_sw128(a), dw = sdesc_mn128(w);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) umma_bf16(d, dmove(da, kstep(kk)), dmove(dw, kk * 2048), idesc, kk ? 1u : 0u);
}

// D (+)= G^T 1 over the tile's 128 rows: the column sums of G (MN-major view)
// into 16 equal accumulator columns; the ones operand is uniform, so every
// K step reads the same 64-element block
__device__ __forceinline__ void ft_mma_colsum(uint32_t d, uint32_t g, uint32_t ones, uint32_t idesc, bool acc) {
  const uint64_t dg = sdesc_mn128(g), d1 = sdesc_sw128(ones);
  const uint32_t acc0 = acc ? 1u : 0u;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) umma_bf16(d, dmove(dg, kk * 2048), dmove(d1, (kk & 3) * 32), idesc, kk ? 1u : acc0);
}

struct FusedArgs {
  const float *X, *t;  // [B][48] features, [B] targets
  int B;
  float clip, inv_batch;
  const uint16_t *w4;                  // BF16 copy of the output weights (the others come by TMA)
  const float *P;                      // FP32 masters (biases)
  float *part;                         // [gridDim.x][PART_STRIDE] partial gradients and loss
  int *err;
  uint32_t spin;
};

__global__ void __launch_bounds__(FT_THREADS, 1)
    k_train_fused(const __grid_constant__ CUtensorMap mW1, const __grid_constant__ CUtensorMap mW2,
                  const __grid_constant__ CUtensorMap mW3, FusedArgs A) {
  extern __shared__ uint8_t smem_raw[];
  // aligned by an offset from the shared array itself, so that the compiler
  // keeps shared-memory (not generic) accesses
  uint8_t *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float *tbuf_all = (float *)(sm + FT_MISC);
  float *acc = (float *)(sm + FT_ACC);  // [0..127] gb1, [128..] gb2, [256..] gb3, [384..] gw4, [512] gb4, [513] loss
  float *yp = (float *)(sm + FT_YP);
  uint64_t *bar = (uint64_t *)(sm + FT_BAR);        // the products' commits
  uint64_t *wbar = (uint64_t *)(sm + FT_BAR + 8);   // the weights' copies
  uint32_t *tmem_slot = (uint32_t *)(sm + FT_BAR + 16);
  uint64_t *bar2 = (uint64_t *)(sm + FT_BAR + 24);  // the weight-gradient products of a backward stage
  uint64_t *dbar = (uint64_t *)(sm + FT_BAR + 32);  // the drain after an expired wait
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int r = quarter * 32 + lane;  // this thread's row of the tile (its tensor-memory lane)
  const int c0 = half * 64;           // and its 64 columns
  float *tbuf = tbuf_all + warp * 32 * 17;
  const uint32_t lim = A.spin ? A.spin : SPIN_LIMIT;
  const uint32_t sbase = smem_u32(sm);
  constexpr uint32_t ID_KK = idesc_bf16(128, 128), ID_MN = idesc_bf16(128, 128) | IDESC_TA | IDESC_TB,
                     ID_MN48 = idesc_bf16(128, 48) | IDESC_TA | IDESC_TB, ID_KMN = idesc_bf16(128, 128) | IDESC_TB,
                     ID_ONES = idesc_bf16(128, 16) | IDESC_TA;

  for (int i = threadIdx.x; i < 4 * 128 + 4; i += blockDim.x) acc[i] = 0.0f;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(wbar, 1);
    mbar_init(bar2, 1);
    mbar_init(dbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the BF16 weights by TMA, 128-row x 64-column boxes in the 128-byte
    // swizzle (the K-major operand layout), while the rest is set up
    mbar_expect_tx(wbar, 5 * FT_TILE);
    tma_load_2d(&mW1, wbar, sm + FT_W1, 0, 0);
    tma_load_2d(&mW2, wbar, sm + FT_W2, 0, 0);
    tma_load_2d(&mW2, wbar, sm + FT_W2 + FT_TILE, 64, 0);
    tma_load_2d(&mW3, wbar, sm + FT_W3, 0, 0);
    tma_load_2d(&mW3, wbar, sm + FT_W3 + FT_TILE, 64, 0);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = threadIdx.x; i < 2048 / 16; i += blockDim.x)
    *(uint4 *)(sm + FT_ONES + 16 * i) = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
  float *bias = (float *)(sm + FT_BIAS);  // the epilogues read these as broadcasts
  if (threadIdx.x < 128) {
    bias[threadIdx.x] = A.P[OFF_B1 + threadIdx.x];
    bias[128 + threadIdx.x] = A.P[OFF_B2 + threadIdx.x];
    bias[256 + threadIdx.x] = A.P[OFF_B3 + threadIdx.x];
    bias[384 + threadIdx.x] = from_bf16(A.w4[threadIdx.x]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);  // this warp's lanes
  const float *b1 = bias, *b2 = bias + 128, *b3 = bias + 256, *w4f = bias + 384;
  const float b4 = A.P[OFF_B4];
  uint32_t phase = 0;
  int tiles_done = 0;
  // the weights have landed (bounded wait; on expiry a second bounded wait
  // for the copies still in flight, then no tile is run)
  bool wok = mbar_wait(wbar, 0, lim);
  wok = __syncthreads_or(!wok) == 0;
  if (!wok && threadIdx.x == 0) {
    mbar_wait(wbar, 0, lim);
    atomicOr(A.err, ERRB_TIMEOUT);
  }

  // every thread: wait for the last commit on bar (bounded); false when it ran out
  auto wait_mma = [&]() -> bool {
    const bool ok = mbar_wait(bar, phase, lim);
    phase ^= 1u;
    const int f = __syncthreads_or(!ok);
    tc_fence_after();
    return f == 0;
  };
  // the same for the commits on bar2
  uint32_t phase2 = 0;
  auto wait_mma2 = [&]() -> bool {
    const bool ok = mbar_wait(bar2, phase2, lim);
    phase2 ^= 1u;
    const int f = __syncthreads_or(!ok);
    tc_fence_after();
    return f == 0;
  };
  // after the threads wrote operand tiles: visible to the tensor cores
  auto publish = [&]() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  };
  // relu(z + bias) of this thread's 64 columns as BF16 into a tile
  auto relu_out = [&](const float *bb, uint8_t *tile) {
#pragma unroll 1
    for (int c = c0; c < c0 + 64; c += 32) {
      float v[32];
      tmem_ld32(trow + TM_Z + c, v);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint16_t h[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) h[j] = to_bf16(fmaxf(v[16 * hh + j] + bb[c + 16 * hh + j], 0.0f));
        st_row16(tile, r, c + 16 * hh, h);
      }
    }
  };
  // G = q [h > 0] of this thread's 64 columns into a tile (BF16; its column
  // sums, the bias gradient, are taken on the tensor cores)
  auto mask_out = [&](const uint8_t *hmask, uint8_t *tile) {
#pragma unroll 1
    for (int c = c0; c < c0 + 64; c += 32) {
      float v[32];
      tmem_ld32(trow + TM_Z + c, v);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint16_t hm[16], gb[16];
        ld_row16(hmask, r, c + 16 * hh, hm);
#pragma unroll
        for (int j = 0; j < 16; ++j) gb[j] = to_bf16(from_bf16(hm[j]) > 0.0f ? v[16 * hh + j] : 0.0f);
        st_row16(tile, r, c + 16 * hh, gb);
      }
    }
  };

  const int n_tiles = A.B / 128;
  bool ok = true;
  // X of the next tile (its 128 x 48 floats, contiguous, coalesced) and this
  // thread's row target, loaded into registers one tile ahead
  constexpr int XQ = 128 * 12 / FT_THREADS;
  static_assert(128 * 12 % FT_THREADS == 0, "X tile split");
  float4 xn[XQ];
  float tn = 0.0f;
  auto load_x = [&](int t) {
    const float4 *xt = (const float4 *)(A.X + (size_t)t * 128 * 48);
#pragma unroll
    for (int k = 0; k < XQ; ++k) xn[k] = __ldg(&xt[threadIdx.x + k * FT_THREADS]);
    tn = __ldg(&A.t[(size_t)t * 128 + r]);
  };
  if (blockIdx.x < n_tiles) load_x(blockIdx.x);
  for (int tile = blockIdx.x; tile < n_tiles && ok && wok; tile += gridDim.x) {
    // ---- X (BF16, zero padded to 64) into its tile, and the clipped target
#pragma unroll
    for (int k = 0; k < XQ; ++k) {
      const int q = threadIdx.x + k * FT_THREADS;
      const float4 v = xn[k];
      const int xrow = q / 12, col = (q - xrow * 12) * 4;
      const uint32_t lo = (uint32_t)to_bf16(v.x) | ((uint32_t)to_bf16(v.y) << 16),
                     hi = (uint32_t)to_bf16(v.z) | ((uint32_t)to_bf16(v.w) << 16);
      *(uint2 *)(sm + FT_X + sw128(xrow, col >> 3) + (col & 7) * 2) = make_uint2(lo, hi);
    }
    if (threadIdx.x < 128) {  // columns 48 .. 63: zero
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      *(uint4 *)(sm + FT_X + sw128(threadIdx.x, 6)) = z;
      *(uint4 *)(sm + FT_X + sw128(threadIdx.x, 7)) = z;
    }
    const float tgt = fminf(fmaxf(tn, -A.clip), A.clip);
    publish();
    if (tile + (int)gridDim.x < n_tiles) load_x(tile + (int)gridDim.x);  // lands while this tile runs
    // ---- z1 = X W1^T; h1 = relu(z1 + b1)
    if (threadIdx.x == 0) {
      ft_mma_kk<1>(tmem + TM_Z, sbase + FT_X, sbase + FT_W1, ID_KK);
      umma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    relu_out(b1, sm + FT_H1);
    publish();
    // ---- z2 = h1 W2^T; h2 = relu(z2 + b2)
    if (threadIdx.x == 0) {
      ft_mma_kk<2>(tmem + TM_Z, sbase + FT_H1, sbase + FT_W2, ID_KK);
      umma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    relu_out(b2, sm + FT_H2);
    publish();
    // ---- z3 = h2 W3^T; h3 = relu(z3 + b3) (BF16); y = h3 . w4 + b4; loss; G3 = dy w4 [h3 > 0]
    if (threadIdx.x == 0) {
      ft_mma_kk<2>(tmem + TM_Z, sbase + FT_H2, sbase + FT_W3, ID_KK);
      umma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    {
      float y = 0.0f;
#pragma unroll 1
      for (int c = c0; c < c0 + 64; c += 32) {
        float v[32];
        tmem_ld32(trow + TM_Z + c, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) y = fmaf(from_bf16(to_bf16(fmaxf(v[j] + b3[c + j], 0.0f))), w4f[c + j], y);
      }
      yp[half * 128 + r] = y;
    }
    __syncthreads();
    const float y = (yp[r] + yp[128 + r]) + b4;
    const float diff = y - tgt, dy = diff * A.inv_batch;
    if (half == 0) {
      const float l = warp_sum_f(0.5f * diff * diff * A.inv_batch), g4 = warp_sum_f(dy);
      if (lane == 0) {
        atomicAdd(&acc[513], l);
        atomicAdd(&acc[512], g4);
      }
    }
#pragma unroll 1
    for (int c = c0; c < c0 + 64; c += 32) {
      float v[32];
      tmem_ld32(trow + TM_Z + c, v);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float wv[16];
        uint16_t gb[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c + 16 * hh + j;
          const float h = from_bf16(to_bf16(fmaxf(v[16 * hh + j] + b3[n], 0.0f)));
          wv[j] = dy * h;
          gb[j] = to_bf16(h > 0.0f ? dy * w4f[n] : 0.0f);
        }
        st_row16(sm + FT_G3, r, c + 16 * hh, gb);
        const float sw = chunk_colsum(tbuf, wv);
        if (lane < 16) atomicAdd(&acc[384 + c + 16 * hh + lane], sw);
      }
    }
    publish();
    // ---- q2 = G3 W3 (committed first), then gW3 += G3^T h2 and gb3 += G3^T 1,
    // which run while the threads form G2 = q2 [h2 > 0] in registers; G2
    // replaces h2 once those products have read it
    if (threadIdx.x == 0) {
      ft_mma_kmn(tmem + TM_Z, sbase + FT_G3, sbase + FT_W3, ID_KMN);
      umma_commit(bar);
      ft_mma_mn(tmem + TM_GW3, sbase + FT_G3, sbase + FT_H2, ID_MN, tiles_done > 0);
      ft_mma_colsum(tmem + TM_GB3, sbase + FT_G3, sbase + FT_ONES, ID_ONES, tiles_done > 0);
      umma_commit(bar2);
    }
    if (!(ok = wait_mma())) break;
    {
      uint32_t g2[32];  // this thread's 64 columns of G2, BF16 pairs
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        float v[32];
        tmem_ld32(trow + TM_Z + c0 + 32 * cc, v);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint16_t hm[16];
          ld_row16(sm + FT_H2, r, c0 + 32 * cc + 16 * hh, hm);
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const uint32_t lo = to_bf16(from_bf16(hm[j]) > 0.0f ? v[16 * hh + j] : 0.0f),
                           hi = to_bf16(from_bf16(hm[j + 1]) > 0.0f ? v[16 * hh + j + 1] : 0.0f);
            g2[16 * cc + 8 * hh + j / 2] = lo | (hi << 16);
          }
        }
      }
      if (!(ok = wait_mma2())) break;  // gW3 and gb3 have read h2
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint8_t *sl = sm + FT_H2 + (uint32_t)(c0 >> 6) * FT_TILE;
        const int j = 2 * q;  // 16-byte chunks j, j + 1 of the row's 64-column slice
        *(uint4 *)(sl + sw128(r, j)) = make_uint4(g2[8 * q], g2[8 * q + 1], g2[8 * q + 2], g2[8 * q + 3]);
        *(uint4 *)(sl + sw128(r, j + 1)) = make_uint4(g2[8 * q + 4], g2[8 * q + 5], g2[8 * q + 6], g2[8 * q + 7]);
      }
    }
    publish();
    // ---- q1 = G2 W2 (committed first), then gW2 += G2^T h1 and gb2 += G2^T 1,
    // which run while the threads form G1 = q1 [h1 > 0] over G3 (free: the
    // products that read G3 are done)
    if (threadIdx.x == 0) {
      ft_mma_kmn(tmem + TM_Z, sbase + FT_H2, sbase + FT_W2, ID_KMN);
      umma_commit(bar);
      ft_mma_mn(tmem + TM_GW2, sbase + FT_H2, sbase + FT_H1, ID_MN, tiles_done > 0);
      ft_mma_colsum(tmem + TM_GB2, sbase + FT_H2, sbase + FT_ONES, ID_ONES, tiles_done > 0);
      umma_commit(bar2);
    }
    if (!(ok = wait_mma())) break;
    mask_out(sm + FT_H1, sm + FT_G3);
    publish();
    // ---- gW1 += G1^T X, gb1 += G1^T 1 (the next tile overwrites X, G1, h1 and
    // G2 only after this; the products complete in issue order)
    if (threadIdx.x == 0) {
      ft_mma_mn(tmem + TM_GW1, sbase + FT_G3, sbase + FT_X, ID_MN48, tiles_done > 0);
      ft_mma_colsum(tmem + TM_GB1, sbase + FT_G3, sbase + FT_ONES, ID_ONES, tiles_done > 0);
      umma_commit(bar);
    }
    if (!(ok = wait_mma())) break;
    if (!(ok = wait_mma2())) break;  // gW2's commit (complete by now)
    ++tiles_done;
  }
  if (!ok) {  // a wait ran out: let the products in flight finish (bounded) before the memory goes
    if (threadIdx.x == 0) {
      umma_commit(dbar);  // arrives once every product this thread issued is done
      mbar_wait(dbar, 0, lim);
      atomicOr(A.err, ERRB_TIMEOUT);
    }
    __syncthreads();
  }
  // ---- this CTA's partial gradients and loss: the weight gradients through
  // shared memory (the operand tiles are free now; rows padded to 132 floats,
  // 16-byte stores and loads without bank conflicts) and out with coalesced
  // 16-byte stores; the bias gradients from their accumulator columns
  float *out = A.part + (size_t)blockIdx.x * PART_STRIDE;
  if (ok && wok && tiles_done > 0) {
    constexpr int LD = 132;
    float *st3 = (float *)sm, *st2 = st3 + 128 * LD, *st1 = st2 + 128 * LD;
#pragma unroll 1
    for (int c = c0; c < c0 + 64; c += 32) {
      float v[32];
      tmem_ld32(trow + TM_GW3 + c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 4) *(float4 *)&st3[r * LD + c + j] = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      tmem_ld32(trow + TM_GW2 + c, v);
#pragma unroll
      for (int j = 0; j < 32; j += 4) *(float4 *)&st2[r * LD + c + j] = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
    if (half == 0) {
#pragma unroll 1
      for (int c = 0; c < 48; c += 16) {
        float v[16];
        tmem_ld16(trow + TM_GW1 + c, v);
#pragma unroll
        for (int j = 0; j < 16; j += 4) *(float4 *)&st1[r * LD + c + j] = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
    } else {  // the bias gradients: column 0 of each accumulator, row r = unit r
      float v[16];
      tmem_ld16(trow + TM_GB1, v);
      acc[r] = v[0];
      tmem_ld16(trow + TM_GB2, v);
      acc[128 + r] = v[0];
      tmem_ld16(trow + TM_GB3, v);
      acc[256 + r] = v[0];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 128 * 128 / 4; i += FT_THREADS) {
      const int o = i >> 5, c = (i & 31) * 4;
      *(float4 *)&out[OFF_W3 + 4 * i] = *(const float4 *)&st3[o * LD + c];
      *(float4 *)&out[OFF_W2 + 4 * i] = *(const float4 *)&st2[o * LD + c];
    }
    for (int i = threadIdx.x; i < 128 * 48 / 4; i += FT_THREADS) {
      const int o = i / 12, c = (i - o * 12) * 4;
      *(float4 *)&out[OFF_W1 + 4 * i] = *(const float4 *)&st1[o * LD + c];
    }
  } else {
    for (int i = threadIdx.x; i < 128 * 128; i += blockDim.x) {
      out[OFF_W3 + i] = 0.0f;
      out[OFF_W2 + i] = 0.0f;
    }
    for (int i = threadIdx.x; i < 128 * 48; i += blockDim.x) out[OFF_W1 + i] = 0.0f;
  }
  __syncthreads();
  if (threadIdx.x < 128) {
    const int t = threadIdx.x;
    out[OFF_B1 + t] = acc[t];
    out[OFF_B2 + t] = acc[128 + t];
    out[OFF_B3 + t] = acc[256 + t];
    out[OFF_W4 + t] = acc[384 + t];
    if (t == 0) {
      out[OFF_B4] = acc[512];
      out[N_PARAMS] = acc[513];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

// Sum of the CTAs' partials in a fixed order (deterministic): a CTA of
// SUM_THREADS threads takes SUM_PAR consecutive parameters; each thread of
// slice s (SUM_SLICES slices) loads 4 consecutive parameters (16 bytes) of the
// partials c = s, s + SUM_SLICES, ... (a few loads per thread), and the slices
// are added in order through shared memory.  Many threads with wide loads
// keep enough bytes in flight to stream the partials at L2 bandwidth.  Returns the sum of parameter blockIdx.x *
// SUM_PAR + threadIdx.x for the first SUM_PAR threads (the partials are padded
// to PART_STRIDE, so the last group of 4 stays inside them).
constexpr int SUM_THREADS = 256, SUM_SLICES = 32, SUM_LANES = SUM_THREADS / SUM_SLICES, SUM_PAR = 4 * SUM_LANES,
              SUM_LOADS = 4;
__device__ __forceinline__ float sum_partials(const float *__restrict__ part, int n_parts, float *red) {
  const int pl = threadIdx.x % SUM_LANES, sl = threadIdx.x / SUM_LANES;
  const int i4 = blockIdx.x * SUM_PAR + 4 * pl;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i4 < PART_STRIDE) {
    for (int c = sl; c < n_parts; c += SUM_LOADS * SUM_SLICES) {
      float4 v[SUM_LOADS];
#pragma unroll
      for (int j = 0; j < SUM_LOADS; ++j) {  // unconditional loads (clamped index): all issued at once
        const int cj = min(c + j * SUM_SLICES, n_parts - 1);
        v[j] = __ldg((const float4 *)&part[(size_t)cj * PART_STRIDE + i4]);
      }
#pragma unroll
      for (int j = 0; j < SUM_LOADS; ++j)
        if (c + j * SUM_SLICES < n_parts) {
          s.x += v[j].x;
          s.y += v[j].y;
          s.z += v[j].z;
          s.w += v[j].w;
        }
    }
  }
  *(float4 *)&red[sl * SUM_PAR + 4 * pl] = s;
  __syncthreads();
  float g = 0.0f;
  if (threadIdx.x < SUM_PAR) {
    g = red[threadIdx.x];
#pragma unroll
    for (int k = 1; k < SUM_SLICES; ++k) g += red[k * SUM_PAR + threadIdx.x];
  }
  return g;
}

// G[i] = sum over the CTAs' partials (fixed order)
__global__ void __launch_bounds__(SUM_THREADS) k_sum_parts(const float *__restrict__ part, int n_parts, float *G) {
  __shared__ __align__(16) float red[SUM_SLICES * SUM_PAR];
  const int i = blockIdx.x * SUM_PAR + threadIdx.x;
  const float g = sum_partials(part, n_parts, red);
  if (threadIdx.x < SUM_PAR && i <= N_PARAMS) G[i] = g;
}

// The step's tail in one launch: the CTAs' partials summed (fixed order), then
// Adam on the masters (the arithmetic of k_adam) and the BF16 copies the
// products take (those of k_weights_bf16; the zero padding of W1p is written
// once at creation).
__global__ void __launch_bounds__(SUM_THREADS) k_sum_adam(const float *__restrict__ part, int n_parts, float *G,
                                                           float *P, float *Mm, float *Vv, float lr, float beta1,
                                                           float beta2, float eps, float c1, float c2, Bf16Copies C) {
  __shared__ __align__(16) float red[SUM_SLICES * SUM_PAR];
  const int i = blockIdx.x * SUM_PAR + threadIdx.x;
  const float g = sum_partials(part, n_parts, red);
  if (threadIdx.x >= SUM_PAR || i > N_PARAMS) return;
  G[i] = g;
  if (i == N_PARAMS) return;  // the loss
  const float m = beta1 * Mm[i] + (1.0f - beta1) * g;
  const float v = beta2 * Vv[i] + (1.0f - beta2) * g * g;
  Mm[i] = m;
  Vv[i] = v;
  const float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  P[i] = p;
  const uint16_t b = to_bf16(p);
  if (i < OFF_B1) {
    const int o = (i - OFF_W1) / MLP_IN, k = (i - OFF_W1) % MLP_IN;
    C.W1p[o * 64 + k] = b;
  } else if (i >= OFF_W2 && i < OFF_B2) {
    const int o = (i - OFF_W2) / MLP_H, k = (i - OFF_W2) % MLP_H;
    C.W2[i - OFF_W2] = b;
    C.W2T[k * MLP_H + o] = b;
  } else if (i >= OFF_W3 && i < OFF_B3) {
    const int o = (i - OFF_W3) / MLP_H, k = (i - OFF_W3) % MLP_H;
    C.W3[i - OFF_W3] = b;
    C.W3T[k * MLP_H + o] = b;
  } else if (i >= OFF_W4 && i < OFF_B4) {
    C.w4[i - OFF_W4] = b;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mutex;

int get_encode() {
  std::lock_guard<std::mutex> lock(g_encode_mutex);
  if (g_encode) return CR_OK;
  cudaDriverEntryPointQueryResult q;
  void *fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return CR_ERR_CUDA;
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return CR_OK;
}

// 2D BF16 tensor [rows][cols] (cols contiguous), box of GK columns x box_rows
int make_map(CUtensorMap *map, const uint16_t *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  if (((uintptr_t)base & 15) || (cols * 2) % 16) return CR_ERR_INVALID_ARG;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)GK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? CR_OK : CR_ERR_INVALID_ARG;
}

template <int BN, int EPI>
int launch_mma(const uint16_t *A, const uint16_t *Bm, int M, int N, int K, int lda, int ldb, int k_split,
               const GemmEpi &E, cudaStream_t s) {
  CUtensorMap ma, mb;
  int rc = make_map(&ma, A, (uint64_t)M, (uint64_t)lda, GM);
  if (rc == CR_OK) rc = make_map(&mb, Bm, (uint64_t)N, (uint64_t)ldb, BN);
  if (rc != CR_OK) return rc;
  static bool attr = false;
  const size_t smem = mma_smem_bytes<BN>();
  if (!attr) {
    if (cudaFuncSetAttribute(k_mma<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return CR_ERR_CUDA;
    attr = true;
  }
  const int splits = (K + k_split - 1) / k_split;
  dim3 grid((M + GM - 1) / GM, (N + BN - 1) / BN, splits);
  k_mma<BN, EPI><<<grid, 128, smem, s>>>(ma, mb, M, N, K, k_split, E);
  return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

// split of a long K (weight gradients) over about one wave of CTAs
int split_for(int K, int tiles) {
  int per = (K + 151) / 152 * std::max(tiles, 1);
  per = (per + GK - 1) / GK * GK;
  return std::max(per, GK);
}

}  // namespace
}  // namespace crmc

using namespace crmc;

struct cr_trainer {
  int max_batch = 0;
  double lr = 1e-3, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, clip = 20.0;
  long long step = 0;
  cudaStream_t stream = nullptr;
  float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr, *loss = nullptr, *tc = nullptr;
  int *err = nullptr;
  uint16_t *Xb = nullptr, *XbT = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *H1T = nullptr, *H2T = nullptr,
           *G3 = nullptr, *G3T = nullptr, *G2 = nullptr, *G2T = nullptr, *G1T = nullptr;
  uint16_t *wb = nullptr;  // BF16 weight copies (one block)
  float *part = nullptr;   // split-K slices of a weight gradient [max_splits][128][128]
  int max_splits = 0;
  bool unfused = false;     // one product per launch (k_mma) instead of the fused step
  float *part_f = nullptr;  // fused step: per-CTA partial gradients and loss [sms][PART_STRIDE]
  int sms = 1;
  Bf16Copies C{};
  CUtensorMap mW1{}, mW2{}, mW3{};  // TMA maps of the BF16 weights (fused step)
  int64_t launches = 0;
};

static void free_trainer(cr_trainer *t) {
  if (!t) return;
  void *ptrs[] = {t->P,  t->G,   t->Mm,  t->Vv, t->tc,  t->err, t->Xb, t->XbT, t->H1, t->H2,
                  t->H3, t->H1T, t->H2T, t->G3, t->G3T, t->G2,  t->G2T, t->G1T, t->wb, t->part, t->part_f};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete t;
}

extern "C" int cr_train_create(cr_trainer **out, const cr_mlp *m, const cr_train_cfg *cfg) {
  if (!out || !m || !cfg || cfg->max_batch <= 0 || cfg->max_batch % 128 || !m->W1 || !m->b1 || !m->W2 || !m->b2 ||
      !m->W3 || !m->b3 || !m->w4)
    return CR_ERR_INVALID_ARG;
  *out = nullptr;
  if (get_encode() != CR_OK) return CR_ERR_CUDA;
  cr_trainer *t = new (std::nothrow) cr_trainer();
  if (!t) return CR_ERR_NOMEM;
  t->max_batch = cfg->max_batch;
  t->lr = cfg->lr;
  t->beta1 = cfg->beta1;
  t->beta2 = cfg->beta2;
  t->eps = cfg->eps;
  t->clip = cfg->target_clip > 0.0 ? cfg->target_clip : 1e30;
  t->unfused = cfg->unfused != 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, dev);
    t->sms = std::max(t->sms, 1);
  }
  const size_t B = (size_t)cfg->max_batch;
  bool ok = true;
  auto al = [&](auto **p, size_t n) {
    if (ok && cudaMalloc((void **)p, n * sizeof(**p)) != cudaSuccess) ok = false;
  };
  al(&t->P, N_PARAMS);
  al(&t->G, N_PARAMS + 1);  // + loss
  al(&t->Mm, N_PARAMS);
  al(&t->Vv, N_PARAMS);
  al(&t->tc, B);
  al(&t->err, 1);
  al(&t->Xb, B * 64);
  al(&t->XbT, B * MLP_IN);
  for (uint16_t **p : {&t->H1, &t->H2, &t->H3, &t->H1T, &t->H2T, &t->G3, &t->G3T, &t->G2, &t->G2T, &t->G1T})
    al(p, B * MLP_H);
  al(&t->wb, (size_t)MLP_H * 64 + 4 * MLP_H * MLP_H + MLP_H);
  {
    const int ks = split_for(cfg->max_batch, 1);
    t->max_splits = (cfg->max_batch + ks - 1) / ks;
    al(&t->part, (size_t)t->max_splits * MLP_H * MLP_H);
  }
  al(&t->part_f, (size_t)std::min(t->sms, cfg->max_batch / 128) * PART_STRIDE);
  if (!ok) {
    free_trainer(t);
    return CR_ERR_NOMEM;
  }
  t->loss = t->G + N_PARAMS;
  t->C.W1p = t->wb;
  t->C.W2 = t->C.W1p + MLP_H * 64;
  t->C.W2T = t->C.W2 + MLP_H * MLP_H;
  t->C.W3 = t->C.W2T + MLP_H * MLP_H;
  t->C.W3T = t->C.W3 + MLP_H * MLP_H;
  t->C.w4 = t->C.W3T + MLP_H * MLP_H;
  if (make_map(&t->mW1, t->C.W1p, MLP_H, 64, 128) != CR_OK || make_map(&t->mW2, t->C.W2, MLP_H, MLP_H, 128) != CR_OK ||
      make_map(&t->mW3, t->C.W3, MLP_H, MLP_H, 128) != CR_OK) {
    free_trainer(t);
    return CR_ERR_CUDA;
  }
  // masters from the BF16 initial weights
  std::vector<float> h(N_PARAMS);
  auto bf = [](uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
  };
  for (int i = 0; i < MLP_H * MLP_IN; ++i) h[OFF_W1 + i] = bf(m->W1[i]);
  for (int i = 0; i < MLP_H * MLP_H; ++i) {
    h[OFF_W2 + i] = bf(m->W2[i]);
    h[OFF_W3 + i] = bf(m->W3[i]);
  }
  for (int i = 0; i < MLP_H; ++i) {
    h[OFF_B1 + i] = m->b1[i];
    h[OFF_B2 + i] = m->b2[i];
    h[OFF_B3 + i] = m->b3[i];
    h[OFF_W4 + i] = bf(m->w4[i]);
  }
  h[OFF_B4] = m->b4;
  if (cudaMemcpy(t->P, h.data(), sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(t->Mm, 0, sizeof(float) * N_PARAMS) != cudaSuccess ||
      cudaMemset(t->Vv, 0, sizeof(float) * N_PARAMS) != cudaSuccess || cudaMemset(t->err, 0, sizeof(int)) != cudaSuccess) {
    free_trainer(t);
    return CR_ERR_CUDA;
  }
  k_weights_bf16<<<(MLP_H * MLP_H + 255) / 256, 256>>>(t->P, t->C);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_trainer(t);
    return CR_ERR_CUDA;
  }
  *out = t;
  return CR_OK;
}

extern "C" void cr_train_destroy(cr_trainer *t) {
  if (!t) return;
  cudaStreamSynchronize(t->stream);
  free_trainer(t);
}

extern "C" int cr_train_set_stream(cr_trainer *t, void *stream) {
  if (!t) return CR_ERR_INVALID_ARG;
  t->stream = (cudaStream_t)stream;
  return CR_OK;
}

// CTAs of the fused step: as many as give every CTA the same number of
// tiles as the busiest one (at most one per SM), so that no CTA writes a
// partial for less work than the kernel's duration allows
static int fused_grid(int B, int sms) {
  const int tiles = B / 128;
  const int per = (tiles + sms - 1) / std::max(sms, 1);
  return (tiles + per - 1) / std::max(per, 1);
}

// the fused kernel alone (per-CTA partials in t->part_f)
static int train_fused_kernel(cr_trainer *t, const float *X, const float *target, int B) {
  if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0) return CR_ERR_INVALID_ARG;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_train_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FT_SMEM) != cudaSuccess)
      return CR_ERR_CUDA;
    attr = true;
  }
  const int grid = fused_grid(B, t->sms);
  FusedArgs A{};
  A.X = X;
  A.t = target;
  A.B = B;
  A.clip = (float)t->clip;
  A.inv_batch = 1.0f / (float)B;
  A.w4 = t->C.w4;
  A.P = t->P;
  A.part = t->part_f;
  A.err = t->err;
  A.spin = 0;
  k_train_fused<<<grid, FT_THREADS, FT_SMEM, t->stream>>>(t->mW1, t->mW2, t->mW3, A);
  t->launches++;
  return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

// the fused step (k_train_fused, then the CTAs' partials summed in order)
static int train_grads_fused(cr_trainer *t, const float *X, const float *target, int B) {
  const int rc = train_fused_kernel(t, X, target, B);
  if (rc != CR_OK) return rc;
  k_sum_parts<<<(N_PARAMS + 1 + SUM_PAR - 1) / SUM_PAR, SUM_THREADS, 0, t->stream>>>(t->part_f,
                                                                                 fused_grid(B, t->sms), t->G);
  t->launches++;
  return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

// forward + backward of one batch into t->G (and t->loss); device inputs
static int train_grads(cr_trainer *t, const float *X, const float *target, int B) {
  if (!t || !X || !target || B <= 0 || B % 128 || B > t->max_batch) return CR_ERR_INVALID_ARG;
  if (!t->unfused) return train_grads_fused(t, X, target, B);
  cudaStream_t s = t->stream;
  if (cudaMemsetAsync(t->G, 0, sizeof(float) * (N_PARAMS + 1), s) != cudaSuccess) return CR_ERR_CUDA;
  k_prep<<<(B * 64 + 255) / 256, 256, 0, s>>>(X, target, B, (float)t->clip, t->Xb, t->XbT, t->tc);
  t->launches++;
  const float *P = t->P;
  float *G = t->G;
  int rc;
  GemmEpi E{};
  E.err = t->err;
  // H1 = relu(X W1^T + b1)
  E.bias = P + OFF_B1;
  E.out = t->H1;
  E.ldo = MLP_H;
  E.outT = t->H1T;
  E.ldt = B;
  if ((rc = launch_mma<128, EPI_RELU>(t->Xb, t->C.W1p, B, MLP_H, 64, 64, 64, 64, E, s)) != CR_OK) return rc;
  // H2 = relu(H1 W2^T + b2)
  E.bias = P + OFF_B2;
  E.out = t->H2;
  E.outT = t->H2T;
  if ((rc = launch_mma<128, EPI_RELU>(t->H1, t->C.W2, B, MLP_H, MLP_H, MLP_H, MLP_H, MLP_H, E, s)) != CR_OK) return rc;
  // H3 = relu(H2 W3^T + b3), then the output layer, the loss and G3 = dL/dz3
  GemmEpi H{};
  H.err = t->err;
  H.bias = P + OFF_B3;
  H.out = t->H3;
  H.ldo = MLP_H;
  H.w4 = t->C.w4;
  H.b4 = P + OFF_B4;
  H.target = t->tc;
  H.inv_batch = 1.0f / (float)B;
  H.g3 = t->G3;
  H.g3T = t->G3T;
  H.ldt3 = B;
  H.gb3 = G + OFF_B3;
  H.gw4 = G + OFF_W4;
  H.gb4 = G + OFF_B4;
  H.loss = t->loss;
  if ((rc = launch_mma<128, EPI_HEAD>(t->H2, t->C.W3, B, MLP_H, MLP_H, MLP_H, MLP_H, MLP_H, H, s)) != CR_OK) return rc;
  // weight gradients: K = batch split over about one wave of CTAs, each split
  // storing its slice, the slices summed in split order
  const int ks = split_for(B, 1);
  const int splits = (B + ks - 1) / ks;
  if (splits > t->max_splits) return CR_ERR_INVALID_ARG;
  GemmEpi A{};
  A.err = t->err;
  A.outF = t->part;
  auto sum_into = [&](float *dst, int count) {
    k_sum_splits<<<(count + 255) / 256, 256, 0, s>>>(t->part, splits, count, dst);
    return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
  };
  // gW3 = G3^T H2
  A.ldf = MLP_H;
  if ((rc = launch_mma<128, EPI_PARTIAL>(t->G3T, t->H2T, MLP_H, MLP_H, B, B, B, ks, A, s)) != CR_OK) return rc;
  if ((rc = sum_into(G + OFF_W3, MLP_H * MLP_H)) != CR_OK) return rc;
  // G2 = (G3 W3) * [H2 > 0]; gb2
  GemmEpi Mk{};
  Mk.err = t->err;
  Mk.mask = t->H2;
  Mk.ldm = MLP_H;
  Mk.out = t->G2;
  Mk.ldo = MLP_H;
  Mk.outT = t->G2T;
  Mk.ldt = B;
  Mk.colsum = G + OFF_B2;
  if ((rc = launch_mma<128, EPI_MASK>(t->G3, t->C.W3T, B, MLP_H, MLP_H, MLP_H, MLP_H, MLP_H, Mk, s)) != CR_OK) return rc;
  // gW2 = G2^T H1
  if ((rc = launch_mma<128, EPI_PARTIAL>(t->G2T, t->H1T, MLP_H, MLP_H, B, B, B, ks, A, s)) != CR_OK) return rc;
  if ((rc = sum_into(G + OFF_W2, MLP_H * MLP_H)) != CR_OK) return rc;
  // G1 = (G2 W2) * [H1 > 0] (transposed only); gb1
  Mk.mask = t->H1;
  Mk.out = nullptr;
  Mk.outT = t->G1T;
  Mk.colsum = G + OFF_B1;
  if ((rc = launch_mma<128, EPI_MASK>(t->G2, t->C.W2T, B, MLP_H, MLP_H, MLP_H, MLP_H, MLP_H, Mk, s)) != CR_OK) return rc;
  // gW1 = G1^T X
  A.ldf = MLP_IN;
  if ((rc = launch_mma<48, EPI_PARTIAL>(t->G1T, t->XbT, MLP_H, MLP_IN, B, B, B, ks, A, s)) != CR_OK) return rc;
  if ((rc = sum_into(G + OFF_W1, MLP_H * MLP_IN)) != CR_OK) return rc;
  t->launches += 3;
  t->launches += 8;
  return CR_OK;
}

static int train_check(cr_trainer *t) {
  int e = 0;
  if (cudaMemcpyAsync(&e, t->err, sizeof(int), cudaMemcpyDeviceToHost, t->stream) != cudaSuccess ||
      cudaStreamSynchronize(t->stream) != cudaSuccess)
    return CR_ERR_CUDA;
  return (e & ERRB_TIMEOUT) ? CR_ERR_TIMEOUT : CR_OK;
}

extern "C" int cr_train_gradients(cr_trainer *t, const float *X, const float *target, int32_t batch, float *grads,
                                  float *loss) {
  int rc = train_grads(t, X, target, batch);
  if (rc != CR_OK) return rc;
  if (grads && cudaMemcpyAsync(grads, t->G, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
    return CR_ERR_CUDA;
  if (loss && cudaMemcpyAsync(loss, t->loss, sizeof(float), cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
    return CR_ERR_CUDA;
  return train_check(t);
}

// Adam on the masters from the gradients in t->G, then the BF16 copies
static int adam_update(cr_trainer *t) {
  t->step++;
  const double c1 = 1.0 - std::pow(t->beta1, (double)t->step), c2 = 1.0 - std::pow(t->beta2, (double)t->step);
  k_adam<<<(N_PARAMS + 255) / 256, 256, 0, t->stream>>>(t->P, t->G, t->Mm, t->Vv, N_PARAMS, (float)t->lr,
                                                         (float)t->beta1, (float)t->beta2, (float)t->eps, (float)c1,
                                                         (float)c2);
  k_weights_bf16<<<(MLP_H * MLP_H + 255) / 256, 256, 0, t->stream>>>(t->P, t->C);
  t->launches += 2;
  return cudaGetLastError() == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

extern "C" int cr_train_step(cr_trainer *t, const float *X, const float *target, int32_t batch, float *loss) {
  int rc;
  if (t && !t->unfused) {  // the fused step, then the partials' sum, Adam and the BF16 copies in one launch
    if (!X || !target || batch <= 0 || batch % 128 || batch > t->max_batch) return CR_ERR_INVALID_ARG;
    if ((rc = train_fused_kernel(t, X, target, batch)) != CR_OK) return rc;
    t->step++;
    const double c1 = 1.0 - std::pow(t->beta1, (double)t->step), c2 = 1.0 - std::pow(t->beta2, (double)t->step);
    k_sum_adam<<<(N_PARAMS + 1 + SUM_PAR - 1) / SUM_PAR, SUM_THREADS, 0, t->stream>>>(
        t->part_f, fused_grid(batch, t->sms), t->G, t->P, t->Mm, t->Vv, (float)t->lr, (float)t->beta1,
        (float)t->beta2, (float)t->eps, (float)c1, (float)c2, t->C);
    t->launches++;
    if (cudaGetLastError() != cudaSuccess) return CR_ERR_CUDA;
  } else {
    if ((rc = train_grads(t, X, target, batch)) != CR_OK) return rc;
    if ((rc = adam_update(t)) != CR_OK) return rc;
  }
  if (loss) {
    if (cudaMemcpyAsync(loss, t->loss, sizeof(float), cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
      return CR_ERR_CUDA;
    return train_check(t);
  }
  return CR_OK;
}

extern "C" int cr_train_apply(cr_trainer *t, const float *grads) {
  if (!t || !grads) return CR_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(t->G, grads, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice, t->stream) != cudaSuccess)
    return CR_ERR_CUDA;
  const int rc = adam_update(t);
  if (rc != CR_OK) return rc;
  return cudaStreamSynchronize(t->stream) == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

extern "C" int cr_train_moments(cr_trainer *t, float *m, float *v) {
  if (!t) return CR_ERR_INVALID_ARG;
  if (m && cudaMemcpyAsync(m, t->Mm, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
    return CR_ERR_CUDA;
  if (v && cudaMemcpyAsync(v, t->Vv, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
    return CR_ERR_CUDA;
  return cudaStreamSynchronize(t->stream) == cudaSuccess ? CR_OK : CR_ERR_CUDA;
}

extern "C" int cr_train_get(cr_trainer *t, float *params, uint16_t *W1, float *b1, uint16_t *W2, float *b2,
                            uint16_t *W3, float *b3, uint16_t *w4, float *b4) {
  if (!t) return CR_ERR_INVALID_ARG;
  std::vector<float> h(N_PARAMS);
  if (cudaMemcpyAsync(h.data(), t->P, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, t->stream) != cudaSuccess ||
      cudaStreamSynchronize(t->stream) != cudaSuccess)
    return CR_ERR_CUDA;
  if (params) std::memcpy(params, h.data(), sizeof(float) * N_PARAMS);
  auto tb = [](float f) {  // round to nearest even BF16
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
  };
  for (int i = 0; i < MLP_H * MLP_IN; ++i)
    if (W1) W1[i] = tb(h[OFF_W1 + i]);
  for (int i = 0; i < MLP_H * MLP_H; ++i) {
    if (W2) W2[i] = tb(h[OFF_W2 + i]);
    if (W3) W3[i] = tb(h[OFF_W3 + i]);
  }
  for (int i = 0; i < MLP_H; ++i) {
    if (b1) b1[i] = h[OFF_B1 + i];
    if (b2) b2[i] = h[OFF_B2 + i];
    if (b3) b3[i] = h[OFF_B3 + i];
    if (w4) w4[i] = tb(h[OFF_W4 + i]);
  }
  if (b4) *b4 = h[OFF_B4];
  return CR_OK;
}

extern "C" int cr_train_stats(const cr_trainer *t, int64_t *steps, int64_t *launches) {
  if (!t) return CR_ERR_INVALID_ARG;
  if (steps) *steps = t->step;
  if (launches) *launches = t->launches;
  return CR_OK;
}

// error word of the exposed products (cr_mma_bf16, cr_selftest_mma_timeout)
static int *mma_err_word() {
  static int *d_err = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!d_err) {
    if (cudaMalloc((void **)&d_err, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(d_err, 0, sizeof(int)) != cudaSuccess) {
      cudaFree(d_err);
      d_err = nullptr;
    }
  }
  return d_err;
}

// read and clear the error word after a product: CR_ERR_TIMEOUT when a
// bounded wait ran out
static int mma_status(int *d_err, cudaStream_t s) {
  int e = 0;
  if (cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CR_ERR_CUDA;
  if (e) {
    if (cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return CR_ERR_CUDA;
    return CR_ERR_TIMEOUT;
  }
  return CR_OK;
}

extern "C" int cr_selftest_mma_timeout(const uint16_t *A, const uint16_t *B, float *D, uint32_t polls, void *stream) {
  if (!A || !B || !D || polls == 0) return CR_ERR_INVALID_ARG;
  if (get_encode() != CR_OK) return CR_ERR_CUDA;
  int *d_err = mma_err_word();
  if (!d_err) return CR_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  GemmEpi E{};
  E.err = d_err;
  E.outF = D;
  E.ldf = 128;
  E.spin = polls;
  E.withhold_first = 1;
  // one 128 x 128 tile, K = 64: a single slice, the one withheld
  const int rc = launch_mma<128, EPI_STORE>(A, B, 128, 128, 64, 64, 64, 64, E, s);
  if (rc != CR_OK) return rc;
  return mma_status(d_err, s);
}

extern "C" int cr_mma_bf16(const uint16_t *A, const uint16_t *B, float *D, int32_t M, int32_t N, int32_t K,
                           int32_t accumulate, void *stream) {
  if (!A || !B || !D || M <= 0 || K <= 0 || K % 8 || !(N == 48 || N == 128)) return CR_ERR_INVALID_ARG;
  if (get_encode() != CR_OK) return CR_ERR_CUDA;
  int *d_err = mma_err_word();
  if (!d_err) return CR_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  GemmEpi E{};
  E.err = d_err;
  E.outF = D;
  E.ldf = N;
  const int tiles = (M + GM - 1) / GM;
  const int ks = accumulate ? split_for(K, tiles) : ((K + GK - 1) / GK) * GK;
  int rc = N == 48 ? (accumulate ? launch_mma<48, EPI_ATOMIC>(A, B, M, N, K, K, K, ks, E, s)
                                 : launch_mma<48, EPI_STORE>(A, B, M, N, K, K, K, ks, E, s))
                   : (accumulate ? launch_mma<128, EPI_ATOMIC>(A, B, M, N, K, K, K, ks, E, s)
                                 : launch_mma<128, EPI_STORE>(A, B, M, N, K, K, K, ks, E, s));
  if (rc != CR_OK) return rc;
  return mma_status(d_err, s);
}
