// Screening network: a 3-layer MLP (BF16 weights, FP32 accumulation) that
// predicts log10|g_k| of every pool operator from per-operator features, so
// that only the predicted top fraction of the pool is evaluated exactly.
//
// Training and the layer-by-layer forward (which keeps the activations for the
// backward pass) run their dense contractions on the 5th-generation tensor
// cores through one kernel, C[M x N] = A[M x K] . B[N x K]^T with A, B BF16
// and K contiguous (inference over the pool uses the fused kernel of
// swcs_mlp_fused.cu instead):
//   - a CTA of 128 threads owns a 128-row tile and all N <= 256 columns;
//   - K is consumed in chunks of 32: the CTA copies the A and B chunks into
//     shared memory in the canonical no-swizzle K-major layout (8x16-byte core
//     matrices; leading byte offset 128 B between K-adjacent core matrices,
//     stride byte offset 512 B between 8-row groups), then one thread issues
//     two tcgen05.mma (K = 16 each) into an FP32 accumulator in tensor memory
//     and commits them to an mbarrier that the CTA waits on (bounded);
//   - the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31, thread t owns row t) and applies bias, ReLU, BF16
//     rounding, the final 256-wide dot product, or plain FP32 output.
// Forward: H1 = bf16(relu(X W1^T + b1)), H2 = bf16(relu(H1 W2^T + b2)),
// y = H2 . w3 + b3.  Backward (mean squared error): dZ2 = bf16(dy w3 (H2>0)),
// dH1 = dZ2 W2 (GEMM with B = W2^T), dZ1 = bf16(dH1 (H1>0)), and the weight
// gradients dW2 = dZ2^T H1, dW1 = dZ1^T X as GEMMs over the batch with
// transposed operands.  Adam updates FP32 master weights and refreshes the
// BF16 copies.
//
// With tensor maps for A and B (every shape the training step uses) the GEMM
// runs pipelined instead (mlp_gemm_tma_kernel): warp 0 (one thread) streams
// K-chunks of A and B into a ring of three shared-memory stages by TMA, warp 1
// (one thread) issues the MMAs of each chunk as soon as it has landed and
// frees the stage with a tcgen05.commit, so copies and MMAs overlap; the
// weight-gradient GEMMs, which have only two 128-row tiles but a long K (the
// batch), also split K over CTAs that add their partial products into the
// zeroed FP32 output.
#include <algorithm>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

namespace {

constexpr int kGemmThreads = 128;
constexpr int kKChunk = 32;
constexpr uint64_t kMbarSpinLimit = 1ull << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle, K-major canonical layout).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (uint64_t i = 0; i < kMbarSpinLimit; ++i) {
    if (mbar_try_wait(addr, parity)) return true;
    if ((i & 63) == 63) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Copies rows [r0, r0+rows) x K-chunk [k0, k0+32) of a K-contiguous BF16
// matrix into the canonical layout: core (r/8, kk/8) at ((r/8)*4 + kk/8)*128 B.
__device__ __forceinline__ void stage_chunk(uint8_t* dst, const __nv_bfloat16* src, int ld, int r0, int rows,
                                            int rows_valid, int k0) {
  for (int seg = threadIdx.x; seg < rows * 4; seg += kGemmThreads) {
    const int r = seg >> 2, kk8 = seg & 3;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r0 + r < rows_valid) v = *reinterpret_cast<const uint4*>(src + (size_t)(r0 + r) * ld + k0 + kk8 * 8);
    *reinterpret_cast<uint4*>(dst + (((r >> 3) * 4 + kk8) * 128) + (r & 7) * 16) = v;
  }
}

__global__ void __launch_bounds__(kGemmThreads) mlp_gemm_kernel(GemmArgs g) {
  __shared__ __align__(128) uint8_t sA[128 * kKChunk * 2];
  __shared__ __align__(128) uint8_t sB[256 * kKChunk * 2];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_holder;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  const int ncols = g.N <= 32 ? 32 : (g.N <= 64 ? 64 : (g.N <= 128 ? 128 : 256));

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_holder;
  const uint32_t idesc = idesc_bf16(128, g.N);
  bool ok = true;
  uint32_t phase = 0;
  const int nchunks = g.K / kKChunk;
  for (int c = 0; c < nchunks && ok; ++c) {
    stage_chunk(sA, g.A, g.lda, m0, 128, g.M, c * kKChunk);
    stage_chunk(sB, g.B, g.ldb, 0, g.N, g.N, c * kKChunk);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int s = 0; s < kKChunk / 16; ++s) {
        const uint64_t da = smem_desc(smem_u32(sA) + s * 256, 128, 512);
        const uint64_t db = smem_desc(smem_u32(sB) + s * 256, 128, 512);
        const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar))
                   : "memory");
    }
    if (!mbar_wait(smem_u32(&mbar), phase)) {
      ok = false;
      if (g.err) set_error(g.err, kDevTimeout);
    }
    phase ^= 1u;
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // ---------------- epilogue: thread t owns row m0 + t (TMEM lane t)
  const int row = m0 + threadIdx.x;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;  // dot-product partial sums (kDotGroups)
  if (ok) {
    for (int c0 = 0; c0 < g.N; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
      int grp = 0;
      while (grp < kDotGroups - 1 && dot_group_begin(grp + 1, g.N / 16) <= c0 / 16) ++grp;
      float part = grp == 0 ? p0 : (grp == 1 ? p1 : (grp == 2 ? p2 : p3));
      if (row < g.M) {
        if (g.mode == kGemmF32) {
          float* o = g.out_f32 + (size_t)row * g.ldo + c0;
#pragma unroll
          for (int i = 0; i < 16; ++i) o[i] = v[i];
        } else {
          __nv_bfloat16* o = g.out_bf16 + (size_t)row * g.ldo + c0;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float z = v[i] + (g.bias ? g.bias[c0 + i] : 0.f);
            z = z > 0.f ? z : 0.f;
            const __nv_bfloat16 hb = __float2bfloat16_rn(z);
            o[i] = hb;
            if (g.mode == kGemmReluBf16Dot) part += __bfloat162float(hb) * __bfloat162float(g.w3[c0 + i]);
          }
        }
      }
      if (grp == 0) p0 = part;
      else if (grp == 1) p1 = part;
      else if (grp == 2) p2 = part;
      else p3 = part;
    }
  }
  if (g.mode == kGemmReluBf16Dot && row < g.M && ok) g.y[row] = (((p0 + p1) + p2) + p3) + g.b3;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------- pipelined GEMM (TMA + tcgen05)
constexpr int kStages = 3;

__device__ __forceinline__ void mbar_init1(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}
// 2-D tile load: box origin (x = K element, y = row) into shared memory, completion on mbar.
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(mbar))
      : "memory");
}

// C = A B^T for one 128-row tile and K-chunks [c0, c1) of kc elements (this CTA's split of K).  Stage s
// holds A as kc/8 column blocks of 128 rows x 16 B (one TMA box each: LBO 2 KB, SBO 128 B) and B as kc/8
// blocks of N x 16 B (LBO N x 16 B, SBO 128 B).
__global__ void __launch_bounds__(kGemmThreads)
mlp_gemm_tma_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b, GemmArgs g,
                    int kc, int splits) {
  extern __shared__ __align__(128) uint8_t dsm[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], fin;
  __shared__ uint32_t tmem_holder;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  const int ncols = g.N <= 32 ? 32 : (g.N <= 64 ? 64 : (g.N <= 128 ? 128 : 256));
  const int nch = g.K / kc, per = (nch + splits - 1) / splits;
  const int c0 = (int)blockIdx.y * per, c1 = min(nch, c0 + per);
  const uint32_t a_bytes = 128u * (uint32_t)kc * 2u, b_bytes = (uint32_t)g.N * (uint32_t)kc * 2u;
  uint8_t* stage[kStages];
#pragma unroll
  for (int s = 0; s < kStages; ++s) stage[s] = dsm + (size_t)s * (a_bytes + b_bytes);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init1(&full[s]);
      mbar_init1(&empty[s]);
    }
    mbar_init1(&fin);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_holder;
  const uint32_t idesc = idesc_bf16(128, g.N);
  bool bad = false;
  if (threadIdx.x == 0) {  // ------------------------------------------------ TMA producer
    bool issued[kStages] = {};
    uint32_t last[kStages] = {};
    for (int c = c0; c < c1; ++c) {
      const int j = c - c0, s = j % kStages;
      const uint32_t par = (uint32_t)(j / kStages) & 1u;
      if (!mbar_wait(smem_u32(&empty[s]), par ^ 1u)) {  // the MMAs that read this stage last have completed
        bad = true;
        break;
      }
      mbar_expect_tx(&full[s], a_bytes + b_bytes);
      for (int q = 0; q < kc / 8; ++q) {
        tma_2d(stage[s] + (size_t)q * 2048, &tm_a, c * kc + 8 * q, m0, &full[s]);
        tma_2d(stage[s] + a_bytes + (size_t)q * g.N * 16, &tm_b, c * kc + 8 * q, 0, &full[s]);
      }
      issued[s] = true;
      last[s] = par;
    }
    // no copy may still be landing when the CTA leaves (returns at once when already consumed)
    for (int s = 0; s < kStages; ++s)
      if (issued[s] && !mbar_wait(smem_u32(&full[s]), last[s])) bad = true;
  } else if (threadIdx.x == 32) {  // ---------------------------------------- MMA issuer
    for (int c = c0; c < c1 && !bad; ++c) {
      const int j = c - c0, s = j % kStages;
      if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(j / kStages) & 1u)) {
        bad = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int k = 0; k < kc / 16; ++k) {
        const uint64_t da = smem_desc(smem_u32(stage[s]) + (uint32_t)k * 2 * 2048, 2048, 128);
        const uint64_t db = smem_desc(smem_u32(stage[s] + a_bytes) + (uint32_t)k * 2 * g.N * 16, (uint32_t)g.N * 16, 128);
        const uint32_t acc = (j > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      mma_commit(&empty[s]);
    }
    mma_commit(&fin);  // every MMA issued above has completed once this phase completes
  }
  __syncwarp();
  if (!mbar_wait(smem_u32(&fin), 0)) bad = true;
  bad = __syncthreads_or(bad) != 0;  // one decision for the whole CTA before the warp-wide tensor-memory loads
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // ---------------- epilogue: thread t owns row m0 + t (TMEM lane t)
  const int row = m0 + threadIdx.x;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;  // dot-product partial sums (kDotGroups)
  const bool empty_split = c0 >= c1;               // no chunk: nothing was accumulated
  if (!bad && !empty_split) {
    for (int cc = 0; cc < g.N; cc += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)cc, v);
      int grp = 0;
      while (grp < kDotGroups - 1 && dot_group_begin(grp + 1, g.N / 16) <= cc / 16) ++grp;
      float part = grp == 0 ? p0 : (grp == 1 ? p1 : (grp == 2 ? p2 : p3));
      if (row < g.M) {
        if (g.mode == kGemmF32) {
          float* o = g.out_f32 + (size_t)row * g.ldo + cc;
          if (splits > 1) {
#pragma unroll
            for (int i = 0; i < 16; ++i) atomicAdd(&o[i], v[i]);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = v[i];
          }
        } else {
          __nv_bfloat16* o = g.out_bf16 + (size_t)row * g.ldo + cc;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float z = v[i] + (g.bias ? g.bias[cc + i] : 0.f);
            z = z > 0.f ? z : 0.f;
            const __nv_bfloat16 hb = __float2bfloat16_rn(z);
            o[i] = hb;
            if (g.mode == kGemmReluBf16Dot) part += __bfloat162float(hb) * __bfloat162float(g.w3[cc + i]);
          }
        }
      }
      if (grp == 0) p0 = part;
      else if (grp == 1) p1 = part;
      else if (grp == 2) p2 = part;
      else p3 = part;
    }
  }
  if (g.mode == kGemmReluBf16Dot && row < g.M && !bad) g.y[row] = (((p0 + p1) + p2) + p3) + g.b3;
  if (bad && g.err) set_error(g.err, kDevTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------- elementwise / reductions
__global__ void mlp_dy_kernel(const float* y, const float* t, int B, float* dy, double* loss) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)B;
    s += (double)d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(loss, s / B);
}

// dZ2 = bf16(dy_i w3_j (H2_ij > 0)),  dw3_j += sum_i dy_i H2_ij,  db3 += sum_i dy_i
__global__ void mlp_dz2_kernel(const float* dy, const __nv_bfloat16* w3, const __nv_bfloat16* H2, int B, int W,
                               __nv_bfloat16* dZ2, float* dw3, float* db3) {
  const int j = threadIdx.x;  // one column per thread (W <= 256)
  if (j >= W) return;
  float a = 0.f, b = 0.f;
  const float wj = __bfloat162float(w3[j]);
  for (int i = blockIdx.x; i < B; i += gridDim.x) {
    const float h = __bfloat162float(H2[(size_t)i * W + j]);
    const float d = dy[i];
    dZ2[(size_t)i * W + j] = __float2bfloat16_rn(h > 0.f ? d * wj : 0.f);
    a += d * h;
    if (j == 0) b += d;
  }
  atomicAdd(&dw3[j], a);
  if (j == 0) atomicAdd(db3, b);
}

// dZ1 = bf16(dH1 (H1 > 0))
__global__ void mlp_dz1_kernel(const float* dH1, const __nv_bfloat16* H1, size_t n, __nv_bfloat16* dZ1) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dZ1[i] = __float2bfloat16_rn(__bfloat162float(H1[i]) > 0.f ? dH1[i] : 0.f);
}

// column sums of a BF16 [B x W] matrix into db (FP32)
__global__ void mlp_colsum_kernel(const __nv_bfloat16* Z, int B, int W, float* db) {
  const int j = threadIdx.x;
  if (j >= W) return;
  float a = 0.f;
  for (int i = blockIdx.x; i < B; i += gridDim.x) a += __bfloat162float(Z[(size_t)i * W + j]);
  atomicAdd(&db[j], a);
}

// out[c][r] = in[r][c] (BF16), rows beyond R are zero up to Rpad
__global__ void mlp_transpose_kernel(const __nv_bfloat16* in, int R, int C, int Rpad, __nv_bfloat16* out) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < C && r < Rpad) out[(size_t)c * Rpad + r] = tile[threadIdx.x][k];
  }
}

// Adam on FP32 master parameters; refreshes the BF16 weight copies.
__global__ void mlp_adam_kernel(MlpParams p, const float* grad, float lr, float b1, float b2, float eps, int step) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n_params; i += gridDim.x * blockDim.x) {
    const float gr = grad[i];
    const float m = b1 * p.m[i] + (1.f - b1) * gr;
    const float v = b2 * p.v[i] + (1.f - b2) * gr * gr;
    p.m[i] = m;
    p.v[i] = v;
    p.master[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// BF16 copies of the weights from the FP32 master: W1b, W2b, W2^T b, w3b.
__global__ void mlp_refresh_kernel(MlpParams p) {
  const int W = p.width, D = p.d_in;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < W * W; i += gridDim.x * blockDim.x) {
    const int o = i / W, k = i % W;
    const __nv_bfloat16 v = __float2bfloat16_rn(p.master[p.off_W2 + i]);
    p.W2b[i] = v;
    p.W2tb[(size_t)k * W + o] = v;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < W * D; i += gridDim.x * blockDim.x)
    p.W1b[i] = __float2bfloat16_rn(p.master[p.off_W1 + i]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < W; i += gridDim.x * blockDim.x)
    p.w3b[i] = __float2bfloat16_rn(p.master[p.off_w3 + i]);
}

}  // namespace

// Each CTA holds up to 256 tensor-memory columns; reserving shared memory
// keeps at most two CTAs per SM so the 512 columns are never oversubscribed.
constexpr int kGemmReserveSmem = 88 * 1024;

cudaError_t launch_mlp_gemm(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N < 16 || g.N > 256 || (g.N & 15) || g.K <= 0 || (g.K % kKChunk) || (g.lda & 7) || (g.ldb & 7))
    return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(mlp_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmReserveSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  mlp_gemm_kernel<<<(g.M + 127) / 128, kGemmThreads, kGemmReserveSmem, st>>>(g);
  return cudaGetLastError();
}

// K-chunk of the pipelined GEMM: 64 where K allows, else 32.
int mlp_gemm_tma_kc(int K) { return K % 64 == 0 ? 64 : 32; }

cudaError_t launch_mlp_gemm_tma(const CUtensorMap& tm_a, const CUtensorMap& tm_b, const GemmArgs& g, int splits,
                                cudaStream_t st) {
  if (g.M <= 0 || g.N < 16 || g.N > 256 || (g.N & 15) || g.K <= 0 || (g.K % kKChunk) || splits < 1 ||
      (splits > 1 && g.mode != kGemmF32))
    return cudaErrorInvalidValue;
  const int kc = mlp_gemm_tma_kc(g.K);
  const size_t stage = (size_t)128 * kc * 2 + (size_t)g.N * kc * 2;
  // at most two CTAs per SM, so their tensor-memory columns (<= 256 each) never oversubscribe the 512
  const size_t smem = std::max((size_t)kStages * stage, (size_t)kGemmReserveSmem);
  static size_t attr = 0;
  if (attr < smem) {
    const cudaError_t e = cudaFuncSetAttribute(mlp_gemm_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  mlp_gemm_tma_kernel<<<dim3((g.M + 127) / 128, splits), kGemmThreads, smem, st>>>(tm_a, tm_b, g, kc, splits);
  return cudaGetLastError();
}

cudaError_t launch_mlp_dy(const float* y, const float* t, int B, float* dy, double* loss, cudaStream_t st) {
  mlp_dy_kernel<<<(B + 255) / 256, 256, 0, st>>>(y, t, B, dy, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_dz2(const float* dy, const __nv_bfloat16* w3, const __nv_bfloat16* H2, int B, int W,
                           __nv_bfloat16* dZ2, float* dw3, float* db3, cudaStream_t st) {
  mlp_dz2_kernel<<<256, W, 0, st>>>(dy, w3, H2, B, W, dZ2, dw3, db3);
  return cudaGetLastError();
}

cudaError_t launch_mlp_dz1(const float* dH1, const __nv_bfloat16* H1, size_t n, __nv_bfloat16* dZ1, cudaStream_t st) {
  mlp_dz1_kernel<<<608, 256, 0, st>>>(dH1, H1, n, dZ1);
  return cudaGetLastError();
}

cudaError_t launch_mlp_colsum(const __nv_bfloat16* Z, int B, int W, float* db, cudaStream_t st) {
  mlp_colsum_kernel<<<256, W, 0, st>>>(Z, B, W, db);
  return cudaGetLastError();
}

cudaError_t launch_mlp_transpose(const __nv_bfloat16* in, int R, int C, int Rpad, __nv_bfloat16* out, cudaStream_t st) {
  dim3 grid((Rpad + 31) / 32, (C + 31) / 32);
  mlp_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, R, C, Rpad, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(const MlpParams& p, const float* grad, float lr, int step, cudaStream_t st) {
  mlp_adam_kernel<<<(p.n_params + 255) / 256, 256, 0, st>>>(p, grad, lr, 0.9f, 0.999f, 1e-8f, step);
  return cudaGetLastError();
}

cudaError_t launch_mlp_refresh(const MlpParams& p, cudaStream_t st) {
  mlp_refresh_kernel<<<256, 256, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace swcs
