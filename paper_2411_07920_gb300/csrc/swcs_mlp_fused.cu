// Screening network, inference: the whole forward pass y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 of
// every pool operator in one persistent kernel on the 5th-generation tensor cores.
//
//   - one CTA per SM (576 threads, about 226 KB of shared memory), looping over 128-row tiles;
//   - the weights W1 [W x D] and W2 [W x W] are loaded once per CTA by TMA and stay in shared memory;
//     feature tiles X [128 x D] stream in by TMA through two stages;
//   - warp 0 (one thread) issues the TMA loads, warp 1 (one thread) the tcgen05.mma, warps 2-17 run the
//     epilogues: four warps per group of columns, one per tensor-memory lane quadrant, so every SM
//     sub-partition has four epilogue warps to hide tensor-memory and shared-memory latency; all hand-offs
//     go through mbarriers with bounded waits;
//   - layer 1 accumulates X W1^T into tensor memory columns [0, W), its epilogue writes
//     H1 = bf16(relu(. + b1)) straight into shared memory in the operand layout of layer 2, and layer 2
//     accumulates H1 W2^T into columns [256, 256 + W); the second epilogue applies b2, ReLU, BF16 and the
//     w3 dot product.  H1 and H2 never leave the SM: HBM sees X (64 B per row) and y (4 B per row).
//   - while the epilogue of layer 2 reads tile t, the tensor cores already run layer 1 of tile t + 1.
//
// Operand layout (K-major, no swizzle): core matrices of 8 rows x 16 bytes; one TMA box of 8 K-elements x
// R rows fills R x 16 contiguous bytes, so K-adjacent core matrices are R x 16 bytes apart (leading byte
// offset) and row-adjacent ones 128 bytes (stride byte offset).  Arithmetic, rounding and summation order
// are those of the layer-by-layer kernels (mlp_gemm_kernel), so y is bit-identical to their result.
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

namespace {

constexpr int kEpiThreads = 128 * kDotGroups;  // warps 2 .. 2 + 4 kDotGroups - 1
constexpr int kFusedThreads = 64 + kEpiThreads;
constexpr int kCtrlBytes = 256;                 // control block, then the dot-product partials
constexpr int kTile = 128;
constexpr uint32_t kT2Col = 256;  // tensor-memory column of the layer-2 accumulator
constexpr uint64_t kSpinLimit = 1ull << 26;

struct FusedCtrl {
  uint64_t full_x[2], empty_x[2], w_full, mma1, mma2, t1_free, h1_ready, t2_free, part_ready, fin;
  uint32_t tmem;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // tcgen05 descriptor version; base offset 0, no swizzle
  return d;
}

__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
  // D = F32 (bit 4), A = B = BF16 (bits 7, 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

// Bounded wait for the phase of the given parity; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity) {
  const uint32_t a = saddr(b);
  for (uint64_t i = 0; i < kSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 63) == 63) __nanosleep(32);
  }
  return false;
}

// 2-D tile load: box origin (x = K element, y = row) into shared memory, completion on mbar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(saddr(mbar))
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(b))
               : "memory");
}

__device__ __forceinline__ void tmem_load16(uint32_t taddr, float* v) {
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

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

}  // namespace

size_t mlp_fused_smem_bytes(int d_in, int width) {
  return 128 /* alignment slack */ + kCtrlBytes + (size_t)kDotGroups * kTile * 4 /* partials */ +
         (size_t)width * d_in * 2 + (size_t)width * width * 2 +
         2 * (size_t)kTile * d_in * 2 + (size_t)kTile * width * 2;
}

__global__ void __launch_bounds__(kFusedThreads, 1)
mlp_fused_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_w1,
                 const __grid_constant__ CUtensorMap tm_w2, FusedArgs f) {
  extern __shared__ uint8_t dsm[];
  const uint32_t pad = (128u - (saddr(dsm) & 127u)) & 127u;
  uint8_t* sm = dsm + pad;
  FusedCtrl& c = *reinterpret_cast<FusedCtrl*>(sm);
  const int D = f.d_in, W = f.width;
  float* sPart = reinterpret_cast<float*>(sm + kCtrlBytes);  // [kDotGroups][kTile]
  uint8_t* sW1 = sm + kCtrlBytes + kDotGroups * kTile * 4;
  uint8_t* sW2 = sW1 + (size_t)W * D * 2;
  uint8_t* sX0 = sW2 + (size_t)W * W * 2;
  uint8_t* sX1 = sX0 + (size_t)kTile * D * 2;
  uint8_t* sH1 = sX1 + (size_t)kTile * D * 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (int)((f.M + kTile - 1) / kTile);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(saddr(&c.tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&c.full_x[s], 1);
      mbar_init(&c.empty_x[s], 1);
    }
    mbar_init(&c.w_full, 1);
    mbar_init(&c.mma1, 1);
    mbar_init(&c.mma2, 1);
    mbar_init(&c.t1_free, kEpiThreads);
    mbar_init(&c.h1_ready, kEpiThreads);
    mbar_init(&c.t2_free, kEpiThreads);
    mbar_init(&c.part_ready, kEpiThreads);
    mbar_init(&c.fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = c.tmem;
  const uint32_t idesc = idesc_f16(kTile, W);
  bool bad = false;

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------------ TMA producer
      mbar_expect_tx(&c.w_full, (uint32_t)(W * D * 2 + W * W * 2));
      for (int g = 0; g < D / 8; ++g) tma_load_2d(sW1 + (size_t)g * W * 16, &tm_w1, 8 * g, 0, &c.w_full);
      for (int g = 0; g < W / 8; ++g) tma_load_2d(sW2 + (size_t)g * W * 16, &tm_w2, 8 * g, 0, &c.w_full);
      bool issued0 = false, issued1 = false;
      uint32_t last0 = 0, last1 = 0;
      int j = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
        const int s = j & 1;
        const uint32_t par = (uint32_t)(j >> 1) & 1u;
        if (!mbar_wait_bounded(&c.empty_x[s], par ^ 1u)) {
          bad = true;
          break;
        }
        uint8_t* dst = s ? sX1 : sX0;
        mbar_expect_tx(&c.full_x[s], (uint32_t)(kTile * D * 2));
        for (int g = 0; g < D / 8; ++g) tma_load_2d(dst + g * (kTile * 16), &tm_x, 8 * g, t * kTile, &c.full_x[s]);
        if (s) { issued1 = true; last1 = par; } else { issued0 = true; last0 = par; }
      }
      // no copy may still be landing when the CTA leaves (returns at once when already consumed)
      if (issued0 && !mbar_wait_bounded(&c.full_x[0], last0)) bad = true;
      if (issued1 && !mbar_wait_bounded(&c.full_x[1], last1)) bad = true;
      if (!mbar_wait_bounded(&c.w_full, 0)) bad = true;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------------ MMA issuer
      if (!mbar_wait_bounded(&c.w_full, 0)) bad = true;
      int j = 0;
      for (int t = blockIdx.x; t < ntiles && !bad; t += gridDim.x, ++j) {
        const int s = j & 1;
        const uint8_t* sx = s ? sX1 : sX0;
        if (!mbar_wait_bounded(&c.full_x[s], (uint32_t)(j >> 1) & 1u)) { bad = true; break; }
        if (j > 0 && !mbar_wait_bounded(&c.t1_free, (uint32_t)(j - 1) & 1u)) { bad = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int k = 0; k < D / 16; ++k)
          mma_f16(tmem, desc_kmajor(saddr(sx) + k * 2 * (kTile * 16), kTile * 16, 128),
                  desc_kmajor(saddr(sW1) + k * 2 * (W * 16), W * 16, 128), idesc, k > 0 ? 1u : 0u);
        mma_commit(&c.empty_x[s]);
        mma_commit(&c.mma1);
        if (!mbar_wait_bounded(&c.h1_ready, (uint32_t)j & 1u)) { bad = true; break; }
        if (j > 0 && !mbar_wait_bounded(&c.t2_free, (uint32_t)(j - 1) & 1u)) { bad = true; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int k = 0; k < W / 16; ++k)
          mma_f16(tmem + kT2Col, desc_kmajor(saddr(sH1) + k * 2 * (kTile * 16), kTile * 16, 128),
                  desc_kmajor(saddr(sW2) + k * 2 * (W * 16), W * 16, 128), idesc, k > 0 ? 1u : 0u);
        mma_commit(&c.mma2);
      }
      mma_commit(&c.fin);  // every MMA issued above has completed once this phase completes
      if (!mbar_wait_bounded(&c.fin, 0)) bad = true;
    }
  } else {  // ------------------------------------------------------------ epilogue, warps 2-17
    const int q = warp & 3;            // a warp reads the tensor-memory lanes 32 (warp % 4) .. + 31
    const int grp = (warp - 2) >> 2;   // its group of 16-column chunks
    const int r = q * 32 + lane;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    const int cb = dot_group_begin(grp, W / 16) * 16, ce = dot_group_begin(grp + 1, W / 16) * 16;
    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      if (!mbar_wait_bounded(&c.mma1, (uint32_t)j & 1u)) { bad = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int c0 = cb; c0 < ce; c0 += 16) {
        float v[16];
        tmem_load16(tmem + lanes + (uint32_t)c0, v);
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float z0 = v[2 * i] + __ldg(&f.b1[c0 + 2 * i]);
          float z1 = v[2 * i + 1] + __ldg(&f.b1[c0 + 2 * i + 1]);
          z0 = z0 > 0.f ? z0 : 0.f;
          z1 = z1 > 0.f ? z1 : 0.f;
          w[i] = pack_bf16x2(__float2bfloat16_rn(z0), __float2bfloat16_rn(z1));
        }
        // row r, K groups c0/8 and c0/8 + 1: 16 bytes each in the layer-2 operand layout
        *reinterpret_cast<uint4*>(sH1 + (size_t)(c0 / 8) * (kTile * 16) + r * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(sH1 + (size_t)(c0 / 8 + 1) * (kTile * 16) + r * 16) =
            make_uint4(w[4], w[5], w[6], w[7]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&c.t1_free);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // H1 visible to the tensor cores
      mbar_arrive(&c.h1_ready);
      if (!mbar_wait_bounded(&c.mma2, (uint32_t)j & 1u)) { bad = true; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float part = 0.f;
      for (int c0 = cb; c0 < ce; c0 += 16) {
        float v[16];
        tmem_load16(tmem + lanes + kT2Col + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float z = v[i] + __ldg(&f.b2[c0 + i]);
          z = z > 0.f ? z : 0.f;
          const __nv_bfloat16 hb = __float2bfloat16_rn(z);
          part += __bfloat162float(hb) * __bfloat162float(f.w3[c0 + i]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&c.t2_free);
      // partials of the row meet in shared memory; group 0 adds them in group order.  Group 0 reads
      // them before it arrives on h1_ready of the next tile, so no group can overwrite them earlier.
      sPart[grp * kTile + r] = part;
      mbar_arrive(&c.part_ready);
      if (grp == 0) {
        if (!mbar_wait_bounded(&c.part_ready, (uint32_t)j & 1u)) { bad = true; break; }
        float dot = sPart[r];
#pragma unroll
        for (int gg = 1; gg < kDotGroups; ++gg) dot += sPart[gg * kTile + r];
        const int64_t row = (int64_t)t * kTile + r;
        if (row < f.M) f.y[row] = dot + __ldg(f.b3);
      }
    }
  }
  if (bad && f.err) set_error(f.err, kDevTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

cudaError_t launch_mlp_fused(const CUtensorMap& tm_x, const CUtensorMap& tm_w1, const CUtensorMap& tm_w2,
                             const FusedArgs& f, int nblocks, cudaStream_t st) {
  const size_t smem = mlp_fused_smem_bytes(f.d_in, f.width);
  static size_t attr = 0;
  if (attr < smem) {
    const cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  mlp_fused_kernel<<<nblocks, kFusedThreads, smem, st>>>(tm_x, tm_w1, tm_w2, f);
  return cudaGetLastError();
}

}  // namespace swcs
