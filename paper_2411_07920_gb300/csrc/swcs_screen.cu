// Per-operator features for the screening network and top-k selection of
// its predictions (ADAPT step 4 over the generalized singles and doubles
// pool, Sec. II.C: only the selected operators' gradients are then formed).
//
// Features of operator k (tau_k removes (p,q) and adds (r,s); singles p -> r),
// all independent of the system size; L(x) = log10(|x| + 1e-12) / 4:
//   0 double?  1-4 indices / n_so  5-8 h_pp, h_qq, h_rr, h_ss  9 orbital-energy gap
//   10 L(<rs||pq>) (singles: Fock_rp on the reference)  11 L(v / max(|gap|, 0.1))
//   12 occupied-in-reference count of (p,q) / 2   13 of (r,s) / 2
//   14 L(c_ref)   15 L(c(tau_k ref))   16 L(c(tau_k^dag ref))
//   17 opposite-spin pair?  18 same-spin double?  19 1/(1+|gap|)  20 L(2 c_ref v)
//   21 L(n_p n_q (1-n_r)(1-n_s)): weight of determinants tau_k acts on, from the
//      state's orbital occupations n_p = <psi|a+_p a_p|psi>/<psi|psi>
//   22 n_e/n_so  23 n_so/64  24 L(n_r n_s (1-n_p)(1-n_q))  25-28 n_p, n_q, n_r, n_s
//   29 L(v (w_up + w_dn))  30-31 zero
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

namespace {

__device__ __forceinline__ float lg(double v) { return (float)(0.25 * log10(fabs(v) + 1e-12)); }

__device__ __forceinline__ double amp_of(const StateDev& S, uint64_t key) {
  const int64_t j = idx_lookup(S.tab, S.tab_mask, key);
  return j >= 0 ? S.amps[j] : 0.0;
}

// occ[p] += sum_D c_D^2 [p in D]
__global__ void occupation_kernel(StateDev S, double* occ) {
  __shared__ double acc[64];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) acc[t] = 0.0;
  __syncthreads();
  const long long n = *S.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    uint64_t d = S.keys[i];
    const double w = S.amps[i] * S.amps[i];
    while (d) {
      const int p = __ffsll((long long)d) - 1;
      d &= d - 1;
      atomicAdd(&acc[p], w);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 64; t += blockDim.x)
    if (acc[t] != 0.0) atomicAdd(&occ[t], acc[t]);
}

__global__ void features_kernel(HamDev H, StateDev S, const uint8_t* pool_ops, int64_t n_pool, const double* occ,
                                __nv_bfloat16* x) {
  __shared__ double nocc[64];
  const int n = H.n;
  double tot = 0.0;
  for (int t = 0; t < n; ++t) tot += occ[t];
  const double n2 = tot / H.ne;
  for (int t = threadIdx.x; t < 64; t += blockDim.x) nocc[t] = t < n ? occ[t] / n2 : 0.0;
  __syncthreads();
  const uint64_t ref = (H.ne >= 64) ? ~0ull : ((1ull << H.ne) - 1ull);
  const double c_ref = amp_of(S, ref);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pool; k += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* o = pool_ops + 5 * k;
    const bool dbl = o[0] == 2;
    const int p = o[1], q = dbl ? o[2] : o[1], r = dbl ? o[3] : o[2], s = dbl ? o[4] : o[2];
    float f[kFeatures];
#pragma unroll
    for (int i = 0; i < kFeatures; ++i) f[i] = 0.f;
    const double ep = H.h[p * n + p], eq = dbl ? H.h[q * n + q] : 0.0;
    const double er = H.h[r * n + r], es = dbl ? H.h[s * n + s] : 0.0;
    const double gap = dbl ? (er + es - ep - eq) : (er - ep);
    double v;
    if (dbl) {
      v = H.G[(size_t)pair_index(p, q, n) * H.npairs + pair_index(r, s, n)];
    } else {  // Fock element on the reference: h_rp + sum_{j in ref} <rj||pj>
      v = H.h[r * n + p];
      for (int j = 0; j < H.ne; ++j) v += H.Ws[((size_t)p * n + r) * n + j];
    }
    const int occ_lo = (p < H.ne) + (dbl && q < H.ne), occ_hi = (r < H.ne) + (dbl && s < H.ne);
    GateOp op = decode_op(o);
    uint64_t partner = 0;
    int sb = 0;
    double c_up = 0.0, c_dn = 0.0;
    const int role = gate_role(op, ref, &partner, &sb);
    if (role > 0) c_up = amp_of(S, partner);
    if (role < 0) c_dn = amp_of(S, partner);
    f[0] = dbl ? 1.f : 0.f;
    f[1] = (float)p / n;
    f[2] = (float)q / n;
    f[3] = (float)r / n;
    f[4] = (float)s / n;
    f[5] = (float)ep;
    f[6] = (float)eq;
    f[7] = (float)er;
    f[8] = (float)es;
    f[9] = (float)gap;
    const double np_ = nocc[p], nq = dbl ? nocc[q] : 1.0, nr = nocc[r], ns = dbl ? nocc[s] : 0.0;
    const double w_up = np_ * nq * (1.0 - nr) * (1.0 - ns), w_dn = nr * (dbl ? ns : 1.0) * (1.0 - np_) * (dbl ? 1.0 - nq : 1.0);
    f[10] = lg(v);
    f[11] = lg(fabs(v) / fmax(fabs(gap), 0.1));
    f[12] = 0.5f * occ_lo;
    f[13] = 0.5f * occ_hi;
    f[14] = lg(c_ref);
    f[15] = lg(c_up);
    f[16] = lg(c_dn);
    f[17] = (dbl && ((p & 1) != (q & 1))) ? 1.f : 0.f;
    f[18] = (dbl && ((p & 1) == (q & 1))) ? 1.f : 0.f;
    f[19] = (float)(1.0 / (1.0 + fabs(gap)));
    f[20] = lg(2.0 * c_ref * v);
    f[21] = lg(w_up);
    f[24] = lg(w_dn);
    f[25] = (float)np_;
    f[26] = (float)(dbl ? nq : np_);
    f[27] = (float)nr;
    f[28] = (float)(dbl ? ns : nr);
    f[29] = lg(fabs(v) * (w_up + w_dn));
    f[22] = (float)H.ne / n;
    f[23] = (float)n / 64.f;
    __nv_bfloat16* row = x + (size_t)k * kFeatures;
#pragma unroll
    for (int i = 0; i < kFeatures; ++i) row[i] = __float2bfloat16_rn(f[i]);
  }
}

__device__ __forceinline__ uint32_t order_key(float y) {
  const uint32_t u = __float_as_uint(y);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // monotone in y
}

// ctl: [0] bucket of the high half, [1] rank still needed inside it, [2] threshold key,
// [3] count strictly above the threshold still needed at the threshold, [4] output counter
__global__ void topk_hist_hi(const float* y, int64_t n, unsigned* hist) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[order_key(y[i]) >> 16], 1u);
}

__global__ void topk_pick_hi(const unsigned* hist, int64_t k, unsigned long long* ctl) {
  if (threadIdx.x || blockIdx.x) return;
  long long cum = 0;
  for (int b = 65535; b >= 0; --b) {
    if (cum + hist[b] >= k) {
      ctl[0] = (unsigned long long)b;
      ctl[1] = (unsigned long long)(k - cum);
      return;
    }
    cum += hist[b];
  }
  ctl[0] = 0;
  ctl[1] = 0;
}

__global__ void topk_hist_lo(const float* y, int64_t n, const unsigned long long* ctl, unsigned* hist) {
  const uint32_t hi = (uint32_t)ctl[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = order_key(y[i]);
    if ((key >> 16) == hi) atomicAdd(&hist[65536 + (key & 0xFFFFu)], 1u);
  }
}

__global__ void topk_pick_lo(const unsigned* hist, unsigned long long* ctl) {
  if (threadIdx.x || blockIdx.x) return;
  const long long need = (long long)ctl[1];
  long long cum = 0;
  for (int b = 65535; b >= 0; --b) {
    const long long h = hist[65536 + b];
    if (cum + h >= need) {
      ctl[2] = (ctl[0] << 16) | (unsigned long long)b;
      ctl[3] = (unsigned long long)(need - cum);  // how many of the threshold-equal keys to admit
      ctl[4] = 0;
      return;
    }
    cum += h;
  }
  ctl[2] = 0;
  ctl[3] = 0;
  ctl[4] = 0;
}

__global__ void topk_compact(const float* y, int64_t n, unsigned long long* ctl, int64_t* out) {
  const uint32_t thr = (uint32_t)ctl[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = order_key(y[i]);
    bool take = key > thr;
    if (key == thr) take = atomicAdd(&ctl[5], 1ull) < ctl[3];
    if (take) out[atomicAdd(&ctl[4], 1ull)] = i;
  }
}

__global__ void subset_bits_kernel(const int64_t* subset, int64_t n, uint32_t* bits, int64_t n_pool) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = subset[i];
    if (k >= 0 && k < n_pool) atomicOr(&bits[k >> 5], 1u << (k & 31));
  }
}

__global__ void log_abs_kernel(const double* g, int64_t n, float* t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    t[i] = (float)fmax(log10(fabs(g[i]) + 1e-12), -10.0);
}

}  // namespace

cudaError_t launch_pool_features(const HamDev& H, const StateDev& S, const uint8_t* pool_ops, int64_t n_pool,
                                 double* occ, __nv_bfloat16* x, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(occ, 0, 64 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  occupation_kernel<<<304, 256, 0, st>>>(S, occ);
  features_kernel<<<(int)((n_pool + 255) / 256), 256, 0, st>>>(H, S, pool_ops, n_pool, occ, x);
  return cudaGetLastError();
}

cudaError_t launch_topk(const float* y, int64_t n, int64_t k, unsigned* hist, unsigned long long* ctl,
                        int64_t* out_idx, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(hist, 0, 2 * 65536 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, 8 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1216);
  topk_hist_hi<<<nb, 256, 0, st>>>(y, n, hist);
  topk_pick_hi<<<1, 32, 0, st>>>(hist, k, ctl);
  topk_hist_lo<<<nb, 256, 0, st>>>(y, n, ctl, hist);
  topk_pick_lo<<<1, 32, 0, st>>>(hist, ctl);
  topk_compact<<<nb, 256, 0, st>>>(y, n, ctl, out_idx);
  return cudaGetLastError();
}

cudaError_t launch_subset_bits(const int64_t* subset, int64_t n, uint32_t* bits, int64_t n_pool, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bits, 0, ((n_pool + 31) / 32) * 4, st);
  if (e != cudaSuccess) return e;
  if (n > 0) subset_bits_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, st>>>(subset, n, bits, n_pool);
  return cudaGetLastError();
}

cudaError_t launch_log_abs(const double* g, int64_t n, float* t, cudaStream_t st) {
  log_abs_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, st>>>(g, n, t);
  return cudaGetLastError();
}

}  // namespace swcs
