// Adjoint of the truncated gate sequence ("analytic gradients", Sec. II.B).
//
// With every truncation held as the fixed projector P_g onto its kept set S_g,
//   psi_{g+1} = P_{g+1} U_g psi_g,  U_g = exp(theta_g A_g),  A_g = tau_g - tau_g^dag,
//   nu_M      = P_M (H - E) psi_M,
//   dE/dtheta_g = 2 <nu_{g+1} | A_g U_g psi_g> / <psi_M|psi_M>,
//   nu_g      = P_g U_g^dag nu_{g+1}.
// A gate couples each determinant only with its partner, so on a block
// {L, U} with tau L = s U (x = psi_g, v = nu_{g+1}, c = cos, sn = sin):
//   <v | A U x>_block = v_L (-sn x_L - s c x_U) + v_U (s c x_L - sn x_U)
//   (U^dag v)_L = c v_L + s sn v_U,   (U^dag v)_U = -s sn v_L + c v_U,
// and determinants without a partner pass nu through unchanged.  One thread
// per determinant of S_g: lookups of its partner in S_g and of itself and its
// partner in S_{g+1}; the block is counted by its lower member when that is in
// S_g, otherwise by its upper member.
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

namespace {

constexpr int kAdjThreads = 256;

__global__ void build_index_kernel(const uint64_t* keys, const long long* n_ptr, IdxSlot* tab, uint64_t mask) {
  const long long n = *n_ptr;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    idx_insert(tab, mask, keys[i], (uint64_t)i);
}

__global__ void nu_init_kernel(const double* amps, const double* sigma, const long long* n_ptr, const double* acc,
                               double* nu) {
  const long long n = *n_ptr;
  const double e = acc[0] / acc[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    nu[i] = sigma[i] - e * amps[i];
}

__device__ __forceinline__ double nu_at(const AdjArgs& a, uint64_t key) {
  const int64_t j = idx_lookup(a.tab_nu, a.mask_nu, key);
  return j >= 0 ? a.nu_in[j] : 0.0;
}

__global__ void __launch_bounds__(kAdjThreads) adjoint_gate_kernel(AdjArgs a) {
  __shared__ double red[kAdjThreads / 32];
  const GateOp op = decode_op(a.op);
  const double c = a.cs[0], sn = a.cs[1];
  const long long n = *a.n;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t d = a.keys[i];
    const double x = a.amps[i];
    uint64_t p = 0;
    int sb = 0;
    const int role = gate_role(op, d, &p, &sb);
    const double vd = nu_at(a, d);
    if (role == 0) {
      a.nu_out[i] = vd;
      continue;
    }
    const double s = sb ? -1.0 : 1.0;
    const double vp = nu_at(a, p);
    if (role > 0) {  // d = L, p = U
      const int64_t j = idx_lookup(a.tab, a.mask, p);
      const double xu = j >= 0 ? a.amps[j] : 0.0;
      a.nu_out[i] = c * vd + s * sn * vp;
      acc += vd * (-sn * x - s * c * xu) + vp * (s * c * x - sn * xu);
    } else {  // d = U, p = L
      a.nu_out[i] = -s * sn * vp + c * vd;
      if (idx_lookup(a.tab, a.mask, p) < 0) acc += vp * (-s * c * x) + vd * (-sn * x);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) t += red[w];
    if (t != 0.0) atomicAdd(a.dtheta, t);
  }
}

__global__ void scale_dtheta_kernel(double* d, int n, const double* acc) {
  const double f = 2.0 / acc[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] *= f;
}

}  // namespace

cudaError_t launch_build_index(const uint64_t* keys, const long long* n, IdxSlot* tab, uint64_t mask, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(tab, 0xff, (mask + 1) * sizeof(IdxSlot), st);
  if (e != cudaSuccess) return e;
  build_index_kernel<<<608, 256, 0, st>>>(keys, n, tab, mask);
  return cudaGetLastError();
}

cudaError_t launch_nu_init(const double* amps, const double* sigma, const long long* n, const double* acc, double* nu,
                           cudaStream_t st) {
  nu_init_kernel<<<608, 256, 0, st>>>(amps, sigma, n, acc, nu);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gate(const AdjArgs& a, int nblocks, cudaStream_t st) {
  adjoint_gate_kernel<<<nblocks, kAdjThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scale_dtheta(double* d, int n, const double* acc, cudaStream_t st) {
  scale_dtheta_kernel<<<(n + 255) / 256, 256, 0, st>>>(d, n, acc);
  return cudaGetLastError();
}

}  // namespace swcs
