// MP2 amplitudes for the UCCSD initial guess (Sec. II.A) and the overlap of
// the context's state with a caller's sparse state (the infidelity of
// Sec. IV.B).
//
//   t(i j -> a b) = <ab||ij> / (e_i + e_j - e_a - e_b),  e_p = h_pp + sum_{k occ} <pk||pk>
//
// One thread per double; the orbital energies are summed over the occupied
// spin-orbitals in index order and the denominator left to right, so the
// amplitudes do not depend on the launch.  The overlap looks each of the
// caller's determinants up in the index table of the state.
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

namespace {

__device__ __forceinline__ double orbital_energy(const HamDev& H, int p) {
  double s = 0.0;
  for (int k = 0; k < H.ne; ++k) s = __dadd_rn(s, H.J[p * H.n + k]);
  return __dadd_rn(H.h[p * H.n + p], s);
}

__global__ void mp2_kernel(HamDev H, const uint8_t* ijab, int64_t nd, double* t) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nd; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = ijab[4 * q], j = ijab[4 * q + 1], a = ijab[4 * q + 2], b = ijab[4 * q + 3];
    const double num = H.G[(size_t)pair_index(i, j, H.n) * H.npairs + pair_index(a, b, H.n)];  // <ab||ij>
    const double den =
        __dadd_rn(__dadd_rn(__dadd_rn(orbital_energy(H, i), orbital_energy(H, j)), -orbital_energy(H, a)),
                  -orbital_energy(H, b));
    t[q] = num / den;
  }
}

// out[0] += sum over the caller's determinants of c_state c_given, out[1] += sum c_given^2
__global__ void overlap_kernel(StateDev S, const uint64_t* keys, const double* amps, int64_t n, double* out) {
  double ab = 0.0, bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double c = amps[i];
    const int64_t j = idx_lookup(S.tab, S.tab_mask, keys[i]);
    if (j >= 0) ab += S.amps[j] * c;
    bb += c * c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ab += __shfl_xor_sync(0xffffffffu, ab, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ab != 0.0) atomicAdd(&out[0], ab);
    if (bb != 0.0) atomicAdd(&out[1], bb);
  }
}

// out[2] += <state|state>
__global__ void norm_kernel(StateDev S, double* out) {
  const long long n = *S.n;
  double aa = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    aa += S.amps[i] * S.amps[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) aa += __shfl_xor_sync(0xffffffffu, aa, o);
  if ((threadIdx.x & 31) == 0 && aa != 0.0) atomicAdd(&out[2], aa);
}

}  // namespace

cudaError_t launch_mp2(const HamDev& H, const uint8_t* ijab, int64_t nd, double* t, cudaStream_t st) {
  if (nd <= 0) return cudaSuccess;
  const int nb = (int)((nd + 255) / 256 < 1024 ? (nd + 255) / 256 : 1024);
  mp2_kernel<<<nb, 256, 0, st>>>(H, ijab, nd, t);
  return cudaGetLastError();
}

cudaError_t launch_overlap(const StateDev& S, const uint64_t* keys, const double* amps, int64_t n, double* out,
                           int nblocks, cudaStream_t st) {
  if (n > 0) overlap_kernel<<<nblocks, 256, 0, st>>>(S, keys, amps, n, out);
  norm_kernel<<<nblocks, 256, 0, st>>>(S, out);
  return cudaGetLastError();
}

}  // namespace swcs
