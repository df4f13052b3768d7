// sigma = H psi kernels (Slater-Condon rules) for the energy and the
// operator-pool gradient.
//
//   energy   sigma_D = <D|H|D> c_D + sum_{E in conn(D) and S} <D|H|E> c_E,
//            E = sum c_D sigma_D / sum c_D^2                (Sec. II, step 7)
//   scatter  sigma_E += <E|H|D> c_D for every E in conn(D) + {D}, D in S,
//            into an external hash table (pass 1 of the pool sweep)
//   gather   g_k += dir * phase * c_D * sigma_E for every connected pair,
//            k = the pool operator that maps D to E                (step 4)
//
// Every single and double excitation of D is one generalized pool operator
// (Sec. II.C): removing pair Pa and adding pair Pb is tau_k of the operator
// {min(Pa,Pb) -> max(Pa,Pb)} when Pa < Pb (dir +1) and tau_k^dag otherwise
// (dir -1), so the gradient is a segmented sum over the same pairs that
// build sigma.
//
// Work layout: one warp per determinant D.  The warp builds D's occupied
// and virtual lists per spin in shared memory, then walks the excitation
// classes (singles, alpha-alpha, beta-beta, alpha-beta doubles) with the
// removed pair warp-uniform and lanes over the added pairs, so a warp reads
// one row G[Pa, *] of the packed integrals at a time.
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

namespace {

constexpr int kWarps = kSigmaThreads / 32;
constexpr unsigned kMaxProbe = 1u << 20;

enum Mode { kEnergy = 0, kScatter = 1, kGather = 2 };

struct WarpLists {
  uint8_t occ[2][kMaxSpin];  // spin-orbital indices, ascending
  uint8_t vir[2][kMaxSpin];
  uint8_t occ_all[64];
};

struct Tables {
  uint16_t tri_o[kMaxSpin * (kMaxSpin - 1) / 2];  // occupied slot pairs (a<b): a | b<<8
  uint16_t tri_v[kMaxSpin * (kMaxSpin - 1) / 2];  // virtual slot pairs
};

__device__ __forceinline__ unsigned bucket_of(uint64_t hb, unsigned log2b) {
  return log2b ? (unsigned)((hb >> 40) & ((1ull << log2b) - 1ull)) : 0u;
}

__device__ __forceinline__ bool ext_add(const ExtTable& T, uint64_t key, uint64_t hb, double v, unsigned& n_new) {
  uint64_t s = hb & T.mask;
  for (unsigned n = 0; n < kMaxProbe; ++n) {
    const uint64_t k = ld_key_relaxed(&T.slots[s].key);
    if (k == key) {
      atomicAdd(&T.slots[s].val, v);
      return true;
    }
    if (k == kEmpty) {
      const unsigned long long prev =
          atomicCAS((unsigned long long*)&T.slots[s].key, (unsigned long long)kEmpty, (unsigned long long)key);
      if (prev == kEmpty || prev == key) {
        atomicAdd(&T.slots[s].val, v);
        if (prev == kEmpty) ++n_new;
        return true;
      }
    }
    s = (s + 1) & T.mask;
  }
  return false;
}

__device__ __forceinline__ bool ext_get(const ExtTable& T, uint64_t key, uint64_t hb, double& v) {
  uint64_t s = hb & T.mask;
  for (unsigned n = 0; n < kMaxProbe; ++n) {
    const ValSlot sl = T.slots[s];
    if (sl.key == key) { v = sl.val; return true; }
    if (sl.key == kEmpty) return false;
    s = (s + 1) & T.mask;
  }
  return false;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One connected pair (D -> E) with removed (p<q) and added (r<s) pairs; q<0 / s<0 for singles.
template <int MODE>
struct PairCtx {
  const HamDev& H;
  const StateDev& S;
  const ExtTable& T;
  double* g;
  uint64_t d;
  double cd;
  double acc;        // energy: sum_E <D|H|E> c_E
  unsigned n_new;    // scatter: new keys inserted by this lane
  bool fail;
};

template <int MODE>
__device__ __forceinline__ void visit_double(PairCtx<MODE>& x, int p, int q, int r, int s) {
  const uint64_t e = x.d ^ ((1ull << p) | (1ull << q) | (1ull << r) | (1ull << s));
  const int n = x.H.n;
  const int pa = pair_index(p, q, n), pb = pair_index(r, s, n);
  if (MODE == kEnergy) {
    const int64_t j = idx_lookup(x.S.tab, x.S.tab_mask, e);
    if (j >= 0) {
      const int sb = double_phase(x.d, p, q, r, s);
      x.acc += apply_sign(x.H.G[(size_t)pa * x.H.npairs + pb], sb) * x.S.amps[j];
    }
  } else {
    const uint64_t hb = mix64(e);
    if (bucket_of(hb, x.T.nbucket_log2) != x.T.bucket) return;
    const int sb = double_phase(x.d, p, q, r, s);
    if (MODE == kScatter) {
      const double v = apply_sign(x.H.G[(size_t)pa * x.H.npairs + pb], sb) * x.cd;
      if (!ext_add(x.T, e, hb, v, x.n_new)) x.fail = true;
    } else {
      double sig;
      if (!ext_get(x.T, e, hb, sig)) { x.fail = true; return; }
      int k;
      bool down;
      if (pa < pb) { k = x.H.opd[(size_t)pa * x.H.npairs + pb]; down = false; }
      else { k = x.H.opd[(size_t)pb * x.H.npairs + pa]; down = true; }
      atomicAdd(&x.g[k], apply_sign(x.cd * sig, sb ^ (int)down));
    }
  }
}

template <int MODE>
__device__ __forceinline__ void visit_single(PairCtx<MODE>& x, const WarpLists& L, int p, int q) {
  const uint64_t e = x.d ^ ((1ull << p) | (1ull << q));
  const int n = x.H.n;
  uint64_t hb = 0;
  if (MODE != kEnergy) {
    hb = mix64(e);
    if (bucket_of(hb, x.T.nbucket_log2) != x.T.bucket) return;
  }
  int64_t j = -1;
  if (MODE == kEnergy) {
    j = idx_lookup(x.S.tab, x.S.tab_mask, e);
    if (j < 0) return;
  }
  const int sb = single_phase(x.d, p, q);
  if (MODE == kGather) {
    double sig;
    if (!ext_get(x.T, e, hb, sig)) { x.fail = true; return; }
    const int lo = p < q ? p : q, hi = p < q ? q : p;
    const int k = x.H.ops1[lo * n + hi];
    atomicAdd(&x.g[k], apply_sign(x.cd * sig, sb ^ (int)(p > q)));
    return;
  }
  // <E|H|D> = phase * (h_qp + sum_{k in D} <qk||pk>)
  double f = x.H.h[q * n + p];
  const double* w = x.H.Ws + ((size_t)p * n + q) * n;
  for (int t = 0; t < x.H.ne; ++t) f += w[L.occ_all[t]];
  f = apply_sign(f, sb);
  if (MODE == kEnergy) x.acc += f * x.S.amps[j];
  else if (!ext_add(x.T, e, hb, f * x.cd, x.n_new)) x.fail = true;
}

template <int MODE>
__global__ void __launch_bounds__(kSigmaThreads)
sigma_kernel(HamDev H, StateDev S, ExtTable T, double* g, double* acc_out, int add_norm, double* sig_out) {
  __shared__ WarpLists lists[kWarps];
  __shared__ Tables tabs;
  __shared__ double s_red[2][kWarps];
  __shared__ unsigned s_new;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int no = H.no, nv = H.nv, n = H.n;
  const int n_to = no * (no - 1) / 2, n_tv = nv * (nv - 1) / 2;
  // triangular decode tables (slot pairs a<b in lexicographic order)
  for (int t = threadIdx.x; t < n_to || t < n_tv; t += blockDim.x) {
    if (t < n_to || t < n_tv) {
      // decode t for a list of length L
      auto dec = [](int t, int L) -> uint16_t {
        int a = 0, base = 0;
        while (base + (L - 1 - a) <= t) { base += L - 1 - a; ++a; }
        return (uint16_t)(a | ((a + 1 + (t - base)) << 8));
      };
      if (t < n_to) tabs.tri_o[t] = dec(t, no);
      if (t < n_tv) tabs.tri_v[t] = dec(t, nv);
    }
  }
  if (threadIdx.x == 0) s_new = 0;
  __syncthreads();

  const long long nd = *S.n;
  const long long gwarp = (long long)blockIdx.x * kWarps + warp;
  const long long nwarps = (long long)gridDim.x * kWarps;
  double e_num = 0.0, e_n2 = 0.0;
  unsigned my_new = 0;
  bool my_fail = false;
  WarpLists& L = lists[warp];

  for (long long i = gwarp; i < nd; i += nwarps) {
    const uint64_t d = S.keys[i];
    const double cd = S.amps[i];
    // occupied / virtual lists per spin (spin-orbital p = 2*spatial + spin)
    {
      const int m = n >> 1;
      for (int sp = 0; sp < 2; ++sp) {
        const bool inr = lane < m;
        const bool occ = inr && ((d >> (2 * lane + sp)) & 1ull);
        const unsigned bo = __ballot_sync(0xffffffffu, occ);
        const unsigned bv = __ballot_sync(0xffffffffu, inr && !occ);
        const unsigned below = (1u << lane) - 1u;
        if (occ) L.occ[sp][__popc(bo & below)] = (uint8_t)(2 * lane + sp);
        else if (inr) L.vir[sp][__popc(bv & below)] = (uint8_t)(2 * lane + sp);
      }
      const unsigned lo = (unsigned)d, hi = (unsigned)(d >> 32);
      const unsigned below = (1u << lane) - 1u;
      if ((lo >> lane) & 1u) L.occ_all[__popc(lo & below)] = (uint8_t)lane;
      if ((hi >> lane) & 1u) L.occ_all[__popc(lo) + __popc(hi & below)] = (uint8_t)(32 + lane);
      __syncwarp();
    }
    PairCtx<MODE> x{H, S, T, g, d, cd, 0.0, 0u, false};

    // singles: 2 * no * nv
    const int n_s = 2 * no * nv;
    for (int t = lane; t < n_s; t += 32) {
      const int sp = t / (no * nv), rem = t - sp * no * nv;
      const int o = rem / nv, v = rem - o * nv;
      visit_single<MODE>(x, L, L.occ[sp][o], L.vir[sp][v]);
    }
    // same-spin doubles
    for (int sp = 0; sp < 2; ++sp) {
      for (int op = 0; op < n_to; ++op) {
        const uint16_t oo = tabs.tri_o[op];
        const int p = L.occ[sp][oo & 255], q = L.occ[sp][oo >> 8];
        for (int t = lane; t < n_tv; t += 32) {
          const uint16_t vv = tabs.tri_v[t];
          visit_double<MODE>(x, p, q, L.vir[sp][vv & 255], L.vir[sp][vv >> 8]);
        }
      }
    }
    // opposite-spin doubles
    for (int oa = 0; oa < no; ++oa) {
      for (int ob = 0; ob < no; ++ob) {
        const int pa = L.occ[0][oa], pb = L.occ[1][ob];
        const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
        for (int t = lane; t < nv * nv; t += 32) {
          const int va = t / nv, vb = t - va * nv;
          const int ra = L.vir[0][va], rb = L.vir[1][vb];
          visit_double<MODE>(x, p, q, ra < rb ? ra : rb, ra < rb ? rb : ra);
        }
      }
    }

    if (MODE == kEnergy) {
      // diagonal <D|H|D> = sum_i h_ii + 1/2 sum_ij <ij||ij>
      double hd = 0.0;
      for (int t = lane; t < H.ne; t += 32) {
        const int a = L.occ_all[t];
        double jj = 0.0;
        for (int u = 0; u < H.ne; ++u) jj += H.J[a * n + L.occ_all[u]];
        hd += H.h[a * n + a] + 0.5 * jj;
      }
      hd = warp_sum(hd);
      const double off = warp_sum(x.acc);
      if (lane == 0) {
        e_num += cd * (hd * cd + off);
        e_n2 += cd * cd;
        if (sig_out) sig_out[i] = hd * cd + off;
      }
    } else if (MODE == kScatter) {
      if (lane == 0) {
        const uint64_t hb = mix64(d);
        if (bucket_of(hb, T.nbucket_log2) == T.bucket) {
          double hd = 0.0;
          for (int t = 0; t < H.ne; ++t) {
            const int a = L.occ_all[t];
            double jj = 0.0;
            for (int u = 0; u < H.ne; ++u) jj += H.J[a * n + L.occ_all[u]];
            hd += H.h[a * n + a] + 0.5 * jj;
          }
          if (!ext_add(T, d, hb, hd * cd, x.n_new)) x.fail = true;
        }
      }
    } else {
      if (lane == 0) {
        const uint64_t hb = mix64(d);
        if (bucket_of(hb, T.nbucket_log2) == T.bucket) {
          double sig;
          if (ext_get(T, d, hb, sig)) e_num += cd * sig;
          else x.fail = true;
        }
        if (add_norm) e_n2 += cd * cd;
      }
    }
    my_new += x.n_new;
    my_fail |= x.fail;
    __syncwarp();
  }

  if (MODE == kScatter) {
    unsigned w = my_new;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0 && w) atomicAdd(&s_new, w);
  }
  if (my_fail && T.err) set_error(T.err, kDevTableFull);
  if (MODE != kScatter) {
    if (lane == 0) {
      s_red[0][warp] = e_num;
      s_red[1][warp] = e_n2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (MODE == kScatter) {
      if (s_new) atomicAdd(T.n_distinct, (unsigned long long)s_new);
    } else {
      double a0 = 0.0, a1 = 0.0;
      for (int w = 0; w < kWarps; ++w) { a0 += s_red[0][w]; a1 += s_red[1][w]; }
      atomicAdd(&acc_out[0], a0);
      atomicAdd(&acc_out[1], a1);
    }
  }
}

__global__ void clear_ext_kernel(ValSlot* s, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    s[i].key = kEmpty;
    s[i].val = 0.0;
  }
}

__global__ void finalize_energy_kernel(const double* acc, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    out[0] = acc[0] / acc[1];
    out[1] = acc[1];
  }
}

__global__ void scale_gradient_kernel(double* g, int64_t n, const double* acc) {
  const double f = 2.0 / acc[1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    g[i] *= f;
}

__global__ void gather_subset_kernel(const double* g, const int64_t* sub, int64_t n, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[sub[i]] = g[sub[i]];
}

// J[i*n+j] = <ij||ij>; Ws[(p*n+q)*n+k] = <qk||pk>; G[P(p,q)*np + P(r,s)] = <rs||pq>
__global__ void pack_kernel(const double* gf, int n, double* J, double* Ws, double* G) {
  const size_t n2 = (size_t)n * n, n3 = n2 * n;
  const int np = n * (n - 1) / 2;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, str = (size_t)gridDim.x * blockDim.x;
  auto at = [&](int p, int q, int r, int s) { return gf[(((size_t)p * n + q) * n + r) * n + s]; };
  for (size_t t = tid; t < n2; t += str) {
    const int i = (int)(t / n), j = (int)(t % n);
    J[t] = at(i, j, i, j);
  }
  for (size_t t = tid; t < n3; t += str) {
    const int p = (int)(t / n2), q = (int)((t / n) % n), k = (int)(t % n);
    Ws[t] = at(q, k, p, k);
  }
  for (size_t t = tid; t < (size_t)np * np; t += str) {
    const int a = (int)(t / np), b = (int)(t % np);
    // decode pair indices
    int p = 0, base = 0;
    while (base + (n - 1 - p) <= a) { base += n - 1 - p; ++p; }
    const int q = p + 1 + (a - base);
    int r = 0;
    base = 0;
    while (base + (n - 1 - r) <= b) { base += n - 1 - r; ++r; }
    const int s = r + 1 + (b - base);
    G[t] = at(r, s, p, q);
  }
}

}  // namespace

int sigma_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sigma_kernel<kScatter>, kSigmaThreads, 0) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

cudaError_t launch_energy(const HamDev& H, const StateDev& S, double* acc, int nblocks, cudaStream_t st) {
  ExtTable T{};
  sigma_kernel<kEnergy><<<nblocks, kSigmaThreads, 0, st>>>(H, S, T, nullptr, acc, 1, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_energy_sigma(const HamDev& H, const StateDev& S, double* acc, double* sig_out, int nblocks,
                                cudaStream_t st) {
  ExtTable T{};
  sigma_kernel<kEnergy><<<nblocks, kSigmaThreads, 0, st>>>(H, S, T, nullptr, acc, 1, sig_out);
  return cudaGetLastError();
}

cudaError_t launch_sigma_scatter(const HamDev& H, const StateDev& S, const ExtTable& T, int nblocks,
                                 cudaStream_t st) {
  sigma_kernel<kScatter><<<nblocks, kSigmaThreads, 0, st>>>(H, S, T, nullptr, nullptr, 0, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_pool_gather(const HamDev& H, const StateDev& S, const ExtTable& T, double* g, double* acc,
                               int add_norm, int nblocks, cudaStream_t st) {
  sigma_kernel<kGather><<<nblocks, kSigmaThreads, 0, st>>>(H, S, T, g, acc, add_norm, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_clear_ext(ValSlot* slots, uint64_t n, cudaStream_t st) {
  clear_ext_kernel<<<1216, 256, 0, st>>>(slots, n);
  return cudaGetLastError();
}

cudaError_t launch_finalize_energy(const double* acc, double* out, cudaStream_t st) {
  finalize_energy_kernel<<<1, 32, 0, st>>>(acc, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_gradient(double* g, int64_t n, const double* acc, cudaStream_t st) {
  scale_gradient_kernel<<<304, 256, 0, st>>>(g, n, acc);
  return cudaGetLastError();
}

cudaError_t launch_gather_subset(const double* g, const int64_t* sub, int64_t n, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  gather_subset_kernel<<<152, 256, 0, st>>>(g, sub, n, out);
  return cudaGetLastError();
}

cudaError_t launch_pack_hamiltonian(const double* g_full, int n, double* J, double* Ws, double* G,
                                    cudaStream_t st) {
  pack_kernel<<<608, 256, 0, st>>>(g_full, n, J, Ws, G);
  return cudaGetLastError();
}

}  // namespace swcs
