// Device pieces of the gate sequence shared by the persistent gate kernel
// (swcs_ansatz.cu) and the batched persistent kernel (swcs_batch.cu): the
// top-N radix select over 12-bit digits and the epoch-tagged index tables.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {
namespace {

// Radix select over 12-bit digits.  |c| (63 bits) in digits [51,63) [39,51)
// [27,39) [15,27) [3,15) [0,3): the first digit is the exponent and the top
// mantissa bit, so it already splits the amplitudes into 2 bins per binade;
// the bitstring (64 bits) for exact ties in [52,64) [40,52) ... [0,4).
constexpr int kBinsLog = 12;
constexpr int kBins = 1 << kBinsLog;
constexpr int kAbsPasses = 6;
constexpr int kKeyPasses = 6;
constexpr int kPasses = kAbsPasses + kKeyPasses;

__device__ __forceinline__ int abs_hi(int q) { return 63 - kBinsLog * q; }
__device__ __forceinline__ int abs_lo(int q) { return max(0, 63 - kBinsLog * (q + 1)); }
__device__ __forceinline__ int key_hi(int q) { return 64 - kBinsLog * q; }
__device__ __forceinline__ int key_lo(int q) { return max(0, 64 - kBinsLog * (q + 1)); }

__device__ __forceinline__ uint64_t abs_bits(double c) {
  return (uint64_t)__double_as_longlong(c) & 0x7fffffffffffffffull;
}


__device__ __forceinline__ bool keep_entry(const SelState& s, uint64_t key, double c, uint64_t min_bits) {
  const uint64_t x = abs_bits(c);
  if (x < min_bits) return false;
  if (s.mode == 0) return true;
  if (s.mode == 1) return (x >> s.shift) >= (s.prefix >> s.shift);
  if (x != s.prefix) return x > s.prefix;
  return (key >> s.kshift) <= (s.kprefix >> s.kshift);
}

// The bin holding the need-th entry in selection order (descending bins for
// |c|, ascending for bitstrings) among nb bins of h; the whole block takes
// part: each thread sums a run of bins, a block scan gives each run's start.
__device__ void find_bin(const unsigned* h, int nb, long long need, bool desc, SelState& sel, long long* scan) {
  const int T = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int per = (nb + T - 1) / T;
  const int o0 = min(nb, t * per), o1 = min(nb, o0 + per);
  long long loc = 0;
  for (int o = o0; o < o1; ++o) loc += h[desc ? nb - 1 - o : o];
  long long inc = loc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long v = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += v;
  }
  if (lane == 31) scan[wid] = inc;
  __syncthreads();
  long long base = 0;
  for (int w = 0; w < wid; ++w) base += scan[w];
  long long cum = base + inc - loc;  // entries before this thread's run
  if (cum < need && cum + loc >= need) {
    for (int o = o0; o < o1; ++o) {
      const int v = desc ? nb - 1 - o : o;
      const long long hv = h[v];
      if (cum + hv >= need) {
        sel.bin = v;
        sel.cum = cum;
        sel.cnt = hv;
        break;
      }
      cum += hv;
    }
  }
  __syncthreads();
}

// Index tables of the states inside one launch: 8-byte slots holding the
// build's epoch in the high 32 bits and the determinant's position in the
// state arrays in the low 32; the key itself is read from the state's key
// array.  A slot whose epoch is not the build's reads as empty, so a table is
// never cleared between gates, and two tables take half the memory of
// key/index slots.  After the last gate the output table is written once in
// the plain key/index form that every other kernel reads.
__device__ __forceinline__ bool ep_insert(uint64_t* t, uint64_t mask, uint64_t key, uint32_t pos, uint32_t ep) {
  uint64_t s = mix64(key) & mask;
  const unsigned long long claim = ((unsigned long long)ep << 32) | pos;
  for (uint64_t n = 0; n <= mask; ++n) {
    unsigned long long* w = (unsigned long long*)&t[s];
    const unsigned long long old = ld_key_relaxed((const uint64_t*)w);
    if ((uint32_t)(old >> 32) != ep && atomicCAS(w, old, claim) == old) return true;
    s = (s + 1) & mask;
  }
  return false;
}

// Position of key in the build `ep` of table t over the state keys (-1: absent); adds the slots visited to *probes.
__device__ __forceinline__ int64_t ep_lookup(const uint64_t* __restrict__ t, uint64_t mask, const uint64_t* keys,
                                             uint64_t key, uint32_t ep, unsigned* probes) {
  uint64_t s = mix64(key) & mask;
  for (uint64_t n = 0; n <= mask; ++n) {
    const uint64_t w = t[s];
    if ((uint32_t)(w >> 32) != ep) {  // a slot this build never claimed ends the probe
      *probes += (unsigned)n + 1u;
      return -1;
    }
    if (keys[(uint32_t)w] == key) {
      *probes += (unsigned)n + 1u;
      return (int64_t)(uint32_t)w;
    }
    s = (s + 1) & mask;
  }
  *probes += (unsigned)(mask + 1);
  return -1;
}

// Counters per gate, in a ring of 3 so that the next gate's set can be
// reset while the current one is live.
enum { kCtrExtra = 0, kCtrZero = 1, kCtrKept = 2, kCtrN = 4 };

}  // namespace
}  // namespace swcs
