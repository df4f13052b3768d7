// Device helpers shared by the SWCS kernels: determinant bit operations and
// fermionic phases, the open-addressing determinant hash, bounded grid
// barriers and the device error word.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace swcs {

constexpr uint64_t kEmpty = ~0ull;  // never a valid determinant (n_so <= 64, n_e < n_so)

// Device error codes (mirrored to SWCS_ERR_* on the host).
enum DevErr : int { kDevOk = 0, kDevTimeout = 1, kDevTableFull = 2, kDevBadState = 3 };

// ----------------------------------------------------------------------------
// Hashing (splitmix64 finaliser).  Determinants differ in few bits, so the
// full avalanche matters for probe lengths.
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// Index table slot: determinant -> position in the state arrays.
struct __align__(16) IdxSlot {
  uint64_t key;
  uint64_t idx;
};

// Value table slot: determinant -> accumulated FP64 value.
struct __align__(16) ValSlot {
  uint64_t key;
  double val;
};

__device__ __forceinline__ uint64_t ld_key_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Lookup in an index table of capacity mask+1.  Returns the stored index or -1.
__device__ __forceinline__ int64_t idx_lookup(const IdxSlot* __restrict__ t, uint64_t mask, uint64_t key) {
  uint64_t s = mix64(key) & mask;
  for (uint64_t n = 0; n <= mask; ++n) {
    const IdxSlot sl = t[s];
    if (sl.key == key) return (int64_t)sl.idx;
    if (sl.key == kEmpty) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}

// The lookup continued from slot s after n0 slots already visited; adds the slots it visited (the n0
// included) to *probes when probes is given.
__device__ __forceinline__ int64_t idx_lookup_at(const IdxSlot* __restrict__ t, uint64_t mask, uint64_t key, uint64_t s,
                                                 uint64_t n0, unsigned* probes) {
  for (uint64_t n = n0; n <= mask; ++n) {
    const IdxSlot sl = t[s];
    if (sl.key == key || sl.key == kEmpty) {
      if (probes) *probes += (unsigned)n + 1u;
      return sl.key == key ? (int64_t)sl.idx : -1;
    }
    s = (s + 1) & mask;
  }
  if (probes) *probes += (unsigned)(mask + 1);
  return -1;
}

// The same lookup, also adding the number of slots it visited to *probes.
__device__ __forceinline__ int64_t idx_lookup_counted(const IdxSlot* __restrict__ t, uint64_t mask, uint64_t key,
                                                      unsigned* probes) {
  uint64_t s = mix64(key) & mask;
  for (uint64_t n = 0; n <= mask; ++n) {
    const IdxSlot sl = t[s];
    if (sl.key == key || sl.key == kEmpty) {
      *probes += (unsigned)n + 1u;
      return sl.key == key ? (int64_t)sl.idx : -1;
    }
    s = (s + 1) & mask;
  }
  *probes += (unsigned)(mask + 1);
  return -1;
}

// Insert (key -> idx); keys are unique per build.  Returns false when the
// table has no free slot (cannot happen at load <= 1/2, checked anyway).
__device__ __forceinline__ bool idx_insert(IdxSlot* t, uint64_t mask, uint64_t key, uint64_t idx) {
  uint64_t s = mix64(key) & mask;
  for (uint64_t n = 0; n <= mask; ++n) {
    unsigned long long prev = atomicCAS((unsigned long long*)&t[s].key, (unsigned long long)kEmpty,
                                        (unsigned long long)key);
    if (prev == kEmpty || prev == key) {
      t[s].idx = idx;
      return true;
    }
    s = (s + 1) & mask;
  }
  return false;
}

// ----------------------------------------------------------------------------
// Fermionic phases.  parity_below(d, p) = number of occupied orbitals < p, mod 2.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int parity_below(uint64_t d, int p) {
  return __popcll(d & ((1ull << p) - 1ull)) & 1;
}

// Phase of a+_{c1} a_{a0} on d (a0 occupied, c1 empty, a0 != c1): returns 0 / 1 (sign bit).
__device__ __forceinline__ int single_phase(uint64_t d, int a0, int c1) {
  int par = parity_below(d, a0);
  uint64_t d1 = d & ~(1ull << a0);
  par ^= parity_below(d1, c1);
  return par;
}

// Phase of a+_{c2} a+_{c3} a_{a1} a_{a0} on d (a0,a1 occupied; c2,c3 empty;
// all distinct): applied right to left.  Returns the sign bit.
__device__ __forceinline__ int double_phase(uint64_t d, int a0, int a1, int c2, int c3) {
  int par = parity_below(d, a0);
  uint64_t x = d & ~(1ull << a0);
  par ^= parity_below(x, a1);
  x &= ~(1ull << a1);
  par ^= parity_below(x, c3);
  x |= (1ull << c3);
  par ^= parity_below(x, c2);
  return par;
}

// -v when sign_bit is set, as a flip of the IEEE-754 sign bit on the integer
// pipe (the same value as negation, zeros and NaNs included).
__device__ __forceinline__ double apply_sign(double v, int sign_bit) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(sign_bit != 0) << 63));
}

// ----------------------------------------------------------------------------
// A gate operator (5 bytes: kind, i0..i3; kind 1: tau = a+_{i1} a_{i0},
// kind 2: tau = a+_{i2} a+_{i3} a_{i1} a_{i0}, kind 0: identity).
// ----------------------------------------------------------------------------
struct GateOp {
  int kind;
  uint64_t mask_a;  // annihilated by tau
  uint64_t mask_c;  // created by tau
  int i0, i1, i2, i3;
};

__device__ __forceinline__ GateOp decode_op(const uint8_t* o) {
  GateOp g;
  g.kind = o[0];
  g.i0 = o[1];
  g.i1 = o[2];
  g.i2 = o[3];
  g.i3 = o[4];
  if (g.kind == 1) {
    g.mask_a = 1ull << g.i0;
    g.mask_c = 1ull << g.i1;
  } else if (g.kind == 2) {
    g.mask_a = (1ull << g.i0) | (1ull << g.i1);
    g.mask_c = (1ull << g.i2) | (1ull << g.i3);
  } else {
    g.mask_a = 0;
    g.mask_c = 0;
  }
  return g;
}

// Role of d under the gate: +1 lower (tau d != 0), -1 upper (tau^dag d != 0),
// 0 neither.  *partner and *sbit (phase of tau d, or of tau^dag d) on +-1.
__device__ __forceinline__ int gate_role(const GateOp& op, uint64_t d, uint64_t* partner, int* sbit) {
  if (!op.kind) return 0;
  const bool up = ((d & op.mask_a) == op.mask_a) && ((d & op.mask_c) == 0);
  const bool dn = ((d & op.mask_c) == op.mask_c) && ((d & op.mask_a) == 0);
  if (!up && !dn) return 0;
  *partner = d ^ op.mask_a ^ op.mask_c;
  if (op.kind == 1) *sbit = up ? single_phase(d, op.i0, op.i1) : single_phase(d, op.i1, op.i0);
  else *sbit = up ? double_phase(d, op.i0, op.i1, op.i2, op.i3) : double_phase(d, op.i2, op.i3, op.i0, op.i1);
  return up ? 1 : -1;
}

// ----------------------------------------------------------------------------
// Global timer and bounded waits.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// Barrier among `nblocks` co-resident CTAs sharing {count, gen}.  Waits at
// most timeout_ns; on timeout sets *err = kDevTimeout.  Returns false when an
// error is pending (caller must leave the kernel).
struct GridBar {
  unsigned count;
  unsigned gen;
};

__device__ __forceinline__ bool grid_barrier(GridBar* b, unsigned nblocks, int* err, uint64_t timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned my_gen = ld_acquire_u32(&b->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const uint64_t t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(&b->gen) == my_gen) {
        if ((++spins & 255u) == 0) {
          if (ld_acquire_i32(err) != 0) { ok = 0; break; }
          if (globaltimer_ns() - t0 > timeout_ns) { set_error(err, kDevTimeout); ok = 0; break; }
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ok && ld_acquire_i32(err) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Warp-aggregated atomic increment: every active lane with `pred` gets a
// distinct slot from *ctr.
__device__ __forceinline__ unsigned long long warp_alloc(unsigned long long* ctr, bool pred) {
  const unsigned mask = __activemask();
  const unsigned ballot = __ballot_sync(mask, pred);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(ballot) - 1;
  unsigned long long base = 0;
  if (ballot && lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(ballot));
  base = __shfl_sync(mask, base, leader < 0 ? 0 : leader);
  return base + __popc(ballot & ((1u << lane) - 1u));
}

}  // namespace swcs
