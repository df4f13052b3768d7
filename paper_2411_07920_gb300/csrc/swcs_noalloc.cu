// swcs_energy_noalloc: the energy of a caller-owned device state without any
// device allocation during the call.
//
// Who needs it: callers that must not call cudaMalloc / cudaFree on their
// hot path -- frameworks that reserve all device memory up front in their
// own caching allocator (a direct cudaMalloc then fails or fragments their
// pool), and latency-critical loops where cudaFree would synchronise the
// whole device.  They load the Hamiltonian once at set-up (that call does
// allocate) and then evaluate energies of states they keep in their own
// buffers.
//
// Scratch: the index table of the caller's state, the two accumulators and
// an input-check word live in one file-scope __device__ array (g_noalloc),
// 2 MiB + 256 B, resident on every GPU that loads this library until the
// process exits.  Host code cannot take the array's name as a device
// address: on the first call on each device the entry point asks the runtime
// for it (cudaGetSymbolAddress, with that device current) and keeps it.  That
// first call should therefore come before any stream capture.  Every call
// clears the whole table (all 131,072 slots, 2 MiB) and the accumulators
// before it indexes the state; calls whose work overlaps on the GPU (two
// streams, two host threads) share the array and race.
//
// The call runs on the device the context was created on: when another
// device is current it switches for the call and switches back.
//
// Input check without a host synchronisation: a determinant that appears
// twice, or one outside the loaded Hamiltonian's sector (a bit at or above
// n_so, a wrong electron count, S_z != 0), makes the call skip the energy
// kernel and write NaN to both outputs.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/swcs.h"
#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

// Access to the loaded Hamiltonian of a context (defined with the context).
int ctx_ham_for_noalloc(swcs_ctx* c, HamDev* H, cudaStream_t* st, int* nblocks, int* dev);
int ctx_fail_for_noalloc(swcs_ctx* c, int code, const char* msg);

namespace {

constexpr int64_t kMaxDets = SWCS_NOALLOC_MAX_DETS;
constexpr uint64_t kSlots = 2 * (uint64_t)kMaxDets;  // load <= 1/2

struct NoAllocScratch {
  IdxSlot tab[kSlots];
  double acc[2];
  long long n;
  int bad;  // set when the input holds a duplicate determinant or one outside the sector
};

static __device__ __align__(256) NoAllocScratch g_noalloc;

__global__ void noalloc_clear(long long n) {
  NoAllocScratch* s = &g_noalloc;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kSlots; i += (uint64_t)gridDim.x * blockDim.x)
    s->tab[i].key = kEmpty;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->acc[0] = 0.0;
    s->acc[1] = 0.0;
    s->n = n;
    s->bad = 0;
  }
}

// Insert that tells a duplicate apart from a fresh key (the shared insert
// treats a key already present as success).  At load <= 1/2 every insert
// finds a free slot; a full table is flagged like a bad input anyway.  Any
// bad determinant sets the state size to 0 before the energy kernel reads it,
// so that kernel never indexes the integrals with an orbital outside the
// sector.
__global__ void noalloc_index(const uint64_t* __restrict__ keys, long long n, int n_so, int n_e) {
  NoAllocScratch* s = &g_noalloc;
  const uint64_t valid = n_so >= 64 ? ~0ull : (1ull << n_so) - 1ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t key = keys[i];
    bool ok = key != kEmpty && (key & ~valid) == 0 && __popcll(key) == n_e &&
              2 * __popcll(key & 0x5555555555555555ull) == n_e;
    if (ok) {
      ok = false;
      uint64_t slot = mix64(key) & (kSlots - 1);
      for (uint64_t probe = 0; probe < kSlots; ++probe) {
        const unsigned long long prev = atomicCAS((unsigned long long*)&s->tab[slot].key,
                                                  (unsigned long long)kEmpty, (unsigned long long)key);
        if (prev == kEmpty) {
          s->tab[slot].idx = (uint64_t)i;
          ok = true;
          break;
        }
        if (prev == key) break;  // the same determinant twice
        slot = (slot + 1) & (kSlots - 1);
      }
    }
    if (!ok) {
      atomicExch(&s->bad, 1);
      atomicExch((unsigned long long*)&s->n, 0ull);
    }
  }
}

// Both outputs become NaN when the input check failed.
__global__ void noalloc_flag(double* out) {
  if (threadIdx.x == 0 && *(volatile int*)&g_noalloc.bad) {
    out[0] = __longlong_as_double(0x7ff8000000000000ll);
    out[1] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

std::mutex g_mu;
NoAllocScratch* g_addr[64] = {};

// Makes the context's device current for the call and restores the caller's.
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  cudaError_t enter(int want) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev == want) return cudaSuccess;
    e = cudaSetDevice(want);
    switched = e == cudaSuccess;
    return e;
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace swcs

using namespace swcs;

extern "C" int swcs_energy_noalloc(swcs_ctx* c, const uint64_t* d_keys, const double* d_amps, int64_t n,
                                   double* d_out) {
  if (!c) return SWCS_ERR_INVALID_ARG;
  if (n < 1 || n > kMaxDets)
    return ctx_fail_for_noalloc(c, SWCS_ERR_INVALID_ARG,
                                "swcs_energy_noalloc: n must be in 1..SWCS_NOALLOC_MAX_DETS (65536)");
  if (!d_keys || !d_amps || !d_out) return ctx_fail_for_noalloc(c, SWCS_ERR_INVALID_ARG, "swcs_energy_noalloc: null pointer");
  HamDev H;
  cudaStream_t st;
  int nblocks = 0, dev = 0;
  int r = ctx_ham_for_noalloc(c, &H, &st, &nblocks, &dev);
  if (r) return r;
  if (dev < 0 || dev >= 64) return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: device index out of range");
  DeviceGuard guard;
  if (guard.enter(dev) != cudaSuccess)
    return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: cannot make the context's device current");
  NoAllocScratch* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
      if (e != cudaSuccess || !p)
        return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: cudaGetSymbolAddress failed");
      g_addr[dev] = (NoAllocScratch*)p;
    }
    s = g_addr[dev];
  }
  noalloc_clear<<<256, 256, 0, st>>>((long long)n);
  if (cudaGetLastError() != cudaSuccess) return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: launch failed");
  noalloc_index<<<(int)((n + 255) / 256), 256, 0, st>>>(d_keys, (long long)n, H.n, H.ne);
  StateDev S;
  S.keys = d_keys;
  S.amps = d_amps;
  S.n = &s->n;
  S.tab = s->tab;
  S.tab_mask = kSlots - 1;
  if (cudaGetLastError() != cudaSuccess || launch_energy(H, S, s->acc, nblocks, st) != cudaSuccess ||
      launch_finalize_energy(s->acc, d_out, st) != cudaSuccess)
    return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: launch failed");
  noalloc_flag<<<1, 32, 0, st>>>(d_out);
  if (cudaGetLastError() != cudaSuccess) return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: launch failed");
  return SWCS_OK;
}
