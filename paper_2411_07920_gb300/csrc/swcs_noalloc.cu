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
// Scratch: the index table of the caller's state and the two accumulators
// live in one file-scope __device__ array (g_noalloc), 2 MiB + 256 B,
// resident on every GPU that loads this library until the process exits.
// Host code cannot take the array's name as a device address: on the first
// call on each device the entry point asks the runtime for it
// (cudaGetSymbolAddress, with that device current) and keeps it.  That first
// call should therefore come before any stream capture.  Every call clears
// the part it uses; calls whose work overlaps on the GPU (two streams, two
// host threads) share the array and race.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/swcs.h"
#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace swcs {

// Access to the loaded Hamiltonian of a context (defined with the context).
int ctx_ham_for_noalloc(swcs_ctx* c, HamDev* H, cudaStream_t* st, int* nblocks);
int ctx_fail_for_noalloc(swcs_ctx* c, int code, const char* msg);

namespace {

constexpr int64_t kMaxDets = SWCS_NOALLOC_MAX_DETS;
constexpr uint64_t kSlots = 2 * (uint64_t)kMaxDets;  // load <= 1/2

struct NoAllocScratch {
  IdxSlot tab[kSlots];
  double acc[2];
  long long n;
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
  }
}

// At load <= 1/2 every insert finds a free slot.
__global__ void noalloc_index(const uint64_t* __restrict__ keys, long long n) {
  NoAllocScratch* s = &g_noalloc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    idx_insert(s->tab, kSlots - 1, keys[i], (uint64_t)i);
}

std::mutex g_mu;
NoAllocScratch* g_addr[64] = {};

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
  int nblocks = 0;
  int r = ctx_ham_for_noalloc(c, &H, &st, &nblocks);
  if (r) return r;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: cannot query the current device");
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
  noalloc_index<<<(int)((n + 255) / 256), 256, 0, st>>>(d_keys, (long long)n);
  StateDev S;
  S.keys = d_keys;
  S.amps = d_amps;
  S.n = &s->n;
  S.tab = s->tab;
  S.tab_mask = kSlots - 1;
  if (cudaGetLastError() != cudaSuccess || launch_energy(H, S, s->acc, nblocks, st) != cudaSuccess ||
      launch_finalize_energy(s->acc, d_out, st) != cudaSuccess)
    return ctx_fail_for_noalloc(c, SWCS_ERR_CUDA, "swcs_energy_noalloc: launch failed");
  return SWCS_OK;
}
