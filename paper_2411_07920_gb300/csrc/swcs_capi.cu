// Host side of the C ABI declared in include/swcs.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swcs.h"
#include "swcs_device.cuh"
#include "swcs_kernels.h"

using namespace swcs;

namespace {

constexpr uint64_t kTimeoutNs = 2000000000ull;  // bounded device waits: 2 s

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct swcs_ctx {
  cudaStream_t st = nullptr;
  int dev = 0;
  int nsm = 0;
  std::string err;

  // Hamiltonian
  int n = 0, ne = 0, no = 0, nv = 0, npairs = 0;
  bool have_ham = false;
  double fci_dim = 0.0;
  int64_t pool_size = 0;
  std::vector<uint8_t> pool_ops;  // 5 bytes each
  DevBuf h, J, Ws, G, opd, ops1, gstage, pool_dev;
  DevBuf selbits, feat, ypred, topk_hist, topk_ctl, occ;

  // state
  DevBuf keys_a, amps_a, keys_b, amps_b, tab0, tab1;
  int64_t cap = 0;
  uint64_t tab_mask = 0;
  int tab_cur = 0;
  bool have_state = false;
  int64_t n_state_host = -1;  // cached size (-1 unknown)

  // control and scratch
  DevBuf ctrl;  // n_state, tab_cur, err, bar, ctr, hist, stats, acc, eout
  DevBuf ops_dev, cs_dev;
  DevBuf gdev, subset_dev, gsub;
  DevBuf ovl_keys, ovl_amps;  // swcs_overlap: the caller's state

  // row sweep: alpha strings of the sector, beta-rank tables, grouped state, rows
  DevBuf alpha_list, rank_tab, atab, gid_of, gcount, goff, gfill, gkey, gamp, grank, rows, rbeta, gab, kab, gorig;
  int NA = 0;
  int64_t NB = 0;
  int opt_sweep = 0;    // 0 auto, 1 hashed external table, 2 alpha-string rows
  int opt_cluster = 1;  // CTAs per row cluster
  int opt_rows_l2 = 0;  // cap concurrent rows to about half of L2
  int opt_threads = 1024;  // threads per CTA of the row sweep
  int opt_row_occ = 2;    // resident 512-thread CTAs per SM asked of the compiler (1, 2 or 3)
  double trunc_eps = 0.0;  // magnitude criterion of the truncation (0: off)
  int opt_energy = 0;     // energy: 0 automatic, 1 probe kernel, 2 alpha-string rows
  uint64_t opt_timeout_ns = kTimeoutNs;  // bound of every device-side wait
  int opt_skip_arrive = -1;              // test hook (see swcs_set_option)
  int opt_count_probes = 0;              // count hash probes of the gate kernel and the row sweep
  uint64_t opt_ext_cap = 0;              // hashed sweep: first table capacity (0: sized from an estimate)
  int opt_gate_blocks = 0;   // CTAs of the gate kernel (0: whole device)
  int opt_gate_threads = kAnsatzThreads;  // threads per gate-kernel CTA (batched instances: kAnsatzThreadsShared)
  int opt_row_clusters = 0;  // clusters of the row sweep (0: as many as fit)

  // adjoint: checkpoints, per-gate snapshots of one segment, sigma, nu, indices, gradient
  DevBuf ck_keys, ck_amps, ck_n, sn_keys, sn_amps, sn_n, sigma, nu0, nu1, atab0, atab1, dth;
  DevBuf prb;  // swcs_sigma_at: requested alpha strings, ranges, beta ranks and outputs
  DevBuf ab_cnt, ab_list;  // screened sweep: selected alpha-beta doubles per alpha pair
  DevBuf selhist;          // gate kernel: radix-select histograms (two sets of 12 passes x 4096 bins)
  int opt_screen_scatter = 1;  // a subset sweep marks and scatters only what the selected operators read
  bool screen_now = false;     // set around a subset sweep whose lists are built

  // external sigma table
  DevBuf ext;
  uint64_t ext_cap = 0;
  double ext_distinct_last = 0.0;
  int64_t stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  // pinned host staging
  void* pin = nullptr;
  size_t pin_bytes = 0;

  // per-kernel event timing (swcs_profile_*) and launch count
  bool prof = false;
  struct Ev {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Ev> ev_pending;
  std::vector<cudaEvent_t> ev_free;
  double prof_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int64_t prof_n[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int64_t launches = 0;
};

namespace {

// Layout of the small control block on the device.
struct Ctrl {
  long long n_state;
  int tab_cur;
  int err;
  GridBar bar;
  unsigned long long ctr[12];
  long long stats[8];
  double acc[2];
  double eout[2];
  unsigned long long n_distinct;
  double ovl[3];  // swcs_overlap: <state|given>, <given|given>, <state|state>
  unsigned long long probes[4];  // hash probes: gate lookups, their slots, row-sweep lookups, their slots
  unsigned row_next;  // the row sweep's next target
};

int fail(swcs_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int cuda_fail(swcs_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SWCS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);   \
  } while (0)

int ensure(swcs_ctx* c, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return SWCS_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SWCS_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return SWCS_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

int ensure_pinned(swcs_ctx* c, size_t bytes) {
  if (c->pin_bytes >= bytes) return SWCS_OK;
  if (c->pin) cudaFreeHost(c->pin);
  c->pin = nullptr;
  c->pin_bytes = 0;
  if (cudaMallocHost(&c->pin, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SWCS_ERR_OOM, "pinned host allocation of %zu bytes failed", bytes);
  }
  c->pin_bytes = bytes;
  return SWCS_OK;
}

Ctrl* ctrl(swcs_ctx* c) { return (Ctrl*)c->ctrl.p; }

// Kernel kinds for swcs_profile_read.
enum Kind { kKAnsatz = 0, kKEnergy = 1, kKScatter = 2, kKGather = 3, kKClear = 4, kKOther = 5, kKRow = 6, kKGroup = 7, kKAdjoint = 8 };

cudaEvent_t take_event(swcs_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launches one kernel through `launch`, counting it and, when profiling is
// on, bracketing it with events on the context's stream.
template <class F>
cudaError_t launch_k(swcs_ctx* c, int kind, F&& launch) {
  c->launches++;
  if (!c->prof) return launch();
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (a) cudaEventRecord(a, c->st);
  cudaError_t e = launch();
  if (b) cudaEventRecord(b, c->st);
  if (a && b) c->ev_pending.push_back({kind, a, b});
  return e;
}

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Reads the device error word and maps it to a status (synchronises).
int check_device(swcs_ctx* c, const char* where) {
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  int derr = 0;
  CK(cudaMemcpy(&derr, &ctrl(c)->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (derr == 0) return SWCS_OK;
  int zero = 0;
  CK(cudaMemcpy(&ctrl(c)->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
  c->have_state = false;
  if (derr == kDevTimeout) return fail(c, SWCS_ERR_TIMEOUT, "%s: a device-side wait timed out", where);
  if (derr == kDevTableFull) return fail(c, SWCS_ERR_TABLE_FULL, "%s: a device hash table or buffer overflowed", where);
  return fail(c, SWCS_ERR_CUDA, "%s: device reported error %d", where, derr);
}

HamDev ham_dev(swcs_ctx* c) {
  HamDev H;
  H.n = c->n;
  H.ne = c->ne;
  H.no = c->no;
  H.nv = c->nv;
  H.npairs = c->npairs;
  H.h = (const double*)c->h.p;
  H.J = (const double*)c->J.p;
  H.Ws = (const double*)c->Ws.p;
  H.G = (const double*)c->G.p;
  H.opd = (const int*)c->opd.p;
  H.ops1 = (const int*)c->ops1.p;
  H.pool_size = c->pool_size;
  return H;
}

StateDev state_dev(swcs_ctx* c) {
  StateDev S;
  S.keys = (const uint64_t*)c->keys_a.p;
  S.amps = (const double*)c->amps_a.p;
  S.n = &ctrl(c)->n_state;
  S.tab = (const IdxSlot*)(c->tab_cur ? c->tab1.p : c->tab0.p);
  S.tab_mask = c->tab_mask;
  return S;
}

// Canonical generalized singles and doubles pool and its (pair, pair) index tables.
void build_pool(swcs_ctx* c, std::vector<int>& opd, std::vector<int>& ops1) {
  const int n = c->n, np = c->npairs;
  c->pool_ops.clear();
  ops1.assign((size_t)n * n, -1);
  opd.assign((size_t)np * np, -1);
  int64_t k = 0;
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q)
      if ((p & 1) == (q & 1)) {
        ops1[(size_t)p * n + q] = (int)k++;
        c->pool_ops.insert(c->pool_ops.end(), {1, (uint8_t)p, (uint8_t)q, 0, 0});
      }
  for (int a = 0; a < np; ++a) {
    int p = 0, base = 0;
    while (base + (n - 1 - p) <= a) { base += n - 1 - p; ++p; }
    const int q = p + 1 + (a - base);
    for (int b = a + 1; b < np; ++b) {
      int r = 0, bb = 0;
      while (bb + (n - 1 - r) <= b) { bb += n - 1 - r; ++r; }
      const int s = r + 1 + (b - bb);
      if (r == p || r == q || s == p || s == q) continue;
      if ((p & 1) + (q & 1) != (r & 1) + (s & 1)) continue;
      opd[(size_t)a * np + b] = (int)k++;
      c->pool_ops.insert(c->pool_ops.end(), {2, (uint8_t)p, (uint8_t)q, (uint8_t)r, (uint8_t)s});
    }
  }
  c->pool_size = k;
}

int validate_ops(swcs_ctx* c, const uint8_t* ops, int n_ops) {
  for (int g = 0; g < n_ops; ++g) {
    const uint8_t* o = ops + 5 * g;
    const int kind = o[0];
    if (kind == 1) {
      if (o[1] >= c->n || o[2] >= c->n || o[1] == o[2] || ((o[1] ^ o[2]) & 1))
        return fail(c, SWCS_ERR_INVALID_ARG, "op %d: invalid single (%d -> %d)", g, o[1], o[2]);
    } else if (kind == 2) {
      const int i0 = o[1], i1 = o[2], i2 = o[3], i3 = o[4];
      if (i0 >= c->n || i1 >= c->n || i2 >= c->n || i3 >= c->n)
        return fail(c, SWCS_ERR_INVALID_ARG, "op %d: index out of range", g);
      if (i0 == i1 || i2 == i3 || i0 == i2 || i0 == i3 || i1 == i2 || i1 == i3)
        return fail(c, SWCS_ERR_INVALID_ARG, "op %d: annihilated and created indices must be distinct", g);
      if ((i0 & 1) + (i1 & 1) != (i2 & 1) + (i3 & 1))
        return fail(c, SWCS_ERR_INVALID_ARG, "op %d: does not conserve S_z", g);
    } else {
      return fail(c, SWCS_ERR_INVALID_ARG, "op %d: kind must be 1 or 2", g);
    }
  }
  return SWCS_OK;
}

// Sizes the state buffers for at most max_state determinants.
int ensure_state_buffers(swcs_ctx* c, int64_t max_state) {
  const int64_t cap = 2 * std::max<int64_t>(max_state, 1) + 64;
  const uint64_t tcap = pow2_at_least((uint64_t)std::max<int64_t>(2 * max_state, 64));
  if (cap > c->cap || tcap - 1 != c->tab_mask) {
    // keep the current state when growing
    int r;
    DevBuf nk, na;
    if ((r = ensure(c, nk, cap * 8))) return r;
    if ((r = ensure(c, na, cap * 8))) { release(nk); return r; }
    if (c->have_state && c->keys_a.p) {
      long long ns = 0;
      CK(cudaMemcpyAsync(&ns, &ctrl(c)->n_state, 8, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      ns = std::min<long long>(ns, cap);
      CK(cudaMemcpyAsync(nk.p, c->keys_a.p, ns * 8, cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(na.p, c->amps_a.p, ns * 8, cudaMemcpyDeviceToDevice, c->st));
      CK(cudaStreamSynchronize(c->st));
    }
    release(c->keys_a);
    release(c->amps_a);
    c->keys_a = nk;
    c->amps_a = na;
    if ((r = ensure(c, c->keys_b, cap * 8))) return r;
    if ((r = ensure(c, c->amps_b, cap * 8))) return r;
    if ((r = ensure(c, c->tab0, tcap * sizeof(IdxSlot)))) return r;
    if ((r = ensure(c, c->tab1, tcap * sizeof(IdxSlot)))) return r;
    c->cap = cap;
    c->tab_mask = tcap - 1;
  }
  return ensure(c, c->selhist, kAnsatzHistWords * 4);  // the gate kernel's select histograms
}

int64_t max_state_for(swcs_ctx* c, int64_t n_keep, int n_ops, int64_t n_now) {
  double bound = c->fci_dim;
  if (n_ops < 60) bound = std::min(bound, (double)n_now * std::ldexp(1.0, n_ops));
  if (n_keep > 0) bound = std::min(bound, (double)n_keep);
  bound = std::max(bound, (double)n_now);
  return (int64_t)bound;
}

// keep_zeros: determinants a gate reaches with an exactly zero amplitude stay
// in the kept set (ranked below every nonzero |c|) unless a criterion cuts
// them -- the projectors of the adjoint need them (a partner at theta = 0 has
// c = 0 but a nonzero derivative); the magnitude criterion still drops them.
// The gate kernel's arguments for this context (no launch).
AnsatzArgs gate_args(swcs_ctx* c, const uint8_t* d_ops, const double* d_cs, int n_ops, int64_t n_keep, bool reset,
                     uint64_t* snap_keys, double* snap_amps, long long* snap_n, int64_t snap_stride, bool keep_zeros) {
  AnsatzArgs a{};
  a.keys_a = (uint64_t*)c->keys_a.p;
  a.amps_a = (double*)c->amps_a.p;
  a.keys_b = (uint64_t*)c->keys_b.p;
  a.amps_b = (double*)c->amps_b.p;
  a.cap = c->cap;
  a.tab[0] = (IdxSlot*)c->tab0.p;
  a.tab[1] = (IdxSlot*)c->tab1.p;
  a.tab_mask = c->tab_mask;
  a.tab_cur = 0;
  a.ops = d_ops;
  a.cs = d_cs;
  a.n_ops = n_ops;
  a.n_keep = n_keep;
  {  // |c| >= eps <=> abs bit pattern >= eps's bit pattern (IEEE-754 order of non-negative doubles)
    uint64_t eb = 0;
    std::memcpy(&eb, &c->trunc_eps, 8);
    a.min_abs_bits = (c->trunc_eps > 0.0) ? eb : (keep_zeros ? 0ull : 1ull);
  }
  a.reset_to_hf = reset ? 1 : 0;
  a.hf = (c->ne >= 64) ? ~0ull : ((1ull << c->ne) - 1ull);
  Ctrl* k = ctrl(c);
  a.n_state = &k->n_state;
  a.tab_cur_out = &k->tab_cur;
  a.ctr = k->ctr;
  a.hist = (unsigned*)c->selhist.p;
  a.bar = &k->bar;
  a.err = &k->err;
  a.timeout_ns = c->opt_timeout_ns;
  a.skip_arrive_block = c->opt_skip_arrive;
  a.probe_ctr = c->opt_count_probes ? &k->probes[0] : nullptr;
  a.snap_keys = snap_keys;
  a.snap_amps = snap_amps;
  a.snap_n = snap_n;
  a.snap_stride = snap_stride;
  a.stats = k->stats;
  return a;
}

int run_gates(swcs_ctx* c, const uint8_t* d_ops, const double* d_cs, int n_ops, int64_t n_keep, bool reset,
              uint64_t* snap_keys = nullptr, double* snap_amps = nullptr, long long* snap_n = nullptr,
              int64_t snap_stride = 0, bool keep_zeros = false) {
  const int gthreads = c->opt_gate_threads;
  const int bps = ansatz_blocks_per_sm(gthreads);
  if (bps <= 0) return fail(c, SWCS_ERR_NO_DEVICE, "ansatz kernel cannot be resident on this device");
  if (!c->selhist.p) return fail(c, SWCS_ERR_CUDA, "gate kernel histograms not allocated");
  const AnsatzArgs a = gate_args(c, d_ops, d_cs, n_ops, n_keep, reset, snap_keys, snap_amps, snap_n, snap_stride,
                                 keep_zeros);
  Ctrl* k = ctrl(c);
  // barrier words must start at zero
  CK(cudaMemsetAsync(&k->bar, 0, sizeof(GridBar), c->st));
  int nblocks = c->nsm * bps;
  if (c->opt_gate_blocks > 0) {
    nblocks = std::min(nblocks, c->opt_gate_blocks);
  } else {  // small states: about two entries per thread, since every grid barrier costs per CTA
    const int64_t want = (c->cap + 2 * gthreads - 1) / (2 * gthreads);
    nblocks = (int)std::max<int64_t>(std::min<int64_t>(nblocks, want), std::min(nblocks, 8));
  }
  CK(launch_k(c, kKAnsatz, [&] { return launch_ansatz(a, nblocks, gthreads, c->st); }));
  // the kernel builds its input index in tab[0], swaps per gate and writes the output's plain table into the other
  c->tab_cur = (int)((((unsigned)n_ops) & 1u) ^ 1u);
  c->have_state = true;
  c->n_state_host = -1;
  return SWCS_OK;
}

int need_ham(swcs_ctx* c) {
  if (!c) return SWCS_ERR_INVALID_ARG;
  if (!c->have_ham) return fail(c, SWCS_ERR_INVALID_ARG, "no Hamiltonian loaded");
  return SWCS_OK;
}

int need_state(swcs_ctx* c) {
  int r = need_ham(c);
  if (r) return r;
  if (!c->have_state) return fail(c, SWCS_ERR_INVALID_ARG, "no state: call swcs_apply_ansatz or swcs_set_state");
  return SWCS_OK;
}

int64_t host_state_size(swcs_ctx* c) {
  if (c->n_state_host >= 0) return c->n_state_host;
  long long ns = 0;
  if (cudaMemcpyAsync(&ns, &ctrl(c)->n_state, 8, cudaMemcpyDeviceToHost, c->st) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return -1;
  c->n_state_host = ns;
  return ns;
}

// Energies and sweeps need at least one determinant.  A state can be empty
// after swcs_set_state with no nonzero amplitude, or after the magnitude
// criterion removed every determinant (count-only truncation keeps the norm).
// The size is read back (one synchronisation) unless already known; the
// sweeps read it anyway to size their launches.
int need_nonempty(swcs_ctx* c) {
  int r = need_state(c);
  if (r) return r;
  const int64_t n = host_state_size(c);
  if (n < 0) return fail(c, SWCS_ERR_CUDA, "cannot read state size");
  if (n == 0) return fail(c, SWCS_ERR_INVALID_ARG, "the state is empty (no determinant with a kept amplitude)");
  return SWCS_OK;
}

int upload_ops(swcs_ctx* c, const uint8_t* h_ops, const double* h_theta, int n_ops) {
  int r;
  if ((r = ensure(c, c->ops_dev, (size_t)5 * n_ops + 16))) return r;
  if ((r = ensure(c, c->cs_dev, (size_t)16 * n_ops + 16))) return r;
  const size_t nb = (size_t)5 * n_ops, cb = (size_t)16 * n_ops;
  if ((r = ensure_pinned(c, nb + cb + 64))) return r;
  CK(cudaStreamSynchronize(c->st));  // staging buffer reuse
  uint8_t* p = (uint8_t*)c->pin;
  double* cs = (double*)(p + ((nb + 15) & ~(size_t)15));
  memcpy(p, h_ops, nb);
  for (int g = 0; g < n_ops; ++g) {  // host cos/sin: one libm call per gate
    cs[2 * g] = std::cos(h_theta[g]);
    cs[2 * g + 1] = std::sin(h_theta[g]);
  }
  CK(cudaMemcpyAsync(c->ops_dev.p, p, nb, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->cs_dev.p, cs, cb, cudaMemcpyHostToDevice, c->st));
  return SWCS_OK;
}

__global__ void sincos_kernel(const double* th, double* cs, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s, co;
    sincos(th[i], &s, &co);
    cs[2 * i] = co;
    cs[2 * i + 1] = s;
  }
}

// Alpha-string row sweep; returns 1 when not applicable (caller falls back).
// nd_bound >= 0: size buffers for that many determinants instead of reading
// the state size (no host synchronisation); enqueue = false: only size.
// Device arrays of a sigma probe (swcs_sigma_at): alpha strings to visit, their
// ranges of requested beta ranks, and the outputs.
struct RowProbe {
  int n = 0;
  const uint32_t* x = nullptr;
  const int* off = nullptr;
  const uint32_t* rank = nullptr;
  double* out = nullptr;
};

// Arguments of the grouping kernels and of the row sweep for this context's
// buffers (alpha-string table of capacity acap); the caller sets the mode fields.
GroupArgs group_args(swcs_ctx* c, uint64_t acap) {
  Ctrl* k = ctrl(c);
  GroupArgs ga{};
  ga.keys = (const uint64_t*)c->keys_a.p;
  ga.amps = (const double*)c->amps_a.p;
  ga.n = &k->n_state;
  ga.atab = (IdxSlot*)c->atab.p;
  ga.amask = acap - 1;
  ga.n_groups = &k->n_distinct;
  ga.gid_of = (uint32_t*)c->gid_of.p;
  ga.gcount = (long long*)c->gcount.p;
  ga.goff = (long long*)c->goff.p;
  ga.gfill = (long long*)c->gfill.p;
  ga.gkey = (uint64_t*)c->gkey.p;
  ga.gamp = (double*)c->gamp.p;
  ga.grank = (uint32_t*)c->grank.p;
  ga.gorig = (uint32_t*)c->gorig.p;
  ga.rank_tab = (const uint32_t*)c->rank_tab.p;
  ga.ks = c->no;
  ga.acc = k->acc;
  return ga;
}

RowArgs row_args(swcs_ctx* c, const GroupArgs& ga, double* d_g, int max_s, int max_d, int twords, int rbeta_packed) {
  Ctrl* k = ctrl(c);
  RowArgs ra{};
  ra.H = ham_dev(c);
  ra.gkey = ga.gkey;
  ra.gamp = ga.gamp;
  ra.grank = ga.grank;
  ra.goff = ga.goff;
  ra.atab = ga.atab;
  ra.amask = ga.amask;
  ra.alpha_list = (const uint32_t*)c->alpha_list.p;
  ra.NA = c->NA;
  ra.rank_tab = ga.rank_tab;
  ra.rows = (double*)c->rows.p;
  ra.NB = c->NB;
  ra.g = d_g;
  ra.acc = k->acc;
  ra.err = &k->err;
  ra.max_ent_s = max_s;
  ra.max_ent_d = max_d;
  ra.touched_words = twords;
  ra.rbeta = (const uint32_t*)c->rbeta.p;
  ra.rbeta_packed = rbeta_packed;
  ra.gab = (const double*)c->gab.p;
  ra.kab = (const int*)c->kab.p;
  ra.gorig = (const uint32_t*)c->gorig.p;
  ra.n_groups = ga.n_groups;
  ra.n_shards = 1;
  ra.ab_cnt = (const int*)c->ab_cnt.p;
  ra.ab_list = (const uint2*)c->ab_list.p;
  return ra;
}

// A shard of the pool sweep (swcs_pool_gradients_partial_dev): target alpha strings of colex rank
// shard (mod n_shards); the gradient is left unscaled and the energy unfinished.
struct RowShard {
  int shard = 0, n_shards = 1;
};

int sweep_rows(swcs_ctx* c, double* d_g, int64_t nd_bound = -1, bool enqueue = true, const uint32_t* sel = nullptr,
               bool energy_only = false, double* sig_out = nullptr, const RowProbe* probe = nullptr,
               const RowShard* shard = nullptr) {
  const int m = c->n / 2;
  if (m > 32 || c->NB <= 0 || c->NB > (1 << 22)) return 1;
  const int64_t nd = nd_bound >= 0 ? nd_bound : host_state_size(c);
  if (nd < 0) return fail(c, SWCS_ERR_CUDA, "cannot read state size");
  Ctrl* k = ctrl(c);
  const int gsz = std::max(1, std::min(16, c->opt_cluster));
  const int ks = c->no, nvs = c->nv;
  const int ns = ks * nvs, ndb = (ks * (ks - 1) / 2) * (nvs * (nvs - 1) / 2);
  // Shared-memory layouts, best first: every CTA of a cluster holds the target's whole entry lists (each
  // stages its own share of the discovery, then the cluster merges them) or only its own share; with the
  // touched-sector bitmap (one bit per 32-byte sector, 4 entries, of the row) or clearing whole rows.
  const int t_same = 1 + ns + ndb;
  const int share_s = (ns + gsz - 1) / gsz + 1, share_d = (ndb + gsz - 1) / gsz + 1;
  const int tw_full = (int)((c->NB + 127) / 128);
  const int nthr = c->opt_threads;
  // dynamic shared memory per CTA: a 1024-thread CTA has an SM to itself, smaller CTAs share one by two
  const size_t smem_cap = nthr == 1024 ? 200 * 1024 : 96 * 1024;
  int max_s = 0, max_d = 0, st_s = 0, st_d = 0, twords = 0;
  size_t smem = 0;
  bool fits = false;
  for (int layout = 0; layout < 4 && !fits; ++layout) {
    const bool merged = gsz > 1 && (layout & 1) == 0;
    twords = layout < 2 ? tw_full : 0;
    max_s = merged ? ns + 1 : share_s;
    max_d = merged ? ndb + 1 : share_d;
    st_s = merged ? share_s : 0;
    st_d = merged ? share_d : 0;
    smem = row_sweep_smem(max_s, max_d, st_s, st_d, t_same, twords);
    fits = smem <= smem_cap;
  }
  if (!fits) return 1;
  int ncl = 0;
  if (row_sweep_max_clusters(nthr, c->opt_row_occ, gsz, smem, &ncl) != cudaSuccess || ncl <= 0) {
    cudaGetLastError();
    return 1;
  }
  // keep the rows of all clusters within about half of L2
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->dev);
  const int64_t row_bytes = c->NB * 8;
  const int l2_rows = (int)std::max<int64_t>(1, (int64_t)l2 / 2 / std::max<int64_t>(row_bytes, 1));
  if (c->opt_rows_l2 && ncl > l2_rows) ncl = l2_rows;
  if (c->opt_row_clusters > 0 && ncl > c->opt_row_clusters) ncl = c->opt_row_clusters;
  int r;
  const uint64_t acap = pow2_at_least((uint64_t)std::max<int64_t>(2 * nd, 64));
  if ((r = ensure(c, c->atab, acap * sizeof(IdxSlot))) || (r = ensure(c, c->gid_of, nd * 4 + 4)) ||
      (r = ensure(c, c->gcount, nd * 8 + 8)) || (r = ensure(c, c->goff, nd * 8 + 16)) ||
      (r = ensure(c, c->gfill, nd * 8 + 8)) || (r = ensure(c, c->gkey, nd * 8 + 8)) ||
      (r = ensure(c, c->gamp, nd * 8 + 8)) || (r = ensure(c, c->grank, nd * 4 + 4)) ||
      (r = ensure(c, c->rows, (size_t)ncl * ((c->NB + 3) & ~(int64_t)3) * 8)) ||
      (r = ensure(c, c->rbeta, (size_t)std::max<int64_t>(nd, 1) * ks * nvs * 4)) ||
      (r = ensure(c, c->gorig, (size_t)std::max<int64_t>(nd, 1) * 4)))
    return r;
  if (!enqueue) return SWCS_OK;
  CK(cudaMemsetAsync(c->atab.p, 0xff, acap * sizeof(IdxSlot), c->st));
  CK(cudaMemsetAsync(c->gcount.p, 0, nd * 8 + 8, c->st));
  CK(cudaMemsetAsync(c->gfill.p, 0, nd * 8 + 8, c->st));
  CK(cudaMemsetAsync(&k->n_distinct, 0, 8, c->st));
  CK(cudaMemsetAsync(k->acc, 0, 16, c->st));
  if (!energy_only && !probe) CK(cudaMemsetAsync(d_g, 0, sizeof(double) * c->pool_size, c->st));
  CK(cudaMemsetAsync(c->rows.p, 0, (size_t)ncl * ((c->NB + 3) & ~(int64_t)3) * 8, c->st));  // rows padded to 32 B
  const GroupArgs ga = group_args(c, acap);
  CK(launch_k(c, kKGroup, [&] { return launch_group_state(ga, c->st); }));
  c->launches += 4;  // five grouping kernels in one call
  // beta-single entries carry the spatial pair i * m + j too when ranks fit 21 bits and pairs 10
  const int rbeta_packed = c->NB <= (1 << 21) && m <= 32 ? 1 : 0;
  CK(launch_k(c, kKGroup, [&] {
    return launch_rbeta(ga.gkey, ga.n, ga.rank_tab, ks, nvs, m, rbeta_packed, (uint32_t*)c->rbeta.p, c->st);
  }));
  RowArgs ra = row_args(c, ga, d_g, max_s, max_d, twords, rbeta_packed);
  ra.stage_ent_s = st_s;
  ra.stage_ent_d = st_d;
  ra.target_ctr = &k->row_next;
  CK(cudaMemsetAsync(&k->row_next, 0, sizeof(unsigned), c->st));
  ra.sel_bits = sel;
  ra.energy_only = energy_only ? 1 : 0;
  ra.sig_out = sig_out;
  ra.n_probe = probe ? probe->n : 0;
  ra.probe_x = probe ? probe->x : nullptr;
  ra.probe_off = probe ? probe->off : nullptr;
  ra.probe_rank = probe ? probe->rank : nullptr;
  ra.probe_out = probe ? probe->out : nullptr;
  ra.shard = shard ? shard->shard : 0;
  ra.n_shards = shard ? shard->n_shards : 1;
  ra.screen = (sel && c->screen_now && twords > 0) ? 1 : 0;
  ra.probe_ctr = c->opt_count_probes ? &k->probes[2] : nullptr;
  CK(launch_k(c, kKRow, [&] { return launch_row_sweep(ra, nthr, c->opt_row_occ, gsz, ncl, smem, c->st); }));
  c->stats[2] = 0;
  c->stats[3] = ncl;
  c->stats[4] = (int64_t)ncl * c->NB;
  if (probe || shard) return SWCS_OK;
  if (!energy_only) CK(launch_k(c, kKOther, [&] { return launch_scale_gradient(d_g, c->pool_size, k->acc, c->st); }));
  CK(launch_k(c, kKOther, [&] { return launch_finalize_energy(k->acc, k->eout, c->st); }));
  return SWCS_OK;
}

// Energy (and optionally sigma_D in state order) through the row machinery;
// 1 when not applicable.
int energy_rows(swcs_ctx* c, double* sig_out) {
  if (c->opt_energy == 1) return 1;
  return sweep_rows(c, nullptr, -1, true, nullptr, true, sig_out);
}

int sweep(swcs_ctx* c, double* d_g, const uint32_t* sel = nullptr) {
  if (c->opt_sweep != 1) {
    const int r = sweep_rows(c, d_g, -1, true, sel);
    if (r != 1) return r;
    if (c->opt_sweep == 2) return fail(c, SWCS_ERR_INVALID_ARG, "row sweep not applicable to this sector");
  }
  const HamDev H = ham_dev(c);
  const StateDev S = state_dev(c);
  Ctrl* k = ctrl(c);
  const int nblk = c->nsm * sigma_blocks_per_sm();
  const int64_t nd = host_state_size(c);
  if (nd < 0) return fail(c, SWCS_ERR_CUDA, "cannot read state size");
  const double nconn = 2.0 * c->no * c->nv + 2.0 * binom(c->no, 2) * binom(c->nv, 2) + (double)c->no * c->no * c->nv * c->nv;
  double est = c->ext_distinct_last > 0 ? 1.25 * c->ext_distinct_last : std::min((double)nd * (nconn + 1.0), c->fci_dim);
  est = std::min(est, c->fci_dim);
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  const double budget = 0.80 * ((double)free_b + (double)c->ext.bytes);
  uint64_t cmax = 1;
  while ((double)(cmax * 2) * sizeof(ValSlot) <= budget) cmax <<= 1;
  const double load = 0.6;
  unsigned lb = 0;
  while (est / (double)(1u << lb) > load * (double)cmax && lb < 20) ++lb;
  for (int attempt = 0; attempt < 8; ++attempt) {
    const double per_bucket = est / (double)(1u << lb);
    uint64_t cap = pow2_at_least((uint64_t)std::max(1024.0, per_bucket / load));
    if (attempt == 0 && c->opt_ext_cap) {
      cap = pow2_at_least(c->opt_ext_cap);
      est = std::min(est, 0.5 * load * (double)cap);
      lb = 0;
    }
    cap = std::min(cap, cmax);
    if (c->ext_cap < cap) {
      release(c->ext);
      int r = ensure(c, c->ext, cap * sizeof(ValSlot));
      if (r) return r;
      c->ext_cap = cap;
    }
    if (!(attempt == 0 && c->opt_ext_cap))
      cap = std::min<uint64_t>(c->ext_cap, pow2_at_least((uint64_t)std::max(1024.0, per_bucket / load)));
    cap = std::min(cap, c->ext_cap);
    CK(cudaMemsetAsync(d_g, 0, sizeof(double) * c->pool_size, c->st));
    CK(cudaMemsetAsync(k->acc, 0, sizeof(double) * 2, c->st));
    bool overflow = false;
    double total_distinct = 0.0;
    for (unsigned b = 0; b < (1u << lb) && !overflow; ++b) {
      ExtTable T;
      T.slots = (ValSlot*)c->ext.p;
      T.mask = cap - 1;
      T.nbucket_log2 = lb;
      T.bucket = b;
      T.n_distinct = &k->n_distinct;
      T.err = &k->err;
      CK(launch_k(c, kKClear, [&] { return launch_clear_ext(T.slots, cap, c->st); }));
      CK(cudaMemsetAsync(&k->n_distinct, 0, 8, c->st));
      CK(launch_k(c, kKScatter, [&] { return launch_sigma_scatter(H, S, T, nblk, c->st); }));
      unsigned long long nd_b = 0;
      CK(cudaMemcpyAsync(&nd_b, &k->n_distinct, 8, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      int derr = 0;
      CK(cudaMemcpy(&derr, &k->err, sizeof(int), cudaMemcpyDeviceToHost));
      if (derr == kDevTableFull || (double)nd_b > 0.85 * (double)cap) {
        int zero = 0;
        CK(cudaMemcpy(&k->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        overflow = true;
        break;
      }
      if (derr) return check_device(c, "pool sweep (scatter)");
      total_distinct += (double)nd_b;
      CK(launch_k(c, kKGather, [&] { return launch_pool_gather(H, S, T, d_g, k->acc, b == 0, nblk, c->st); }));
    }
    if (overflow) {
      est = std::max(est * 4.0, 2.0 * (double)cap);
      while (est / (double)(1u << lb) > load * (double)cmax && lb < 20) ++lb;
      continue;
    }
    c->ext_distinct_last = total_distinct;
    c->stats[2] = (int64_t)total_distinct;
    c->stats[3] = (int64_t)(1u << lb);
    c->stats[4] = (int64_t)cap;
    CK(launch_k(c, kKOther, [&] { return launch_scale_gradient(d_g, c->pool_size, k->acc, c->st); }));
    CK(launch_k(c, kKOther, [&] { return launch_finalize_energy(k->acc, k->eout, c->st); }));
    return SWCS_OK;
  }
  return fail(c, SWCS_ERR_TABLE_FULL, "external sigma table could not be sized (device memory too small)");
}

}  // namespace

namespace swcs {

// Used by swcs_energy_noalloc (its own translation unit): the loaded
// Hamiltonian, the context's stream, the energy kernel's grid size and the
// device the context was created on.
int ctx_ham_for_noalloc(swcs_ctx* c, HamDev* H, cudaStream_t* st, int* nblocks, int* dev) {
  const int r = need_ham(c);
  if (r) return r;
  *H = ham_dev(c);
  *st = c->st;
  *nblocks = c->nsm * sigma_blocks_per_sm();
  *dev = c->dev;
  return SWCS_OK;
}

int ctx_fail_for_noalloc(swcs_ctx* c, int code, const char* msg) { return fail(c, code, "%s", msg); }

}  // namespace swcs

// =============================================================================
extern "C" {

int swcs_create(swcs_ctx** out, void* cuda_stream) {
  if (!out) return SWCS_ERR_INVALID_ARG;
  *out = nullptr;
  swcs_ctx* c = new swcs_ctx();
  c->st = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->dev) != cudaSuccess) { delete c; return SWCS_ERR_NO_DEVICE; }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->dev) != cudaSuccess) { delete c; return SWCS_ERR_NO_DEVICE; }
  if (prop.major != 10 || prop.minor != 3) {
    cudaGetLastError();
    delete c;
    return SWCS_ERR_NO_DEVICE;
  }
  c->nsm = prop.multiProcessorCount;
  if (ensure(c, c->ctrl, sizeof(Ctrl)) != SWCS_OK) { delete c; return SWCS_ERR_OOM; }
  if (cudaMemset(c->ctrl.p, 0, sizeof(Ctrl)) != cudaSuccess) { delete c; return SWCS_ERR_CUDA; }
  *out = c;
  return SWCS_OK;
}

int swcs_destroy(swcs_ctx* c) {
  if (!c) return SWCS_OK;
  cudaStreamSynchronize(c->st);
  DevBuf* bufs[] = {&c->h, &c->J, &c->Ws, &c->G, &c->opd, &c->ops1, &c->gstage, &c->keys_a, &c->amps_a,
                    &c->keys_b, &c->amps_b, &c->tab0, &c->tab1, &c->ctrl, &c->ops_dev, &c->cs_dev,
                    &c->gdev, &c->subset_dev, &c->gsub, &c->ovl_keys, &c->ovl_amps, &c->ext, &c->alpha_list,
                    &c->rank_tab, &c->atab,
                    &c->gid_of, &c->gcount, &c->goff, &c->gfill, &c->gkey, &c->gamp, &c->grank, &c->rows,
                    &c->rbeta, &c->gab, &c->kab, &c->gorig,
                    &c->ck_keys, &c->ck_amps, &c->ck_n, &c->sn_keys, &c->sn_amps, &c->sn_n, &c->sigma, &c->nu0,
                    &c->nu1, &c->atab0, &c->atab1, &c->dth, &c->pool_dev, &c->selbits, &c->feat,
                    &c->ypred, &c->topk_hist, &c->topk_ctl, &c->occ, &c->prb, &c->ab_cnt, &c->ab_list,
                    &c->selhist};
  for (DevBuf* b : bufs) release(*b);
  if (c->pin) cudaFreeHost(c->pin);
  for (auto& e : c->ev_pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  delete c;
  return SWCS_OK;
}

const char* swcs_last_error(const swcs_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

int swcs_load_hamiltonian(swcs_ctx* c, const double* h_h, const double* h_g, int n_so, int n_elec) {
  if (!c) return SWCS_ERR_INVALID_ARG;
  if (!h_h || !h_g) return fail(c, SWCS_ERR_INVALID_ARG, "null integral pointer");
  if (n_so < 4 || n_so > 64 || (n_so & 1)) return fail(c, SWCS_ERR_INVALID_ARG, "n_so must be even, 4..64 (got %d)", n_so);
  if (n_elec < 2 || n_elec >= n_so || (n_elec & 1))
    return fail(c, SWCS_ERR_INVALID_ARG, "n_elec must be even with 2 <= n_elec < n_so (got %d)", n_elec);
  const int n = n_so;
  c->n = n;
  c->ne = n_elec;
  c->no = n_elec / 2;
  c->nv = n / 2 - c->no;
  c->npairs = n * (n - 1) / 2;
  c->fci_dim = binom(n / 2, c->no) * binom(n / 2, c->no);
  const size_t n2 = (size_t)n * n, n3 = n2 * n, n4 = n3 * n, np2 = (size_t)c->npairs * c->npairs;
  int r;
  if ((r = ensure(c, c->h, n2 * 8)) || (r = ensure(c, c->J, n2 * 8)) || (r = ensure(c, c->Ws, n3 * 8)) ||
      (r = ensure(c, c->G, np2 * 8)) || (r = ensure(c, c->opd, np2 * 4)) || (r = ensure(c, c->ops1, n2 * 4)) ||
      (r = ensure(c, c->gstage, n4 * 8)))
    return r;
  CK(cudaMemcpyAsync(c->h.p, h_h, n2 * 8, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->gstage.p, h_g, n4 * 8, cudaMemcpyHostToDevice, c->st));
  CK(launch_k(c, kKOther, [&] { return launch_pack_hamiltonian((const double*)c->gstage.p, n, (double*)c->J.p, (double*)c->Ws.p, (double*)c->G.p, c->st); }));
  std::vector<int> opd, ops1;
  build_pool(c, opd, ops1);
  {
    // alpha strings of the sector and per-byte colex rank tables of one spin
    const int m = n / 2, ks = c->no;
    std::vector<uint32_t> al;
    if (m <= 32) {
      uint64_t v = (1ull << ks) - 1ull;
      while (v < (1ull << m)) {
        al.push_back((uint32_t)v);
        const uint64_t t = v | (v - 1);
        v = (t + 1) | (((~t & -~t) - 1) >> (__builtin_ctzll(v) + 1));
      }
    }
    c->NA = (int)al.size();
    c->NB = (int64_t)al.size();
    std::vector<uint32_t> T((size_t)4 * (ks + 1) * 256, 0u);
    for (int ch = 0; ch < 4; ++ch)
      for (int j = 0; j <= ks; ++j)
        for (int byte = 0; byte < 256; ++byte) {
          int i = j;
          double r = 0.0;
          bool ok = true;
          for (int b = 0; b < 8; ++b)
            if ((byte >> b) & 1) {
              const int pos = 8 * ch + b;
              if (pos >= m || i >= ks) { ok = false; break; }
              r += binom(pos, i + 1);
              ++i;
            }
          T[((size_t)ch * (ks + 1) + j) * 256 + byte] = ok ? (uint32_t)r : 0u;
        }
    if ((r = ensure(c, c->alpha_list, al.size() * 4 + 4)) || (r = ensure(c, c->rank_tab, T.size() * 4))) return r;
    // alpha-beta double tables by spatial indices: the phase of the double on
    // any D is (beta single on D) ^ (alpha single on D) ^ e(a,b,i,j), and e
    // depends on the indices only, so it is read off a minimal determinant
    if (m <= 32) {
      const size_t m4 = (size_t)m * m * m * m;
      std::vector<double> gab(m4, 0.0);
      std::vector<int> kab(m4, -1);
      auto par_below = [](uint64_t d, int p) { return __builtin_popcountll(d & ((1ull << p) - 1ull)) & 1; };
      auto sphase = [&](uint64_t d, int a0, int c1) { return par_below(d, a0) ^ par_below(d & ~(1ull << a0), c1); };
      auto dphase = [&](uint64_t d, int p, int q, int rr, int ss) {
        int par = par_below(d, p);
        uint64_t x = d & ~(1ull << p);
        par ^= par_below(x, q);
        x &= ~(1ull << q);
        par ^= par_below(x, ss);
        x |= (1ull << ss);
        par ^= par_below(x, rr);
        return par;
      };
      const size_t n1 = (size_t)n;
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
          if (a == b) continue;
          for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
              if (i == j) continue;
              const int A2 = 2 * a, B2 = 2 * b, I1 = 2 * i + 1, J1 = 2 * j + 1;
              const int p = std::min(A2, I1), q = std::max(A2, I1), rr = std::min(B2, J1), ss = std::max(B2, J1);
              const uint64_t d0 = (1ull << A2) | (1ull << I1);
              const int e = dphase(d0, p, q, rr, ss) ^ sphase(d0, I1, J1) ^ sphase(d0, A2, B2);
              const double v = h_g[((rr * n1 + ss) * n1 + p) * n1 + q];  // <rs||pq>
              const size_t ti = (((size_t)a * m + b) * m + i) * m + j;
              gab[ti] = e ? -v : v;
              const int pa = pair_index(p, q, n), pb = pair_index(rr, ss, n);
              const bool down = pa > pb;
              const int k = down ? opd[(size_t)pb * c->npairs + pa] : opd[(size_t)pa * c->npairs + pb];
              kab[ti] = k | (int)((unsigned)(e ^ (int)down) << 31);
            }
        }
      if ((r = ensure(c, c->gab, m4 * 8)) || (r = ensure(c, c->kab, m4 * 4))) return r;
      CK(cudaMemcpyAsync(c->gab.p, gab.data(), m4 * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(c->kab.p, kab.data(), m4 * 4, cudaMemcpyHostToDevice, c->st));
      CK(cudaStreamSynchronize(c->st));
    }
    if (!al.empty()) CK(cudaMemcpyAsync(c->alpha_list.p, al.data(), al.size() * 4, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->rank_tab.p, T.data(), T.size() * 4, cudaMemcpyHostToDevice, c->st));
  }
  CK(cudaMemcpyAsync(c->opd.p, opd.data(), np2 * 4, cudaMemcpyHostToDevice, c->st));
  if ((r = ensure(c, c->pool_dev, c->pool_ops.size() + 16))) return r;
  CK(cudaMemcpyAsync(c->pool_dev.p, c->pool_ops.data(), c->pool_ops.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->ops1.p, ops1.data(), n2 * 4, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->have_ham = true;
  c->have_state = false;
  c->ext_distinct_last = 0.0;
  return SWCS_OK;
}

int swcs_pool_size(swcs_ctx* c, int64_t* n_out) {
  int r = need_ham(c);
  if (r) return r;
  if (!n_out) return fail(c, SWCS_ERR_INVALID_ARG, "null output");
  *n_out = c->pool_size;
  return SWCS_OK;
}

int swcs_pool_ops(swcs_ctx* c, uint8_t* out) {
  int r = need_ham(c);
  if (r) return r;
  if (!out) return fail(c, SWCS_ERR_INVALID_ARG, "null output");
  memcpy(out, c->pool_ops.data(), c->pool_ops.size());
  return SWCS_OK;
}

// Spin complement of every pool operator (Sec. III uses spin-complemented
// operators for the closed-shell molecules): spin-orbital p = 2i + s maps to
// 2i + (1 - s).  The flipped generator equals sign[k] times the generator of
// pool operator partner[k]; it is found as the flipped string brought to the
// pool's index order, or as the adjoint of a pool operator (then the
// generator changes sign).
int swcs_pool_spin_pairs(swcs_ctx* c, int64_t* partner, int8_t* sign) {
  int r = need_ham(c);
  if (r) return r;
  if (!partner || !sign) return fail(c, SWCS_ERR_INVALID_ARG, "null output");
  auto pack = [](int kind, int a, int b, int x, int y) {
    return ((uint64_t)kind << 32) | ((uint64_t)a << 24) | ((uint64_t)b << 16) | ((uint64_t)x << 8) | (uint64_t)y;
  };
  std::unordered_map<uint64_t, int64_t> at;
  at.reserve((size_t)c->pool_size * 2);
  for (int64_t k = 0; k < c->pool_size; ++k) {
    const uint8_t* o = &c->pool_ops[(size_t)5 * k];
    at.emplace(pack(o[0], o[1], o[2], o[3], o[4]), k);
  }
  for (int64_t k = 0; k < c->pool_size; ++k) {
    const uint8_t* o = &c->pool_ops[(size_t)5 * k];
    int p = o[1] ^ 1, q = o[2] ^ 1, x = o[3] ^ 1, y = o[4] ^ 1, sg = 1;
    auto it = at.end();
    if (o[0] == 1) {
      it = at.find(pack(1, p, q, 0, 0));  // same spin: the flip keeps p < q
    } else {
      if (p > q) { std::swap(p, q); sg = -sg; }  // a_q a_p with p < q
      if (x > y) { std::swap(x, y); sg = -sg; }  // a+_x a+_y with x < y
      it = at.find(pack(2, p, q, x, y));
      if (it == at.end()) {
        it = at.find(pack(2, x, y, p, q));  // adjoint of a pool operator
        sg = -sg;
      }
    }
    if (it == at.end()) return fail(c, SWCS_ERR_INVALID_ARG, "pool operator %lld has no spin complement", (long long)k);
    partner[k] = it->second;
    sign[k] = (int8_t)sg;
  }
  return SWCS_OK;
}

// MP2-ordered UCCSD ansatz (Sec. II.A): doubles i<j -> a<b of the reference with
// their first-order amplitudes, largest |t| first (stable: equal |t| keep the
// canonical order), then the singles at zero.
int swcs_mp2_uccsd(swcs_ctx* c, uint8_t* h_ops, double* h_theta, int64_t cap, int64_t* n_out) {
  int r = need_ham(c);
  if (r) return r;
  const int n = c->n, ne = c->ne;
  std::vector<uint8_t> ijab;
  for (int i = 0; i < ne; ++i)
    for (int j = i + 1; j < ne; ++j)
      for (int a = ne; a < n; ++a)
        for (int b = a + 1; b < n; ++b)
          if ((i & 1) + (j & 1) == (a & 1) + (b & 1))
            ijab.insert(ijab.end(), {(uint8_t)i, (uint8_t)j, (uint8_t)a, (uint8_t)b});
  std::vector<uint8_t> singles;
  for (int i = 0; i < ne; ++i)
    for (int a = ne; a < n; ++a)
      if ((i & 1) == (a & 1)) singles.insert(singles.end(), {(uint8_t)i, (uint8_t)a});
  const int64_t nd = (int64_t)ijab.size() / 4, ns = (int64_t)singles.size() / 2;
  if (n_out) *n_out = nd + ns;
  if (!h_ops || !h_theta || cap < nd + ns) return SWCS_OK;
  std::vector<double> t(nd);
  if (nd > 0) {
    if ((r = ensure(c, c->gsub, ijab.size())) || (r = ensure(c, c->subset_dev, (size_t)nd * 8))) return r;
    CK(cudaMemcpyAsync(c->gsub.p, ijab.data(), ijab.size(), cudaMemcpyHostToDevice, c->st));
    CK(launch_k(c, kKOther, [&] {
      return launch_mp2(ham_dev(c), (const uint8_t*)c->gsub.p, nd, (double*)c->subset_dev.p, c->st);
    }));
    CK(cudaMemcpyAsync(t.data(), c->subset_dev.p, (size_t)nd * 8, cudaMemcpyDeviceToHost, c->st));
    if ((r = check_device(c, "swcs_mp2_uccsd"))) return r;
  }
  std::vector<int64_t> ord(nd);
  for (int64_t q = 0; q < nd; ++q) ord[q] = q;
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return std::fabs(t[x]) > std::fabs(t[y]); });
  for (int64_t q = 0; q < nd; ++q) {
    const uint8_t* e = &ijab[4 * ord[q]];
    uint8_t* o = h_ops + 5 * q;
    o[0] = 2; o[1] = e[0]; o[2] = e[1]; o[3] = e[2]; o[4] = e[3];
    h_theta[q] = t[ord[q]];
  }
  for (int64_t q = 0; q < ns; ++q) {
    uint8_t* o = h_ops + 5 * (nd + q);
    o[0] = 1; o[1] = singles[2 * q]; o[2] = singles[2 * q + 1]; o[3] = 0; o[4] = 0;
    h_theta[nd + q] = 0.0;
  }
  return SWCS_OK;
}

// <state|given>, <state|state>, <given|given> and 1 - |<state|given>|^2 / (<state|state> <given|given>).
int swcs_overlap(swcs_ctx* c, const uint64_t* h_keys, const double* h_amps, int64_t n, double* out4) {
  int r = need_state(c);
  if (r) return r;
  if (!out4 || n < 0 || (n > 0 && (!h_keys || !h_amps))) return fail(c, SWCS_ERR_INVALID_ARG, "bad overlap arguments");
  if ((r = ensure(c, c->ovl_keys, (size_t)std::max<int64_t>(n, 1) * 8)) ||
      (r = ensure(c, c->ovl_amps, (size_t)std::max<int64_t>(n, 1) * 8)))
    return r;
  Ctrl* k = ctrl(c);
  if (n > 0) {
    CK(cudaMemcpyAsync(c->ovl_keys.p, h_keys, (size_t)n * 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->ovl_amps.p, h_amps, (size_t)n * 8, cudaMemcpyHostToDevice, c->st));
  }
  CK(cudaMemsetAsync(k->ovl, 0, 24, c->st));
  CK(launch_k(c, kKOther, [&] {
    return launch_overlap(state_dev(c), (const uint64_t*)c->ovl_keys.p, (const double*)c->ovl_amps.p, n, k->ovl,
                          c->nsm * 4, c->st);
  }));
  double v[3];
  CK(cudaMemcpyAsync(v, k->ovl, 24, cudaMemcpyDeviceToHost, c->st));
  if ((r = check_device(c, "swcs_overlap"))) return r;
  out4[0] = v[0];
  out4[1] = v[2];
  out4[2] = v[1];
  out4[3] = (v[1] > 0.0 && v[2] > 0.0) ? 1.0 - v[0] * v[0] / (v[2] * v[1]) : 1.0;
  return SWCS_OK;
}

static int apply_common(swcs_ctx* c, const uint8_t* h_ops, const double* h_theta, int n_ops, int64_t n_keep,
                        bool reset) {
  int r = reset ? need_ham(c) : need_state(c);
  if (r) return r;
  if (n_ops < 0 || (n_ops > 0 && (!h_ops || !h_theta))) return fail(c, SWCS_ERR_INVALID_ARG, "bad ops / theta");
  if ((r = validate_ops(c, h_ops, n_ops))) return r;
  const int64_t n_now = reset ? 1 : host_state_size(c);
  const int64_t ms = max_state_for(c, n_keep, n_ops, n_now);
  if (ms > ((int64_t)1 << 31)) return fail(c, SWCS_ERR_INVALID_ARG, "state bound %lld too large: give n_keep", (long long)ms);
  if ((r = ensure_state_buffers(c, ms))) return r;
  if (n_ops == 0 && !reset) return SWCS_OK;
  if ((r = upload_ops(c, h_ops, h_theta, n_ops))) return r;
  if (reset) {
    long long one = 1;
    CK(cudaMemcpyAsync(&ctrl(c)->n_state, &one, 8, cudaMemcpyHostToDevice, c->st));
  }
  if (n_ops == 0) {  // reference determinant only
    const uint8_t id[5] = {0, 0, 0, 0, 0};
    const double z = 0.0;
    if ((r = upload_ops(c, id, &z, 1))) return r;
    if ((r = run_gates(c, (const uint8_t*)c->ops_dev.p, (const double*)c->cs_dev.p, 1, n_keep, true))) return r;
    return check_device(c, "swcs_apply_ansatz");
  }
  if ((r = run_gates(c, (const uint8_t*)c->ops_dev.p, (const double*)c->cs_dev.p, n_ops, n_keep, reset))) return r;
  return check_device(c, "swcs_apply_ansatz");
}

int swcs_apply_ansatz(swcs_ctx* c, const uint8_t* h_ops, const double* h_theta, int n_ops, int64_t n_keep) {
  return apply_common(c, h_ops, h_theta, n_ops, n_keep, true);
}

int swcs_apply_gates(swcs_ctx* c, const uint8_t* h_ops, const double* h_theta, int n_ops, int64_t n_keep) {
  return apply_common(c, h_ops, h_theta, n_ops, n_keep, false);
}

int swcs_apply_ansatz_dev(swcs_ctx* c, const uint8_t* d_ops, const double* d_theta, int n_ops, int64_t n_keep) {
  int r = need_ham(c);
  if (r) return r;
  if (n_ops <= 0 || !d_ops || !d_theta) return fail(c, SWCS_ERR_INVALID_ARG, "bad ops / theta");
  const int64_t ms = max_state_for(c, n_keep, n_ops, 1);
  if (ms > ((int64_t)1 << 31)) return fail(c, SWCS_ERR_INVALID_ARG, "state bound too large: give n_keep");
  if ((r = ensure_state_buffers(c, ms))) return r;
  if ((r = ensure(c, c->cs_dev, (size_t)16 * n_ops + 16))) return r;
  CK(launch_k(c, kKOther, [&] {
    sincos_kernel<<<(n_ops + 255) / 256, 256, 0, c->st>>>(d_theta, (double*)c->cs_dev.p, n_ops);
    return cudaGetLastError();
  }));
  return run_gates(c, d_ops, (const double*)c->cs_dev.p, n_ops, n_keep, true);
}

int swcs_truncate(swcs_ctx* c, int64_t n_keep) {
  int r = need_state(c);
  if (r) return r;
  const uint8_t id[5] = {0, 0, 0, 0, 0};
  const double z = 0.0;
  if ((r = upload_ops(c, id, &z, 1))) return r;
  if ((r = run_gates(c, (const uint8_t*)c->ops_dev.p, (const double*)c->cs_dev.p, 1, n_keep, false))) return r;
  return check_device(c, "swcs_truncate");
}

int swcs_energy_dev(swcs_ctx* c, double* d_out) {
  int r = need_nonempty(c);
  if (r) return r;
  Ctrl* k = ctrl(c);
  if ((r = energy_rows(c, nullptr)) != 1) {
    if (r) return r;
    if (d_out) CK(cudaMemcpyAsync(d_out, k->eout, 16, cudaMemcpyDeviceToDevice, c->st));
    return SWCS_OK;
  }
  CK(cudaMemsetAsync(k->acc, 0, 16, c->st));
  CK(launch_k(c, kKEnergy, [&] { return launch_energy(ham_dev(c), state_dev(c), k->acc, c->nsm * sigma_blocks_per_sm(), c->st); }));
  CK(launch_k(c, kKOther, [&] { return launch_finalize_energy(k->acc, d_out ? d_out : k->eout, c->st); }));
  return SWCS_OK;
}

int swcs_energy(swcs_ctx* c, double* e_out, double* n2_out) {
  int r = swcs_energy_dev(c, nullptr);
  if (r) return r;
  double out[2];
  CK(cudaMemcpyAsync(out, ctrl(c)->eout, 16, cudaMemcpyDeviceToHost, c->st));
  if ((r = check_device(c, "swcs_energy"))) return r;
  if (e_out) *e_out = out[0];
  if (n2_out) *n2_out = out[1];
  return SWCS_OK;
}

int swcs_pool_gradients_dev(swcs_ctx* c, double* d_g_out, const int64_t* d_subset, int64_t n_subset) {
  int r = need_nonempty(c);
  if (r) return r;
  if (!d_g_out) return fail(c, SWCS_ERR_INVALID_ARG, "null output");
  double* g = d_g_out;
  const uint32_t* sel = nullptr;
  if (d_subset) {
    if ((r = ensure(c, c->gdev, sizeof(double) * c->pool_size))) return r;
    g = (double*)c->gdev.p;
    if ((r = ensure(c, c->selbits, ((c->pool_size + 31) / 32) * 4 + 4))) return r;
    CK(launch_k(c, kKOther, [&] { return launch_subset_bits(d_subset, n_subset, (uint32_t*)c->selbits.p, c->pool_size, c->st); }));
    sel = (const uint32_t*)c->selbits.p;
    const int m = c->n / 2;
    if (c->opt_screen_scatter && c->kab.p && m <= 32) {  // selected alpha-beta doubles per alpha pair
      const size_t m2 = (size_t)m * m;
      if ((r = ensure(c, c->ab_cnt, m2 * 4)) || (r = ensure(c, c->ab_list, m2 * m2 * 8))) return r;
      CK(launch_k(c, kKOther, [&] {
        return launch_screen_lists((const int*)c->kab.p, m, sel, (int*)c->ab_cnt.p, (uint2*)c->ab_list.p, c->st);
      }));
      c->screen_now = true;
    }
  }
  r = sweep(c, g, sel);
  c->screen_now = false;
  if (r) return r;
  if (d_subset) CK(launch_k(c, kKOther, [&] { return launch_gather_subset(g, d_subset, n_subset, d_g_out, c->st); }));
  return SWCS_OK;
}

int swcs_pool_gradients_partial_dev(swcs_ctx* c, int shard, int n_shards, double* d_graw, double* d_acc) {
  int r = need_nonempty(c);
  if (r) return r;
  if (!d_graw || !d_acc) return fail(c, SWCS_ERR_INVALID_ARG, "null output");
  if (n_shards < 1 || shard < 0 || shard >= n_shards) return fail(c, SWCS_ERR_INVALID_ARG, "shard must be in 0..n_shards-1");
  RowShard sh;
  sh.shard = shard;
  sh.n_shards = n_shards;
  r = sweep_rows(c, d_graw, -1, true, nullptr, false, nullptr, nullptr, &sh);
  if (r == 1) return fail(c, SWCS_ERR_INVALID_ARG, "the sharded sweep needs the alpha-string row sweep (not applicable to this sector)");
  if (r) return r;
  CK(cudaMemcpyAsync(d_acc, ctrl(c)->acc, 16, cudaMemcpyDeviceToDevice, c->st));
  return SWCS_OK;
}

int swcs_pool_gradients(swcs_ctx* c, double* h_g_out, const int64_t* h_subset, int64_t n_subset) {
  int r = need_nonempty(c);
  if (r) return r;
  if (!h_g_out) return fail(c, SWCS_ERR_INVALID_ARG, "null output");
  if ((r = ensure(c, c->gdev, sizeof(double) * c->pool_size))) return r;
  if ((r = sweep(c, (double*)c->gdev.p))) return r;
  if ((r = check_device(c, "swcs_pool_gradients"))) return r;
  if (!h_subset) {
    CK(cudaMemcpy(h_g_out, c->gdev.p, sizeof(double) * c->pool_size, cudaMemcpyDeviceToHost));
  } else {
    std::vector<double> all(c->pool_size);
    CK(cudaMemcpy(all.data(), c->gdev.p, sizeof(double) * c->pool_size, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n_subset; ++i) {
      if (h_subset[i] < 0 || h_subset[i] >= c->pool_size) return fail(c, SWCS_ERR_INVALID_ARG, "subset index out of range");
      h_g_out[h_subset[i]] = all[h_subset[i]];
    }
  }
  return SWCS_OK;
}

int swcs_state_size(swcs_ctx* c, int64_t* n_out) {
  int r = need_state(c);
  if (r) return r;
  const int64_t n = host_state_size(c);
  if (n < 0) return fail(c, SWCS_ERR_CUDA, "cannot read state size");
  *n_out = n;
  return SWCS_OK;
}

int swcs_get_state(swcs_ctx* c, uint64_t* keys, double* amps, int64_t cap, int64_t* n_out) {
  int r = need_state(c);
  if (r) return r;
  if ((r = check_device(c, "swcs_get_state"))) return r;
  const int64_t n = host_state_size(c);
  if (n < 0) return fail(c, SWCS_ERR_CUDA, "cannot read state size");
  if (n_out) *n_out = n;
  if (cap < n || n == 0) return SWCS_OK;
  std::vector<uint64_t> k(n);
  std::vector<double> a(n);
  CK(cudaMemcpy(k.data(), c->keys_a.p, 8 * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(a.data(), c->amps_a.p, 8 * n, cudaMemcpyDeviceToHost));
  std::vector<int64_t> ord(n);
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return k[x] < k[y]; });
  for (int64_t i = 0; i < n; ++i) {
    keys[i] = k[ord[i]];
    amps[i] = a[ord[i]];
  }
  return SWCS_OK;
}

int swcs_set_state(swcs_ctx* c, const uint64_t* keys, const double* amps, int64_t n) {
  int r = need_ham(c);
  if (r) return r;
  if (n < 0 || (n > 0 && (!keys || !amps))) return fail(c, SWCS_ERR_INVALID_ARG, "bad state arrays");
  std::vector<std::pair<uint64_t, double>> v;
  v.reserve(n);
  const uint64_t valid = (c->n >= 64) ? ~0ull : ((1ull << c->n) - 1ull);
  for (int64_t i = 0; i < n; ++i) {
    if (keys[i] & ~valid) return fail(c, SWCS_ERR_INVALID_ARG, "determinant %lld has bits >= n_so", (long long)i);
    if (__builtin_popcountll(keys[i]) != c->ne) return fail(c, SWCS_ERR_INVALID_ARG, "determinant %lld has wrong electron count", (long long)i);
    if (__builtin_popcountll(keys[i] & 0x5555555555555555ull) != c->no)
      return fail(c, SWCS_ERR_INVALID_ARG, "determinant %lld is outside the S_z = 0 sector", (long long)i);
    v.emplace_back(keys[i], amps[i]);
  }
  std::sort(v.begin(), v.end(), [](const std::pair<uint64_t, double>& x, const std::pair<uint64_t, double>& y) { return x.first < y.first; });
  std::vector<uint64_t> k;
  std::vector<double> a;
  for (size_t i = 0; i < v.size();) {
    size_t j = i;
    double s = 0.0;
    while (j < v.size() && v[j].first == v[i].first) s += v[j++].second;
    if (s != 0.0) { k.push_back(v[i].first); a.push_back(s); }
    i = j;
  }
  const int64_t m = (int64_t)k.size();
  c->have_state = false;
  if ((r = ensure_state_buffers(c, std::max<int64_t>(m, 1)))) return r;
  if (m > 0) {
    CK(cudaMemcpyAsync(c->keys_a.p, k.data(), 8 * m, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->amps_a.p, a.data(), 8 * m, cudaMemcpyHostToDevice, c->st));
  }
  long long mm = m;
  CK(cudaMemcpyAsync(&ctrl(c)->n_state, &mm, 8, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->have_state = true;
  c->n_state_host = m;
  // rebuild the index table: a truncation-free identity pass
  const uint8_t id[5] = {0, 0, 0, 0, 0};
  const double z = 0.0;
  if ((r = upload_ops(c, id, &z, 1))) return r;
  if ((r = run_gates(c, (const uint8_t*)c->ops_dev.p, (const double*)c->cs_dev.p, 1, 0, false))) return r;
  return check_device(c, "swcs_set_state");
}

int swcs_probe_counts(swcs_ctx* c, int64_t* h_out4, int reset) {
  if (!c || !h_out4) return SWCS_ERR_INVALID_ARG;
  unsigned long long v[4];
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(v, ctrl(c)->probes, sizeof v, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 4; ++i) h_out4[i] = (int64_t)v[i];
  if (reset) CK(cudaMemset(ctrl(c)->probes, 0, sizeof v));
  return SWCS_OK;
}

int swcs_stats(swcs_ctx* c, int64_t* out8) {
  if (!c || !out8) return SWCS_ERR_INVALID_ARG;
  long long dev[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  CK(cudaMemcpy(dev, ctrl(c)->stats, sizeof dev, cudaMemcpyDeviceToHost));
  out8[0] = dev[0];
  out8[1] = dev[1];
  out8[2] = c->stats[2];
  out8[3] = c->stats[3];
  out8[4] = c->stats[4];
  out8[5] = c->launches;
  out8[6] = dev[6];
  out8[7] = dev[7];
  return SWCS_OK;
}

int swcs_sweep_energy(swcs_ctx* c, double* e_out, double* n2_out) {
  int r = need_nonempty(c);
  if (r) return r;
  double out[2];
  CK(cudaMemcpyAsync(out, ctrl(c)->eout, 16, cudaMemcpyDeviceToHost, c->st));
  if ((r = check_device(c, "swcs_sweep_energy"))) return r;
  if (e_out) *e_out = out[0];
  if (n2_out) *n2_out = out[1];
  return SWCS_OK;
}

int swcs_get_sigma(swcs_ctx* c, uint64_t* keys, double* sigma, int64_t cap, int64_t* n_out) {
  int r = need_nonempty(c);
  if (r) return r;
  const int64_t n = host_state_size(c);
  if (n < 0) return fail(c, SWCS_ERR_CUDA, "cannot read state size");
  if (n_out) *n_out = n;
  if (cap < n) return SWCS_OK;
  if ((r = ensure(c, c->sigma, (size_t)std::max<int64_t>(n, 1) * 8))) return r;
  Ctrl* k = ctrl(c);
  CK(cudaMemsetAsync(k->acc, 0, 16, c->st));
  CK(launch_k(c, kKEnergy, [&] {
    return launch_energy_sigma(ham_dev(c), state_dev(c), k->acc, (double*)c->sigma.p, c->nsm * sigma_blocks_per_sm(), c->st);
  }));
  std::vector<uint64_t> kk(n);
  std::vector<double> ss(n);
  CK(cudaMemcpyAsync(kk.data(), c->keys_a.p, 8 * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(ss.data(), c->sigma.p, 8 * n, cudaMemcpyDeviceToHost, c->st));
  if ((r = check_device(c, "swcs_get_sigma"))) return r;
  std::vector<int64_t> ord(n);
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return kk[x] < kk[y]; });
  for (int64_t i = 0; i < n; ++i) {
    keys[i] = kk[ord[i]];
    sigma[i] = ss[ord[i]];
  }
  return SWCS_OK;
}

int swcs_sigma_at(swcs_ctx* c, const uint64_t* keys, int64_t n, double* sigma) {
  int r = need_nonempty(c);
  if (r) return r;
  if (n < 0 || (n > 0 && (!keys || !sigma))) return fail(c, SWCS_ERR_INVALID_ARG, "bad sigma_at arrays");
  if (n == 0) return SWCS_OK;
  if (n > (int64_t)1 << 30) return fail(c, SWCS_ERR_INVALID_ARG, "too many determinants for sigma_at");
  const uint64_t valid = c->n >= 64 ? ~0ull : (1ull << c->n) - 1ull;
  const int m = c->n / 2;
  // alpha string, beta-string colex rank (sum over occupied spatial orbitals p_i, ascending, of C(p_i, i+1))
  std::vector<uint32_t> xa(n), rb(n);
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t d = keys[i];
    if (d & ~valid) return fail(c, SWCS_ERR_INVALID_ARG, "determinant %lld has bits >= n_so", (long long)i);
    if (__builtin_popcountll(d) != c->ne) return fail(c, SWCS_ERR_INVALID_ARG, "determinant %lld has wrong electron count", (long long)i);
    if (__builtin_popcountll(d & 0x5555555555555555ull) != c->no)
      return fail(c, SWCS_ERR_INVALID_ARG, "determinant %lld is outside the S_z = 0 sector", (long long)i);
    uint32_t x = 0, rank = 0;
    int nb = 0;
    for (int p = 0; p < m; ++p) {
      if ((d >> (2 * p)) & 1ull) x |= 1u << p;
      if ((d >> (2 * p + 1)) & 1ull) rank += (uint32_t)binom(p, ++nb);
    }
    xa[i] = x;
    rb[i] = rank;
  }
  std::vector<int64_t> ord(n);
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return xa[a] < xa[b]; });
  std::vector<uint32_t> ux, rk(n);
  std::vector<int> off;
  for (int64_t t = 0; t < n; ++t) {
    if (t == 0 || xa[ord[t]] != xa[ord[t - 1]]) {
      ux.push_back(xa[ord[t]]);
      off.push_back((int)t);
    }
    rk[t] = rb[ord[t]];
  }
  off.push_back((int)n);
  const int nx = (int)ux.size();
  const size_t bx = ((size_t)nx * 4 + 15) & ~(size_t)15, bo = ((size_t)(nx + 1) * 4 + 15) & ~(size_t)15;
  const size_t br = ((size_t)n * 4 + 15) & ~(size_t)15;
  if ((r = ensure(c, c->prb, bx + bo + br + (size_t)n * 8))) return r;
  uint8_t* base = (uint8_t*)c->prb.p;
  RowProbe pr;
  pr.n = nx;
  pr.x = (const uint32_t*)base;
  pr.off = (const int*)(base + bx);
  pr.rank = (const uint32_t*)(base + bx + bo);
  pr.out = (double*)(base + bx + bo + br);
  CK(cudaMemcpyAsync((void*)pr.x, ux.data(), (size_t)nx * 4, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync((void*)pr.off, off.data(), (size_t)(nx + 1) * 4, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync((void*)pr.rank, rk.data(), (size_t)n * 4, cudaMemcpyHostToDevice, c->st));
  r = sweep_rows(c, nullptr, -1, true, nullptr, false, nullptr, &pr);
  if (r == 1) return fail(c, SWCS_ERR_INVALID_ARG, "sigma_at needs the alpha-string row sweep (not applicable to this sector)");
  if (r) return r;
  std::vector<double> out(n);
  CK(cudaMemcpyAsync(out.data(), pr.out, (size_t)n * 8, cudaMemcpyDeviceToHost, c->st));
  if ((r = check_device(c, "swcs_sigma_at"))) return r;
  for (int64_t t = 0; t < n; ++t) sigma[ord[t]] = out[t];
  return SWCS_OK;
}

int swcs_pool_features_dev(swcs_ctx* c, uint16_t* d_x) {
  int r = need_nonempty(c);
  if (r) return r;
  if (!d_x) return fail(c, SWCS_ERR_INVALID_ARG, "null output");
  if ((r = ensure(c, c->occ, 64 * sizeof(double)))) return r;
  CK(launch_k(c, kKOther, [&] {
    return launch_pool_features(ham_dev(c), state_dev(c), (const uint8_t*)c->pool_dev.p, c->pool_size, (double*)c->occ.p,
                                (__nv_bfloat16*)d_x, c->st);
  }));
  c->launches += 1;
  return SWCS_OK;
}

int swcs_pool_screen_dev(swcs_ctx* c, swcs_mlp* m, double frac, int64_t* d_subset, int64_t* h_n_subset) {
  int r = need_nonempty(c);
  if (r) return r;
  if (!m || !d_subset || !(frac > 0.0) || frac > 1.0) return fail(c, SWCS_ERR_INVALID_ARG, "bad screening arguments");
  const int64_t P = c->pool_size;
  const int64_t k = std::max<int64_t>(1, (int64_t)std::ceil(frac * (double)P));
  if ((r = ensure(c, c->feat, (size_t)P * kFeatures * 2)) || (r = ensure(c, c->ypred, (size_t)P * 4)) ||
      (r = ensure(c, c->topk_hist, 2 * 65536 * 4)) || (r = ensure(c, c->topk_ctl, 8 * 8)))
    return r;
  if ((r = swcs_pool_features_dev(c, (uint16_t*)c->feat.p))) return r;
  if ((r = swcs_mlp_predict_dev(m, (const uint16_t*)c->feat.p, P, (float*)c->ypred.p)))
    return fail(c, r, "screening network: %s", swcs_mlp_last_error(m));
  CK(launch_k(c, kKOther, [&] {
    return launch_topk((const float*)c->ypred.p, P, k, (unsigned*)c->topk_hist.p, (unsigned long long*)c->topk_ctl.p,
                       d_subset, c->st);
  }));
  c->launches += 4;
  if (h_n_subset) *h_n_subset = k;
  return SWCS_OK;
}

int swcs_set_truncation_threshold(swcs_ctx* c, double eps) {
  if (!c) return SWCS_ERR_INVALID_ARG;
  if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(c, SWCS_ERR_INVALID_ARG, "threshold must be finite and >= 0");
  c->trunc_eps = eps;
  return SWCS_OK;
}

int swcs_set_option(swcs_ctx* c, const char* name, int64_t value) {
  if (!c || !name) return SWCS_ERR_INVALID_ARG;
  const std::string k(name);
  if (k == "sweep") {
    if (value < 0 || value > 2) return fail(c, SWCS_ERR_INVALID_ARG, "sweep must be 0, 1 or 2");
    c->opt_sweep = (int)value;
  } else if (k == "gate_blocks") {
    if (value < 0) return fail(c, SWCS_ERR_INVALID_ARG, "gate_blocks must be >= 0");
    c->opt_gate_blocks = (int)value;
  } else if (k == "screen_scatter") {
    if (value != 0 && value != 1) return fail(c, SWCS_ERR_INVALID_ARG, "screen_scatter must be 0 or 1");
    c->opt_screen_scatter = (int)value;
  } else if (k == "row_clusters") {
    if (value < 0) return fail(c, SWCS_ERR_INVALID_ARG, "row_clusters must be >= 0");
    c->opt_row_clusters = (int)value;
  } else if (k == "wait_timeout_ms") {
    if (value < 1 || value > 60000) return fail(c, SWCS_ERR_INVALID_ARG, "wait_timeout_ms must be 1..60000");
    c->opt_timeout_ns = (uint64_t)value * 1000000ull;
  } else if (k == "count_probes") {
    if (value != 0 && value != 1) return fail(c, SWCS_ERR_INVALID_ARG, "count_probes must be 0 or 1");
    c->opt_count_probes = (int)value;
  } else if (k == "test_skip_arrive") {
    c->opt_skip_arrive = value < 0 ? -1 : (int)value;
  } else if (k == "ext_capacity") {
    if (value < 0) return fail(c, SWCS_ERR_INVALID_ARG, "ext_capacity must be >= 0");
    c->opt_ext_cap = (uint64_t)value;
  } else if (k == "energy") {
    if (value < 0 || value > 2) return fail(c, SWCS_ERR_INVALID_ARG, "energy must be 0, 1 or 2");
    c->opt_energy = (int)value;
  } else if (k == "row_occupancy") {
    if (value < 1 || value > 3) return fail(c, SWCS_ERR_INVALID_ARG, "row_occupancy must be 1, 2 or 3");
    c->opt_row_occ = (int)value;
  } else if (k == "threads") {
    if (value != 128 && value != 256 && value != 512 && value != 1024)
      return fail(c, SWCS_ERR_INVALID_ARG, "threads must be 128, 256, 512 or 1024");
    c->opt_threads = (int)value;
  } else if (k == "rows_l2") {
    c->opt_rows_l2 = value != 0;
  } else if (k == "cluster") {
    if (value < 1 || value > 16) return fail(c, SWCS_ERR_INVALID_ARG, "cluster must be 1..16");
    c->opt_cluster = (int)value;
  } else {
    return fail(c, SWCS_ERR_INVALID_ARG, "unknown option '%s'", name);
  }
  return SWCS_OK;
}

int swcs_profile_enable(swcs_ctx* c, int on) {
  if (!c) return SWCS_ERR_INVALID_ARG;
  c->prof = on != 0;
  return SWCS_OK;
}

int swcs_profile_read(swcs_ctx* c, double* ms8, int64_t* n8, int reset) {
  if (!c) return SWCS_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->st));
  for (auto& e : c->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      c->prof_ms[e.kind] += ms;
      c->prof_n[e.kind] += 1;
    }
    c->ev_free.push_back(e.a);
    c->ev_free.push_back(e.b);
  }
  c->ev_pending.clear();
  for (int i = 0; i < 9; ++i) {
    if (ms8) ms8[i] = c->prof_ms[i];
    if (n8) n8[i] = c->prof_n[i];
    if (reset) {
      c->prof_ms[i] = 0;
      c->prof_n[i] = 0;
    }
  }
  if (reset) {
    c->launches = 0;
    long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpy(ctrl(c)->stats, z, sizeof z, cudaMemcpyHostToDevice));
  }
  return SWCS_OK;
}

int swcs_energy_grad(swcs_ctx* c, const uint8_t* h_ops, const double* h_theta, int n_ops, int64_t n_keep,
                     int ckpt_every, double* h_e_out, double* h_dtheta_out) {
  int r = need_ham(c);
  if (r) return r;
  if (n_ops <= 0 || !h_ops || !h_theta) return fail(c, SWCS_ERR_INVALID_ARG, "energy_grad needs at least one gate");
  if ((r = validate_ops(c, h_ops, n_ops))) return r;
  const int ck = ckpt_every > 0 ? ckpt_every : 20;
  const int ncp = (n_ops + ck - 1) / ck;
  const int64_t ms = max_state_for(c, n_keep, n_ops, 1);
  if (ms > ((int64_t)1 << 31)) return fail(c, SWCS_ERR_INVALID_ARG, "state bound too large: give n_keep");
  if ((r = ensure_state_buffers(c, ms))) return r;
  const int64_t stride = ms + 64;
  const uint64_t tcap = c->tab_mask + 1;
  if ((r = ensure(c, c->ck_keys, (size_t)(ncp + 1) * stride * 8)) || (r = ensure(c, c->ck_amps, (size_t)(ncp + 1) * stride * 8)) ||
      (r = ensure(c, c->ck_n, (size_t)(ncp + 1) * 8)) || (r = ensure(c, c->sn_keys, (size_t)ck * stride * 8)) ||
      (r = ensure(c, c->sn_amps, (size_t)ck * stride * 8)) || (r = ensure(c, c->sn_n, (size_t)ck * 8)) ||
      (r = ensure(c, c->sigma, (size_t)stride * 8)) || (r = ensure(c, c->nu0, (size_t)stride * 8)) ||
      (r = ensure(c, c->nu1, (size_t)stride * 8)) || (r = ensure(c, c->atab0, tcap * sizeof(IdxSlot))) ||
      (r = ensure(c, c->atab1, tcap * sizeof(IdxSlot))) || (r = ensure(c, c->dth, (size_t)n_ops * 8)))
    return r;
  if ((r = upload_ops(c, h_ops, h_theta, n_ops))) return r;
  Ctrl* k = ctrl(c);
  uint64_t* ckk = (uint64_t*)c->ck_keys.p;
  double* cka = (double*)c->ck_amps.p;
  long long* ckn = (long long*)c->ck_n.p;
  const uint8_t* dops = (const uint8_t*)c->ops_dev.p;
  const double* dcs = (const double*)c->cs_dev.p;
  auto save_slot = [&](int slot) -> int {
    CK(cudaMemcpyAsync(ckk + (size_t)slot * stride, c->keys_a.p, stride * 8, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(cka + (size_t)slot * stride, c->amps_a.p, stride * 8, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(ckn + slot, &k->n_state, 8, cudaMemcpyDeviceToDevice, c->st));
    return SWCS_OK;
  };
  auto load_slot = [&](int slot) -> int {
    CK(cudaMemcpyAsync(c->keys_a.p, ckk + (size_t)slot * stride, stride * 8, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(c->amps_a.p, cka + (size_t)slot * stride, stride * 8, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(&k->n_state, ckn + slot, 8, cudaMemcpyDeviceToDevice, c->st));
    return SWCS_OK;
  };
  // ---- forward with a checkpoint before every segment and after the last gate
  {
    const uint64_t hf = (c->ne >= 64) ? ~0ull : ((1ull << c->ne) - 1ull);
    const double one = 1.0;
    const long long n1 = 1;
    CK(cudaMemcpyAsync(ckk, &hf, 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(cka, &one, 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(ckn, &n1, 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(&k->n_state, &n1, 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));  // host staging above
  }
  for (int seg = 0; seg < ncp; ++seg) {
    const int g0 = seg * ck, g1 = std::min(n_ops, g0 + ck);
    if (seg > 0 && (r = save_slot(seg))) return r;
    if ((r = run_gates(c, dops + 5 * g0, dcs + 2 * g0, g1 - g0, n_keep, seg == 0, nullptr, nullptr, nullptr, 0, true)))
      return r;
  }
  if ((r = save_slot(ncp))) return r;
  c->have_state = true;
  if ((r = need_nonempty(c))) return r;
  // ---- energy, sigma and nu_M = P_M (H - E) psi_M on the final state
  CK(cudaMemsetAsync(k->acc, 0, 16, c->st));
  const int nblk = c->nsm * sigma_blocks_per_sm();
  c->have_state = true;
  if ((r = energy_rows(c, (double*)c->sigma.p)) == 1) {
    CK(cudaMemsetAsync(k->acc, 0, 16, c->st));
    CK(launch_k(c, kKEnergy, [&] { return launch_energy_sigma(ham_dev(c), state_dev(c), k->acc, (double*)c->sigma.p, nblk, c->st); }));
  } else if (r) {
    return r;
  }
  IdxSlot* atab[2] = {(IdxSlot*)c->atab0.p, (IdxSlot*)c->atab1.p};
  double* nu[2] = {(double*)c->nu0.p, (double*)c->nu1.p};
  CK(launch_k(c, kKOther, [&] { return launch_nu_init((const double*)c->amps_a.p, (const double*)c->sigma.p, &k->n_state, k->acc, nu[0], c->st); }));
  CK(launch_k(c, kKOther, [&] { return launch_build_index(ckk + (size_t)ncp * stride, ckn + ncp, atab[0], tcap - 1, c->st); }));
  CK(cudaMemsetAsync(c->dth.p, 0, (size_t)n_ops * 8, c->st));
  int cur = 0;
  const int adj_blocks = c->nsm * 8;
  // ---- backward, one segment at a time
  for (int seg = ncp - 1; seg >= 0; --seg) {
    const int g0 = seg * ck, g1 = std::min(n_ops, g0 + ck);
    if ((r = load_slot(seg))) return r;
    if (g1 - g0 > 1) {
      if ((r = run_gates(c, dops + 5 * g0, dcs + 2 * g0, g1 - g0 - 1, n_keep, false, (uint64_t*)c->sn_keys.p,
                         (double*)c->sn_amps.p, (long long*)c->sn_n.p, stride, true)))
        return r;
    }
    for (int g = g1 - 1; g >= g0; --g) {
      const uint64_t* keys_g;
      const double* amps_g;
      const long long* n_g;
      if (g == g0) {
        keys_g = ckk + (size_t)seg * stride;
        amps_g = cka + (size_t)seg * stride;
        n_g = ckn + seg;
      } else {
        keys_g = (const uint64_t*)c->sn_keys.p + (size_t)(g - g0 - 1) * stride;
        amps_g = (const double*)c->sn_amps.p + (size_t)(g - g0 - 1) * stride;
        n_g = (const long long*)c->sn_n.p + (g - g0 - 1);
      }
      CK(launch_k(c, kKOther, [&] { return launch_build_index(keys_g, n_g, atab[cur ^ 1], tcap - 1, c->st); }));
      AdjArgs a;
      a.op = dops + 5 * g;
      a.cs = dcs + 2 * g;
      a.keys = keys_g;
      a.amps = amps_g;
      a.n = n_g;
      a.tab = atab[cur ^ 1];
      a.mask = tcap - 1;
      a.tab_nu = atab[cur];
      a.mask_nu = tcap - 1;
      a.nu_in = nu[cur];
      a.nu_out = nu[cur ^ 1];
      a.dtheta = (double*)c->dth.p + g;
      CK(launch_k(c, kKAdjoint, [&] { return launch_adjoint_gate(a, adj_blocks, c->st); }));
      cur ^= 1;
    }
  }
  CK(launch_k(c, kKOther, [&] { return launch_scale_dtheta((double*)c->dth.p, n_ops, k->acc, c->st); }));
  CK(launch_k(c, kKOther, [&] { return launch_finalize_energy(k->acc, k->eout, c->st); }));
  // leave psi_M as the context's state (an identity pass rebuilds the index
  // table and drops the zero amplitudes the projectors kept)
  if ((r = load_slot(ncp))) return r;
  {
    const uint8_t id[5] = {0, 0, 0, 0, 0};
    if ((r = ensure(c, c->gsub, 16))) return r;
    CK(cudaMemcpyAsync(c->gsub.p, id, 5, cudaMemcpyHostToDevice, c->st));
    const double z[2] = {1.0, 0.0};
    if ((r = ensure(c, c->subset_dev, 16))) return r;
    CK(cudaMemcpyAsync(c->subset_dev.p, z, 16, cudaMemcpyHostToDevice, c->st));
    if ((r = run_gates(c, (const uint8_t*)c->gsub.p, (const double*)c->subset_dev.p, 1, 0, false))) return r;
  }
  double out[2];
  CK(cudaMemcpyAsync(out, k->eout, 16, cudaMemcpyDeviceToHost, c->st));
  if (h_dtheta_out) CK(cudaMemcpyAsync(h_dtheta_out, c->dth.p, (size_t)n_ops * 8, cudaMemcpyDeviceToHost, c->st));
  if ((r = check_device(c, "swcs_energy_grad"))) return r;
  if (h_e_out) *h_e_out = out[0];
  return SWCS_OK;
}


// =============================================================================
// Batched launch: many independent instances in one CUDA graph.
// =============================================================================
struct swcs_batch {
  cudaStream_t origin = nullptr;
  bool own_origin = false;  // created here: the legacy default stream cannot be captured
  int dev = 0;
  std::string err;
  std::vector<swcs_ctx*> inst;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  std::vector<int64_t> n_keep, max_state;
  std::vector<int> n_ops;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double share = 1.0;
  int cluster = 2;
  float tuned_ms = 0.f;
  // persistent launch (mode 0, default) and its tuning; mode 1 is the graph of per-instance stream branches
  int mode = 0;
  int tile = 4096, occ = 2, hash_factor = 2;
  void* d_inst = nullptr;
  BatchSched* d_sched = nullptr;
  BatchSched* d_sched0 = nullptr;  // the initial scheduler state, copied in before every launch
  double* d_rows = nullptr;
  int* d_status = nullptr;
  size_t rows_bytes = 0, inst_bytes = 0;
  int nblocks = 0;
  uint64_t timeout_ns = kTimeoutNs;  // bound of the persistent kernel's wait for work
  int stall_instance = -1;           // test hook: this instance's first phase is never picked up
};

namespace {

int bfail(swcs_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

void batch_drop_graph(swcs_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Work of an instance: gate applications + connected pairs of its sweep.
double inst_work(swcs_ctx* c, int n_ops, int64_t ms) {
  const double nconn = 2.0 * c->no * c->nv + 2.0 * binom(c->no, 2) * binom(c->nv, 2) + (double)c->no * c->no * c->nv * c->nv;
  return (double)n_ops * (double)ms + (double)ms * (nconn + 1.0);
}

// Captures every instance's pipeline (persistent gate kernel, grouping, row
// sweep, finalisation) on its own stream branch; grid sizes are the
// instance's share of the device, proportional to its work.
int batch_capture(swcs_batch* b, double share, int cluster) {
  batch_drop_graph(b);
  const int n = (int)b->inst.size();
  double wsum = 0.0;
  std::vector<double> w(n);
  for (int i = 0; i < n; ++i) wsum += (w[i] = inst_work(b->inst[i], b->n_ops[i], b->max_state[i]));
  swcs_ctx* c0 = b->inst[0];
  const int gate_total = c0->nsm * std::max(1, ansatz_blocks_per_sm(kAnsatzThreadsShared));
  for (int i = 0; i < n; ++i) {
    swcs_ctx* c = b->inst[i];
    c->opt_gate_threads = kAnsatzThreadsShared;
    const double f = std::min(1.0, share * w[i] / wsum);
    c->opt_gate_blocks = std::max(1, (int)std::lround(f * gate_total));
    c->opt_cluster = cluster;
    c->opt_row_clusters = std::max(1, (int)std::lround(f * gate_total / (2.0 * cluster)));
    int r = sweep_rows(c, (double*)c->gdev.p, b->max_state[i], false);  // size only
    if (r == 1) return bfail(b, SWCS_ERR_INVALID_ARG, "batch: an instance's sector does not fit the row sweep");
    if (r) return bfail(b, r, std::string("batch sizing: ") + c->err);
  }
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bfail(b, SWCS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  cudaEventRecord(b->fork, b->origin);
  int status = SWCS_OK;
  for (int i = 0; i < n && status == SWCS_OK; ++i) {
    swcs_ctx* c = b->inst[i];
    cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    int r = run_gates(c, (const uint8_t*)c->ops_dev.p, (const double*)c->cs_dev.p, b->n_ops[i], b->n_keep[i], true);
    if (!r) r = sweep_rows(c, (double*)c->gdev.p, b->max_state[i], true);
    if (r) {
      status = bfail(b, r == 1 ? SWCS_ERR_INVALID_ARG : r, std::string("batch capture: ") + c->err);
      break;
    }
    cudaEventRecord(b->done[i], b->streams[i]);
    cudaStreamWaitEvent(b->origin, b->done[i], 0);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->origin, &g);
  if (status) {
    if (g) cudaGraphDestroy(g);
    return status;
  }
  if (e != cudaSuccess) return bfail(b, SWCS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) return bfail(b, SWCS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  for (int i = 0; i < n; ++i) b->inst[i]->have_state = true;
  b->mode = 1;
  return SWCS_OK;
}

void batch_free_persistent(swcs_batch* b) {
  for (void* p : {(void*)b->d_inst, (void*)b->d_sched, (void*)b->d_sched0, (void*)b->d_rows, (void*)b->d_status})
    if (p) cudaFree(p);
  b->d_inst = nullptr;
  b->d_sched = b->d_sched0 = nullptr;
  b->d_rows = nullptr;
  b->d_status = nullptr;
  b->rows_bytes = b->inst_bytes = 0;
}

// The persistent launch: per-instance descriptors (gate, grouping and row-sweep
// arguments over the instance's own buffers), the initial scheduler words, and
// a graph of {scheduler reset, status reset, row reset, the kernel}.
int batch_build_persistent(swcs_batch* b, int tile, int occ, int hash_factor) {
  batch_drop_graph(b);
  const int n = (int)b->inst.size();
  std::vector<BatchInst> hi(n);
  std::vector<BatchSched> hs(n);
  size_t dyn = 0;
  int64_t max_nb = 4;
  for (int i = 0; i < n; ++i) {
    swcs_ctx* c = b->inst[i];
    const int m = c->n / 2;
    if (m > 32 || c->NB <= 0 || c->NB > (1 << 22)) return bfail(b, SWCS_ERR_INVALID_ARG, "batch: an instance's sector does not fit the row sweep");
    const int64_t nd = b->max_state[i];
    const int ks = c->no, nvs = c->nv;
    const int ns = ks * nvs, ndb = (ks * (ks - 1) / 2) * (nvs * (nvs - 1) / 2);
    const int max_s = ns + 1, max_d = ndb + 1, t_same = 1 + ns + ndb;  // one CTA per target: all its entries
    int twords = (int)((c->NB + 127) / 128);
    size_t smem = row_sweep_smem(max_s, max_d, 0, 0, t_same, twords);
    if (smem > 96 * 1024) {
      twords = 0;
      smem = row_sweep_smem(max_s, max_d, 0, 0, t_same, 0);
    }
    if (smem > 96 * 1024) return bfail(b, SWCS_ERR_INVALID_ARG, "batch: an instance's sector does not fit the row sweep");
    dyn = std::max(dyn, smem);
    max_nb = std::max<int64_t>(max_nb, c->NB);
    const uint64_t acap = pow2_at_least((uint64_t)std::max<int64_t>((int64_t)hash_factor * nd, 64));
    int r;
    if ((r = ensure(c, c->atab, acap * sizeof(IdxSlot))) || (r = ensure(c, c->gid_of, nd * 4 + 4)) ||
        (r = ensure(c, c->gcount, nd * 8 + 8)) || (r = ensure(c, c->goff, nd * 8 + 16)) ||
        (r = ensure(c, c->gfill, nd * 8 + 8)) || (r = ensure(c, c->gkey, nd * 8 + 8)) ||
        (r = ensure(c, c->gamp, nd * 8 + 8)) || (r = ensure(c, c->grank, nd * 4 + 4)) ||
        (r = ensure(c, c->rbeta, (size_t)std::max<int64_t>(nd, 1) * ks * nvs * 4)) ||
        (r = ensure(c, c->gorig, (size_t)std::max<int64_t>(nd, 1) * 4)))
      return bfail(b, r, "batch: " + c->err);
    const int packed = c->NB <= (1 << 21) && m <= 32 ? 1 : 0;
    BatchInst& I = hi[i];
    I.ga = gate_args(c, (const uint8_t*)c->ops_dev.p, (const double*)c->cs_dev.p, b->n_ops[i], b->n_keep[i], true,
                     nullptr, nullptr, nullptr, 0, false);
    I.gr = group_args(c, acap);
    I.ra = row_args(c, I.gr, (double*)c->gdev.p, max_s, max_d, twords, packed);
    I.n_ops = b->n_ops[i];
    I.tile = tile;
    I.ks = ks;
    I.nvs = nvs;
    I.m = m;
    I.packed = packed;
    I.acap = acap;
    I.g = (double*)c->gdev.p;
    I.pool_size = c->pool_size;
    I.eout = ctrl(c)->eout;
    BatchSched& S = hs[i];
    S = BatchSched{};
    S.tab_cur = 0;
    S.ep = 1;
    S.slot[0].phase = 0;
    S.slot[0].type = kPhInit;
    S.slot[0].ntiles = (unsigned)((c->tab_mask + 1 + tile - 1) / tile);
    S.slot[1].phase = 0xFFFFFFFFu;
    S.slot[1].type = kPhDone;
    if (i == b->stall_instance) S.slot[0].phase = 1;  // never matches the phase word: no CTA takes its tiles
  }
  const int bps = std::min(occ, batch_blocks_per_sm(dyn));
  if (bps <= 0) return bfail(b, SWCS_ERR_NO_DEVICE, "batch: the persistent kernel cannot be resident on this device");
  const int nblocks = b->inst[0]->nsm * bps;
  const int64_t row_stride = (max_nb + 3) & ~(int64_t)3;
  const size_t rows_bytes = (size_t)nblocks * row_stride * 8;
  batch_free_persistent(b);
  if (cudaMalloc(&b->d_inst, n * sizeof(BatchInst)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_sched, n * sizeof(BatchSched)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_sched0, n * sizeof(BatchSched)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_rows, rows_bytes) != cudaSuccess || cudaMalloc((void**)&b->d_status, 16) != cudaSuccess) {
    batch_free_persistent(b);
    return bfail(b, SWCS_ERR_OOM, "batch: device memory for the persistent launch");
  }
  b->rows_bytes = rows_bytes;
  b->nblocks = nblocks;
  if (cudaMemcpy(b->d_inst, hi.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_sched0, hs.data(), n * sizeof(BatchSched), cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, SWCS_ERR_CUDA, "batch: descriptor upload failed");
  const uint64_t timeout = b->timeout_ns;
  cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bfail(b, SWCS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  cudaMemcpyAsync(b->d_sched, b->d_sched0, n * sizeof(BatchSched), cudaMemcpyDeviceToDevice, b->origin);
  cudaMemsetAsync(b->d_status, 0, 16, b->origin);
  cudaMemsetAsync(b->d_rows, 0, rows_bytes, b->origin);
  e = launch_batch((const BatchInst*)b->d_inst, b->d_sched, n, b->d_rows, row_stride, b->d_status, nblocks, dyn, timeout,
                   b->origin);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, SWCS_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) return bfail(b, SWCS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  b->tile = tile;
  b->occ = occ;
  b->hash_factor = hash_factor;
  b->mode = 0;
  for (int i = 0; i < n; ++i) b->inst[i]->have_state = false;  // the index tables stay in the launch's internal form
  return SWCS_OK;
}

int batch_check(swcs_batch* b) {
  cudaError_t e = cudaStreamSynchronize(b->origin);
  if (e != cudaSuccess) return bfail(b, SWCS_ERR_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
  if (b->mode == 0 && b->d_status) {
    int st[2] = {0, 0};
    if (cudaMemcpy(st, b->d_status, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return bfail(b, SWCS_ERR_CUDA, "batch run: status read failed");
    if (st[1] != 0) return bfail(b, SWCS_ERR_TIMEOUT, "batch run: a bounded wait for work ran out");
    if (st[0] != (int)b->inst.size()) return bfail(b, SWCS_ERR_CUDA, "batch run: not every instance finished");
  }
  for (swcs_ctx* c : b->inst) {
    int r = check_device(c, "batch instance");
    if (r) return bfail(b, r, c->err);
  }
  return SWCS_OK;
}

}  // namespace

int swcs_batch_create(swcs_batch** out, void* cuda_stream) {
  if (!out) return SWCS_ERR_INVALID_ARG;
  swcs_batch* b = new swcs_batch();
  b->origin = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&b->dev) != cudaSuccess || cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return SWCS_ERR_NO_DEVICE;
  }
  if (!b->origin) {  // a blocking stream: ordered with the legacy default stream
    if (cudaStreamCreate(&b->origin) != cudaSuccess) {
      cudaEventDestroy(b->fork);
      delete b;
      return SWCS_ERR_CUDA;
    }
    b->own_origin = true;
  }
  *out = b;
  return SWCS_OK;
}

int swcs_batch_destroy(swcs_batch* b) {
  if (!b) return SWCS_OK;
  cudaStreamSynchronize(b->origin);
  batch_drop_graph(b);
  batch_free_persistent(b);
  for (swcs_ctx* c : b->inst) swcs_destroy(c);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_origin) cudaStreamDestroy(b->origin);
  delete b;
  return SWCS_OK;
}

const char* swcs_batch_last_error(const swcs_batch* b) { return b ? b->err.c_str() : "no batch"; }

int swcs_batch_add(swcs_batch* b, const double* h_h, const double* h_g, int n_so, int n_elec, const uint8_t* h_ops,
                   const double* h_theta, int n_ops, int64_t n_keep, int* index_out) {
  if (!b) return SWCS_ERR_INVALID_ARG;
  if (n_ops <= 0 || !h_ops || !h_theta) return bfail(b, SWCS_ERR_INVALID_ARG, "batch_add: needs at least one gate");
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    return bfail(b, SWCS_ERR_CUDA, "batch_add: stream creation failed");
  swcs_ctx* c = nullptr;
  int r = swcs_create(&c, st);
  if (r) {
    cudaStreamDestroy(st);
    return bfail(b, r, "batch_add: context creation failed");
  }
  auto undo = [&](int code) {
    const std::string m = c->err;
    swcs_destroy(c);
    cudaStreamDestroy(st);
    return bfail(b, code, "batch_add: " + m);
  };
  if ((r = swcs_load_hamiltonian(c, h_h, h_g, n_so, n_elec))) return undo(r);
  if ((r = validate_ops(c, h_ops, n_ops))) return undo(r);
  const int64_t ms = max_state_for(c, n_keep, n_ops, 1);
  if (ms > ((int64_t)1 << 31)) return undo(fail(c, SWCS_ERR_INVALID_ARG, "state bound too large: give n_keep"));
  if ((r = ensure_state_buffers(c, ms)) || (r = upload_ops(c, h_ops, h_theta, n_ops)) ||
      (r = ensure(c, c->gdev, sizeof(double) * c->pool_size)))
    return undo(r);
  if (cudaStreamSynchronize(st) != cudaSuccess) return undo(SWCS_ERR_CUDA);
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  b->inst.push_back(c);
  b->streams.push_back(st);
  b->done.push_back(ev);
  b->n_keep.push_back(n_keep);
  b->max_state.push_back(ms);
  b->n_ops.push_back(n_ops);
  batch_drop_graph(b);
  if (index_out) *index_out = (int)b->inst.size() - 1;
  return SWCS_OK;
}

int swcs_batch_set_option(swcs_batch* b, const char* name, int64_t value) {
  if (!b || !name) return SWCS_ERR_INVALID_ARG;
  const std::string k = name;
  if (k == "wait_timeout_ms") {
    if (value < 1 || value > 60000) return bfail(b, SWCS_ERR_INVALID_ARG, "wait_timeout_ms must be 1..60000");
    b->timeout_ns = (uint64_t)value * 1000000ull;
  } else if (k == "test_stall_instance") {
    if (value < -1 || value >= (int64_t)b->inst.size()) return bfail(b, SWCS_ERR_INVALID_ARG, "test_stall_instance out of range");
    b->stall_instance = (int)value;
  } else {
    return bfail(b, SWCS_ERR_INVALID_ARG, "unknown batch option " + k);
  }
  batch_drop_graph(b);
  return SWCS_OK;
}

int swcs_batch_set_tuning(swcs_batch* b, int mode, int tile, int ctas_per_sm, int hash_factor) {
  if (!b) return SWCS_ERR_INVALID_ARG;
  if ((mode != 0 && mode != 1) || tile < 256 || tile > (1 << 20) || ctas_per_sm < 1 || ctas_per_sm > 2 ||
      (hash_factor != 2 && hash_factor != 4 && hash_factor != 8))
    return bfail(b, SWCS_ERR_INVALID_ARG, "batch_set_tuning: mode 0|1, tile 256..2^20, ctas_per_sm 1|2, hash_factor 2|4|8");
  b->mode = mode;
  b->tile = tile;
  b->occ = ctas_per_sm;
  b->hash_factor = hash_factor;
  return SWCS_OK;
}

int swcs_batch_build(swcs_batch* b, int autotune) {
  if (!b || b->inst.empty()) return bfail(b, SWCS_ERR_INVALID_ARG, "batch_build: no instances");
  if (!autotune && b->mode == 0) return batch_build_persistent(b, b->tile, b->occ, b->hash_factor);
  if (autotune && b->mode == 0) {
    // autotuner of the persistent launch: items per tile, CTAs per SM and the
    // alpha-string table's size (capacity = factor x state bound), timed whole
    const int tiles[] = {2048, 4096, 8192, 16384};
    const int occs[] = {1, 2};
    const int factors[] = {2, 4};
    double best_ms = 1e30;
    int bt = 4096, bo = 2, bf = 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int t : tiles)
      for (int o : occs)
        for (int f : factors) {
          if (batch_build_persistent(b, t, o, f)) continue;
          cudaGraphLaunch(b->exec, b->origin);  // warm-up
          if (batch_check(b)) continue;
          float best = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, b->origin);
            cudaGraphLaunch(b->exec, b->origin);
            cudaEventRecord(e1, b->origin);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
          }
          if (best < best_ms) {
            best_ms = best;
            bt = t;
            bo = o;
            bf = f;
          }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30) return bfail(b, SWCS_ERR_CUDA, "batch autotune: no configuration ran");
    b->tuned_ms = (float)best_ms;
    return batch_build_persistent(b, bt, bo, bf);
  }
  if (!autotune) return batch_capture(b, b->share, b->cluster);
  // autotuner: device share per unit of work and cluster size of the row
  // sweep, timed on the whole graph
  const double shares[] = {1.0, 2.0, 4.0, 8.0, 16.0, 32.0};
  const int clusters[] = {1, 2};
  double best_ms = 1e30, best_share = 1.0;
  int best_cl = 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (double sh : shares)
    for (int cl : clusters) {
      int r = batch_capture(b, sh, cl);
      if (r) continue;
      cudaGraphLaunch(b->exec, b->origin);  // warm-up
      if (batch_check(b)) continue;
      float best = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, b->origin);
        cudaGraphLaunch(b->exec, b->origin);
        cudaEventRecord(e1, b->origin);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
      }
      if (best < best_ms) {
        best_ms = best;
        best_share = sh;
        best_cl = cl;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_ms >= 1e30) return bfail(b, SWCS_ERR_CUDA, "batch autotune: no configuration ran");
  b->share = best_share;
  b->cluster = best_cl;
  b->tuned_ms = (float)best_ms;
  return batch_capture(b, best_share, best_cl);
}

int swcs_batch_run(swcs_batch* b) {
  if (!b || !b->exec) return bfail(b, SWCS_ERR_INVALID_ARG, "batch_run: call swcs_batch_build first");
  const cudaError_t e = cudaGraphLaunch(b->exec, b->origin);
  if (e != cudaSuccess) return bfail(b, SWCS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return SWCS_OK;
}

int swcs_batch_size(swcs_batch* b, int* n_out) {
  if (!b || !n_out) return SWCS_ERR_INVALID_ARG;
  *n_out = (int)b->inst.size();
  return SWCS_OK;
}

int swcs_batch_pool_size(swcs_batch* b, int i, int64_t* n_out) {
  if (!b || !n_out || i < 0 || i >= (int)b->inst.size()) return bfail(b, SWCS_ERR_INVALID_ARG, "bad instance index");
  *n_out = b->inst[i]->pool_size;
  return SWCS_OK;
}

int swcs_batch_results(swcs_batch* b, int i, double* h_e, double* h_n2, double* h_g) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return bfail(b, SWCS_ERR_INVALID_ARG, "bad instance index");
  int r = batch_check(b);
  if (r) return r;
  swcs_ctx* c = b->inst[i];
  double out[2];
  if (cudaMemcpy(out, ctrl(c)->eout, 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
      (h_g && cudaMemcpy(h_g, c->gdev.p, sizeof(double) * c->pool_size, cudaMemcpyDeviceToHost) != cudaSuccess))
    return bfail(b, SWCS_ERR_CUDA, "batch_results: copy failed");
  if (h_e) *h_e = out[0];
  if (h_n2) *h_n2 = out[1];
  return SWCS_OK;
}

int swcs_batch_tuning(swcs_batch* b, double* h_out8) {
  if (!b || !h_out8) return SWCS_ERR_INVALID_ARG;
  h_out8[0] = b->mode;
  h_out8[1] = b->tile;
  h_out8[2] = b->occ;
  h_out8[3] = b->hash_factor;
  h_out8[4] = b->tuned_ms;
  h_out8[5] = (double)b->inst.size();
  h_out8[6] = b->share;
  h_out8[7] = b->cluster;
  return SWCS_OK;
}

int swcs_batch_run_serial(swcs_batch* b) {
  if (!b || b->inst.empty()) return bfail(b, SWCS_ERR_INVALID_ARG, "batch_run_serial: no instances");
  for (size_t i = 0; i < b->inst.size(); ++i) {
    swcs_ctx* c = b->inst[i];
    const cudaStream_t own = c->st;
    c->st = b->origin;  // every instance's kernels back to back on one stream, no synchronisation between them
    c->opt_gate_threads = kAnsatzThreads;
    c->opt_gate_blocks = 0;
    c->opt_cluster = 1;  // the single-context default shape
    c->opt_threads = 1024;
    c->opt_row_clusters = 0;
    int r = run_gates(c, (const uint8_t*)c->ops_dev.p, (const double*)c->cs_dev.p, b->n_ops[i], b->n_keep[i], true);
    if (!r) r = sweep_rows(c, (double*)c->gdev.p, b->max_state[i], true);
    c->st = own;
    if (r) return bfail(b, r == 1 ? SWCS_ERR_INVALID_ARG : r, "batch_run_serial: " + c->err);
  }
  return SWCS_OK;
}

}  // extern "C"
