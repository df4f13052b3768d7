// Batched persistent launch (the many-instances workload): one kernel runs
// every instance's whole hot path -- the gate sequence of Eq. 1 with merge and
// truncation after every gate (Sec. II.B), then the pool sweep of ADAPT step 4
// (Sec. II.C) -- for all instances at once.
//
// Work items are (instance, phase, tile).  Each instance walks a chain of
// phases (BatchPhase): initial index tables; per gate the gate pass (which also
// counts the first select digit), the select passes still needed and the
// compaction into the next state; the grouping of the state by alpha string;
// the beta-single tables; the row sweep with one target alpha string per tile;
// the finish.  An instance's current phase and the next free tile of it share
// one 64-bit word, so a CTA takes a tile with one atomic add and sees which
// phase the tile belongs to.  The CTA that finishes a phase's last tile runs
// the phase's epilogue (the select's bin search, the sizes of the next phase)
// and publishes the next phase.  A CTA never waits on another CTA inside a
// tile; it only polls the instances' words for work, with a bounded wait.
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"
#include "swcs_rowsweep.cuh"
#include "swcs_select.cuh"

namespace swcs {

namespace {

constexpr int kBatchThreads = 512;
constexpr size_t kHistSet = (size_t)kPasses * kBins;  // select histograms of one gate

// The tile a CTA is working on, shared by its threads.
struct BatchTask {
  int inst;
  unsigned phase, tile, ntiles;
  int type, gate, pass;
  long long n, m;
  int epilogue, exit;
  // the instance's scheduler state as published with this phase (read once, with volatile loads)
  int tab_cur;
  unsigned ep;
  SelState sel;
};

// Field-wise volatile read of a select state written by another CTA.
__device__ __forceinline__ void load_sel(const SelState* p, SelState& o) {
  const volatile SelState* v = p;
  o.prefix = v->prefix;
  o.kprefix = v->kprefix;
  o.need = v->need;
  o.shift = v->shift;
  o.kshift = v->kshift;
  o.mode = v->mode;
  o.pass = v->pass;
  o.bin = v->bin;
  o.cum = v->cum;
  o.cnt = v->cnt;
}

__device__ __forceinline__ unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}

// Items [b, e) of a phase's tile t over `count` items in tiles of `per`.
__device__ __forceinline__ void tile_range(long long count, long long per, unsigned t, long long& b, long long& e) {
  b = (long long)t * per;
  e = min(count, b + per);
}

// ---------------------------------------------------------------- gate sequence tiles
// Initial tables: both (epoch, position) index tables empty (epoch 0), the first gate's
// histograms and the counters zero, the reference determinant as the state.
__device__ void tile_init(const BatchInst& I, const BatchTask& k) {
  const AnsatzArgs& a = I.ga;
  const long long cap = (long long)a.tab_mask + 1;
  long long b, e;
  tile_range(cap, I.tile, k.tile, b, e);
  for (long long i = b + threadIdx.x; i < e; i += blockDim.x) {  // (epoch, position) slots, epoch 0: no build
    ((uint64_t*)a.tab[0])[i] = 0;
    ((uint64_t*)a.tab[1])[i] = 0;
  }
  const long long chunk = (long long)ceil_div((long long)kHistSet, k.ntiles);
  for (long long i = (long long)k.tile * chunk + threadIdx.x; i < min((long long)kHistSet, (long long)(k.tile + 1) * chunk);
       i += blockDim.x)
    a.hist[i] = 0;
  if (k.tile == 0) {
    for (int i = threadIdx.x; i < 12; i += blockDim.x) a.ctr[i] = 0;
    if (threadIdx.x == 0) {
      a.keys_a[0] = a.hf;
      a.amps_a[0] = 1.0;
    }
  }
}

// Gate pass (P1 of the gate kernel) over the state's items [b, e): rotation of
// each two-determinant block, partners not in the state appended, exact drops
// counted, the first select digit of every kept |c| counted.
__device__ void tile_gate(const BatchInst& I, const BatchSched& S, const BatchTask& k, unsigned* s_hist) {
  const AnsatzArgs& a = I.ga;
  const int g = k.gate;
  unsigned long long* ctr = a.ctr + (g % 3) * kCtrN;
  const GateOp op = decode_op(a.ops + 5 * g);
  const double cs = a.cs[2 * g], sn = a.cs[2 * g + 1];
  const uint64_t* tcur = (const uint64_t*)a.tab[k.tab_cur];
  const long long n = k.n;
  long long b, e;
  tile_range(n, I.tile, k.tile, b, e);
  unsigned* H = a.hist + (size_t)(g & 1) * kHistSet;
  {  // the next gate's histograms, last read by the previous gate
    unsigned* Hn = a.hist + (size_t)((g + 1) & 1) * kHistSet;
    const long long chunk = (long long)ceil_div((long long)kHistSet, k.ntiles);
    for (long long i = (long long)k.tile * chunk + threadIdx.x;
         i < min((long long)kHistSet, (long long)(k.tile + 1) * chunk); i += blockDim.x)
      Hn[i] = 0;
    if (k.tile == 0 && threadIdx.x < kCtrN) a.ctr[((g + 1) % 3) * kCtrN + threadIdx.x] = 0;
  }
  for (int t = threadIdx.x; t < kBins; t += blockDim.x) s_hist[t] = 0;
  __syncthreads();
  const long long span = e - b;
  const long long n_iter = (span + blockDim.x - 1) / blockDim.x * blockDim.x;  // warp-converged loop
  unsigned probes = 0;
  for (long long r = threadIdx.x; r < n_iter; r += blockDim.x) {
    const long long i = b + r;
    const bool live = r < span;
    uint64_t d = 0, partner = 0;
    double c = 0.0, out = 0.0, extra = 0.0;
    bool has_extra = false;
    if (live) {
      d = a.keys_a[i];
      c = a.amps_a[i];
      const bool up = op.kind && ((d & op.mask_a) == op.mask_a) && ((d & op.mask_c) == 0);
      const bool dn = op.kind && ((d & op.mask_c) == op.mask_c) && ((d & op.mask_a) == 0);
      if (up || dn) {
        int sbit;
        if (op.kind == 1) sbit = up ? single_phase(d, op.i0, op.i1) : single_phase(d, op.i1, op.i0);
        else sbit = up ? double_phase(d, op.i0, op.i1, op.i2, op.i3) : double_phase(d, op.i2, op.i3, op.i0, op.i1);
        partner = d ^ op.mask_a ^ op.mask_c;
        const double t1 = __dmul_rn(c, cs);
        const int64_t j = ep_lookup(tcur, a.tab_mask, a.keys_a, partner, k.ep, &probes);
        if (j >= 0) {
          const double t2 = __dmul_rn(a.amps_a[j], sn);
          out = __dadd_rn(t1, up ? apply_sign(t2, !sbit) : apply_sign(t2, sbit));
        } else {
          out = t1;
          const double t = __dmul_rn(c, sn);
          extra = up ? apply_sign(t, sbit) : apply_sign(t, !sbit);
          has_extra = abs_bits(extra) >= a.min_abs_bits;
        }
      } else {
        out = c;
      }
      a.keys_b[i] = d;
      a.amps_b[i] = out;
      if (abs_bits(out) >= a.min_abs_bits) atomicAdd(&s_hist[abs_bits(out) >> abs_lo(0)], 1u);
      if (has_extra) atomicAdd(&s_hist[abs_bits(extra) >> abs_lo(0)], 1u);
    }
    const unsigned long long slot = warp_alloc(&ctr[kCtrExtra], has_extra);
    if (has_extra) {
      const unsigned long long pos = (unsigned long long)n + slot;
      if (pos < (unsigned long long)a.cap) {
        a.keys_b[pos] = partner;
        a.amps_b[pos] = extra;
      } else {
        set_error(a.err, kDevTableFull);
      }
    }
    const bool zero = live && abs_bits(out) < a.min_abs_bits;
    const unsigned zb = __ballot_sync(__activemask(), zero);
    if ((threadIdx.x & 31) == 0 && zb) atomicAdd(&ctr[kCtrZero], (unsigned long long)__popc(zb));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kBins; t += blockDim.x)
    if (s_hist[t]) atomicAdd(&H[t], s_hist[t]);
}

// Select pass p over the merged items [b, e): digit p of the entries that
// still match the decided prefix.
__device__ void tile_select(const BatchInst& I, const BatchSched& S, const BatchTask& k, unsigned* s_hist) {
  const AnsatzArgs& a = I.ga;
  const int p = k.pass;
  const bool keyphase = p >= kAbsPasses;
  const int q = keyphase ? p - kAbsPasses : p;
  const int lo = keyphase ? key_lo(q) : abs_lo(q), hi = keyphase ? key_hi(q) : abs_hi(q);
  const unsigned dmask = (1u << (hi - lo)) - 1u;
  const unsigned long long prefix = k.sel.prefix, kprefix = k.sel.kprefix;
  const unsigned long long pre = keyphase ? kprefix : prefix;
  long long b, e;
  tile_range(k.m, I.tile, k.tile, b, e);
  for (int t = threadIdx.x; t < kBins; t += blockDim.x) s_hist[t] = 0;
  __syncthreads();
  for (long long i = b + threadIdx.x; i < e; i += blockDim.x) {
    const uint64_t x = abs_bits(a.amps_b[i]);
    if (x < a.min_abs_bits) continue;
    uint64_t v;
    if (!keyphase) {
      if ((x >> hi) != (pre >> hi)) continue;
      v = x;
    } else {
      if (x != prefix) continue;
      const uint64_t key = a.keys_b[i];
      if (hi < 64 && (key >> hi) != (pre >> hi)) continue;
      v = key;
    }
    atomicAdd(&s_hist[(v >> lo) & dmask], 1u);
  }
  __syncthreads();
  unsigned* gh = a.hist + (size_t)(k.gate & 1) * kHistSet + (size_t)p * kBins;
  for (int t = threadIdx.x; t < kBins; t += blockDim.x)
    if (s_hist[t]) atomicAdd(&gh[t], s_hist[t]);
}

// Compaction (P3) over the merged items [b, e): the kept entries into the next
// state and its index table (the next epoch).
__device__ void tile_compact(const BatchInst& I, const BatchSched& S, const BatchTask& k) {
  const AnsatzArgs& a = I.ga;
  unsigned long long* ctr = a.ctr + (k.gate % 3) * kCtrN;
  uint64_t* tnxt = (uint64_t*)a.tab[k.tab_cur ^ 1];
  const uint32_t ep_nxt = k.ep + 1;
  const SelState s = k.sel;
  long long b, e;
  tile_range(k.m, I.tile, k.tile, b, e);
  const long long span = e - b;
  const long long n_iter = (span + blockDim.x - 1) / blockDim.x * blockDim.x;
  for (long long r = threadIdx.x; r < n_iter; r += blockDim.x) {
    const long long i = b + r;
    bool keep = false;
    uint64_t key = 0;
    double c = 0.0;
    if (r < span) {
      key = a.keys_b[i];
      c = a.amps_b[i];
      keep = keep_entry(s, key, c, a.min_abs_bits);
    }
    const unsigned long long pos = warp_alloc(&ctr[kCtrKept], keep);
    if (keep) {
      a.keys_a[pos] = key;
      a.amps_a[pos] = c;
      if (!ep_insert(tnxt, a.tab_mask, key, (uint32_t)pos, ep_nxt)) set_error(a.err, kDevTableFull);
    }
  }
}

// ---------------------------------------------------------------- sweep tiles
// Before the grouping: alpha-string table empty, group counts, the gradient
// and the accumulators zero.
__device__ void tile_group_clear(const BatchInst& I, const BatchTask& k) {
  const long long items = max(max((long long)I.acap, (long long)I.pool_size), k.n + 1);
  long long b, e;
  tile_range(items, I.tile, k.tile, b, e);
  for (long long i = b + threadIdx.x; i < e; i += blockDim.x) {
    if (i < (long long)I.acap) {
      I.gr.atab[i].key = kEmpty;
      I.gr.atab[i].idx = ~0ull;
    }
    if (i <= k.n) {
      I.gr.gcount[i] = 0;
      I.gr.gfill[i] = 0;
    }
    if (i < I.pool_size) I.g[i] = 0.0;
  }
  if (k.tile == 0 && threadIdx.x == 0) {
    *I.gr.n_groups = 0;
    I.gr.acc[0] = 0.0;
    I.gr.acc[1] = 0.0;
  }
}

// The row sweep's target tile: one alpha string of the instance's sector, swept
// by this CTA alone (its own row, a block barrier between the passes).
template <int kRowThreads>
__device__ void tile_row(const BatchInst& I, const BatchTask& k, unsigned char* dyn, RowShared& sh, double* row,
                         int& row_inst) {
  const RowArgs& A = I.ra;
  const RowDyn dy = row_dyn(dyn, A);
  if (row_inst != k.inst) {  // the sector's tables in shared memory
    row_cta_init<kRowThreads>(A, sh, dy);
    row_inst = k.inst;
  }
  BlockSync sy;
  double e_acc = 0.0;
  unsigned n_lookups = 0, n_probe_slots = 0;
  row_target<kRowThreads>(A, sh, dy, row, (int)k.tile, false, false, 0, 1, sy, e_acc, n_lookups, n_probe_slots,
                          false);  // the row is clean again for the next work item, whichever instance it belongs to
  row_flush<kRowThreads>(A, sh, e_acc, n_lookups, n_probe_slots);
}

__device__ void tile_finish(const BatchInst& I) {
  const double n2 = I.gr.acc[1];
  const double f = 2.0 / n2;
  for (long long i = threadIdx.x; i < I.pool_size; i += blockDim.x) I.g[i] *= f;
  if (threadIdx.x == 0) {
    I.eout[0] = I.gr.acc[0] / n2;
    I.eout[1] = n2;
  }
}

// ---------------------------------------------------------------- epilogues
// The bin search of select digit p on the histogram H: updates the instance's
// select state; returns 1 when the cut is decided.  All threads take part.
__device__ int select_step(const AnsatzArgs& a, BatchSched& S, int gate, int p, unsigned* s_hist, SelState& sel,
                           long long* s_scan) {
  const bool keyphase = p >= kAbsPasses;
  const int q = keyphase ? p - kAbsPasses : p;
  const int lo = keyphase ? key_lo(q) : abs_lo(q), hi = keyphase ? key_hi(q) : abs_hi(q);
  const unsigned* gh = a.hist + (size_t)(gate & 1) * kHistSet + (size_t)p * kBins;
  for (int t = threadIdx.x; t < kBins; t += blockDim.x) s_hist[t] = __ldcg(&gh[t]);
  if (threadIdx.x == 0) {
    load_sel(&S.sel, sel);
    sel.bin = -1;
  }
  __syncthreads();
  find_bin(s_hist, 1 << (hi - lo), sel.need, !keyphase, sel, s_scan);
  __shared__ int decided;
  if (threadIdx.x == 0) {
    int chosen = sel.bin;
    if (chosen < 0) {  // cannot happen: total >= need
      set_error(a.err, kDevBadState);
      chosen = 0;
    }
    const long long need = sel.need - sel.cum, cnt = sel.cnt;
    sel.need = need;
    sel.pass = p + 1;
    int dec = 0;
    if (!keyphase) {
      sel.prefix |= (unsigned long long)chosen << lo;
      sel.shift = lo;
      if (cnt == need) dec = 1;
      else if (lo == 0) sel.mode = 2;
    } else {
      sel.kprefix |= (unsigned long long)chosen << lo;
      sel.kshift = lo;
      if (cnt == need || lo == 0) dec = 1;
    }
    S.sel = sel;
    decided = dec;
  }
  __syncthreads();
  return decided;
}

// The phase after the one just finished, and its tile count (thread 0 publishes it).
__device__ void epilogue(const BatchInst& I, BatchSched& S, const BatchTask& k, BatchSlot& nx, unsigned* s_hist,
                         SelState& sel, long long* s_scan) {
  const AnsatzArgs& a = I.ga;
  const long long tile = I.tile;
  nx = BatchSlot{};
  nx.phase = k.phase + 1;
  nx.gate = k.gate;
  nx.pass = 0;
  nx.n = k.n;
  nx.m = k.m;
  auto gate_or_sweep = [&](long long n_state) {
    nx.n = n_state;
    if (nx.gate < I.n_ops) {
      nx.type = kPhGate;
      nx.ntiles = max(1u, ceil_div(n_state, tile));
    } else {
      nx.type = kPhGroupClear;
      nx.ntiles = ceil_div(max(max((long long)I.acap, (long long)I.pool_size), n_state + 1), tile);
    }
  };
  if (ld_acquire_i32(a.err) != 0) {  // an error in one of the tiles: this instance stops
    nx.type = kPhDone;
    nx.ntiles = 0;
    return;
  }
  switch (k.type) {
    case kPhInit:
      nx.type = kPhBuild0;
      nx.ntiles = 1;
      break;
    case kPhBuild0:
      nx.gate = 0;
      gate_or_sweep(1);
      break;
    case kPhGate: {
      unsigned long long* ctr = a.ctr + (k.gate % 3) * kCtrN;
      const long long m = k.n + (long long)ld_key_relaxed((const uint64_t*)&ctr[kCtrExtra]);
      const long long nz = m - (long long)ld_key_relaxed((const uint64_t*)&ctr[kCtrZero]);
      if (m > a.cap) {
        if (threadIdx.x == 0) set_error(a.err, kDevTableFull);
        nx.type = kPhDone;
        nx.ntiles = 0;
        break;
      }
      nx.m = m;
      if (threadIdx.x == 0) {
        SelState s0{};
        s0.mode = (a.n_keep > 0 && nz > a.n_keep) ? 1 : 0;
        s0.need = a.n_keep;
        s0.shift = 63;
        s0.kshift = 64;
        S.sel = s0;
        sel = s0;
        __threadfence();
      }
      __syncthreads();
      const int dec = sel.mode == 0 ? 1 : select_step(a, S, k.gate, 0, s_hist, sel, s_scan);
      nx.type = dec ? kPhCompact : kPhSelect;
      nx.pass = 1;
      nx.ntiles = max(1u, ceil_div(m, tile));
      break;
    }
    case kPhSelect: {
      const int dec = select_step(a, S, k.gate, k.pass, s_hist, sel, s_scan);
      if (!dec && k.pass + 1 >= kPasses) {
        if (threadIdx.x == 0) set_error(a.err, kDevBadState);
        nx.type = kPhDone;
        nx.ntiles = 0;
        break;
      }
      nx.type = dec ? kPhCompact : kPhSelect;
      nx.pass = k.pass + 1;
      nx.ntiles = max(1u, ceil_div(k.m, tile));
      break;
    }
    case kPhCompact: {
      unsigned long long* ctr = a.ctr + (k.gate % 3) * kCtrN;
      const long long n = (long long)ld_key_relaxed((const uint64_t*)&ctr[kCtrKept]);
      if (threadIdx.x == 0) {
        S.tab_cur = k.tab_cur ^ 1;
        S.ep = k.ep + 1;
      }
      nx.gate = k.gate + 1;
      gate_or_sweep(n);
      if (nx.type != kPhGate && threadIdx.x == 0) {
        *a.n_state = n;
        *a.tab_cur_out = k.tab_cur ^ 1;
      }
      break;
    }
    case kPhGroupClear:
      nx.type = kPhGroupInsert;
      nx.ntiles = max(1u, ceil_div(k.n, tile));
      break;
    case kPhGroupInsert:
      nx.type = kPhGroupIds;
      nx.ntiles = ceil_div((long long)I.acap, tile);
      break;
    case kPhGroupIds:
      nx.type = kPhGroupCount;
      nx.ntiles = max(1u, ceil_div(k.n, tile));
      break;
    case kPhGroupCount:
      nx.type = kPhGroupScan;
      nx.ntiles = 1;
      break;
    case kPhGroupScan:
      nx.type = kPhGroupScatter;
      nx.ntiles = max(1u, ceil_div(k.n, tile));
      break;
    case kPhGroupScatter:
      nx.type = kPhRbeta;
      nx.ntiles = max(1u, ceil_div(k.n, tile / 8));
      break;
    case kPhRbeta:
      nx.type = kPhRow;
      nx.ntiles = (unsigned)I.ra.NA;
      break;
    case kPhRow:
      nx.type = kPhFinish;
      nx.ntiles = 1;
      break;
    default:
      nx.type = kPhDone;
      nx.ntiles = 0;
      break;
  }
}

// ---------------------------------------------------------------- the persistent kernel
// status[0]: instances finished; status[1]: a bounded wait for work ran out;
// status[2..3]: global time of the last phase published (the wait is bounded by
// the time since then, so CTAs idle behind a long phase of another instance do
// not give up while work is still moving).
__global__ void __launch_bounds__(kBatchThreads, 2)
batch_kernel(const BatchInst* __restrict__ insts, BatchSched* scheds, int n_inst, double* rows, int64_t row_stride,
             int* status, uint64_t timeout_ns) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ BatchTask task;
  __shared__ BatchSlot next;
  __shared__ SelState sel;
  __shared__ unsigned s_hist[kBins];
  __shared__ long long s_scan[32];
  __shared__ long long s_part[kBatchThreads];
  __shared__ RowShared sh;
  double* row = rows + (size_t)blockIdx.x * (size_t)row_stride;
  int row_inst = -1;
  int start = (int)(blockIdx.x % (unsigned)n_inst);
  for (;;) {
    // ---- find a tile (thread 0)
    if (threadIdx.x == 0) {
      task.exit = 0;
      task.epilogue = 0;
      const uint64_t t0 = globaltimer_ns();
      unsigned spins = 0;
      bool found = false;
      while (!found) {
        if (ld_acquire_i32(&status[1]) != 0 || ld_acquire_i32(&status[0]) >= n_inst) {
          task.exit = 1;
          break;
        }
        for (int kk = 0; kk < n_inst && !found; ++kk) {
          const int i = (start + kk) % n_inst;
          BatchSched& S = scheds[i];
          const unsigned long long w = ld_volatile_u64(&S.word);
          const unsigned ph = (unsigned)(w >> 32), nt = (unsigned)w;
          const volatile BatchSlot* sl = &S.slot[ph & 1];
          if (sl->phase != ph || sl->type == kPhDone || nt >= sl->ntiles) continue;
          const unsigned long long w2 = atomicAdd(&S.word, 1ull);
          __threadfence();
          const unsigned ph2 = (unsigned)(w2 >> 32), t = (unsigned)w2;
          const volatile BatchSlot* s2 = &S.slot[ph2 & 1];
          if (s2->phase != ph2 || s2->type == kPhDone || t >= s2->ntiles) continue;
          task.inst = i;
          task.phase = ph2;
          task.tile = t;
          task.ntiles = s2->ntiles;
          task.type = s2->type;
          task.gate = s2->gate;
          task.pass = s2->pass;
          task.n = s2->n;
          task.m = s2->m;
          task.tab_cur = *(volatile int*)&S.tab_cur;
          task.ep = *(volatile unsigned*)&S.ep;
          load_sel(&S.sel, task.sel);
          found = true;
        }
        if (!found) {
          if ((++spins & 63u) == 0) {
            const uint64_t last = ld_key_relaxed((const uint64_t*)(status + 2));
            const uint64_t ref = last > t0 ? last : t0;
            const uint64_t now = globaltimer_ns();  // another SM's stamp may read a little ahead of this one
            if (now > ref && now - ref > timeout_ns) {
              atomicCAS(&status[1], 0, 1);
              task.exit = 1;
              break;
            }
          }
          __nanosleep(256);
        }
      }
      start = (start + 1) % n_inst;
    }
    __syncthreads();
    if (task.exit) break;
    const BatchTask k = task;
    const BatchInst& I = insts[k.inst];
    BatchSched& S = scheds[k.inst];
    // ---- run it (all threads)
    switch (k.type) {
      case kPhInit:
        tile_init(I, k);
        break;
      case kPhBuild0:
        if (threadIdx.x == 0 && !ep_insert((uint64_t*)I.ga.tab[k.tab_cur], I.ga.tab_mask, I.ga.hf, 0u, k.ep))
          set_error(I.ga.err, kDevTableFull);
        break;
      case kPhGate:
        tile_gate(I, S, k, s_hist);
        break;
      case kPhSelect:
        tile_select(I, S, k, s_hist);
        break;
      case kPhCompact:
        tile_compact(I, S, k);
        break;
      case kPhGroupClear:
        tile_group_clear(I, k);
        break;
      case kPhGroupInsert: {
        long long b, e;
        tile_range(k.n, I.tile, k.tile, b, e);
        group_insert_items(I.gr.keys, e, I.gr.atab, I.gr.amask, I.gr.amps, I.gr.acc, b + threadIdx.x, blockDim.x);
        break;
      }
      case kPhGroupIds: {
        long long b, e;
        tile_range((long long)I.acap, I.tile, k.tile, b, e);
        group_ids_items(I.gr.atab, (uint64_t)e, I.gr.n_groups, (uint64_t)(b + threadIdx.x), blockDim.x);
        break;
      }
      case kPhGroupCount: {
        long long b, e;
        tile_range(k.n, I.tile, k.tile, b, e);
        group_count_items(I.gr.keys, e, I.gr.atab, I.gr.amask, I.gr.gid_of, I.gr.gcount, b + threadIdx.x, blockDim.x);
        break;
      }
      case kPhGroupScan:
        group_scan_block(I.gr.gcount, (long long)*(volatile unsigned long long*)I.gr.n_groups, I.gr.goff, s_part);
        break;
      case kPhGroupScatter: {
        long long b, e;
        tile_range(k.n, I.tile, k.tile, b, e);
        group_scatter_items(I.gr.keys, I.gr.amps, e, I.gr.gid_of, I.gr.goff, I.gr.gfill, I.gr.gkey, I.gr.gamp,
                            I.gr.grank, I.gr.gorig, I.gr.rank_tab, I.gr.ks, b + threadIdx.x, blockDim.x);
        break;
      }
      case kPhRbeta: {
        long long b, e;
        tile_range(k.n, I.tile / 8, k.tile, b, e);
        rbeta_dets(I.gr.gkey, e, I.gr.rank_tab, I.ks, I.nvs, I.m, I.packed, (uint32_t*)I.ra.rbeta,
                   b + (threadIdx.x >> 5), blockDim.x >> 5);
        break;
      }
      case kPhRow:
        tile_row<kBatchThreads>(I, k, dyn, sh, row, row_inst);
        break;
      case kPhFinish:
        tile_finish(I);
        break;
      default:
        break;
    }
    // ---- count it; the phase's last tile runs the epilogue and publishes the next phase
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned d = atomicAdd(&S.done, 1u) + 1u;
      task.epilogue = d == k.ntiles;
      if (task.epilogue) __threadfence();
    }
    __syncthreads();
    if (task.epilogue) {
      epilogue(I, S, k, next, s_hist, sel, s_scan);
      __syncthreads();
      if (threadIdx.x == 0) {
        S.slot[next.phase & 1] = next;
        S.done = 0;
        __threadfence();
        atomicExch(&S.word, (unsigned long long)next.phase << 32);
        atomicMax((unsigned long long*)(status + 2), (unsigned long long)globaltimer_ns());
        if (next.type == kPhDone) atomicAdd(&status[0], 1);
      }
    }
    __syncthreads();
  }
}

}  // namespace

size_t batch_dyn_smem(int max_ent_s, int max_ent_d, int t_same, int touched_words) {
  return row_sweep_smem(max_ent_s, max_ent_d, 0, 0, t_same, touched_words);
}

int batch_blocks_per_sm(size_t dyn_smem) {
  int nb = 0;
  if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel, kBatchThreads, dyn_smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_batch(const BatchInst* d_inst, BatchSched* d_sched, int n_inst, double* d_rows, int64_t row_stride,
                         int* d_status, int nblocks, size_t dyn_smem, uint64_t timeout_ns, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
  if (e != cudaSuccess) return e;
  batch_kernel<<<nblocks, kBatchThreads, dyn_smem, st>>>(d_inst, d_sched, n_inst, d_rows, row_stride, d_status,
                                                          timeout_ns);
  return cudaGetLastError();
}

}  // namespace swcs
