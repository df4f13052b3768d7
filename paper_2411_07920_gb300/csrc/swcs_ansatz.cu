// Gate sequence on the sparse determinant state: one persistent cooperative
// launch runs every gate of the ansatz (Eq. 1), each as
//   P1  gate apply + merge   (Eqs. 2-3, exact on each two-determinant block)
//   P2  top-N radix select   (Sec. II.B truncation, Fig. 1)
//   P3  compaction + re-index of the kept set
// separated by bounded grid barriers.
//
// Merge without a merge table: a gate exp(theta (tau - tau^dag)) couples a
// determinant D only to its partner tau D (or tau^dag D), and that partner
// is unique.  Each thread owns one D of the input state S, looks up its
// partner in the index table of S and writes D's new amplitude from the two
// old ones; a partner that is not in S is appended (it can be produced by
// exactly one D, so no duplicates arise).  Every new amplitude is the sum of
// at most two separately rounded products, so the result does not depend on
// the order of work: bit-identical to any correct sequential evaluation.
//
// Truncation: entries below the magnitude threshold (or exactly zero) are
// dropped, then the n_keep largest |c| of the rest are kept, ties at the cut
// by smaller bitstring.  |c| as an IEEE-754 bit pattern with the sign cleared orders
// like the value, so an MSD radix select over 12-bit digits finds the cut (the
// first digit, the exponent and top mantissa bit, is counted while P1 writes
// the amplitudes); when the cut lands on several equal |c| a second radix
// select over the bitstrings of the tied entries picks the smallest.
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"
#include "swcs_select.cuh"

namespace swcs {

template <int kThreads>
__global__ void __launch_bounds__(kThreads)
ansatz_kernel(AnsatzArgs a) {
  __shared__ SelState sel;
  __shared__ unsigned s_hist[kBins];
  __shared__ long long s_scan[32];
  __shared__ long long s_n;
  __shared__ unsigned long long s_base;

  const unsigned nblocks = gridDim.x;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t gstride = (size_t)nblocks * blockDim.x;
  uint64_t* keysA = a.keys_a;
  double* ampsA = a.amps_a;
  uint64_t* keysB = a.keys_b;
  double* ampsB = a.amps_b;
  int tab_cur = a.tab_cur;
  const size_t hist_set = (size_t)kPasses * kBins;  // two sets, alternating between gates
  unsigned n_lookups = 0, n_probe_slots = 0;  // partner lookups and the slots they visited

  // ---------------------------------------------------------------- prologue
  if (threadIdx.x == 0) {
    s_n = a.reset_to_hf ? 1 : (long long)*a.n_state;
  }
  __syncthreads();
  long long n = s_n;
  if (a.reset_to_hf && gtid == 0) {
    keysA[0] = a.hf;
    ampsA[0] = 1.0;
  }
  // the launch's index tables: 8-byte (epoch, position) slots in the first half of each table buffer
  uint64_t* ct[2] = {(uint64_t*)a.tab[0], (uint64_t*)a.tab[1]};
  for (size_t i = gtid; i <= a.tab_mask; i += gstride) {
    ct[0][i] = 0;  // epoch 0: no build
    ct[1][i] = 0;
  }
  for (size_t i = gtid; i < 3 * kCtrN; i += gstride) a.ctr[i] = 0;
  for (size_t i = gtid; i < hist_set; i += gstride) a.hist[i] = 0;  // the first gate's set
  // test hook: the named CTA leaves without arriving, so every other CTA's
  // bounded wait runs out and the kernel reports kDevTimeout
  if ((int)blockIdx.x == a.skip_arrive_block) return;
  if (!grid_barrier(a.bar, nblocks, a.err, a.timeout_ns)) return;
  uint32_t ep = 1;  // epoch of the build of tab[tab_cur]
  for (size_t i = gtid; i < (size_t)n; i += gstride) {
    if (!ep_insert(ct[tab_cur], a.tab_mask, keysA[i], (uint32_t)i, ep)) set_error(a.err, kDevTableFull);
  }
  if (!grid_barrier(a.bar, nblocks, a.err, a.timeout_ns)) return;

  for (int g = 0; g < a.n_ops; ++g) {
    const long long s_gate_in = n;
    unsigned long long* ctr = a.ctr + (g % 3) * kCtrN;
    const GateOp op = decode_op(a.ops + 5 * g);
    const double cs = a.cs[2 * g], sn = a.cs[2 * g + 1];
    const uint64_t* tcur = ct[tab_cur];
    uint64_t* tnxt = ct[tab_cur ^ 1];
    const uint32_t ep_nxt = ep + 1;
    unsigned* H = a.hist + (size_t)(g & 1) * hist_set;  // this gate's histograms (pass 0 filled below)

    // ------------------------------------------------------------ P1 gate + merge (+ first select digit)
    if (gtid < kCtrN) a.ctr[((g + 1) % 3) * kCtrN + gtid] = 0;
    {
      unsigned* Hn = a.hist + (size_t)((g + 1) & 1) * hist_set;  // the next gate's set, last read by gate g-1
      for (size_t i = gtid; i < hist_set; i += gstride) Hn[i] = 0;
    }
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) s_hist[t] = 0;
    __syncthreads();
    const size_t n_iter = ((size_t)n + gstride - 1) / gstride * gstride;  // warp-converged loop
    for (size_t i = gtid; i < n_iter; i += gstride) {
      const bool live = i < (size_t)n;
      uint64_t d = 0, partner = 0;
      double c = 0.0, out = 0.0, extra = 0.0;
      bool has_extra = false;
      if (live) {
        d = keysA[i];
        c = ampsA[i];
        const bool up = op.kind && ((d & op.mask_a) == op.mask_a) && ((d & op.mask_c) == 0);
        const bool dn = op.kind && ((d & op.mask_c) == op.mask_c) && ((d & op.mask_a) == 0);
        if (up || dn) {
          int sbit;
          if (op.kind == 1) sbit = up ? single_phase(d, op.i0, op.i1) : single_phase(d, op.i1, op.i0);
          else sbit = up ? double_phase(d, op.i0, op.i1, op.i2, op.i3) : double_phase(d, op.i2, op.i3, op.i0, op.i1);
          partner = d ^ op.mask_a ^ op.mask_c;
          const double t1 = __dmul_rn(c, cs);
          const int64_t j = ep_lookup(tcur, a.tab_mask, keysA, partner, ep, &n_probe_slots);
          ++n_lookups;
          if (j >= 0) {
            const double t2 = __dmul_rn(ampsA[j], sn);
            // lower D: c' = c cos - s sin c_U ; upper D: c' = c cos + s sin c_L
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
        keysB[i] = d;
        ampsB[i] = out;
        if (abs_bits(out) >= a.min_abs_bits) atomicAdd(&s_hist[abs_bits(out) >> abs_lo(0)], 1u);
        if (has_extra) atomicAdd(&s_hist[abs_bits(extra) >> abs_lo(0)], 1u);
      }
      const unsigned long long slot = warp_alloc(&ctr[kCtrExtra], has_extra);
      if (has_extra) {
        const unsigned long long pos = (unsigned long long)n + slot;
        if (pos < (unsigned long long)a.cap) {
          keysB[pos] = partner;
          ampsB[pos] = extra;
        } else {
          set_error(a.err, kDevTableFull);
        }
      }
      const bool zero = live && abs_bits(out) < a.min_abs_bits;  // dropped: zero or below threshold
      const unsigned zb = __ballot_sync(__activemask(), zero);
      if ((threadIdx.x & 31) == 0 && zb) atomicAdd(&ctr[kCtrZero], (unsigned long long)__popc(zb));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kBins; t += blockDim.x)
      if (s_hist[t]) atomicAdd(&H[t], s_hist[t]);
    if (!grid_barrier(a.bar, nblocks, a.err, a.timeout_ns)) return;

    const long long m = n + (long long)ld_key_relaxed((const uint64_t*)&ctr[kCtrExtra]);
    const long long nz = m - (long long)ld_key_relaxed((const uint64_t*)&ctr[kCtrZero]);
    if (m > a.cap) return;  // error already flagged

    // ------------------------------------------------------------ P2 radix select
    if (threadIdx.x == 0) {
      sel.mode = (a.n_keep > 0 && nz > a.n_keep) ? 1 : 0;
      sel.prefix = 0;
      sel.kprefix = 0;
      sel.need = a.n_keep;
      sel.shift = 63;
      sel.kshift = 64;
      sel.pass = 0;
    }
    __syncthreads();
    if (sel.mode != 0) {
      bool decided = false;
      for (int p = 0; p < kPasses && !decided; ++p) {
        const bool keyphase = p >= kAbsPasses;
        const int q = keyphase ? p - kAbsPasses : p;
        const int lo = keyphase ? key_lo(q) : abs_lo(q), hi = keyphase ? key_hi(q) : abs_hi(q);
        const unsigned dmask = (1u << (hi - lo)) - 1u;
        unsigned* gh = H + (size_t)p * kBins;
        if (p > 0) {  // digit 0 of |c| was counted during P1
          for (int t = threadIdx.x; t < kBins; t += blockDim.x) s_hist[t] = 0;
          __syncthreads();
          const unsigned long long pre = keyphase ? sel.kprefix : sel.prefix;
          for (size_t i = gtid; i < (size_t)m; i += gstride) {
            const double c = ampsB[i];
            const uint64_t x = abs_bits(c);
            if (x < a.min_abs_bits) continue;
            uint64_t v;
            if (!keyphase) {
              if ((x >> hi) != (pre >> hi)) continue;
              v = x;
            } else {
              if (x != sel.prefix) continue;
              const uint64_t k = keysB[i];
              if (hi < 64 && (k >> hi) != (pre >> hi)) continue;
              v = k;
            }
            atomicAdd(&s_hist[(v >> lo) & dmask], 1u);
          }
          __syncthreads();
          for (int t = threadIdx.x; t < kBins; t += blockDim.x)
            if (s_hist[t]) atomicAdd(&gh[t], s_hist[t]);
          if (!grid_barrier(a.bar, nblocks, a.err, a.timeout_ns)) return;
        }
        // the whole block pulls the global bins (past the barrier, from L2) into shared memory
        for (int t = threadIdx.x; t < kBins; t += blockDim.x) s_hist[t] = __ldcg(&gh[t]);
        if (threadIdx.x == 0) sel.bin = -1;
        __syncthreads();
        find_bin(s_hist, (int)dmask + 1, sel.need, !keyphase, sel, s_scan);
        if (threadIdx.x == 0) {
          int chosen = sel.bin;
          if (chosen < 0) {  // cannot happen: total >= need
            set_error(a.err, kDevBadState);
            chosen = 0;
          }
          const long long need = sel.need - sel.cum, cnt = sel.cnt;
          sel.need = need;
          sel.pass = p + 1;
          if (!keyphase) {
            sel.prefix |= (unsigned long long)chosen << lo;
            sel.shift = lo;
            if (cnt == need) decided = true;          // whole bucket kept
            else if (lo == 0) sel.mode = 2;            // exact |c| ties at the cut
          } else {
            sel.kprefix |= (unsigned long long)chosen << lo;
            sel.kshift = lo;
            if (cnt == need || lo == 0) decided = true;
          }
          if (decided) sel.pass |= 0x100;
        }
        __syncthreads();
        decided = (sel.pass & 0x100) != 0;
        if (ld_acquire_i32(a.err) != 0) return;
      }
    }
    __syncthreads();
    const SelState s = sel;

    // ------------------------------------------------------------ P3 compaction + re-index
    // Output positions by block, in rounds of up to 32 items per thread: each thread marks which of its
    // items are kept, the block scans the counts and takes its range of the output with one atomic (a
    // counter per warp would put tens of thousands of atomics per gate on one address), then the kept
    // items are read again and written, indexed and snapshotted.
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (size_t r0 = 0; r0 < (size_t)m; r0 += (size_t)32 * gstride) {
      uint32_t kmask = 0;
      unsigned cnt = 0;
      for (int it = 0; it < 32; ++it) {
        const size_t i = r0 + (size_t)it * gstride + gtid;
        if (i >= (size_t)m) break;
        const uint64_t k = s.mode == 2 ? keysB[i] : 0;  // the bitstring decides only exact ties at the cut
        if (keep_entry(s, k, ampsB[i], a.min_abs_bits)) {
          kmask |= 1u << it;
          ++cnt;
        }
      }
      unsigned inc = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += v;
      }
      if (lane == 31) s_scan[wid] = inc;
      __syncthreads();
      if (threadIdx.x == 0) {
        long long run = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
          const long long v = s_scan[w];
          s_scan[w] = run;
          run += v;
        }
        s_base = run ? atomicAdd(&ctr[kCtrKept], (unsigned long long)run) : 0ull;
      }
      __syncthreads();
      unsigned long long pos = s_base + (unsigned long long)s_scan[wid] + (inc - cnt);
      __syncthreads();  // s_scan and s_base are rewritten next round
      while (kmask) {
        const int it = __ffs(kmask) - 1;
        kmask &= kmask - 1u;
        const size_t i = r0 + (size_t)it * gstride + gtid;
        const uint64_t k = keysB[i];
        const double c = ampsB[i];
        keysA[pos] = k;
        ampsA[pos] = c;
        if (!ep_insert(tnxt, a.tab_mask, k, (uint32_t)pos, ep_nxt)) set_error(a.err, kDevTableFull);
        if (a.snap_keys) {
          a.snap_keys[(size_t)g * a.snap_stride + pos] = k;
          a.snap_amps[(size_t)g * a.snap_stride + pos] = c;
        }
        ++pos;
      }
    }
    if (!grid_barrier(a.bar, nblocks, a.err, a.timeout_ns)) return;
    n = (long long)ld_key_relaxed((const uint64_t*)&ctr[kCtrKept]);
    if (a.snap_n && gtid == 0) a.snap_n[g] = n;
    if (gtid == 0 && a.stats) {
      atomicAdd((unsigned long long*)&a.stats[0], 1ull);
      atomicAdd((unsigned long long*)&a.stats[1], (unsigned long long)(s.pass & 0xff));
      atomicMax((unsigned long long*)&a.stats[6], (unsigned long long)m);
      atomicAdd((unsigned long long*)&a.stats[7], (unsigned long long)s_gate_in);
    }
    tab_cur ^= 1;
    ep = ep_nxt;
  }
  // the output state's table in the plain key/index form, written into the other buffer
  {
    const uint64_t* t = ct[tab_cur];
    IdxSlot* plain = a.tab[tab_cur ^ 1];
    for (size_t i = gtid; i <= a.tab_mask; i += gstride) {
      const uint64_t w = t[i];
      if ((uint32_t)(w >> 32) == ep) {
        plain[i].key = keysA[(uint32_t)w];
        plain[i].idx = (uint32_t)w;
      } else {
        plain[i].key = kEmpty;
        plain[i].idx = 0;
      }
    }
    tab_cur ^= 1;
  }
  if (a.probe_ctr && (n_lookups | n_probe_slots)) {
    atomicAdd(&a.probe_ctr[0], (unsigned long long)n_lookups);
    atomicAdd(&a.probe_ctr[1], (unsigned long long)n_probe_slots);
  }
  if (gtid == 0) {
    *a.n_state = n;
    *a.tab_cur_out = tab_cur;
  }
}

// One 1024-thread CTA per SM for a single state (fewest CTAs at the grid
// barriers); 256-thread CTAs where many instances share the device (several
// instances' CTAs can then be resident on one SM).
int ansatz_blocks_per_sm(int threads) {
  int nb = 0;
  const cudaError_t e = threads == kAnsatzThreadsShared
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ansatz_kernel<kAnsatzThreadsShared>, threads, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ansatz_kernel<kAnsatzThreads>, threads, 0);
  return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_ansatz(const AnsatzArgs& args, int nblocks, int threads, cudaStream_t st) {
  if (threads != kAnsatzThreads && threads != kAnsatzThreadsShared) return cudaErrorInvalidValue;
  // cooperative launch (all CTAs co-resident, as the grid barrier needs); the
  // launch-attribute form is also valid inside stream capture
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(threads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (threads == kAnsatzThreadsShared) return cudaLaunchKernelEx(&cfg, ansatz_kernel<kAnsatzThreadsShared>, args);
  return cudaLaunchKernelEx(&cfg, ansatz_kernel<kAnsatzThreads>, args);
}

}  // namespace swcs
