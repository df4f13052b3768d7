// Device code of the alpha-string row sweep (the pool sweep, energy, sigma
// probes), shared by its cluster kernel (swcs_rowsweep.cu) and the batched
// persistent kernel (swcs_batch.cu): the per-target passes, the grouping of a
// state by alpha string and the beta-single tables, each as device functions
// over a strided set of items.  Included once per translation unit.
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"

namespace cg = cooperative_groups;

namespace swcs {

namespace {

constexpr int kRowMaxWarps = 32;  // CTA sizes 128, 256, 512 or 1024 threads
constexpr int kSameChunk = 128;  // targets of one determinant per work item (4 per lane)
constexpr int kDblChunk = 1;     // determinants per alpha-double work item

__device__ __forceinline__ uint32_t even_bits(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)x;
}

// Colex rank of a string of one spin: sum_i C(p_i, i+1) over its set bits,
// from per-byte tables T[chunk][bits below chunk][byte].
__device__ __forceinline__ uint32_t str_rank(const uint32_t* __restrict__ T, int ks, uint32_t m) {
  uint32_t r = 0;
  int below = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint32_t byte = (m >> (8 * c)) & 255u;
    if (byte) r += __ldg(&T[(c * (ks + 1) + below) * 256 + byte]);
    below += __popc(byte);
  }
  return r;
}

struct RowEnt {
  uint32_t off;   // first determinant of the group (grouped order)
  uint32_t flat;  // the group's size when found; then the exclusive prefix of work items within its list
  uint8_t o[4];   // spin-orbitals removed from D (o[0], o[1]) and added (o[2], o[3]); singles use o[0], o[2]
};

struct RowShared {
  uint16_t tri_o[kMaxSpin * (kMaxSpin - 1) / 2];
  uint16_t tri_v[kMaxSpin * (kMaxSpin - 1) / 2];
  uint8_t occx[kMaxSpin], virx[kMaxSpin];
  uint8_t bocc[kRowMaxWarps][kMaxSpin], bvir[kRowMaxWarps][kMaxSpin];  // beta spatial lists per warp
  uint8_t occ_all[kRowMaxWarps][64];
  int n_s, n_d;              // entries of the target (all CTAs of the cluster)
  int n_s_loc, n_d_loc;      // entries this CTA found (its staged share)
  uint32_t tot_s, tot_d;     // work items (singles: entry x determinant; doubles: entry x chunk)
  long long gx_off, gx_cnt;  // the alpha group of X itself
  unsigned scan_tmp[kRowMaxWarps];
  double red[kRowMaxWarps];
  unsigned next_item[3][2];  // per pass: the next alpha-beta item and alpha-double item to hand out
};

// Dynamic shared memory: entry lists, the staged share of the discovery, the
// decode table of X's own targets and the bitmap of row entries this CTA
// touched.
struct RowDyn {
  RowEnt* ents_s;  // the target's entries, in the same order in every CTA of the cluster
  RowEnt* ents_d;
  RowEnt* stage_s;  // entries this CTA found (the lists themselves when one CTA sweeps a target)
  RowEnt* stage_d;
  uint32_t* same_tab;  // target t >= 1 of a determinant in X's group: o1 | o2<<8 | v1<<16 | v2<<24 (o2 = 255: single)
  unsigned* touched;   // NB bits (nullptr: clear whole rows)
};

__device__ __forceinline__ double fock_single(const RowArgs& A, const uint8_t* occ_all, int p, int q) {
  const int n = A.H.n;
  double f = __ldg(&A.H.h[q * n + p]);
  const double* w = A.H.Ws + ((size_t)p * n + q) * n;
  for (int t = 0; t < A.H.ne; ++t) f += __ldg(&w[occ_all[t]]);
  return f;
}

// The touched bitmap holds one bit per 32-byte sector (4 entries) of the row:
// clearing works in whole sectors anyway, and a sector is usually hit by
// several contributions.
__device__ __forceinline__ uint32_t sector_word(uint32_t i) { return i >> 7; }
__device__ __forceinline__ unsigned sector_bit(uint32_t i) { return 1u << ((i >> 2) & 31u); }

// Whether a scatter to row entry i is needed, recording its sector as touched.
// The bit is set atomically only while it still reads as clear (two lanes that
// both see it clear both set it).  In energy-only mode (filt) only the sectors
// of X's own determinants are read back: their bits are set before the
// scatter, every other sector is skipped.
__device__ __forceinline__ bool take(unsigned* touched, bool filt, uint32_t i) {
  if (!touched) return true;
  const unsigned bit = sector_bit(i);
  const unsigned w = touched[sector_word(i)];
  if (filt) return (w & bit) != 0u;
  if (!(w & bit)) atomicOr(&touched[sector_word(i)], bit);
  return true;
}

// One connected pair, scatter or gather.  (p<q) removed, (r<s) added for
// doubles; q = s = -1 marks a single p -> r.
template <bool SCATTER>
__device__ __forceinline__ void row_pair(const RowArgs& A, double* row, unsigned* touched, bool filt, uint64_t d,
                                         double cd, uint32_t rank_e, int p, int q, int r, int s,
                                         const uint8_t* occ_all) {
  const int n = A.H.n;
  if (q < 0) {
    if (SCATTER) {
      if (!take(touched, filt, rank_e)) return;
      const int sb = single_phase(d, p, r);
      atomicAdd(&row[rank_e], apply_sign(fock_single(A, occ_all, p, r), sb) * cd);
    } else {
      const int lo = p < r ? p : r, hi = p < r ? r : p;
      const int k = __ldg(&A.H.ops1[lo * n + hi]);
      if (A.sel_bits && !((__ldg(&A.sel_bits[k >> 5]) >> (k & 31)) & 1u)) return;
      const int sb = single_phase(d, p, r);
      atomicAdd(&A.g[k], apply_sign(cd * row[rank_e], sb ^ (int)(p > r)));
    }
    return;
  }
  const int pa = pair_index(p, q, n), pb = pair_index(r, s, n);
  if (SCATTER) {
    if (!take(touched, filt, rank_e)) return;
    const int sb = double_phase(d, p, q, r, s);
    atomicAdd(&row[rank_e], apply_sign(__ldg(&A.H.G[(size_t)pa * A.H.npairs + pb]), sb) * cd);
  } else {
    const bool down = pa > pb;
    const int k = __ldg(&A.H.opd[down ? (size_t)pb * A.H.npairs + pa : (size_t)pa * A.H.npairs + pb]);
    if (A.sel_bits && !((__ldg(&A.sel_bits[k >> 5]) >> (k & 31)) & 1u)) return;
    const int sb = double_phase(d, p, q, r, s);
    atomicAdd(&A.g[k], apply_sign(cd * row[rank_e], sb ^ (int)down));
  }
}

__device__ __forceinline__ void warp_lists(RowShared& sh, int warp, int lane, uint64_t d, int m) {
  const bool inr = lane < m;
  const bool ob = inr && ((d >> (2 * lane + 1)) & 1ull);
  const unsigned bo = __ballot_sync(0xffffffffu, ob);
  const unsigned bv = __ballot_sync(0xffffffffu, inr && !ob);
  const unsigned below = (1u << lane) - 1u;
  if (ob) sh.bocc[warp][__popc(bo & below)] = (uint8_t)lane;
  else if (inr) sh.bvir[warp][__popc(bv & below)] = (uint8_t)lane;
  const unsigned lo = (unsigned)d, hi = (unsigned)(d >> 32);
  if ((lo >> lane) & 1u) sh.occ_all[warp][__popc(lo & below)] = (uint8_t)lane;
  if ((hi >> lane) & 1u) sh.occ_all[warp][__popc(lo) + __popc(hi & below)] = (uint8_t)(32 + lane);
  __syncwarp();
}

// Block-wide exclusive scan, in list order, of the work items of each entry:
// ceil(group size / chunk).
template <int kRowThreads>
__device__ void scan_items(RowShared& sh, RowEnt* ents, int cnt, int chunk, uint32_t* total) {
  const int per = (cnt + kRowThreads - 1) / kRowThreads;
  const int b = threadIdx.x * per, e = min(cnt, b + per);
  auto items = [&](int i) { return (ents[i].flat + chunk - 1) / chunk; };  // flat still holds the size
  unsigned sum = 0;
  for (int i = b; i < e; ++i) sum += items(i);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) sh.scan_tmp[warp] = inc;
  __syncthreads();
  unsigned wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += sh.scan_tmp[w];
  unsigned run = wbase + inc - sum;
  for (int i = b; i < e; ++i) {
    const unsigned it = items(i);
    ents[i].flat = run;
    run += it;
  }
  if (threadIdx.x == kRowThreads - 1) *total = run;
  __syncthreads();
}

// The last entry whose first work item is at or before item t (entries in
// list order, prefixes increasing), found by the whole warp: 32-ary search
// steps, one ballot each; every lane of the warp must call it.  ents[lo].flat
// <= t holds throughout (ents[0].flat = 0), so lane 0's probe is always true
// and the ballot never empty.
__device__ __forceinline__ int warp_find_entry(const RowEnt* ents, int cnt, uint32_t t, int lane) {
  int lo = 0, span = cnt;  // the entry lies in [lo, lo + span)
  while (span > 32) {
    const int stride = (span + 31) >> 5;
    const bool le = lane * stride < span && ents[lo + lane * stride].flat <= t;
    const int k = 31 - __clz(__ballot_sync(0xffffffffu, le));
    lo += k * stride;
    span = min(stride, span - k * stride);
  }
  const bool le = lane < span && ents[lo + lane].flat <= t;
  return lo + 31 - __clz(__ballot_sync(0xffffffffu, le));
}

// Passes over a target's pairs: scatter sigma into the row, gather gradients from it, or (screened sweep)
// mark the row sectors that selected operators will read.
enum RowPass { kPassScatter = 0, kPassGather = 1, kPassMark = 2 };

// n work items from a counter in shared memory, for the whole warp (every lane must call it).
__device__ __forceinline__ uint32_t take_items(unsigned* ctr, uint32_t n, int lane) {
  uint32_t v = 0;
  if (lane == 0) v = atomicAdd(ctr, n);
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ void mark_sector(unsigned* touched, uint32_t i) {
  const unsigned bit = sector_bit(i);
  if (!(touched[sector_word(i)] & bit)) atomicOr(&touched[sector_word(i)], bit);
}

__device__ __forceinline__ bool selected(const RowArgs& A, int k) {
  return !A.sel_bits || ((__ldg(&A.sel_bits[k >> 5]) >> (k & 31)) & 1u);
}

// items: the counters that hand out the alpha-beta and alpha-double work items of each pass (next_item of
// this CTA, or of the cluster's first CTA when the cluster shares the target's lists).
template <int kRowThreads, int PASS>
__device__ void row_phase(const RowArgs& A, RowShared& sh, const RowDyn& dy, double* row, int crank, int gsz,
                          double& e_acc, unsigned* items) {
  constexpr bool SCATTER = PASS == kPassScatter;
  constexpr bool MARK = PASS == kPassMark;
  constexpr int kRowWarps = kRowThreads / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = A.H.n >> 1, ks = A.H.no, nvs = A.H.nv;
  const int n_tv = nvs * (nvs - 1) / 2;
  const int t_same = 1 + ks * nvs + (ks * (ks - 1) / 2) * n_tv;
  const int nch = (t_same + kSameChunk - 1) / kSameChunk;
  unsigned* touched = SCATTER ? dy.touched : nullptr;
  // beta-single table entries: rank | phase << 31, and when packed also the (occupied, virtual) spatial
  // pair i * m + j in bits 21..30 (rows of at most 2^21 entries)
  const bool packed = A.rbeta_packed != 0;
  const uint32_t rmask = packed ? 0x1FFFFFu : 0x7FFFFFFFu;
  const bool filt = SCATTER && (A.energy_only || A.n_probe > 0 || A.screen) && dy.touched != nullptr;
  // ---------------- X's own group: diagonal, beta singles, beta-beta doubles; items (determinant, chunk)
  const long long n_items_same = sh.gx_cnt * nch;
  for (long long u = (long long)crank * kRowWarps + warp; u < n_items_same; u += (long long)gsz * kRowWarps) {
    const long long j = u / nch;
    const int ch = (int)(u - j * nch);
    const long long di = sh.gx_off + j;
    const uint64_t d = __ldg(&A.gkey[di]);
    const double cd = __ldg(&A.gamp[di]);
    const uint32_t db = even_bits(d >> 1);
    warp_lists(sh, warp, lane, d, m);
    const uint8_t* oa = sh.occ_all[warp];
    if (ch == 0 && !MARK) {  // diagonal <D|H|D> = sum_i h_ii + 1/2 sum_ij <ij||ij>
      double hd = 0.0;
      for (int t2 = lane; t2 < A.H.ne; t2 += 32) {
        const int a = oa[t2];
        double jj = 0.0;
        for (int u2 = 0; u2 < A.H.ne; ++u2) jj += __ldg(&A.H.J[a * A.H.n + oa[u2]]);
        hd += __ldg(&A.H.h[a * A.H.n + a]) + 0.5 * jj;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hd += __shfl_xor_sync(0xffffffffu, hd, o);
      if (lane == 0) {
        const uint32_t rd = __ldg(&A.grank[di]);
        if (SCATTER) {
          if (take(touched, filt, rd)) atomicAdd(&row[rd], hd * cd);
        } else if (!MARK) {
          e_acc += cd * row[rd];
        }
      }
    }
    const int t_end = min(t_same, (ch + 1) * kSameChunk);
    const int ns1 = 1 + ks * nvs;  // targets 1 .. ns are the beta singles, then the beta-beta doubles
    for (int t = max(1, ch * kSameChunk) + lane; t < min(t_end, ns1); t += 32) {
      // beta single: rank and phase precomputed for this determinant
      const uint32_t code = dy.same_tab[t];
      const int o1 = code & 255, v1 = (code >> 16) & 255;
      const int i = sh.bocc[warp][o1], jv = sh.bvir[warp][v1];
      const uint32_t wb = __ldg(&A.rbeta[(size_t)di * (ks * nvs) + o1 * nvs + v1]);
      const uint32_t re = wb & rmask;
      const int sb = (int)(wb >> 31);
      const int p = 2 * i + 1, r = 2 * jv + 1;
      if (SCATTER) {
        if (take(touched, filt, re)) atomicAdd(&row[re], apply_sign(fock_single(A, oa, p, r), sb) * cd);
      } else {
        const int k = __ldg(&A.H.ops1[(p < r ? p : r) * A.H.n + (p < r ? r : p)]);
        if (selected(A, k)) {
          if (MARK) mark_sector(dy.touched, re);
          else atomicAdd(&A.g[k], apply_sign(cd * row[re], sb ^ (int)(p > r)));
        }
      }
    }
    // beta-beta doubles, four per lane: every target's loads are issued before the first atomic
    for (int t0 = max(ns1, ch * kSameChunk); t0 < t_end; t0 += 128) {
      uint32_t re[4];
      int ix[4], sg[4];
      double val[4];
      bool ok[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + u * 32 + lane;
        ok[u] = t < t_end;
        re[u] = 0;
        ix[u] = 0;
        sg[u] = 0;
        val[u] = 0.0;
        if (!ok[u]) continue;
        const uint32_t code = dy.same_tab[t];
        const int i1 = sh.bocc[warp][code & 255], i2 = sh.bocc[warp][(code >> 8) & 255];
        const int j1 = sh.bvir[warp][(code >> 16) & 255], j2 = sh.bvir[warp][code >> 24];
        re[u] = str_rank(A.rank_tab, ks, db ^ (1u << i1) ^ (1u << i2) ^ (1u << j1) ^ (1u << j2));
        if (SCATTER && filt && !take(touched, true, re[u])) { ok[u] = false; continue; }
        const int p = 2 * i1 + 1, q = 2 * i2 + 1, r = 2 * j1 + 1, s2 = 2 * j2 + 1;
        const int pa = pair_index(p, q, A.H.n), pb = pair_index(r, s2, A.H.n);
        sg[u] = double_phase(d, p, q, r, s2);
        if (SCATTER) {
          val[u] = __ldg(&A.H.G[(size_t)pa * A.H.npairs + pb]);
        } else {
          const bool down = pa > pb;
          ix[u] = __ldg(&A.H.opd[down ? (size_t)pb * A.H.npairs + pa : (size_t)pa * A.H.npairs + pb]);
          sg[u] ^= (int)down;
          if (!MARK) val[u] = row[re[u]];  // read alongside the operator index, used only if selected
        }
      }
      if (!SCATTER) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (!ok[u]) continue;
          if (!selected(A, ix[u])) ok[u] = false;
          else if (MARK) { mark_sector(dy.touched, re[u]); ok[u] = false; }
        }
      } else if (!filt) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (ok[u]) take(touched, false, re[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!ok[u]) continue;
        if (SCATTER) atomicAdd(&row[re[u]], apply_sign(val[u], sg[u]) * cd);
        else atomicAdd(&A.g[ix[u]], apply_sign(cd * val[u], sg[u]));
      }
    }
    __syncwarp();
  }
  // ---------------- alpha-single neighbours, the alpha single itself: one determinant per lane.  Each
  // lane sums its own Fock element h_qp + sum_{k in D} <qk||pk> (no warp reduction per determinant)
  // items of the neighbour groups: the alpha singles split by a fixed stride (over the cluster when every
  // CTA holds the target's whole lists, else within the CTA over the groups it found); the warps take the
  // items of the alpha-beta and alpha-double loops from shared counters (in the cluster's first CTA when
  // the lists are shared), so a warp that finishes early takes more and the waits at the barrier after the
  // pass stay short
  const bool merged = A.stage_ent_s > 0;
  const bool dyn = true;
  const uint32_t gwarp = (uint32_t)((merged ? crank * kRowWarps : 0) + warp);
  const uint32_t gwarps = (uint32_t)((merged ? gsz : 1) * kRowWarps);
  unsigned* const ctr_ab = items + 2 * PASS;
  unsigned* const ctr_d = items + 2 * PASS + 1;
  for (uint32_t t0 = gwarp * 32; t0 < sh.tot_s; t0 += gwarps * 32) {
    int e1 = warp_find_entry(dy.ents_s, sh.n_s, t0, lane);
    const int ej = e1 + lane;
    const uint32_t st = (lane > 0 && ej < sh.n_s) ? dy.ents_s[ej].flat - t0 : 32u;
    const unsigned starts = __reduce_or_sync(0xffffffffu, st < 32u ? 1u << st : 0u);
    e1 += __popc(starts & ((2u << lane) - 1u));
    const uint32_t t = t0 + lane;
    if (t >= sh.tot_s) continue;
    while (e1 + 1 < sh.n_s && dy.ents_s[e1 + 1].flat <= t) ++e1;
    const RowEnt en = dy.ents_s[e1];
    const long long di = (long long)en.off + (t - en.flat);
    const uint32_t rd = __ldg(&A.grank[di]);
    const int pa = en.o[0], pb = en.o[2];  // alpha spin-orbitals: removed, added
    if (SCATTER) {
      if (!take(touched, filt, rd)) continue;
      const uint64_t d = __ldg(&A.gkey[di]);
      const double cd = __ldg(&A.gamp[di]);
      const int n = A.H.n;
      const double* wv = A.H.Ws + ((size_t)pa * n + pb) * n;
      double f = __ldg(&A.H.h[pb * n + pa]);
      for (uint64_t x = d; x; x &= x - 1ull) f += __ldg(&wv[__ffsll((long long)x) - 1]);
      atomicAdd(&row[rd], apply_sign(f, single_phase(d, pa, pb)) * cd);
    } else if (MARK) {
      const int k = __ldg(&A.H.ops1[(pa < pb ? pa : pb) * A.H.n + (pa < pb ? pb : pa)]);
      if (selected(A, k)) mark_sector(dy.touched, rd);
    } else {
      row_pair<false>(A, row, touched, filt, __ldg(&A.gkey[di]), __ldg(&A.gamp[di]), rd, pa, -1, pb, -1, nullptr);
    }
  }
  // ---------------- alpha-single neighbours, alpha-beta doubles (warp per determinant).
  // Software pipeline over a warp's items: the next item's determinant, amplitude and first 128
  // beta-single entries are loaded while the current one is processed, so the item's chain of dependent
  // loads (state -> beta-single list -> integral -> row) overlaps the previous item's work.
  const int nsb = ks * nvs;
  int e = 0;  // entry of the prefetched item: a warp's items only increase, so walk forward
  long long di_n = 0;
  uint64_t d_n = 0;
  double cd_n = 0.0;
  uint32_t wb_n[4] = {0u, 0u, 0u, 0u};
  auto fetch = [&](uint32_t tt) {
    while (e + 1 < sh.n_s && dy.ents_s[e + 1].flat <= tt) ++e;
    const RowEnt en = dy.ents_s[e];
    di_n = (long long)en.off + (tt - en.flat);
    d_n = __ldg(&A.gkey[di_n]);
    cd_n = __ldg(&A.gamp[di_n]);
    const uint32_t* rb = A.rbeta + (size_t)di_n * nsb;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t2 = u * 32 + lane;
      wb_n[u] = t2 < nsb ? __ldg(&rb[t2]) : 0u;
    }
  };
  uint32_t t = dyn ? take_items(ctr_ab, 1, lane) : gwarp;
  if (t < sh.tot_s) fetch(t);
  while (t < sh.tot_s) {
    const uint32_t tn = dyn ? take_items(ctr_ab, 1, lane) : t + gwarps;  // this warp's next item
    const RowEnt en = dy.ents_s[e];
    const long long di = di_n;
    const uint64_t d = d_n;
    const double cd = cd_n;
    uint32_t wb0[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) wb0[u] = wb_n[u];
    if (tn < sh.tot_s) fetch(tn);
    if (!packed) warp_lists(sh, warp, lane, d, m);  // unpacked entries: pair indices from the beta lists
    const int pa = en.o[0], pb = en.o[2];  // alpha spin-orbitals: removed, added
    // alpha-beta doubles: phase = (beta single on D) ^ (alpha single on D) ^ (index-only bit in the tables);
    // four targets per lane with their loads issued together
    const int sa = single_phase(d, pa, pb);
    const size_t base = ((size_t)(pa >> 1) * m + (pb >> 1)) * (size_t)m * m;
    const uint32_t* rb = A.rbeta + (size_t)di * nsb;
    if (!SCATTER && A.screen) {  // screened: only the selected beta pairs (i -> j) of this alpha pair
      const int ab = (pa >> 1) * m + (pb >> 1);
      const int cnt = __ldg(&A.ab_cnt[ab]);
      const uint2* L = A.ab_list + (size_t)ab * m * m;
      const uint32_t dbs = even_bits(d >> 1);
      const uint32_t mmask = m >= 32 ? 0xFFFFFFFFu : (1u << m) - 1u;
      for (int q = lane; q < cnt; q += 32) {
        const uint2 ent = __ldg(&L[q]);
        const int i = (int)ent.x / m, j = (int)ent.x - i * m;
        if (!((dbs >> i) & 1u) || ((dbs >> j) & 1u)) continue;  // i must be occupied, j empty in D
        // slots of i among D's occupied and of j among its empty beta orbitals: D's beta-single entry
        const int o = __popc(dbs & ((1u << i) - 1u)), v = __popc(~dbs & mmask & ((1u << j) - 1u));
        const uint32_t wb = __ldg(&rb[o * nvs + v]);
        const uint32_t re = wb & rmask;
        if (MARK) {
          mark_sector(dy.touched, re);
        } else {
          const int kk = (int)ent.y;
          atomicAdd(&A.g[kk & 0x7FFFFFFF], apply_sign(cd * row[re], (int)(wb >> 31) ^ sa ^ (int)((unsigned)kk >> 31)));
        }
      }
      __syncwarp();
      t = tn;
      continue;
    }
    for (int t0 = 0; t0 < nsb; t0 += 128) {
      uint32_t wv[4];
      bool ok[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t2 = t0 + u * 32 + lane;
        ok[u] = t2 < nsb;
        wv[u] = t0 == 0 ? wb0[u] : (ok[u] ? __ldg(&rb[t2]) : 0u);
      }
      auto pair_ij = [&](int u) -> uint32_t {
        const int t2 = t0 + u * 32 + lane;
        return packed ? (wv[u] >> 21) & 1023u : (uint32_t)(sh.bocc[warp][t2 / nvs] * m + sh.bvir[warp][t2 % nvs]);
      };
      if (SCATTER) {
        if (filt) {  // energy only: almost every target is skipped, so test before loading the integral
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (!ok[u]) continue;
            const uint32_t re = wv[u] & rmask;
            if (!take(touched, true, re)) continue;
            atomicAdd(&row[re], apply_sign(__ldg(&A.gab[base + pair_ij(u)]), (int)(wv[u] >> 31) ^ sa) * cd);
          }
        } else {  // the four integral loads issued up front, off the atomics' dependency chain
          double gv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) gv[u] = ok[u] ? __ldg(&A.gab[base + pair_ij(u)]) : 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (!ok[u]) continue;
            const uint32_t re = wv[u] & rmask;
            take(touched, false, re);
            atomicAdd(&row[re], apply_sign(gv[u], (int)(wv[u] >> 31) ^ sa) * cd);
          }
        }
      } else {
        uint32_t re[4];
        int kk[4], sb[4];
        double sv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          re[u] = 0;
          kk[u] = 0;
          sb[u] = 0;
          sv[u] = 0.0;
          if (ok[u]) {  // the operator index and the row entry read together
            re[u] = wv[u] & rmask;
            sb[u] = (int)(wv[u] >> 31) ^ sa;
            kk[u] = __ldg(&A.kab[base + pair_ij(u)]);
            sv[u] = row[re[u]];
          }
        }
        if (A.sel_bits) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = kk[u] & 0x7FFFFFFF;
            if (ok[u] && !((__ldg(&A.sel_bits[k >> 5]) >> (k & 31)) & 1u)) ok[u] = false;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (ok[u]) atomicAdd(&A.g[kk[u] & 0x7FFFFFFF], apply_sign(cd * sv[u], sb[u] ^ (int)((unsigned)kk[u] >> 31)));
      }
    }
    __syncwarp();
    t = tn;
  }
  // ---------------- alpha-double neighbours: one determinant per lane; the warp finds the entry of
  // its first item, then each lane counts the entries that start at or before its own item (lane j
  // marks where entry e + j starts inside the warp's 32 items: groups hold at least one determinant,
  // so the starts are distinct and the walk below takes no step).  Every item of an entry is the same
  // pool operator, so the gather sums each entry's lanes in the warp and its first lane adds the total.
  const int npairs = A.H.npairs, n = A.H.n;
  for (uint32_t t0 = dyn ? take_items(ctr_d, 32, lane) : gwarp * 32; t0 < sh.tot_d;
       t0 = dyn ? take_items(ctr_d, 32, lane) : t0 + gwarps * 32) {
    int e = warp_find_entry(dy.ents_d, sh.n_d, t0, lane);
    const int ej = e + lane;
    const uint32_t st = (lane > 0 && ej < sh.n_d) ? dy.ents_d[ej].flat - t0 : 32u;
    const unsigned starts = __reduce_or_sync(0xffffffffu, st < 32u ? 1u << st : 0u) | 1u;
    e += __popc(starts & ((2u << lane) - 1u) & ~1u);
    const uint32_t t = t0 + lane;
    const bool live = t < sh.tot_d;
    double v = 0.0;
    int k = -1;
    if (live) {
      const RowEnt en = dy.ents_d[e];
      const long long di = (long long)en.off + (t - en.flat);
      const int p = en.o[0], q = en.o[1], r = en.o[2], s2 = en.o[3];
      const int pa = pair_index(p, q, n), pb = pair_index(r, s2, n);
      const uint32_t rd = __ldg(&A.grank[di]);
      if (SCATTER) {
        if (filt) {  // energy only: most pairs are skipped, so test before the other loads
          if (take(touched, true, rd)) {
            const double gv = __ldg(&A.H.G[(size_t)pa * npairs + pb]);
            const uint64_t d = __ldg(&A.gkey[di]);
            const double cd = __ldg(&A.gamp[di]);
            atomicAdd(&row[rd], apply_sign(gv, double_phase(d, p, q, r, s2)) * cd);
          }
        } else {  // every load issued together, off the rank's dependency chain
          const double gv = __ldg(&A.H.G[(size_t)pa * npairs + pb]);
          const uint64_t d = __ldg(&A.gkey[di]);
          const double cd = __ldg(&A.gamp[di]);
          take(touched, false, rd);
          atomicAdd(&row[rd], apply_sign(gv, double_phase(d, p, q, r, s2)) * cd);
        }
      } else {
        const bool down = pa > pb;
        k = __ldg(&A.H.opd[down ? (size_t)pb * npairs + pa : (size_t)pa * npairs + pb]);
        if (MARK) {
          if (!selected(A, k)) k = -1;
          if (k >= 0) mark_sector(dy.touched, rd);
        } else {  // the determinant and its row entry read alongside the operator index
          const uint64_t d = __ldg(&A.gkey[di]);
          const double cd = __ldg(&A.gamp[di]);
          const double sv = row[rd];
          if (!selected(A, k)) k = -1;
          if (k >= 0) v = apply_sign(cd * sv, double_phase(d, p, q, r, s2) ^ (int)down);
        }
      }
    }
    if (!SCATTER && !MARK) {
      // segmented sum over the lanes of each entry: lane + o is added while it is in the same entry
      const unsigned later = starts & ~((2u << lane) - 1u);  // starts after this lane
      const int seg_end = later ? __ffs(later) - 1 : 32;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + o < seg_end) v += w;
      }
      if (live && k >= 0 && ((starts >> lane) & 1u) && v != 0.0) atomicAdd(&A.g[k], v);
    }
  }
}

// Synchronisation of the CTAs that share a target's row: a thread-block cluster
// (the pool sweep's launch) or a single CTA (the batched persistent kernel).
struct ClusterSync {
  cg::cluster_group cl;
  __device__ void sync() {
    if (cl.num_blocks() == 1) __syncthreads();  // a cluster of one CTA: the CTA barrier orders the same accesses
    else cl.sync();
  }
  template <class T>
  __device__ T* remote(T* p, int r) { return cl.map_shared_rank(p, r); }
};
struct BlockSync {
  __device__ void sync() { __syncthreads(); }
  template <class T>
  __device__ T* remote(T* p, int) { return p; }
};

// Dynamic shared memory of a row-sweep CTA, laid out for A's sector.
__device__ __forceinline__ RowDyn row_dyn(unsigned char* dyn, const RowArgs& A) {
  const int ks = A.H.no, nvs = A.H.nv;
  const int t_same = 1 + ks * nvs + (ks * (ks - 1) / 2) * (nvs * (nvs - 1) / 2);
  RowDyn dy;
  dy.ents_s = (RowEnt*)dyn;
  dy.ents_d = dy.ents_s + A.max_ent_s;
  dy.stage_s = A.stage_ent_s > 0 ? dy.ents_d + A.max_ent_d : dy.ents_s;
  dy.stage_d = A.stage_ent_s > 0 ? dy.stage_s + A.stage_ent_s : dy.ents_d;
  dy.same_tab = (uint32_t*)(A.stage_ent_s > 0 ? dy.stage_d + A.stage_ent_d : dy.ents_d + A.max_ent_d);
  dy.touched = A.touched_words > 0 ? (unsigned*)(dy.same_tab + t_same) : nullptr;
  return dy;
}

// Per-CTA tables of a sector: pair decodings, the decode table of a target's own
// excitations, a clean touched bitmap.
template <int kRowThreads>
__device__ void row_cta_init(const RowArgs& A, RowShared& sh, const RowDyn& dy) {
  const int ks = A.H.no, nvs = A.H.nv;
  const int n_to = ks * (ks - 1) / 2, n_tv = nvs * (nvs - 1) / 2;
  const int ns = ks * nvs, nd = n_to * n_tv;
  const int t_same = 1 + ns + nd;
  const int nwords = A.touched_words;
  for (int t = threadIdx.x; t < n_to || t < n_tv; t += blockDim.x) {
    auto dec = [](int t, int L) -> uint16_t {
      int a = 0, base = 0;
      while (base + (L - 1 - a) <= t) { base += L - 1 - a; ++a; }
      return (uint16_t)(a | ((a + 1 + (t - base)) << 8));
    };
    if (t < n_to) sh.tri_o[t] = dec(t, ks);
    if (t < n_tv) sh.tri_v[t] = dec(t, nvs);
  }
  for (int w = threadIdx.x; w < nwords; w += kRowThreads) dy.touched[w] = 0u;
  __syncthreads();
  for (int t = 1 + threadIdx.x; t < t_same; t += kRowThreads) {
    uint32_t code;
    if (t - 1 < ns) {
      code = (uint32_t)((t - 1) / nvs) | (255u << 8) | ((uint32_t)((t - 1) % nvs) << 16);
    } else {
      const int dd = t - 1 - ns;
      const uint16_t oo = sh.tri_o[dd / n_tv], vv = sh.tri_v[dd % n_tv];
      code = (uint32_t)(oo & 255) | ((uint32_t)(oo >> 8) << 8) | ((uint32_t)(vv & 255) << 16) | ((uint32_t)(vv >> 8) << 24);
    }
    dy.same_tab[t] = code;
  }
  __syncthreads();
}

// Zeroes the row entries this CTA touched for its last target (each CTA clears its own sectors), or its
// slice of the whole row when there is no touched bitmap.
template <int kRowThreads>
__device__ void row_clear(const RowArgs& A, const RowDyn& dy, double* row, int crank, int gsz) {
  const int nwords = A.touched_words;
  if (dy.touched) {  // clear the entries this CTA touched (others clear theirs)
    for (int w = threadIdx.x; w < nwords; w += kRowThreads) {
      unsigned bits = dy.touched[w];
      if (!bits) continue;
      dy.touched[w] = 0u;
      while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        const int64_t e0 = ((int64_t)w * 32 + b) * 4;  // first entry of the sector
        if (e0 + 3 < A.NB) {  // a whole sector in one 32-byte store: rows start on 32-byte boundaries
          asm volatile("st.global.v4.b64 [%0], {%1, %1, %1, %1};" ::"l"(__cvta_generic_to_global(row + e0)), "l"(0ull)
                       : "memory");
        } else {
          for (int64_t e = e0; e < A.NB; ++e) row[e] = 0.0;
        }
      }
    }
  } else {  // clear this CTA's slice of the row
    const int64_t per = (A.NB + gsz - 1) / gsz;
    const int64_t b = per * crank, e = (A.NB < b + per) ? A.NB : b + per;
    for (int64_t i = b + threadIdx.x; i < e; i += kRowThreads) row[i] = 0.0;
  }
}

// One target alpha string xi of the sweep: discovery of its neighbour groups,
// scatter, gather (or the energy / probe read-back), clear.  Every CTA of the
// target's group calls it with the same xi.
template <int kRowThreads, class Sync>
__device__ void row_target(const RowArgs& A, RowShared& sh, const RowDyn& dy, double* row, int xi, bool probe,
                           bool screen, int crank, int gsz, Sync& sy, double& e_acc, unsigned& n_lookups,
                           unsigned& n_probe_slots, bool defer_clear) {
  const int m = A.H.n >> 1, ks = A.H.no, nvs = A.H.nv;
  const int n_to = ks * (ks - 1) / 2, n_tv = nvs * (nvs - 1) / 2;
  const int ns = ks * nvs, nd = n_to * n_tv;
  const int nwords = A.touched_words;
  const bool merged = A.stage_ent_s > 0;  // the cluster merges its CTAs' entries (clusters of 2 or more)
  (void)n_to;
  const uint32_t X = probe ? __ldg(&A.probe_x[xi]) : A.alpha_list[xi];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const bool inr = lane < m;
    const bool o = inr && ((X >> lane) & 1u);
    const unsigned bo = __ballot_sync(0xffffffffu, o), bv = __ballot_sync(0xffffffffu, inr && !o);
    const unsigned below = (1u << lane) - 1u;
    if (o) sh.occx[__popc(bo & below)] = (uint8_t)lane;
    else if (inr) sh.virx[__popc(bv & below)] = (uint8_t)lane;
    if (lane < 6) (&sh.next_item[0][0])[lane] = 0u;  // every CTA of the cluster is past the last target's passes
    if (lane == 0) {
      sh.n_s_loc = 0;
      sh.n_d_loc = 0;
      const int64_t g = idx_lookup(A.atab, A.amask, (uint64_t)X);
      sh.gx_off = g >= 0 ? A.goff[g] : 0;
      sh.gx_cnt = g >= 0 ? A.goff[g + 1] - A.goff[g] : 0;
    }
  }
  __syncthreads();
  if (A.energy_only && sh.gx_cnt == 0) return;  // same decision in every CTA of the cluster
  // Candidates c = 0 .. ns+nd-1 (alpha singles then doubles of X); this CTA takes c = crank (mod gsz), each
  // thread up to kDisc at a time with their home slots read together.  A clear of the previous target that
  // was deferred to here runs while those reads are in flight.
  constexpr int kDisc = 3;
  const int n_cand = ns + nd;
  for (int r = 0;; ++r) {
    const int cb = (int)threadIdx.x + r * kDisc * kRowThreads;
    if (r > 0 && crank + cb * gsz >= n_cand) break;
    uint32_t Yk[kDisc], ok4[kDisc];
    IdxSlot sl[kDisc];
#pragma unroll
    for (int k = 0; k < kDisc; ++k) {
      const int c = crank + (cb + k * kRowThreads) * gsz;
      Yk[k] = 0u;
      ok4[k] = 0u;
      sl[k].key = kEmpty;
      sl[k].idx = 0;
      if (c >= n_cand) continue;
      uint32_t Y;
      uint8_t o4[4];
      if (c < ns) {
        const int b = sh.occx[c / nvs], a = sh.virx[c % nvs];
        Y = X ^ (1u << b) ^ (1u << a);
        o4[0] = (uint8_t)(2 * a); o4[1] = 0; o4[2] = (uint8_t)(2 * b); o4[3] = 0;
      } else {
        const int dd = c - ns;
        const uint16_t oo = sh.tri_o[dd / n_tv], vv = sh.tri_v[dd % n_tv];
        const int b1 = sh.occx[oo & 255], b2 = sh.occx[oo >> 8];
        const int a1 = sh.virx[vv & 255], a2 = sh.virx[vv >> 8];
        Y = X ^ (1u << b1) ^ (1u << b2) ^ (1u << a1) ^ (1u << a2);
        o4[0] = (uint8_t)(2 * a1); o4[1] = (uint8_t)(2 * a2); o4[2] = (uint8_t)(2 * b1); o4[3] = (uint8_t)(2 * b2);
      }
      Yk[k] = Y;
      ok4[k] = (uint32_t)o4[0] | ((uint32_t)o4[1] << 8) | ((uint32_t)o4[2] << 16) | ((uint32_t)o4[3] << 24);
      sl[k] = A.atab[mix64((uint64_t)Y) & A.amask];
    }
    if (r == 0 && defer_clear) row_clear<kRowThreads>(A, dy, row, crank, gsz);
#pragma unroll
    for (int k = 0; k < kDisc; ++k) {
      const int c = crank + (cb + k * kRowThreads) * gsz;
      if (c >= n_cand) continue;
      const uint64_t Y = Yk[k];
      int64_t g;
      unsigned* pc = A.probe_ctr ? &n_probe_slots : nullptr;
      if (sl[k].key == Y || sl[k].key == kEmpty) {
        g = sl[k].key == Y ? (int64_t)sl[k].idx : -1;
        if (pc) *pc += 1u;
      } else {
        g = idx_lookup_at(A.atab, A.amask, Y, (mix64(Y) + 1) & A.amask, 1, pc);
      }
      if (A.probe_ctr) ++n_lookups;
      if (g >= 0) {
        RowEnt en;
        en.off = (uint32_t)A.goff[g];
        en.flat = (uint32_t)(A.goff[g + 1] - A.goff[g]);
        en.o[0] = (uint8_t)ok4[k]; en.o[1] = (uint8_t)(ok4[k] >> 8);
        en.o[2] = (uint8_t)(ok4[k] >> 16); en.o[3] = (uint8_t)(ok4[k] >> 24);
        const int cap_s = merged ? A.stage_ent_s : A.max_ent_s, cap_d = merged ? A.stage_ent_d : A.max_ent_d;
        if (c < ns) {
          const int slot = atomicAdd(&sh.n_s_loc, 1);
          if (slot < cap_s) dy.stage_s[slot] = en;
        } else {
          const int slot = atomicAdd(&sh.n_d_loc, 1);
          if (slot < cap_d) dy.stage_d[slot] = en;
        }
      }
    }
  }
  __syncthreads();
  // the entries that will be read back (after this CTA's clear of the previous target's sectors)
  if (A.energy_only && dy.touched) {  // X's own determinants
    for (long long t = threadIdx.x; t < sh.gx_cnt; t += kRowThreads) {
      const uint32_t rk = __ldg(&A.grank[sh.gx_off + t]);
      atomicOr(&dy.touched[sector_word(rk)], sector_bit(rk));
    }
  }
  if (probe && dy.touched) {  // the requested entries of X
    for (int t = __ldg(&A.probe_off[xi]) + threadIdx.x; t < __ldg(&A.probe_off[xi + 1]); t += kRowThreads) {
      const uint32_t rk = __ldg(&A.probe_rank[t]);
      atomicOr(&dy.touched[sector_word(rk)], sector_bit(rk));
    }
  }
  if (threadIdx.x == 0) {
    const int cap_s = merged ? A.stage_ent_s : A.max_ent_s, cap_d = merged ? A.stage_ent_d : A.max_ent_d;
    if (sh.n_s_loc > cap_s || sh.n_d_loc > cap_d) set_error(A.err, kDevBadState);
    sh.n_s_loc = min(sh.n_s_loc, cap_s);
    sh.n_d_loc = min(sh.n_d_loc, cap_d);
    if (!merged) {
      sh.n_s = sh.n_s_loc;
      sh.n_d = sh.n_d_loc;
    }
  }
  // every CTA's share of the discovery is complete, and so is every CTA's clear of the previous target's
  // sectors (the clear flows straight into this target's discovery)
  sy.sync();
  if (merged) {
    // the cluster's entries in rank order, copied into every CTA, so that the work items of the whole
    // target can be split evenly over all CTAs whatever the sizes of the groups each CTA found
    int bs = 0, bd = 0;
    for (int r = 0; r < gsz; ++r) {
      const int ns_r = *sy.remote(&sh.n_s_loc, r), nd_r = *sy.remote(&sh.n_d_loc, r);
      const RowEnt* ss = sy.remote(dy.stage_s, r);
      const RowEnt* sd = sy.remote(dy.stage_d, r);
      for (int t = threadIdx.x; t < ns_r && bs + t < A.max_ent_s; t += kRowThreads) dy.ents_s[bs + t] = ss[t];
      for (int t = threadIdx.x; t < nd_r && bd + t < A.max_ent_d; t += kRowThreads) dy.ents_d[bd + t] = sd[t];
      bs += ns_r;
      bd += nd_r;
    }
    if (threadIdx.x == 0) {
      if (bs > A.max_ent_s || bd > A.max_ent_d) set_error(A.err, kDevBadState);
      sh.n_s = min(bs, A.max_ent_s);
      sh.n_d = min(bd, A.max_ent_d);
    }
  }
  __syncthreads();
  scan_items<kRowThreads>(sh, dy.ents_s, sh.n_s, 1, &sh.tot_s);
  scan_items<kRowThreads>(sh, dy.ents_d, sh.n_d, kDblChunk, &sh.tot_d);
  unsigned* items = merged ? sy.remote(&sh.next_item[0][0], 0) : &sh.next_item[0][0];

  if (screen) {
    // the sectors the selected operators read (and the state's own determinants, for the energy),
    // marked by every CTA for its share of the pairs, then merged over the cluster
    for (long long t = threadIdx.x; t < sh.gx_cnt; t += kRowThreads) mark_sector(dy.touched, __ldg(&A.grank[sh.gx_off + t]));
    row_phase<kRowThreads, kPassMark>(A, sh, dy, row, crank, gsz, e_acc, items);
    sy.sync();  // every CTA's marks are complete
    for (int w = threadIdx.x; w < nwords; w += kRowThreads) {
      unsigned bits = 0u;
      for (int r = 0; r < gsz; ++r)
        if (r != crank) bits |= sy.remote(dy.touched, r)[w];
      if (bits) atomicOr(&dy.touched[w], bits);
    }
    __syncthreads();
  }
  row_phase<kRowThreads, kPassScatter>(A, sh, dy, row, crank, gsz, e_acc, items);
  sy.sync();
  if (probe) {  // the requested entries, split over the cluster
    const int t0 = __ldg(&A.probe_off[xi]), t1 = __ldg(&A.probe_off[xi + 1]);
    for (int t = t0 + crank * kRowThreads + (int)threadIdx.x; t < t1; t += gsz * kRowThreads)
      A.probe_out[t] = row[__ldg(&A.probe_rank[t])];
  } else if (A.energy_only) {  // sigma_D of the determinants of X's own group
    for (long long t = (long long)crank * kRowThreads + threadIdx.x; t < sh.gx_cnt; t += (long long)gsz * kRowThreads) {
      const long long di = sh.gx_off + t;
      const double sg = row[__ldg(&A.grank[di])];
      e_acc += __ldg(&A.gamp[di]) * sg;
      if (A.sig_out) A.sig_out[A.gorig[di]] = sg;
    }
  } else {
    row_phase<kRowThreads, kPassGather>(A, sh, dy, row, crank, gsz, e_acc, items);
  }
  sy.sync();
  if (!defer_clear) row_clear<kRowThreads>(A, dy, row, crank, gsz);
}

// End of a CTA's sweep: hash-probe counters and its part of the energy numerator.
template <int kRowThreads>
__device__ void row_flush(const RowArgs& A, RowShared& sh, double e_acc, unsigned n_lookups, unsigned n_probe_slots) {
  constexpr int kRowWarps = kRowThreads / 32;
  if (A.probe_ctr && (n_lookups | n_probe_slots)) {
    atomicAdd(&A.probe_ctr[0], (unsigned long long)n_lookups);
    atomicAdd(&A.probe_ctr[1], (unsigned long long)n_probe_slots);
  }
  // energy numerator
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
  if (lane == 0) sh.red[warp] = e_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kRowWarps; ++w) s += sh.red[w];
    if (s != 0.0) atomicAdd(&A.acc[0], s);
  }
}

// ---------------------------------------------------------------- grouping by alpha string
// Each step works on the items i = i0, i0 + step, ... below its count: the
// kernels below pass the grid's stride, the batched persistent kernel a tile's.
__device__ __forceinline__ void group_insert_items(const uint64_t* keys, long long n, IdxSlot* tab, uint64_t mask,
                                                   const double* amps, double* acc, long long i0, long long step) {
  double s2 = 0.0;
  for (long long i = i0; i < n; i += step) {
    const uint64_t a = even_bits(keys[i]);
    uint64_t s = mix64(a) & mask;
    for (uint64_t k = 0; k <= mask; ++k) {
      const unsigned long long prev =
          atomicCAS((unsigned long long*)&tab[s].key, (unsigned long long)kEmpty, (unsigned long long)a);
      if (prev == kEmpty || prev == a) break;
      s = (s + 1) & mask;
    }
    s2 += amps[i] * amps[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31) == 0 && s2 != 0.0) atomicAdd(&acc[1], s2);
}

__device__ __forceinline__ void group_ids_items(IdxSlot* tab, uint64_t cap, unsigned long long* n_groups,
                                                uint64_t i0, uint64_t step) {
  for (uint64_t i = i0; i < cap; i += step)
    if (tab[i].key != kEmpty) tab[i].idx = atomicAdd(n_groups, 1ull);
}

__device__ __forceinline__ void group_count_items(const uint64_t* keys, long long n, const IdxSlot* tab, uint64_t mask,
                                                  uint32_t* gid_of, long long* gcount, long long i0, long long step) {
  for (long long i = i0; i < n; i += step) {
    const int64_t g = idx_lookup(tab, mask, (uint64_t)even_bits(keys[i]));
    gid_of[i] = (uint32_t)g;
    atomicAdd((unsigned long long*)&gcount[g], 1ull);
  }
}

// Exclusive scan of gcount[0..G) into goff[0..G] by one block (part: blockDim.x longs of shared memory).
__device__ __forceinline__ void group_scan_block(const long long* gcount, long long G, long long* goff, long long* part) {
  const long long per = (G + blockDim.x - 1) / blockDim.x;
  const long long b = threadIdx.x * per, e = min(G, b + per);
  long long s = 0;
  for (long long i = b; i < e; ++i) s += gcount[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const long long v = part[t];
      part[t] = run;
      run += v;
    }
    goff[G] = run;
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (long long i = b; i < e; ++i) {
    goff[i] = run;
    run += gcount[i];
  }
}

__device__ __forceinline__ void group_scatter_items(const uint64_t* keys, const double* amps, long long n,
                                                    const uint32_t* gid_of, const long long* goff, long long* gfill,
                                                    uint64_t* gkey, double* gamp, uint32_t* grank, uint32_t* gorig,
                                                    const uint32_t* rank_tab, int ks, long long i0, long long step) {
  for (long long i = i0; i < n; i += step) {
    const uint32_t g = gid_of[i];
    const long long pos = goff[g] + (long long)atomicAdd((unsigned long long*)&gfill[g], 1ull);
    const uint64_t d = keys[i];
    gkey[pos] = d;
    gamp[pos] = amps[i];
    grank[pos] = str_rank(rank_tab, ks, even_bits(d >> 1));
    gorig[pos] = (uint32_t)i;
  }
}

// Beta single excitations of grouped determinants di = w0, w0 + nw, ... (one warp each): rank of the
// new beta string and the phase bit of a+_{2j+1} a_{2i+1} on D, t = occ_slot*nv + vir_slot.
__device__ __forceinline__ void rbeta_dets(const uint64_t* gkey, long long n, const uint32_t* rank_tab, int ks, int nv,
                                           int m, int packed, uint32_t* rbeta, long long w0, long long nw) {
  const int lane = threadIdx.x & 31;
  for (long long di = w0; di < n; di += nw) {
    const uint64_t d = gkey[di];
    const uint32_t db = even_bits(d >> 1);
    // slot -> orbital via the o-th set / unset bit of the beta string
    for (int t = lane; t < ks * nv; t += 32) {
      const int o = t / nv, v = t - o * nv;
      uint32_t x = db;
      for (int c = 0; c < o; ++c) x &= x - 1;
      const int i = __ffs(x) - 1;
      uint32_t y = ~db & ((m >= 32) ? 0xFFFFFFFFu : ((1u << m) - 1u));
      for (int c = 0; c < v; ++c) y &= y - 1;
      const int j = __ffs(y) - 1;
      const uint32_t re = str_rank(rank_tab, ks, db ^ (1u << i) ^ (1u << j));
      const int sb = single_phase(d, 2 * i + 1, 2 * j + 1);
      const uint32_t ij = packed ? ((uint32_t)(i * m + j) << 21) : 0u;
      rbeta[(size_t)di * (ks * nv) + t] = re | ij | ((uint32_t)sb << 31);
    }
  }
}

}  // namespace
}  // namespace swcs
