// Pool-gradient sweep organised by alpha strings ("row sweep").
//
// The quantity is the same as the hashed sweep (ADAPT step 4, Sec. II.C):
//   sigma_E = sum_{D in S} <E|H|D> c_D   for every E connected to S,
//   g_k     = (2/<psi|psi>) sum_{(D,E)} dir * phase * c_D * sigma_E,
// but the external space is walked one target alpha string X at a time.
// Every determinant is a pair (alpha string, beta string); a connected pair
// (D, E) with E_alpha = X has D_alpha = X (beta-side excitation or the
// diagonal), D_alpha one alpha single away from X (alpha single or
// alpha-beta double) or one alpha double away (alpha-alpha double).  For a
// fixed X all sigma_E therefore live in one dense row indexed by the
// combinatorial rank of E_beta (C(n/2, n_e/2) doubles, 1.84 MB at 52/12),
// owned by one thread-block cluster while it works on X:
//   1. the cluster finds the alpha groups of S at distance 0, 1, 2 from X
//      (alpha-string hash table of S);
//   2. scatter: every pair adds <E|H|D> c_D into row[rank(E_beta)], marking
//      the 32-byte sector it touched;
//   3. cluster barrier; gather: every pair adds dir*phase*c_D*row[...] to
//      g_k, and the diagonal pairs give the energy numerator;
//   4. cluster barrier; each CTA zeroes the sectors it touched, finds the
//      next X's neighbours, and waits at the barrier before its scatter.
// No hashing or compare-and-swap on sigma.  The rows of all clusters share L2;
// when they exceed it (228 rows at 52/12) their sectors spill to HBM.
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "swcs_device.cuh"
#include "swcs_kernels.h"
#include "swcs_rowsweep.cuh"

namespace cg = cooperative_groups;

namespace swcs {

namespace {

template <int kRowThreads, int kMinBlocks>
__global__ void __launch_bounds__(kRowThreads, kMinBlocks)
row_sweep_kernel(RowArgs A) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ RowShared sh;
  __shared__ int s_next[2];
  ClusterSync sy{cg::this_cluster()};
  const int crank = (int)sy.cl.block_rank();
  const int gsz = (int)sy.cl.num_blocks();
  const int cid = blockIdx.x / gsz, ncl = gridDim.x / gsz;
  double* row = A.rows + (size_t)cid * (size_t)((A.NB + 3) & ~(int64_t)3);  // rows padded to whole 32-byte sectors
  const RowDyn dy = row_dyn(dyn, A);
  row_cta_init<kRowThreads>(A, sh, dy);
  double e_acc = 0.0;
  unsigned n_lookups = 0, n_probe_slots = 0;  // hash-probe counters (when requested)

  // targets: every alpha string of the sector in colex order (in energy-only mode those that hold no
  // determinant of the state return at once: nothing of theirs is read back), in probe mode the listed ones
  const bool probe = A.n_probe > 0;
  const bool screen = A.screen && A.sel_bits && dy.touched && !probe && !A.energy_only;
  const int n_targets = probe ? A.n_probe : A.NA;
  // a shard of the pool sweep visits the alpha strings xi = shard (mod n_shards) only (alpha_list is in
  // colex order, so xi is the string's rank)
  const int n_sh = (probe || A.energy_only || A.n_shards < 1) ? 1 : A.n_shards;
  const int sh0 = n_sh > 1 ? A.shard : 0;
  const int n_own = n_targets > sh0 ? (n_targets - sh0 + n_sh - 1) / n_sh : 0;
  // rows are zeroed before the launch, so the clear of a CTA's last target can be left out (deferred clears)
  if (A.target_ctr) {
    // targets handed out in rank order from a counter, so a CTA (or cluster) whose targets were cheap takes
    // more and all finish together (a fixed share of the targets each left the last ones working alone for
    // several percent of the launch).  The cluster's first CTA takes the index and every CTA reads it there;
    // the two slots alternate, so a slot is rewritten only after the barriers of the target that read it.
    for (int it = 0;; ++it) {
      if (crank == 0 && threadIdx.x == 0) s_next[it & 1] = (int)atomicAdd(A.target_ctr, 1u);
      sy.sync();
      const int jx = *sy.remote(&s_next[it & 1], 0);
      if (jx >= n_own) {
        sy.sync();  // no CTA leaves while another still reads its shared memory
        break;
      }
      row_target<kRowThreads>(A, sh, dy, row, sh0 + jx * n_sh, probe, screen, crank, gsz, sy, e_acc, n_lookups,
                              n_probe_slots, true);
    }
  } else {
    for (int jx = cid; jx < n_own; jx += ncl)
      row_target<kRowThreads>(A, sh, dy, row, sh0 + jx * n_sh, probe, screen, crank, gsz, sy, e_acc, n_lookups,
                              n_probe_slots, true);
  }
  row_flush<kRowThreads>(A, sh, e_acc, n_lookups, n_probe_slots);
}

__global__ void group_insert_kernel(const uint64_t* keys, const long long* n_ptr, IdxSlot* tab, uint64_t mask,
                                    const double* amps, double* acc) {
  group_insert_items(keys, *n_ptr, tab, mask, amps, acc, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                     (long long)gridDim.x * blockDim.x);
}

__global__ void group_ids_kernel(IdxSlot* tab, uint64_t cap, unsigned long long* n_groups) {
  group_ids_items(tab, cap, n_groups, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

__global__ void group_count_kernel(const uint64_t* keys, const long long* n_ptr, const IdxSlot* tab, uint64_t mask,
                                   uint32_t* gid_of, long long* gcount) {
  group_count_items(keys, *n_ptr, tab, mask, gid_of, gcount, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                    (long long)gridDim.x * blockDim.x);
}

__global__ void group_scan_kernel(const long long* gcount, const unsigned long long* n_groups, long long* goff) {
  __shared__ long long part[1024];
  group_scan_block(gcount, (long long)*n_groups, goff, part);
}

__global__ void group_scatter_kernel(const uint64_t* keys, const double* amps, const long long* n_ptr,
                                     const uint32_t* gid_of, const long long* goff, long long* gfill,
                                     uint64_t* gkey, double* gamp, uint32_t* grank, uint32_t* gorig,
                                     const uint32_t* rank_tab, int ks) {
  group_scatter_items(keys, amps, *n_ptr, gid_of, goff, gfill, gkey, gamp, grank, gorig, rank_tab, ks,
                      (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

__global__ void rbeta_kernel(const uint64_t* gkey, const long long* n_ptr, const uint32_t* rank_tab, int ks, int nv,
                             int m, int packed, uint32_t* rbeta) {
  rbeta_dets(gkey, *n_ptr, rank_tab, ks, nv, m, packed, rbeta, ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
             ((long long)gridDim.x * blockDim.x) >> 5);
}

// Per alpha pair (a, b) the selected alpha-beta doubles: (beta pair i*m + j, kab entry) for every
// (i, j) whose pool operator is selected; one block per alpha pair, order within a pair arbitrary.
__global__ void screen_lists_kernel(const int* kab, int m, const uint32_t* sel_bits, int* ab_cnt, uint2* ab_list) {
  __shared__ int cnt;
  const int ab = blockIdx.x, m2 = m * m;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int ij = threadIdx.x; ij < m2; ij += blockDim.x) {
    const int kk = kab[(size_t)ab * m2 + ij];
    if (kk == -1) continue;  // a = b or i = j: no operator
    const int k = kk & 0x7FFFFFFF;
    if (!((sel_bits[k >> 5] >> (k & 31)) & 1u)) continue;
    const int pos = atomicAdd(&cnt, 1);
    ab_list[(size_t)ab * m2 + pos] = make_uint2((unsigned)ij, (unsigned)kk);
  }
  __syncthreads();
  if (threadIdx.x == 0) ab_cnt[ab] = cnt;
}

}  // namespace

cudaError_t launch_screen_lists(const int* kab, int m, const uint32_t* sel_bits, int* ab_cnt, uint2* ab_list,
                                cudaStream_t st) {
  screen_lists_kernel<<<m * m, 256, 0, st>>>(kab, m, sel_bits, ab_cnt, ab_list);
  return cudaGetLastError();
}

cudaError_t launch_rbeta(const uint64_t* gkey, const long long* n, const uint32_t* rank_tab, int ks, int nv, int m,
                         int packed, uint32_t* rbeta, cudaStream_t st) {
  rbeta_kernel<<<1216, 256, 0, st>>>(gkey, n, rank_tab, ks, nv, m, packed, rbeta);
  return cudaGetLastError();
}

size_t row_sweep_smem(int max_ent_s, int max_ent_d, int stage_ent_s, int stage_ent_d, int t_same, int touched_words) {
  return sizeof(RowEnt) * (size_t)(max_ent_s + max_ent_d + stage_ent_s + stage_ent_d) + 4 * (size_t)t_same +
         4 * (size_t)touched_words;
}

namespace {
template <int NT, int MB>
cudaError_t max_clusters_t(int gsz, size_t smem, int* n_clusters) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gsz * 64);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = gsz;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaFuncSetAttribute(row_sweep_kernel<NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (gsz > 8) {
    e = cudaFuncSetAttribute(row_sweep_kernel<NT, MB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveClusters(n_clusters, row_sweep_kernel<NT, MB>, &cfg);
}

template <int NT, int MB>
cudaError_t launch_t(const RowArgs& a, int gsz, int n_clusters, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gsz * n_clusters);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = gsz;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, row_sweep_kernel<NT, MB>, a);
}
}  // namespace

// threads: 128, 256, 512 or 1024 per CTA; resident 512-thread CTAs per SM requested
// from the compiler: 1 (no register cap), 2 (64 registers) or 3 (40 registers); 1024-thread CTAs: one
// per SM (64 registers)
cudaError_t row_sweep_max_clusters(int threads, int occ, int gsz, size_t smem, int* n_clusters) {
  if (threads == 128) return max_clusters_t<128, 1>(gsz, smem, n_clusters);
  if (threads == 256) return max_clusters_t<256, 1>(gsz, smem, n_clusters);
  if (threads == 512) return occ >= 3 ? max_clusters_t<512, 3>(gsz, smem, n_clusters)
                             : occ == 2 ? max_clusters_t<512, 2>(gsz, smem, n_clusters)
                                        : max_clusters_t<512, 1>(gsz, smem, n_clusters);
  if (threads == 1024) return max_clusters_t<1024, 1>(gsz, smem, n_clusters);
  return cudaErrorInvalidValue;
}

cudaError_t launch_row_sweep(const RowArgs& a, int threads, int occ, int gsz, int n_clusters, size_t smem,
                             cudaStream_t st) {
  if (threads == 128) return launch_t<128, 1>(a, gsz, n_clusters, smem, st);
  if (threads == 256) return launch_t<256, 1>(a, gsz, n_clusters, smem, st);
  if (threads == 512) return occ >= 3 ? launch_t<512, 3>(a, gsz, n_clusters, smem, st)
                             : occ == 2 ? launch_t<512, 2>(a, gsz, n_clusters, smem, st)
                                        : launch_t<512, 1>(a, gsz, n_clusters, smem, st);
  if (threads == 1024) return launch_t<1024, 1>(a, gsz, n_clusters, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_group_state(const GroupArgs& g, cudaStream_t st) {
  const int nb = 1216;
  group_insert_kernel<<<nb, 256, 0, st>>>(g.keys, g.n, g.atab, g.amask, g.amps, g.acc);
  group_ids_kernel<<<nb, 256, 0, st>>>(g.atab, g.amask + 1, g.n_groups);
  group_count_kernel<<<nb, 256, 0, st>>>(g.keys, g.n, g.atab, g.amask, g.gid_of, g.gcount);
  group_scan_kernel<<<1, 1024, 0, st>>>(g.gcount, g.n_groups, g.goff);
  group_scatter_kernel<<<nb, 256, 0, st>>>(g.keys, g.amps, g.n, g.gid_of, g.goff, g.gfill, g.gkey, g.gamp, g.grank,
                                           g.gorig, g.rank_tab, g.ks);
  return cudaGetLastError();
}

}  // namespace swcs
