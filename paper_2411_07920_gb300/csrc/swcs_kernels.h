// Internal interface between the C-ABI host code and the kernels.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include "swcs_device.cuh"

namespace swcs {

constexpr int kAnsatzThreads = 1024;        // gate kernel CTA, one state on the device
constexpr int kAnsatzThreadsShared = 256;   // gate kernel CTA, instances sharing the device
constexpr int kSigmaThreads = 256;
constexpr int kMaxSpin = 32;  // spin-orbitals of one spin (n_so <= 64)
constexpr size_t kAnsatzHistWords = 2 * 12 * 4096;  // radix-select histograms of the gate kernel

struct AnsatzArgs {
  uint64_t* keys_a;  // state S (input and output), capacity cap
  double* amps_a;
  uint64_t* keys_b;  // merged set Phi (scratch), capacity cap
  double* amps_b;
  int64_t cap;
  IdxSlot* tab[2];  // index tables of S; tab[tab_cur] indexes the input state
  uint64_t tab_mask;
  int tab_cur;
  const uint8_t* ops;  // 5 bytes per gate
  const double* cs;    // (cos theta, sin theta) per gate
  int n_ops;
  int64_t n_keep;      // <= 0: no size criterion
  uint64_t min_abs_bits;  // |c| bit patterns below this are dropped (1: exact zeros; 0: none; else the magnitude criterion)
  int reset_to_hf;
  uint64_t hf;
  long long* n_state;  // in: input size (unless reset_to_hf); out: output size
  int* tab_cur_out;    // out: which table indexes the output state
  unsigned long long* ctr;  // 12 counters
  unsigned* hist;           // kAnsatzHistWords: two sets of 12 passes x 4096 bins
  GridBar* bar;
  int* err;
  uint64_t timeout_ns;
  // optional per-gate snapshots of the kept state (adjoint replay)
  uint64_t* snap_keys;
  double* snap_amps;
  long long* snap_n;
  int64_t snap_stride;
  long long* stats;  // optional: [0] gates, [1] select passes, [6] max |Phi|, [7] sum of input sizes
  int skip_arrive_block;  // test hook: this CTA never arrives at its first grid barrier (-1: off)
  unsigned long long* probe_ctr;  // optional (nullptr: off): [0] partner lookups, [1] slots they visited
};

int ansatz_blocks_per_sm(int threads);
cudaError_t launch_ansatz(const AnsatzArgs& a, int nblocks, int threads, cudaStream_t st);

// Hamiltonian and pool tables on the device.
struct HamDev {
  int n;        // spin-orbitals
  int ne;       // electrons
  int no;       // occupied per spin (ne/2)
  int nv;       // virtual per spin (n/2 - no)
  int npairs;   // n(n-1)/2
  const double* h;     // [n*n]        h[p*n+q]
  const double* J;     // [n*n]        <ij||ij>
  const double* Ws;    // [n*n*n]      Ws[(p*n+q)*n+k] = <qk||pk>
  const double* G;     // [npairs^2]   G[P(p,q)*npairs + P(r,s)] = <rs||pq>
  const int* opd;      // [npairs^2]   pool index of doubles (lower pair, upper pair) or -1
  const int* ops1;     // [n*n]        pool index of singles (lo, hi) or -1
  int64_t pool_size;
};

__host__ __device__ __forceinline__ int pair_index(int p, int q, int n) {  // p < q
  return p * (2 * n - p - 1) / 2 + (q - p - 1);
}

struct StateDev {
  const uint64_t* keys;
  const double* amps;
  long long* n;  // device count
  const IdxSlot* tab;
  uint64_t tab_mask;
};

struct ExtTable {
  ValSlot* slots;
  uint64_t mask;
  unsigned nbucket_log2;  // buckets B = 2^nbucket_log2
  unsigned bucket;        // current bucket
  unsigned long long* n_distinct;
  int* err;
};

// Energy (sigma restricted to S): acc[0] += sum c_D sigma_D, acc[1] += sum c_D^2.
cudaError_t launch_energy(const HamDev& H, const StateDev& S, double* acc, int nblocks, cudaStream_t st);
// Energy as above and sigma_D for each determinant of S (state order) into sig_out.
cudaError_t launch_energy_sigma(const HamDev& H, const StateDev& S, double* acc, double* sig_out, int nblocks,
                                cudaStream_t st);
// Pool sweep pass 1: sigma_E += <E|H|D> c_D for E in bucket.
cudaError_t launch_sigma_scatter(const HamDev& H, const StateDev& S, const ExtTable& T, int nblocks,
                                 cudaStream_t st);
// Pool sweep pass 2: g[k(D,E)] += dir * phase * c_D * sigma_E for E in bucket;
// acc[0] += c_D sigma_D, acc[1] += c_D^2 (only once: when add_norm).
cudaError_t launch_pool_gather(const HamDev& H, const StateDev& S, const ExtTable& T, double* g, double* acc,
                               int add_norm, int nblocks, cudaStream_t st);
cudaError_t launch_clear_ext(ValSlot* slots, uint64_t n, cudaStream_t st);
cudaError_t launch_finalize_energy(const double* acc, double* out, cudaStream_t st);
cudaError_t launch_scale_gradient(double* g, int64_t n, const double* acc, cudaStream_t st);
cudaError_t launch_gather_subset(const double* g, const int64_t* subset, int64_t n, double* out, cudaStream_t st);
int sigma_blocks_per_sm();

// Row sweep (alpha-string rows): see swcs_rowsweep.cu.
struct RowArgs {
  HamDev H;
  const uint64_t* gkey;   // state grouped by alpha string
  const double* gamp;
  const uint32_t* grank;  // rank of each determinant's beta string
  const long long* goff;  // [G+1] group offsets
  const IdxSlot* atab;    // alpha string -> group id
  uint64_t amask;
  const uint32_t* alpha_list;  // every alpha string of the sector
  int NA;
  const uint32_t* rank_tab;    // [4][ks+1][256]
  double* rows;                // [clusters][NB rounded up to a multiple of 4]
  int64_t NB;
  double* g;
  double* acc;                 // acc[0] += sum c_D sigma_D
  int* err;
  int max_ent_s, max_ent_d;  // capacity of the target's entry lists (all CTAs of its cluster together)
  int stage_ent_s, stage_ent_d;
  unsigned* target_ctr;  // zeroed before the launch: hands out the targets of one-CTA rows (nullptr: fixed shares)  // capacity of one CTA's share before the cluster merges them (0: one CTA per target)
  int touched_words;  // words of the per-CTA touched-sector bitmap, one bit per 4 entries (0: clear whole rows)
  const uint32_t* sel_bits;  // pool operators to evaluate (nullptr: all)
  // beta single excitations of each grouped determinant, t = occ_slot*nv + vir_slot:
  // rank of the new beta string | (phase bit << 31)
  const uint32_t* rbeta;
  int rbeta_packed;  // entries also carry the spatial pair i * m + j in bits 21..30 (NB <= 2^21)
  // alpha-beta doubles by spatial indices (a -> b alpha, i -> j beta), [m^4]:
  // integral with the index-only part of the phase folded in, and the pool
  // index | (direction and index-only phase bit << 31)
  const double* gab;
  const int* kab;
  // energy-only mode: visit only alpha strings of the state, gather only the
  // diagonal entries sigma_D (into sig_out[gorig[D]] when sig_out is given)
  int energy_only;
  double* sig_out;
  const uint32_t* gorig;
  const unsigned long long* n_groups;  // groups of the state (energy only: the targets are these alpha strings)
  // probe mode (n_probe > 0): visit only the listed alpha strings, scatter only into the row sectors of
  // the listed beta ranks and read those entries back: sigma_E at arbitrary determinants E
  int n_probe;                 // alpha strings to visit
  const uint32_t* probe_x;     // [n_probe] the alpha strings
  const int* probe_off;        // [n_probe + 1] each string's range in probe_rank / probe_out
  const uint32_t* probe_rank;  // beta-string ranks of the requested determinants
  double* probe_out;           // sigma of each requested determinant
  // sharded pool sweep (n_shards > 1): only the target alpha strings of colex rank = shard (mod n_shards),
  // i.e. every E whose alpha string that rank owns; g and acc[0] are then that shard's partial sums
  int shard, n_shards;
  // screened sweep (screen != 0, with sel_bits): before each target's scatter the row sectors of every
  // E = A_k D with k selected, and of the state's own determinants, are marked (the cluster's marks
  // merged); the scatter then forms sigma only in marked sectors, skipping every other pair before its
  // integral load, and the alpha-beta gather walks, per alpha pair a*m + b, only the selected
  // (beta pair i*m + j, kab entry) of ab_list[(a*m + b) * m*m ...] (ab_cnt of them)
  int screen;
  const int* ab_cnt;
  const uint2* ab_list;
  // optional hash-probe counters (nullptr: off): [0] alpha-string lookups, [1] slots they visited
  unsigned long long* probe_ctr;
};

struct GroupArgs {
  const uint64_t* keys;
  const double* amps;
  const long long* n;
  IdxSlot* atab;
  uint64_t amask;
  unsigned long long* n_groups;
  uint32_t* gid_of;
  long long* gcount;
  long long* goff;
  long long* gfill;
  uint64_t* gkey;
  double* gamp;
  uint32_t* grank;
  uint32_t* gorig;  // original state index of each grouped determinant
  const uint32_t* rank_tab;
  int ks;
  double* acc;  // acc[1] += sum c^2
};

size_t row_sweep_smem(int max_ent_s, int max_ent_d, int stage_ent_s, int stage_ent_d, int t_same, int touched_words);
cudaError_t row_sweep_max_clusters(int threads, int occ, int gsz, size_t smem, int* n_clusters);
cudaError_t launch_row_sweep(const RowArgs& a, int threads, int occ, int gsz, int n_clusters, size_t smem,
                             cudaStream_t st);
cudaError_t launch_group_state(const GroupArgs& g, cudaStream_t st);
// State of the top-N radix select (gate kernel: every CTA keeps an identical copy in shared memory;
// batched kernel: one copy per instance in global memory).
struct SelState {
  unsigned long long prefix;   // |c| bits decided so far
  unsigned long long kprefix;  // bitstring bits decided so far (tie mode)
  long long need;              // rank still to place within the current bucket
  int shift;                   // lowest bit of the last decided |c| digit
  int kshift;                  // lowest bit of the last decided key digit
  int mode;                    // 0 none (keep all nonzero), 1 cut on |c|, 2 cut on |c| then key
  int pass;                    // passes run
  int bin;                     // result of the last bin search
  long long cum, cnt;          // entries before that bin in selection order, entries in it
};

// ---------------------------------------------------------------------------
// Batched persistent launch (swcs_batch.cu).  Every instance runs through a
// chain of phases -- initial tables; per gate the gate pass, the select passes
// still needed and the compaction; the grouping by alpha string; the beta-single
// tables; the row sweep, one target alpha string per tile; the finish -- and
// each phase is split into tiles.  One persistent kernel drains all instances'
// tiles: a CTA takes the next tile of some instance's current phase from that
// instance's (phase, next tile) word; the CTA that finishes a phase's last tile
// runs its epilogue and publishes the next phase.
enum BatchPhase : int {
  kPhInit = 0, kPhBuild0, kPhGate, kPhSelect, kPhCompact, kPhGroupClear, kPhGroupInsert, kPhGroupIds,
  kPhGroupCount, kPhGroupScan, kPhGroupScatter, kPhRbeta, kPhRow, kPhFinish, kPhDone
};

struct BatchInst {
  AnsatzArgs ga;       // gate sequence: state, tables, ops, cos/sin, n_keep, counters, histograms, error word
  GroupArgs gr;        // grouping by alpha string (gr.n unused: the phase passes the state size)
  RowArgs ra;          // row sweep (ra.rows unused: every CTA has its own row)
  int n_ops;
  int tile;            // items per tile of the element-wise phases
  int ks, nvs, m, packed;
  uint64_t acap;       // alpha-string table capacity
  double* g;           // pool gradient [pool_size]
  int64_t pool_size;
  double* eout;        // E, <psi|psi>
};

// One published phase of an instance (two slots, by parity of the phase number).
struct BatchSlot {
  unsigned phase;      // phase number this slot describes
  int type;            // BatchPhase
  unsigned ntiles;
  int gate, pass;
  long long n, m;      // state size entering the gate, merged size
};

struct BatchSched {
  unsigned long long word;  // phase number << 32 | next tile
  unsigned done;            // tiles of the current phase finished
  int tab_cur;
  unsigned ep;              // epoch of tab[tab_cur]'s build
  int pad;
  BatchSlot slot[2];
  SelState sel;             // the current gate's radix select
};

size_t batch_dyn_smem(int max_ent_s, int max_ent_d, int t_same, int touched_words);
int batch_blocks_per_sm(size_t dyn_smem);
cudaError_t launch_batch(const BatchInst* d_inst, BatchSched* d_sched, int n_inst, double* d_rows, int64_t row_stride,
                         int* d_status, int nblocks, size_t dyn_smem, uint64_t timeout_ns, cudaStream_t st);

// Selected alpha-beta doubles per alpha pair for the screened sweep (see RowArgs::screen).
cudaError_t launch_screen_lists(const int* kab, int m, const uint32_t* sel_bits, int* ab_cnt, uint2* ab_list,
                                cudaStream_t st);
cudaError_t launch_rbeta(const uint64_t* gkey, const long long* n, const uint32_t* rank_tab, int ks, int nv, int m,
                         int packed, uint32_t* rbeta, cudaStream_t st);

// Adjoint (swcs_adjoint.cu).
cudaError_t launch_build_index(const uint64_t* keys, const long long* n, IdxSlot* tab, uint64_t mask, cudaStream_t st);
cudaError_t launch_nu_init(const double* amps, const double* sigma, const long long* n, const double* acc, double* nu,
                           cudaStream_t st);
struct AdjArgs {
  const uint8_t* op;     // this gate
  const double* cs;      // its (cos, sin)
  const uint64_t* keys;  // S_g (before the gate), with its index table
  const double* amps;
  const long long* n;
  const IdxSlot* tab;
  uint64_t mask;
  const IdxSlot* tab_nu;  // index of the arrays nu_in is aligned with (S_{g+1})
  uint64_t mask_nu;
  const double* nu_in;
  double* nu_out;         // aligned with S_g
  double* dtheta;         // accumulates the (unscaled) gradient of this gate
};
cudaError_t launch_adjoint_gate(const AdjArgs& a, int nblocks, cudaStream_t st);
cudaError_t launch_scale_dtheta(double* d, int n, const double* acc, cudaStream_t st);

// Screening network (swcs_mlp.cu).
enum GemmMode { kGemmF32 = 0, kGemmReluBf16 = 1, kGemmReluBf16Dot = 2 };
struct GemmArgs {
  const __nv_bfloat16* A;  // [M x K], row stride lda (elements), K contiguous
  const __nv_bfloat16* B;  // [N x K], row stride ldb
  int lda, ldb;
  int M, N, K;             // N in [16, 256], N % 16 == 0, K % 32 == 0
  int mode;
  const float* bias;       // [N] (ReLU modes)
  float* out_f32;          // kGemmF32: [M x N], row stride ldo
  __nv_bfloat16* out_bf16; // ReLU modes: [M x N], row stride ldo
  int ldo;
  const __nv_bfloat16* w3; // kGemmReluBf16Dot: y[row] = sum_j out[row][j] w3[j] + b3
  float b3;
  float* y;
  int* err;
};
struct MlpParams {
  float* master;
  float* m;
  float* v;
  int n_params, d_in, width;
  int off_W1, off_b1, off_W2, off_b2, off_w3, off_b3;
  __nv_bfloat16* W1b;
  __nv_bfloat16* W2b;
  __nv_bfloat16* W2tb;
  __nv_bfloat16* w3b;
};
cudaError_t launch_mlp_gemm(const GemmArgs& g, cudaStream_t st);
// Pipelined form with tensor maps of A ([M x K], boxes of 8 x 128) and B ([N x K], boxes of 8 x N); splits > 1
// (kGemmF32 only) adds partial products into out_f32, which must hold zeros.
cudaError_t launch_mlp_gemm_tma(const CUtensorMap& tm_a, const CUtensorMap& tm_b, const GemmArgs& g, int splits,
                                cudaStream_t st);
int mlp_gemm_tma_kc(int K);
// The w3 dot product of the last layer is summed as kDotGroups partial sums over
// consecutive 16-column chunks (chunk c of n belongs to group g when
// dot_group_begin(g, n) <= c < dot_group_begin(g + 1, n)), combined as
// ((p0 + p1) + p2) + p3; the fused kernel gives each group its own warps, the
// layer-by-layer kernel sums the same way, so both round identically.
constexpr int kDotGroups = 4;
__host__ __device__ __forceinline__ int dot_group_begin(int g, int nchunks) { return g * nchunks / kDotGroups; }
// UCCSD guess and overlap (swcs_guess.cu).
cudaError_t launch_mp2(const HamDev& H, const uint8_t* ijab, int64_t nd, double* t, cudaStream_t st);
cudaError_t launch_overlap(const StateDev& S, const uint64_t* keys, const double* amps, int64_t n, double* out,
                           int nblocks, cudaStream_t st);
// Fused inference forward (all three layers in one persistent tcgen05 kernel).
struct FusedArgs {
  int64_t M;                // rows (pool operators)
  int d_in, width;          // d_in % 16 == 0, 16..64; width % 16 == 0, 16..256
  const float* b1;          // [width]
  const float* b2;          // [width]
  const __nv_bfloat16* w3;  // [width]
  const float* b3;          // [1]
  float* y;                 // [M]
  int* err;
};
size_t mlp_fused_smem_bytes(int d_in, int width);
cudaError_t launch_mlp_fused(const CUtensorMap& tm_x, const CUtensorMap& tm_w1, const CUtensorMap& tm_w2,
                             const FusedArgs& f, int nblocks, cudaStream_t st);
cudaError_t launch_mlp_dy(const float* y, const float* t, int B, float* dy, double* loss, cudaStream_t st);
cudaError_t launch_mlp_dz2(const float* dy, const __nv_bfloat16* w3, const __nv_bfloat16* H2, int B, int W,
                           __nv_bfloat16* dZ2, float* dw3, float* db3, cudaStream_t st);
cudaError_t launch_mlp_dz1(const float* dH1, const __nv_bfloat16* H1, size_t n, __nv_bfloat16* dZ1, cudaStream_t st);
cudaError_t launch_mlp_colsum(const __nv_bfloat16* Z, int B, int W, float* db, cudaStream_t st);
cudaError_t launch_mlp_transpose(const __nv_bfloat16* in, int R, int C, int Rpad, __nv_bfloat16* out, cudaStream_t st);
cudaError_t launch_mlp_adam(const MlpParams& p, const float* grad, float lr, int step, cudaStream_t st);
cudaError_t launch_mlp_refresh(const MlpParams& p, cudaStream_t st);

// Pool features and top-k selection (swcs_screen.cu).
constexpr int kFeatures = 32;
cudaError_t launch_pool_features(const HamDev& H, const StateDev& S, const uint8_t* pool_ops, int64_t n_pool,
                                 double* occ, __nv_bfloat16* x, cudaStream_t st);
cudaError_t launch_topk(const float* y, int64_t n, int64_t k, unsigned* hist, unsigned long long* ctl,
                        int64_t* out_idx, cudaStream_t st);
cudaError_t launch_subset_bits(const int64_t* subset, int64_t n, uint32_t* bits, int64_t n_pool, cudaStream_t st);
cudaError_t launch_log_abs(const double* g, int64_t n, float* t, cudaStream_t st);

// Hamiltonian preparation from the full <pq||rs> array on the device.
cudaError_t launch_pack_hamiltonian(const double* g_full, int n, double* J, double* Ws, double* G,
                                    cudaStream_t st);

}  // namespace swcs
