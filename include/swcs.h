/*
 * swcs.h -- C ABI of the GB300 sparse wavefunction circuit solver (SWCS).
 *
 * The operations are those of ADAPT-VQE with a sparse determinant state
 * (arXiv 2411.07920):
 *   - the factorized ansatz prod_I U_I(theta_I) |Psi_0> with one-parameter
 *     unitaries U = exp(theta (tau - tau^dag)) over single and double
 *     excitations (Sec. II.A, Eqs. 1-3), each evaluated exactly (Sec. II.B);
 *   - truncation of the state to the N_CUT largest |amplitude| after every
 *     gate (Sec. II.B, Fig. 1);
 *   - the energy <psi|H|psi>/<psi|psi> (Sec. II, Fig. 1 step 7);
 *   - the operator-pool gradient over the generalized singles and doubles
 *     pool, g_k = dE/dtheta_k for U_k appended at the end (Sec. II.C, step 4);
 *   - the analytic gradient dE/dtheta of the truncated circuit (Sec. II.B).
 *
 * Conventions
 *   Determinant: uint64_t occupation bitstring, bit p = spin-orbital p,
 *     p = 2*spatial + spin (spin 0 = alpha).  The reference |Psi_0> has bits
 *     0..n_elec-1 set.  Bits >= n_so are zero.
 *   Operator: 5 bytes {kind, i0, i1, i2, i3}
 *     kind 1: tau = a+_{i1} a_{i0}
 *     kind 2: tau = a+_{i2} a+_{i3} a_{i1} a_{i0}
 *     phase of a_p / a+_p on D = (-1)^(occupied spin-orbitals below p).
 *     The index sets {i0,i1} and {i2,i3} must be disjoint and S_z-conserving.
 *   ops[0] acts first on |Psi_0>.
 *   Pool (canonical order): singles (p<q, same spin) tau = a+_q a_p by (p,q);
 *     then doubles over disjoint pairs (p<q) < (r<s) with equal spin content,
 *     tau = a+_r a+_s a_q a_p, by ((p,q),(r,s)).
 *   Truncation keeps the n_keep largest |c|; equal |c| at the cut keep the
 *     smaller bitstring; exact zeros are removed.  The state is not
 *     renormalised; energies and gradients use the Rayleigh quotient.
 *
 * Memory and streams
 *   A context owns its device memory (allocated on first need, grown, freed
 *   by swcs_destroy) and issues all work on the CUDA stream given at
 *   creation (NULL = legacy default stream).  Pointers named h_* are host
 *   memory, d_* device memory; both stay owned by the caller and are not
 *   retained after the call returns.  Functions that return values in host
 *   memory synchronise the stream; *_dev variants only enqueue work.
 *   A context must not be used from two host threads at once.
 *
 * Errors
 *   Every function returns SWCS_OK (0) or a negative SWCS_ERR_* code and
 *   records a message readable with swcs_last_error().  On error the state
 *   held by the context is unspecified until the next swcs_apply_ansatz or
 *   swcs_set_state.  No call aborts the process or traps the GPU: device
 *   waits are bounded and report SWCS_ERR_TIMEOUT.
 */
#ifndef SWCS_H
#define SWCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swcs_ctx swcs_ctx;

enum swcs_status {
  SWCS_OK = 0,
  SWCS_ERR_INVALID_ARG = -1, /* bad size, index, op, or missing Hamiltonian/state */
  SWCS_ERR_OOM = -2,         /* device or pinned-host allocation failed */
  SWCS_ERR_TABLE_FULL = -3,  /* a hash table could not be grown enough */
  SWCS_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
  SWCS_ERR_CUDA = -5,        /* a CUDA runtime call failed (message has details) */
  SWCS_ERR_NO_DEVICE = -6    /* no sm_103 device / kernel image for this device */
};

/* Create a context bound to the current CUDA device and to cuda_stream
 * (a cudaStream_t, or NULL).  *out receives the handle. */
int swcs_create(swcs_ctx** out, void* cuda_stream);
int swcs_destroy(swcs_ctx* ctx);
/* Last error message of this context (static string when ctx is NULL). */
const char* swcs_last_error(const swcs_ctx* ctx);

/* Hamiltonian H = sum h_pq a+_p a_q + 1/4 sum <pq||rs> a+_p a+_q a_s a_r
 * (Sec. II; integrals as produced for Sec. III).
 *   h_h   [n_so*n_so]       h[p*n_so + q], real symmetric
 *   h_g   [n_so^4]          <pq||rs> at ((p*n_so + q)*n_so + r)*n_so + s,
 *                           antisymmetric in (p,q) and (r,s), <pq||rs> = <rs||pq>
 *   n_so  even, 4 <= n_so <= 64;  n_elec even, 2 <= n_elec < n_so
 *         (closed-shell S_z = 0 sector: n_elec/2 electrons of each spin).
 * Copies the data; clears the state. */
int swcs_load_hamiltonian(swcs_ctx* ctx, const double* h_h, const double* h_g, int n_so, int n_elec);

/* Size and operators of the generalized singles and doubles pool (Sec. II.C). */
int swcs_pool_size(swcs_ctx* ctx, int64_t* n_out);
int swcs_pool_ops(swcs_ctx* ctx, uint8_t* h_ops_out /* 5*pool_size bytes */);

/* Spin complements of the pool operators (Sec. III: spin-complemented
 * operators for closed-shell molecules).  With F the spin flip of every
 * spin-orbital (2i + s -> 2i + 1 - s), the flipped generator F(kappa_k) equals
 * sign[k] * kappa_{partner[k]}, kappa = tau - tau^dag.  The spin-complemented
 * operator of the pair is kappa_k + sign[k] kappa_{partner[k]} (2 kappa_k when
 * partner[k] == k and sign[k] == +1; zero, hence not an operator, when
 * partner[k] == k and sign[k] == -1); its gradient is g_k + sign[k] g_partner.
 *   partner  [pool_size] host, int64;  sign  [pool_size] host, +1 or -1. */
int swcs_pool_spin_pairs(swcs_ctx* ctx, int64_t* partner, int8_t* sign);

/* MP2-ordered UCCSD ansatz (Sec. II.A, operators of Eqs. 2-3 relative to the
 * reference): every S_z-conserving double i<j -> a<b (i, j occupied, a, b
 * virtual; op bytes {2, i, j, a, b}) with its first-order amplitude as initial
 * parameter, t = <ab||ij> / (e_i + e_j - e_a - e_b), e_p = h_pp + sum over the
 * occupied k of <pk||pk>, largest |t| first (equal |t| keep the canonical
 * (i, j, a, b) order); then every S_z-conserving single i -> a ({1, i, a, 0, 0})
 * with parameter 0.  *n_out receives the operator count; h_ops [5*cap] and
 * h_theta [cap] are written only when cap is large enough (pass NULL to size).
 * Feed the result to swcs_apply_ansatz / swcs_energy_grad. */
int swcs_mp2_uccsd(swcs_ctx* ctx, uint8_t* h_ops, double* h_theta, int64_t cap, int64_t* n_out);

/* Overlap of the context's state with a sparse state given by the caller
 * (distinct determinants, real amplitudes), for the infidelity against a
 * reference wavefunction (Sec. IV.B): out4 = {<state|given>, <state|state>,
 * <given|given>, 1 - <state|given>^2 / (<state|state> <given|given>)}.
 * h_keys, h_amps [n] host; out4 [4] host.  Synchronises. */
int swcs_overlap(swcs_ctx* ctx, const uint64_t* h_keys, const double* h_amps, int64_t n, double* out4);

/* Evaluate the ansatz (Eq. 1) from |Psi_0>, truncating to n_keep after every
 * gate (n_keep <= 0: no truncation).  h_ops: 5*n_ops bytes; h_theta: n_ops.
 * The resulting state stays on the device in the context. */
int swcs_apply_ansatz(swcs_ctx* ctx, const uint8_t* h_ops, const double* h_theta, int n_ops, int64_t n_keep);
int swcs_apply_ansatz_dev(swcs_ctx* ctx, const uint8_t* d_ops, const double* d_theta, int n_ops, int64_t n_keep);
/* Continue from the current state (no reset to |Psi_0>). */
int swcs_apply_gates(swcs_ctx* ctx, const uint8_t* h_ops, const double* h_theta, int n_ops, int64_t n_keep);
/* Truncate the current state alone (same rule as after a gate). */
int swcs_truncate(swcs_ctx* ctx, int64_t n_keep);

/* Magnitude criterion of the truncation (Sec. II.B, the alternative to a
 * fixed determinant count): from now on every truncation of this context
 * (after each gate of swcs_apply_ansatz / swcs_apply_gates / swcs_truncate,
 * and in the forward replays of swcs_energy_grad, whose projectors are the
 * kept sets) first drops every determinant with |c| < eps, then keeps the
 * n_keep largest of the rest (n_keep <= 0: all of them; n_keep also bounds
 * the memory).  eps = 0 (the default) restores the count-only rule.
 * SWCS_ERR_INVALID_ARG for a negative or non-finite eps. */
int swcs_set_truncation_threshold(swcs_ctx* ctx, double eps);

/* E = <psi|H|psi>/<psi|psi> and <psi|psi> of the current state. */
int swcs_energy(swcs_ctx* ctx, double* h_e_out, double* h_norm2_out);
/* Device variant: d_out[0] = E, d_out[1] = <psi|psi>. */
int swcs_energy_dev(swcs_ctx* ctx, double* d_out);

/* Pool gradient g_k = 2 <psi|H A_k|psi>/<psi|psi>, A_k = tau_k - tau_k^dag,
 * for the canonical pool (ADAPT step 4, Sec. II.C).  h_subset == NULL:
 * all pool entries are written to h_g_out[pool_size]; otherwise only
 * h_g_out[h_subset[i]] for i < n_subset (other entries untouched).  With a
 * subset the device variant's alpha-string row sweep first marks, for each
 * target alpha string, the row sectors that the selected operators read (and
 * those of the state's own determinants, so the energy stays exact), forms
 * sigma only there -- every other connected pair is skipped before its
 * integral is loaded -- and contracts only the selected operators (option
 * "screen_scatter" 0: form sigma in full, filter the contractions only).
 * The host variant evaluates the whole pool and copies the subset out. */
int swcs_pool_gradients(swcs_ctx* ctx, double* h_g_out, const int64_t* h_subset, int64_t n_subset);
int swcs_pool_gradients_dev(swcs_ctx* ctx, double* d_g_out, const int64_t* d_subset, int64_t n_subset);
/* One shard of the pool sweep for a run over n_shards GPUs (one process per
 * GPU, each holding the same state).  The shards partition the external
 * determinants E by the colex rank of their alpha string (rank mod n_shards
 * = shard), so every sigma_E is formed by exactly one shard and a single
 * sum over the shards completes the sweep (ADAPT step 4, Sec. II.C, spread
 * over devices):
 *   d_graw  [pool_size] device: sum over this shard's connected pairs of
 *           dir * phase * c_D * sigma_E (the gradient before its factor
 *           2/<psi|psi>), overwritten
 *   d_acc   [2] device: this shard's part of sum_D c_D sigma_D (the energy
 *           numerator), and <psi|psi> (the whole state's, the same on every shard)
 * After an all-reduce (sum) of d_graw and d_acc[0] over the shards:
 * g = 2 d_graw / d_acc[1], E = d_acc[0] / d_acc[1].  Only enqueues work on the
 * context's stream.  SWCS_ERR_INVALID_ARG unless 0 <= shard < n_shards, or
 * where the alpha-string row sweep does not apply. */
int swcs_pool_gradients_partial_dev(swcs_ctx* ctx, int shard, int n_shards, double* d_graw, double* d_acc);
/* The pool sweep forms sigma on every determinant of the state as well, so it
 * also yields E = <psi|H|psi>/<psi|psi>: returns that value from the last
 * swcs_pool_gradients* call (synchronises). */
int swcs_sweep_energy(swcs_ctx* ctx, double* h_e_out, double* h_norm2_out);

/* Energy and dE/dtheta of the truncated ansatz, each truncation held as a
 * fixed projector onto its kept set (Sec. II.B, "analytic gradients").  A
 * kept set holds every determinant the gate reaches, exact-zero amplitudes
 * included (they rank below every nonzero |c| for the size criterion; the
 * magnitude criterion drops them): without a cut the projector is the
 * identity on the reachable determinants, so the derivative is exact, also
 * at theta_g = 0 where the gate's partner determinants have c = 0.
 * The forward pass keeps a copy of the state every ckpt_every gates
 * (ckpt_every <= 0: 20); the backward pass replays each segment from its
 * checkpoint.  Leaves the final state in the context. */
int swcs_energy_grad(swcs_ctx* ctx, const uint8_t* h_ops, const double* h_theta, int n_ops, int64_t n_keep,
                     int ckpt_every, double* h_e_out, double* h_dtheta_out);

/* Current state size; copy-out sorted by bitstring (returns the size in *n_out;
 * writes only when cap >= size); copy-in (duplicates are summed, zeros dropped). */
int swcs_state_size(swcs_ctx* ctx, int64_t* n_out);
int swcs_get_state(swcs_ctx* ctx, uint64_t* h_keys, double* h_amps, int64_t cap, int64_t* n_out);
int swcs_set_state(swcs_ctx* ctx, const uint64_t* h_keys, const double* h_amps, int64_t n);
/* sigma_D = (H psi)_D for every determinant D of the current state (the
 * vector the energy kernel forms), with the bitstrings, sorted by bitstring;
 * same size/cap convention as swcs_get_state. */
int swcs_get_sigma(swcs_ctx* ctx, uint64_t* h_keys, double* h_sigma, int64_t cap, int64_t* n_out);
/* sigma_E = (H psi)_E = sum_{D in S} <E|H|D> c_D at arbitrary determinants E
 * of the sector, in or outside the state: the external sigma the pool
 * gradient contracts (ADAPT step 4, Sec. II.C), read out of the pool sweep's
 * own alpha-string rows.  The sweep visits only the alpha strings of the
 * given determinants and scatters only into the row sectors they occupy.
 *   h_keys   [n] determinants (any order, repeats allowed); a key outside the
 *            sector (bits >= n_so, wrong electron count, S_z != 0) gives
 *            SWCS_ERR_INVALID_ARG and nothing is computed
 *   h_sigma  [n] output, in the order of h_keys
 * Needs a non-empty state; SWCS_ERR_INVALID_ARG where the row sweep does
 * not apply (beta-string space above 2^22 strings).  Synchronises. */
int swcs_sigma_at(swcs_ctx* ctx, const uint64_t* h_keys, int64_t n, double* h_sigma);

/* Diagnostics accumulated since the last swcs_profile_read(.., reset=1):
 * {gates applied, radix-select passes, distinct determinants in the last
 * external sigma table, its bucket count, its capacity, kernel launches,
 * largest merged set |Phi|, sum over gates of the input state size
 * (gate x determinant applications)}. */
int swcs_stats(swcs_ctx* ctx, int64_t* h_out8);
/* Hash-probe counts accumulated while option "count_probes" is 1 (off by
 * default; counting adds a few integer operations per lookup):
 * {partner lookups of the gate kernel (merge of Sec. II.B), index slots they
 * visited, alpha-string lookups of the row sweep's neighbour discovery, slots
 * they visited}.  Synchronises; reset != 0 clears them.  The paper has no
 * counterpart: a measurement of the open-addressing tables. */
int swcs_probe_counts(swcs_ctx* ctx, int64_t* h_out4, int reset);

/* Tuning options (no effect on results beyond FP64 summation order):
 *   "sweep"    0 automatic (default), 1 hashed external-sigma table,
 *              2 alpha-string rows (SWCS_ERR_INVALID_ARG when the sector's
 *              beta-string space exceeds 2^22 or clusters cannot launch)
 *   "cluster"  CTAs per alpha-string row in the row sweep, 1..16 (default 1)
 *   "threads"  threads per CTA of the row sweep: 128, 256, 512 or 1024 (default 1024)
 *   "energy"   energy and sigma_D: 0 automatic (alpha-string rows when the
 *              sector allows, default), 1 probe kernel (connections of each D
 *              looked up in the state's index), 2 rows
 *   "row_occupancy" resident 512-thread CTAs per SM the row sweep is compiled
 *              for: 2 (default, 64 registers), 3 (40 registers) or 1 (no cap)
 *   "wait_timeout_ms"  bound of every device-side wait (default 2000)
 *   "ext_capacity"  hashed sweep: capacity of its first external table (0,
 *              default: from an estimate); a too-small table is regrown
 *   "test_skip_arrive"  test hook: the given CTA of the gate kernel leaves
 *              before its first grid barrier so the others' bounded waits
 *              run out (-1, default: off); the call then returns
 *              SWCS_ERR_TIMEOUT and the context stays usable
 *   "gate_blocks"   CTAs of the persistent gate kernel (0, default: whole device)
 *   "row_clusters"  clusters of the row sweep (0, default: as many as fit)
 *   "count_probes"  1: count hash probes (swcs_probe_counts); 0 (default)
 *   "screen_scatter" subset sweeps of swcs_pool_gradients_dev: 1 (default)
 *              scatter sigma only into the sectors the subset reads, 0 form
 *              sigma in full
 *   "rows_l2"  1: cap the row sweep's concurrent rows to about half of L2;
 *              0 (default): as many rows as clusters fit on the device */
int swcs_set_option(swcs_ctx* ctx, const char* name, int64_t value);

/* Largest state accepted by swcs_energy_noalloc. */
#define SWCS_NOALLOC_MAX_DETS 65536

/* Energy of a state held in the caller's own device buffers, for callers
 * that must not allocate device memory on their hot path (frameworks that
 * reserve all device memory in their own allocator, so cudaMalloc fails or
 * fragments their pool; latency-critical loops where cudaFree would
 * synchronise the device).  The paper has no counterpart: this is a service
 * of the library, same quantity as swcs_energy.
 *   d_keys, d_amps  [n] device arrays: distinct determinants of the loaded
 *                   Hamiltonian's sector and their amplitudes (no zeros needed)
 *   n               1 <= n <= SWCS_NOALLOC_MAX_DETS, else SWCS_ERR_INVALID_ARG
 *   d_out           [2] device: E and <psi|psi>; both NaN when a determinant
 *                   appears twice or lies outside the sector (bits >= n_so,
 *                   wrong electron count, S_z != 0): the check runs on the
 *                   device, so the call itself still returns SWCS_OK
 * Needs a loaded Hamiltonian (swcs_load_hamiltonian allocates; this call
 * does not: no cudaMalloc, cudaFree or allocating library routine).  Its
 * scratch (index table and accumulators, about 2 MiB) is one static device
 * array per GPU, held from library load until process exit; every call
 * clears the whole table first.  The first call on each device looks up that
 * array's device address; make that first call before any stream capture.
 * The call runs on the context's device (switching to it and back when
 * another device is current).  Work is only enqueued on the context's
 * stream; calls that overlap on the GPU share the array and race. */
int swcs_energy_noalloc(swcs_ctx* ctx, const uint64_t* d_keys, const double* d_amps, int64_t n, double* d_out);

/* Per-kernel device time with CUDA events recorded on the context's stream
 * around each launch (off by default).  Kinds: 0 gate/select kernel,
 * 1 energy, 2 hashed sigma scatter, 3 hashed pool gather, 4 table clear,
 * 5 other, 6 alpha-string row sweep, 7 grouping of the state by alpha string,
 * 8 adjoint gate.  swcs_profile_read synchronises, returns accumulated
 * milliseconds and launch counts per kind (9 entries each; NULL to skip) and,
 * when reset != 0,
 * clears them together with the swcs_stats counters. */
int swcs_profile_enable(swcs_ctx* ctx, int on);
int swcs_profile_read(swcs_ctx* ctx, double* h_ms8, int64_t* h_launches8, int reset);

/* Learned pool screening.  The pool gradient of ADAPT step 4 is the dominant
 * cost of the method (Sec. II.C; gradient evaluations take 43-57% of the
 * time in Sec. III.D).  A small network predicts log10|g_k| from
 * per-operator features so that only the predicted top fraction of the
 * pool is evaluated exactly; the paper has no such network.
 *   Network: 3 layers, width W (<= 256, multiple of 32), input d_in (multiple
 *   of 32): H1 = bf16(relu(x W1^T + b1)), H2 = bf16(relu(H1 W2^T + b2)),
 *   y = H2 . w3 + b3.  BF16 weights (rounded from FP32 master weights),
 *   FP32 accumulation on the tensor cores.  Parameters, FP32, in the order
 *   W1[W][d_in], b1[W], W2[W][W], b2[W], w3[W], b3.
 *   x: BF16 bit patterns, [n][d_in] row-major, on the device.
 *   swcs_mlp_grad_dev: gradients of the mean squared error to targets t[n]
 *   into d_grad (parameter order; NULL to skip) and the loss into d_loss[0].
 *   swcs_mlp_train_step_dev: the same gradients and one Adam step
 *   (beta 0.9 / 0.999, eps 1e-8) of learning rate lr.
 *   swcs_mlp_activations: H1, H2 (BF16 bits) and y of the last grad/train call.
 *   swcs_pool_features_dev: SWCS_MLP_FEATURES features of every pool operator
 *   for the context's current state, BF16 bits [pool_size][32].
 *   swcs_pool_screen_dev: features, network (the fused inference kernel of
 *   swcs_mlp_predict_dev), and the indices of the
 *   ceil(frac * pool_size) largest predictions into d_subset (device,
 *   pool_size capacity, unordered); *h_n_subset receives the count.
 *   Feed them to swcs_pool_gradients_dev to evaluate only those operators.
 *   swcs_log_abs_dev: t[i] = max(log10(|g[i]| + 1e-12), -10) (training targets). */
#define SWCS_MLP_FEATURES 32
typedef struct swcs_mlp swcs_mlp;
int swcs_mlp_create(swcs_mlp** out, void* cuda_stream, int d_in, int width);
int swcs_mlp_destroy(swcs_mlp* m);
const char* swcs_mlp_last_error(const swcs_mlp* m);
int swcs_mlp_param_count(swcs_mlp* m, int64_t* n_out);
int swcs_mlp_set_params(swcs_mlp* m, const float* h_params);
int swcs_mlp_get_params(swcs_mlp* m, float* h_params);
int swcs_mlp_forward_dev(swcs_mlp* m, const uint16_t* d_x, int64_t n, float* d_y);
/* Inference: the same y as swcs_mlp_forward_dev (bit for bit) from one fused
 * kernel that keeps both hidden layers on chip (TMA loads, tcgen05 MMAs into
 * tensor memory); the activations of swcs_mlp_activations are not written.
 * Networks whose weights and tiles exceed one SM's shared memory (d_in = 64
 * with width 256) run layer by layer instead.  d_x: [n x d_in] BF16 bits,
 * 16-byte aligned; d_y: [n] device. */
int swcs_mlp_predict_dev(swcs_mlp* m, const uint16_t* d_x, int64_t n, float* d_y);
int swcs_mlp_grad_dev(swcs_mlp* m, const uint16_t* d_x, const float* d_t, int64_t n, float* d_grad, double* d_loss);
int swcs_mlp_train_step_dev(swcs_mlp* m, const uint16_t* d_x, const float* d_t, int64_t n, float lr, double* d_loss);
int swcs_mlp_activations(swcs_mlp* m, uint16_t* h_H1, uint16_t* h_H2, float* h_y, int64_t n);
int swcs_mlp_sync(swcs_mlp* m);
/* Options of the network's training path (no effect on results beyond the
 * FP32 summation order of the weight gradients):
 *   "gemm_pipeline"  1 (default): the layer-by-layer GEMMs stream their
 *              operands by TMA through a ring of shared-memory stages and
 *              split K over CTAs for the weight gradients, wherever both
 *              operands admit a tensor map; 0: every GEMM stages its operands
 *              with plain loads, one K chunk at a time.
 * Unknown keys or values: SWCS_ERR_INVALID_ARG. */
int swcs_mlp_set_option(swcs_mlp* m, const char* key, int64_t value);
int swcs_log_abs_dev(const double* d_g, int64_t n, float* d_t, void* cuda_stream);
int swcs_pool_features_dev(swcs_ctx* ctx, uint16_t* d_x);
int swcs_pool_screen_dev(swcs_ctx* ctx, swcs_mlp* m, double frac, int64_t* d_subset, int64_t* h_n_subset);

/* Batched launch: many independent instances (each its own Hamiltonian,
 * ansatz and N_keep) evaluated together -- ansatz with truncation after every
 * gate (Eq. 1, Sec. II.B), energy and full pool gradient (Sec. II.C) -- by one
 * launch.  By default (mode 0) that launch is one persistent kernel: every
 * instance walks a chain of phases (index tables; per gate the gate pass, the
 * select passes it needs and the compaction; grouping by alpha string;
 * beta-single tables; the row sweep, one target alpha string per tile;
 * finish), each phase is split into tiles, and the kernel's CTAs take
 * (instance, phase, tile) work items from per-instance atomic words; the CTA
 * that finishes a phase's last tile runs its epilogue and publishes the next
 * phase.  Waits for work are bounded (SWCS_ERR_TIMEOUT).  The launch is
 * captured in a CUDA graph together with the reset of its scheduler words.
 * Mode 1 instead captures each instance's own kernels on a branch of a graph.
 *   swcs_batch_add     copies the inputs (same meaning as swcs_load_hamiltonian
 *                      and swcs_apply_ansatz); *index_out = instance index
 *   swcs_batch_set_tuning  mode (0 persistent, 1 graph branches), items per
 *                      tile (256..2^20), CTAs per SM (1 or 2) and the
 *                      alpha-string table's capacity factor (2, 4 or 8 times
 *                      the state bound) used by the next non-autotuned build
 *   swcs_batch_build   sizes every buffer and captures the graph; autotune != 0
 *                      first times candidate settings on whole launches and
 *                      keeps the fastest (mode 0: tile x CTAs per SM x table
 *                      factor; mode 1: device shares x row-sweep cluster sizes)
 *   swcs_batch_run     one cudaGraphLaunch on the stream given at creation (when
 *                      that is NULL, on a blocking stream owned by the batch)
 *   swcs_batch_run_serial  the library's own per-instance kernels for every
 *                      instance back to back on that stream (no graph, no
 *                      synchronisation between instances): the comparator
 *   swcs_batch_results synchronises; E, <psi|psi> and the pool gradient
 *                      (swcs_batch_pool_size entries) of instance i
 *   swcs_batch_tuning  {mode, tile, CTAs per SM, table factor, tuned ms,
 *                      instances, device share, cluster size}
 * Instances whose beta-string space exceeds 2^22 are rejected at build.  The
 * paper has no batched launch: this is a throughput service of the library. */
typedef struct swcs_batch swcs_batch;
int swcs_batch_create(swcs_batch** out, void* cuda_stream);
int swcs_batch_destroy(swcs_batch* b);
const char* swcs_batch_last_error(const swcs_batch* b);
int swcs_batch_add(swcs_batch* b, const double* h_h, const double* h_g, int n_so, int n_elec, const uint8_t* h_ops,
                   const double* h_theta, int n_ops, int64_t n_keep, int* index_out);
int swcs_batch_set_tuning(swcs_batch* b, int mode, int tile, int ctas_per_sm, int hash_factor);
/* Options of the next build: "wait_timeout_ms" bounds the persistent kernel's
 * wait for work (default 2000; running out: SWCS_ERR_TIMEOUT from the next
 * synchronising call, every CTA leaves); "test_stall_instance" (test hook, -1
 * off) publishes that instance's first phase in a form no CTA takes, so the
 * others finish and the bounded wait runs out without any fault. */
int swcs_batch_set_option(swcs_batch* b, const char* name, int64_t value);
int swcs_batch_build(swcs_batch* b, int autotune);
int swcs_batch_run(swcs_batch* b);
int swcs_batch_run_serial(swcs_batch* b);
int swcs_batch_size(swcs_batch* b, int* n_out);
int swcs_batch_pool_size(swcs_batch* b, int i, int64_t* n_out);
int swcs_batch_results(swcs_batch* b, int i, double* h_e, double* h_norm2, double* h_g);
int swcs_batch_tuning(swcs_batch* b, double* h_out8);

#ifdef __cplusplus
}
#endif
#endif /* SWCS_H */
