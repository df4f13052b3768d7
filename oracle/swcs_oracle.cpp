// Plain CPU reference ("oracle") for the sparse wavefunction circuit solver.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load this library.  The CUDA product path
// shares no code with it: no headers, helpers or tables in common.
//
// Everything here is the slow, literal definition, in FP64, compiled with
// -ffp-contract=off so that every product and sum is rounded separately:
//   * fermionic operators act on occupation bitstrings by their definition
//     (phase = (-1)^(number of occupied spin-orbitals below the index));
//   * a gate exp(theta (tau - tau^dag)) (Eqs. 1-3) acts exactly on each
//     two-determinant block (Sec. II.B, "evaluated exactly");
//   * duplicates are merged in a std::map, exact zeros are dropped and the
//     state is truncated to the N largest |c| after every gate (Sec. II.B,
//     Fig. 1); ties at the cut keep the smaller bitstring;
//   * E = <psi|H|psi>/<psi|psi> from the Slater-Condon rules (Sec. II);
//   * the operator-pool gradient of ADAPT step 4 (Sec. II.C) over the
//     generalized singles and doubles pool, g_k = 2 <psi|H A_k|psi>/<psi|psi>;
//   * the gradient dE/dtheta of the truncated circuit with each truncation
//     held as a fixed projector ("analytic gradients", Sec. II.B).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <utility>
#include <vector>

typedef uint64_t det_t;
typedef std::map<det_t, double> State;

namespace {

// ---------------------------------------------------------------------------
// Second quantisation on one determinant, by definition.
// ---------------------------------------------------------------------------
struct Term {
  det_t det;
  int sign;   // +1 / -1
  bool zero;  // operator annihilated the determinant
};

int occupied_below(det_t d, int p) {
  int n = 0;
  for (int k = 0; k < p; ++k)
    if ((d >> k) & 1ull) ++n;
  return n;
}

void annihilate(Term& t, int p) {
  if (t.zero) return;
  if (!((t.det >> p) & 1ull)) { t.zero = true; return; }
  if (occupied_below(t.det, p) % 2) t.sign = -t.sign;
  t.det &= ~(1ull << p);
}

void create(Term& t, int p) {
  if (t.zero) return;
  if ((t.det >> p) & 1ull) { t.zero = true; return; }
  if (occupied_below(t.det, p) % 2) t.sign = -t.sign;
  t.det |= (1ull << p);
}

// Operator record: kind 1: tau = a+_{i1} a_{i0};  kind 2: tau = a+_{i2} a+_{i3} a_{i1} a_{i0}.
struct Op {
  int kind;
  int i[4];
};

Op op_from_bytes(const uint8_t* b) {
  Op o;
  o.kind = b[0];
  for (int k = 0; k < 4; ++k) o.i[k] = b[1 + k];
  return o;
}

// tau |d>, operators applied right to left.
Term apply_tau(const Op& o, det_t d) {
  Term t{d, 1, false};
  if (o.kind == 1) {
    annihilate(t, o.i[0]);
    create(t, o.i[1]);
  } else {
    annihilate(t, o.i[0]);
    annihilate(t, o.i[1]);
    create(t, o.i[3]);
    create(t, o.i[2]);
  }
  return t;
}

// tau^dagger |d>:  (a+_{i1} a_{i0})^dag = a+_{i0} a_{i1};
//                  (a+_{i2} a+_{i3} a_{i1} a_{i0})^dag = a+_{i0} a+_{i1} a_{i3} a_{i2}.
Term apply_tau_dag(const Op& o, det_t d) {
  Term t{d, 1, false};
  if (o.kind == 1) {
    annihilate(t, o.i[1]);
    create(t, o.i[0]);
  } else {
    annihilate(t, o.i[2]);
    annihilate(t, o.i[3]);
    create(t, o.i[1]);
    create(t, o.i[0]);
  }
  return t;
}

void drop_zeros(State& s) {
  for (auto it = s.begin(); it != s.end();) {
    if (it->second == 0.0) it = s.erase(it);
    else ++it;
  }
}

// One gate exp(theta kappa), kappa = tau - tau^dag, on a sparse state.
// On a block {D, D'} with tau D = s D':  kappa D = s D', kappa D' = -s D and
// kappa^2 = -1, so exp(theta kappa) D = cos D + s sin D' and
// exp(theta kappa) D' = cos D' - s sin D.  Determinants outside every block
// are left unchanged.  Each output receives at most two products, summed in
// the merge map.
State gate_apply(const State& in, const Op& o, double c, double sn, bool keep_zeros = false) {
  State out;
  for (const auto& kv : in) {
    const det_t d = kv.first;
    const double amp = kv.second;
    Term up = apply_tau(o, d);
    Term dn = apply_tau_dag(o, d);
    if (!up.zero) {
      out[d] += amp * c;
      double t = amp * sn;
      out[up.det] += (up.sign > 0) ? t : -t;
    } else if (!dn.zero) {
      out[d] += amp * c;
      double t = amp * sn;
      out[dn.det] += (dn.sign > 0) ? -t : t;
    } else {
      out[d] += amp;
    }
  }
  if (!keep_zeros) drop_zeros(out);
  return out;
}

// Keep the n_keep largest |c| (ties: smaller bitstring first); n_keep <= 0 keeps all.
State truncate_top(const State& in, int64_t n_keep) {
  if (n_keep <= 0 || (int64_t)in.size() <= n_keep) return in;
  std::vector<std::pair<det_t, double>> v(in.begin(), in.end());
  std::sort(v.begin(), v.end(), [](const std::pair<det_t, double>& a, const std::pair<det_t, double>& b) {
    const double aa = std::fabs(a.second), bb = std::fabs(b.second);
    if (aa != bb) return aa > bb;
    return a.first < b.first;
  });
  State out;
  for (int64_t k = 0; k < n_keep; ++k) out.insert(v[k]);
  return out;
}

// Truncation after a gate (Sec. II.B): the magnitude criterion first (drop
// every |c| < eps; eps <= 0 keeps all nonzero amplitudes), then the size
// criterion (top n_keep of what is left, as truncate_top).
State truncate(const State& in, int64_t n_keep, double eps) {
  if (eps <= 0.0) return truncate_top(in, n_keep);
  State kept;
  for (const auto& kv : in)
    if (std::fabs(kv.second) >= eps) kept.insert(kv);
  return truncate_top(kept, n_keep);
}

// ---------------------------------------------------------------------------
// Hamiltonian H = sum h_pq a+_p a_q + 1/4 sum <pq||rs> a+_p a+_q a_s a_r.
// ---------------------------------------------------------------------------
struct Ham {
  int n;
  const double* h;  // h[p*n + q]
  const double* g;  // g[((p*n + q)*n + r)*n + s] = <pq||rs>
  double H1(int p, int q) const { return h[p * n + q]; }
  double G(int p, int q, int r, int s) const { return g[(((size_t)p * n + q) * n + r) * n + s]; }
};

std::vector<int> occ_list(det_t d, int n) {
  std::vector<int> o;
  for (int p = 0; p < n; ++p)
    if ((d >> p) & 1ull) o.push_back(p);
  return o;
}

// <D|H|D> = sum_i h_ii + 1/2 sum_ij <ij||ij>
double sc_diag(const Ham& H, det_t d) {
  std::vector<int> o = occ_list(d, H.n);
  double e1 = 0.0, e2 = 0.0;
  for (int i : o) e1 += H.H1(i, i);
  for (int i : o)
    for (int j : o) e2 += H.G(i, j, i, j);
  return e1 + 0.5 * e2;
}

// E = a+_q a_p D (times its phase): <E|H|D> = phase (h_qp + sum_{k in D} <qk||pk>).
double sc_single(const Ham& H, det_t d, int p, int q, det_t* e_out) {
  Term t{d, 1, false};
  annihilate(t, p);
  create(t, q);
  if (t.zero) { *e_out = 0; return 0.0; }
  *e_out = t.det;
  double v = H.H1(q, p);
  for (int k : occ_list(d, H.n)) v += H.G(q, k, p, k);
  return t.sign * v;
}

// E = a+_r a+_s a_q a_p D (times its phase): <E|H|D> = phase <rs||pq>.
double sc_double(const Ham& H, det_t d, int p, int q, int r, int s, det_t* e_out) {
  Term t{d, 1, false};
  annihilate(t, p);
  annihilate(t, q);
  create(t, s);
  create(t, r);
  if (t.zero) { *e_out = 0; return 0.0; }
  *e_out = t.det;
  return t.sign * H.G(r, s, p, q);
}

// Generic <E|H|D> for any two determinants (Slater-Condon by excitation level).
double sc_element(const Ham& H, det_t e, det_t d) {
  if (e == d) return sc_diag(H, d);
  det_t rem = d & ~e, add = e & ~d;
  int nr = __builtin_popcountll(rem), na = __builtin_popcountll(add);
  if (nr != na || nr > 2) return 0.0;
  std::vector<int> R = occ_list(rem, H.n), A = occ_list(add, H.n);
  det_t out = 0;
  if (nr == 1) return sc_single(H, d, R[0], A[0], &out);
  return sc_double(H, d, R[0], R[1], A[0], A[1], &out);
}

bool same_spin(int p, int q) { return (p % 2) == (q % 2); }

// Visit every single and double excitation E of D with <E|H|D>.
template <class F>
void for_each_connection(const Ham& H, det_t d, F&& f) {
  const int n = H.n;
  std::vector<int> occ = occ_list(d, n), vir;
  for (int p = 0; p < n; ++p)
    if (!((d >> p) & 1ull)) vir.push_back(p);
  det_t e;
  for (int p : occ)
    for (int q : vir)
      if (same_spin(p, q)) {
        double v = sc_single(H, d, p, q, &e);
        f(e, v);
      }
  for (size_t a = 0; a < occ.size(); ++a)
    for (size_t b = a + 1; b < occ.size(); ++b)
      for (size_t c = 0; c < vir.size(); ++c)
        for (size_t dd = c + 1; dd < vir.size(); ++dd) {
          int p = occ[a], q = occ[b], r = vir[c], s = vir[dd];
          if ((p % 2) + (q % 2) != (r % 2) + (s % 2)) continue;  // S_z
          double v = sc_double(H, d, p, q, r, s, &e);
          f(e, v);
        }
}

State state_from(const uint64_t* keys, const double* amps, int64_t n) {
  State s;
  for (int64_t i = 0; i < n; ++i) s[keys[i]] += amps[i];
  return s;
}

double norm2(const State& s) {
  double x = 0.0;
  for (const auto& kv : s) x += kv.second * kv.second;
  return x;
}

// sigma_D = (H psi)_D for D in the state (internal part of sigma).
std::map<det_t, double> sigma_internal(const Ham& H, const State& s) {
  std::map<det_t, double> sig;
  for (const auto& kv : s) {
    const det_t d = kv.first;
    double acc = sc_diag(H, d) * kv.second;
    for_each_connection(H, d, [&](det_t e, double v) {
      auto it = s.find(e);
      if (it != s.end()) acc += v * it->second;  // <D|H|E> = <E|H|D> (real symmetric)
    });
    sig[d] = acc;
  }
  return sig;
}

double energy_of(const Ham& H, const State& s, double* n2_out) {
  std::map<det_t, double> sig = sigma_internal(H, s);
  double num = 0.0;
  for (const auto& kv : s) num += kv.second * sig[kv.first];
  double n2 = norm2(s);
  if (n2_out) *n2_out = n2;
  return num / n2;
}

// Generalized singles and doubles pool in canonical order:
// singles (p<q, same spin) tau = a+_q a_p, by (p,q);
// doubles over disjoint pairs (p<q) < (r<s) with equal spin content,
// tau = a+_r a+_s a_q a_p, by ((p,q),(r,s)).
std::vector<Op> gsd_pool(int n) {
  std::vector<Op> pool;
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q)
      if (same_spin(p, q)) pool.push_back(Op{1, {p, q, 0, 0}});
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q)
      for (int r = p; r < n; ++r)
        for (int s = r + 1; s < n; ++s) {
          if (r == p && s <= q) continue;  // (r,s) must come after (p,q)
          if (r == p || r == q || s == p || s == q) continue;  // disjoint
          if ((p % 2) + (q % 2) != (r % 2) + (s % 2)) continue;  // S_z
          pool.push_back(Op{2, {p, q, r, s}});
        }
  return pool;
}

// Full external sigma: sigma_E = sum_{D in S} <E|H|D> c_D for E in S and conn(S).
std::unordered_map<det_t, double> sigma_external(const Ham& H, const State& s) {
  std::unordered_map<det_t, double> sig;
  sig.reserve(s.size() * 64);
  for (const auto& kv : s) {
    const det_t d = kv.first;
    const double c = kv.second;
    sig[d] += sc_diag(H, d) * c;
    for_each_connection(H, d, [&](det_t e, double v) { sig[e] += v * c; });
  }
  return sig;
}

}  // namespace

// ===========================================================================
// C interface (ctypes)
// ===========================================================================
extern "C" {

// Gate sequence from the reference determinant (bits 0..n_e-1), Eq. 1, with
// ops[0] acting first; truncation to n_keep after every gate (n_keep <= 0:
// none).  Writes up to cap determinants sorted by bitstring; returns the
// state size (may exceed cap, then nothing is written).
// orc_apply_ansatz_eps also drops |c| < eps after every gate (the magnitude
// criterion of Sec. II.B), before the size criterion.
int64_t orc_apply_ansatz_eps(int n_so, int n_e, const uint8_t* ops, const double* theta, int n_ops,
                             int64_t n_keep, double eps, uint64_t* keys_out, double* amps_out, int64_t cap) {
  (void)n_so;
  State s;
  det_t hf = (n_e >= 64) ? ~0ull : ((1ull << n_e) - 1ull);
  s[hf] = 1.0;
  for (int k = 0; k < n_ops; ++k) {
    Op o = op_from_bytes(ops + 5 * k);
    s = gate_apply(s, o, std::cos(theta[k]), std::sin(theta[k]));
    s = truncate(s, n_keep, eps);
  }
  int64_t n = (int64_t)s.size();
  if (n <= cap) {
    int64_t i = 0;
    for (const auto& kv : s) { keys_out[i] = kv.first; amps_out[i] = kv.second; ++i; }
  }
  return n;
}

int64_t orc_apply_ansatz(int n_so, int n_e, const uint8_t* ops, const double* theta, int n_ops,
                         int64_t n_keep, uint64_t* keys_out, double* amps_out, int64_t cap) {
  return orc_apply_ansatz_eps(n_so, n_e, ops, theta, n_ops, n_keep, 0.0, keys_out, amps_out, cap);
}

// One gate (given cos/sin) and truncation on an arbitrary state.
int64_t orc_gate(const uint64_t* keys, const double* amps, int64_t n, const uint8_t* op, double c,
                 double sn, int64_t n_keep, uint64_t* keys_out, double* amps_out, int64_t cap) {
  State s = gate_apply(state_from(keys, amps, n), op_from_bytes(op), c, sn);
  s = truncate_top(s, n_keep);
  int64_t m = (int64_t)s.size();
  if (m <= cap) {
    int64_t i = 0;
    for (const auto& kv : s) { keys_out[i] = kv.first; amps_out[i] = kv.second; ++i; }
  }
  return m;
}

// Truncation alone (top-n_keep by |c|, ties to the smaller bitstring, exact zeros dropped).
int64_t orc_truncate(const uint64_t* keys, const double* amps, int64_t n, int64_t n_keep,
                     uint64_t* keys_out, double* amps_out, int64_t cap) {
  State s = state_from(keys, amps, n);
  drop_zeros(s);
  s = truncate_top(s, n_keep);
  int64_t m = (int64_t)s.size();
  if (m <= cap) {
    int64_t i = 0;
    for (const auto& kv : s) { keys_out[i] = kv.first; amps_out[i] = kv.second; ++i; }
  }
  return m;
}

double orc_h_element(int n_so, const double* h, const double* g, uint64_t e, uint64_t d) {
  Ham H{n_so, h, g};
  return sc_element(H, e, d);
}

// E = <psi|H|psi>/<psi|psi>; also returns <psi|psi>.
void orc_energy(int n_so, const double* h, const double* g, const uint64_t* keys, const double* amps,
                int64_t n, double* e_out, double* n2_out) {
  Ham H{n_so, h, g};
  State s = state_from(keys, amps, n);
  *e_out = energy_of(H, s, n2_out);
}

// sigma_D = (H psi)_D for each input determinant, in input order.
void orc_sigma_internal(int n_so, const double* h, const double* g, const uint64_t* keys,
                        const double* amps, int64_t n, double* sigma_out) {
  Ham H{n_so, h, g};
  State s = state_from(keys, amps, n);
  std::map<det_t, double> sig = sigma_internal(H, s);
  for (int64_t i = 0; i < n; ++i) sigma_out[i] = sig[keys[i]];
}

int64_t orc_pool_size(int n_so) { return (int64_t)gsd_pool(n_so).size(); }

void orc_pool_ops(int n_so, uint8_t* out) {
  std::vector<Op> pool = gsd_pool(n_so);
  for (size_t k = 0; k < pool.size(); ++k) {
    out[5 * k] = (uint8_t)pool[k].kind;
    for (int j = 0; j < 4; ++j) out[5 * k + 1 + j] = (uint8_t)pool[k].i[j];
  }
}

// Pool gradient g_k = 2 <psi|H A_k|psi>/<psi|psi> (ADAPT step 4) through the
// full external sigma: <H psi|A_k psi> = sum_D c_D (s sigma_{tau D} - s' sigma_{tau^dag D}).
// If subset != NULL only those pool entries are written (others untouched).
void orc_pool_gradients(int n_so, const double* h, const double* g, const uint64_t* keys,
                        const double* amps, int64_t n, const int64_t* subset, int64_t n_subset,
                        double* g_out) {
  Ham H{n_so, h, g};
  State s = state_from(keys, amps, n);
  std::unordered_map<det_t, double> sig = sigma_external(H, s);
  const double n2 = norm2(s);
  std::vector<Op> pool = gsd_pool(n_so);
  auto lookup = [&](det_t e) {
    auto it = sig.find(e);
    return it == sig.end() ? 0.0 : it->second;
  };
  auto one = [&](int64_t k) {
    const Op& o = pool[k];
    double acc = 0.0;
    for (const auto& kv : s) {
      Term up = apply_tau(o, kv.first);
      if (!up.zero) acc += kv.second * (up.sign * lookup(up.det));
      Term dn = apply_tau_dag(o, kv.first);
      if (!dn.zero) acc -= kv.second * (dn.sign * lookup(dn.det));
    }
    g_out[k] = 2.0 * acc / n2;
  };
  if (subset) {
    for (int64_t i = 0; i < n_subset; ++i) one(subset[i]);
  } else {
    for (int64_t k = 0; k < (int64_t)pool.size(); ++k) one(k);
  }
}

// Same quantity by brute force: chi = A_k psi formed explicitly, then
// 2 sum_{D in S, E in chi} c_D <D|H|E> chi_E / <psi|psi> with the generic
// matrix element.  O(pool * N^2): tiny inputs only.
void orc_pool_gradients_brute(int n_so, const double* h, const double* g, const uint64_t* keys,
                              const double* amps, int64_t n, double* g_out) {
  Ham H{n_so, h, g};
  State s = state_from(keys, amps, n);
  const double n2 = norm2(s);
  std::vector<Op> pool = gsd_pool(n_so);
  for (size_t k = 0; k < pool.size(); ++k) {
    State chi;
    for (const auto& kv : s) {
      Term up = apply_tau(pool[k], kv.first);
      if (!up.zero) chi[up.det] += up.sign * kv.second;
      Term dn = apply_tau_dag(pool[k], kv.first);
      if (!dn.zero) chi[dn.det] -= dn.sign * kv.second;
    }
    double acc = 0.0;
    for (const auto& a : s)
      for (const auto& b : chi) acc += a.second * sc_element(H, a.first, b.first) * b.second;
    g_out[k] = 2.0 * acc / n2;
  }
}

// dE/dtheta of the truncated circuit, each truncation a fixed projector P_g
// onto the kept set S_g:  psi_g = P_g U_g psi_{g-1},  phi_g = U_g psi_{g-1}.
// S_g holds every determinant of phi_g that the criteria keep, exact zeros
// included (ranked below every nonzero |c|): with no cut the projector is the
// identity on phi_g's support and the derivative is exact, also at theta = 0.
//   nu_M = P_M (H - E) psi_M,  nu_{g-1} = P_{g-1} U_g^dag nu_g,
//   dE/dtheta_g = 2 <nu_g | A_g phi_g> / <psi_M|psi_M>.
void orc_energy_grad_eps(int n_so, int n_e, const double* h, const double* g, const uint8_t* ops,
                         const double* theta, int n_ops, int64_t n_keep, double eps, double* e_out,
                         double* dtheta_out) {
  Ham H{n_so, h, g};
  std::vector<State> psi(n_ops + 1);
  det_t hf = (n_e >= 64) ? ~0ull : ((1ull << n_e) - 1ull);
  psi[0][hf] = 1.0;
  for (int k = 0; k < n_ops; ++k) {
    Op o = op_from_bytes(ops + 5 * k);
    // the projectors keep every determinant the gate reaches, zero amplitude
    // or not, unless a criterion cuts it (a partner at theta = 0 has c = 0
    // but a nonzero derivative); zeros rank below every nonzero |c|
    psi[k + 1] = truncate(gate_apply(psi[k], o, std::cos(theta[k]), std::sin(theta[k]), true), n_keep, eps);
  }
  double n2 = 0.0;
  const double e = energy_of(H, psi[n_ops], &n2);
  *e_out = e;
  std::map<det_t, double> sig = sigma_internal(H, psi[n_ops]);
  State nu;
  for (const auto& kv : psi[n_ops]) nu[kv.first] = sig[kv.first] - e * kv.second;
  for (int k = n_ops - 1; k >= 0; --k) {
    Op o = op_from_bytes(ops + 5 * k);
    const double c = std::cos(theta[k]), sn = std::sin(theta[k]);
    // A phi, phi = U psi_{k}
    State phi = gate_apply(psi[k], o, c, sn, true);
    State aphi;
    for (const auto& kv : phi) {
      Term up = apply_tau(o, kv.first);
      if (!up.zero) aphi[up.det] += up.sign * kv.second;
      Term dn = apply_tau_dag(o, kv.first);
      if (!dn.zero) aphi[dn.det] -= dn.sign * kv.second;
    }
    double dot = 0.0;
    for (const auto& kv : nu) {
      auto it = aphi.find(kv.first);
      if (it != aphi.end()) dot += kv.second * it->second;
    }
    dtheta_out[k] = 2.0 * dot / n2;
    // nu <- P_{k} U^dag nu,  U^dag = U(-theta)
    State back = gate_apply(nu, o, c, -sn, true);
    State proj;
    for (const auto& kv : psi[k]) {
      auto it = back.find(kv.first);
      proj[kv.first] = (it == back.end()) ? 0.0 : it->second;
    }
    nu.swap(proj);
  }
}

void orc_energy_grad(int n_so, int n_e, const double* h, const double* g, const uint8_t* ops,
                     const double* theta, int n_ops, int64_t n_keep, double* e_out,
                     double* dtheta_out) {
  orc_energy_grad_eps(n_so, n_e, h, g, ops, theta, n_ops, n_keep, 0.0, e_out, dtheta_out);
}

// sigma_E = sum_{D in S} <E|H|D> c_D at arbitrary determinants E, each
// computed on its own from E's connections (pull form): E itself and every
// single and double excitation of E that is in the state.
void orc_sigma_at(int n_so, const double* h, const double* g, const uint64_t* keys, const double* amps, int64_t n,
                  const uint64_t* at, int64_t n_at, double* out) {
  Ham H{n_so, h, g};
  std::unordered_map<det_t, double> s;
  s.reserve(2 * n);
  for (int64_t i = 0; i < n; ++i) s[keys[i]] += amps[i];
  for (int64_t t = 0; t < n_at; ++t) {
    const det_t e = at[t];
    double acc = 0.0;
    auto it = s.find(e);
    if (it != s.end()) acc += sc_diag(H, e) * it->second;
    // <E|H|D> for D = excitation of E equals <D|H|E> (real symmetric H)
    for_each_connection(H, e, [&](det_t d, double v) {
      auto jt = s.find(d);
      if (jt != s.end()) acc += v * jt->second;
    });
    out[t] = acc;
  }
}

// Pool gradient of the listed operators with sigma pulled at each needed E:
// g_k = 2/<psi|psi> sum_D c_D (s sigma(tau_k D) - s' sigma(tau_k^dag D)).
void orc_pool_gradients_pull(int n_so, const double* h, const double* g, const uint64_t* keys, const double* amps,
                             int64_t n, const int64_t* subset, int64_t n_subset, double* g_out) {
  Ham H{n_so, h, g};
  std::unordered_map<det_t, double> s;
  s.reserve(2 * n);
  double n2 = 0.0;
  for (int64_t i = 0; i < n; ++i) { s[keys[i]] += amps[i]; n2 += amps[i] * amps[i]; }
  std::vector<Op> pool = gsd_pool(n_so);
  auto sigma = [&](det_t e) {
    double acc = 0.0;
    auto it = s.find(e);
    if (it != s.end()) acc += sc_diag(H, e) * it->second;
    for_each_connection(H, e, [&](det_t d, double v) {
      auto jt = s.find(d);
      if (jt != s.end()) acc += v * jt->second;
    });
    return acc;
  };
  for (int64_t t = 0; t < n_subset; ++t) {
    const Op& o = pool[subset[t]];
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      Term up = apply_tau(o, keys[i]);
      if (!up.zero) acc += amps[i] * (up.sign * sigma(up.det));
      Term dn = apply_tau_dag(o, keys[i]);
      if (!dn.zero) acc -= amps[i] * (dn.sign * sigma(dn.det));
    }
    g_out[t] = 2.0 * acc / n2;
  }
}

}  // extern "C"
