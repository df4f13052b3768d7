"""Python binding of the C ABI in include/swcs.h (argument marshalling only).

Every computation runs in the CUDA library ``libswcs.so`` built in this
package directory (``python -m paper_2411_07920_gb300._build``).  There is no
CPU fallback: importing this module raises when the library is missing.

``Context`` methods carry the C function names without the ``swcs_``
prefix; host arrays are numpy, device arrays are torch CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libswcs.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "swcs.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2411_07920_gb300._build` "
                      "(or __graft_entry__.build()) on a machine with nvcc")

lib = ctypes.CDLL(LIB_PATH)

STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "TABLE_FULL", -4: "TIMEOUT", -5: "CUDA", -6: "NO_DEVICE"}

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_p64 = ctypes.POINTER(ctypes.c_int64)
_pd = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "swcs_create": ([ctypes.POINTER(_vp), _vp], _i),
    "swcs_destroy": ([_vp], _i),
    "swcs_last_error": ([_vp], ctypes.c_char_p),
    "swcs_load_hamiltonian": ([_vp, _vp, _vp, _i, _i], _i),
    "swcs_pool_size": ([_vp, _p64], _i),
    "swcs_pool_ops": ([_vp, _vp], _i),
    "swcs_pool_spin_pairs": ([_vp, _vp, _vp], _i),
    "swcs_mp2_uccsd": ([_vp, _vp, _vp, _i64, _p64], _i),
    "swcs_overlap": ([_vp, _vp, _vp, _i64, _vp], _i),
    "swcs_apply_ansatz": ([_vp, _vp, _vp, _i, _i64], _i),
    "swcs_apply_ansatz_dev": ([_vp, _vp, _vp, _i, _i64], _i),
    "swcs_apply_gates": ([_vp, _vp, _vp, _i, _i64], _i),
    "swcs_truncate": ([_vp, _i64], _i),
    "swcs_set_truncation_threshold": ([_vp, ctypes.c_double], _i),
    "swcs_energy": ([_vp, _pd, _pd], _i),
    "swcs_energy_dev": ([_vp, _vp], _i),
    "swcs_pool_gradients": ([_vp, _vp, _vp, _i64], _i),
    "swcs_pool_gradients_dev": ([_vp, _vp, _vp, _i64], _i),
    "swcs_energy_grad": ([_vp, _vp, _vp, _i, _i64, _i, _pd, _vp], _i),
    "swcs_state_size": ([_vp, _p64], _i),
    "swcs_get_state": ([_vp, _vp, _vp, _i64, _p64], _i),
    "swcs_set_state": ([_vp, _vp, _vp, _i64], _i),
    "swcs_stats": ([_vp, _vp], _i),
    "swcs_profile_enable": ([_vp, _i], _i),
    "swcs_profile_read": ([_vp, _vp, _vp, _i], _i),
    "swcs_energy_noalloc": ([_vp, _vp, _vp, _i64, _vp], _i),
    "swcs_set_option": ([_vp, ctypes.c_char_p, _i64], _i),
    "swcs_sweep_energy": ([_vp, _pd, _pd], _i),
    "swcs_batch_create": ([ctypes.POINTER(_vp), _vp], _i),
    "swcs_batch_destroy": ([_vp], _i),
    "swcs_batch_last_error": ([_vp], ctypes.c_char_p),
    "swcs_batch_add": ([_vp, _vp, _vp, _i, _i, _vp, _vp, _i, _i64, ctypes.POINTER(_i)], _i),
    "swcs_batch_build": ([_vp, _i], _i),
    "swcs_batch_set_tuning": ([_vp, _i, _i, _i, _i], _i),
    "swcs_batch_set_option": ([_vp, ctypes.c_char_p, _i64], _i),
    "swcs_batch_run": ([_vp], _i),
    "swcs_batch_run_serial": ([_vp], _i),
    "swcs_batch_size": ([_vp, ctypes.POINTER(_i)], _i),
    "swcs_batch_pool_size": ([_vp, _i, _p64], _i),
    "swcs_batch_results": ([_vp, _i, _pd, _pd, _vp], _i),
    "swcs_batch_tuning": ([_vp, _vp], _i),
    "swcs_mlp_create": ([ctypes.POINTER(_vp), _vp, _i, _i], _i),
    "swcs_mlp_destroy": ([_vp], _i),
    "swcs_mlp_last_error": ([_vp], ctypes.c_char_p),
    "swcs_mlp_param_count": ([_vp, _p64], _i),
    "swcs_mlp_set_params": ([_vp, _vp], _i),
    "swcs_mlp_get_params": ([_vp, _vp], _i),
    "swcs_mlp_forward_dev": ([_vp, _vp, _i64, _vp], _i),
    "swcs_mlp_predict_dev": ([_vp, _vp, _i64, _vp], _i),
    "swcs_mlp_grad_dev": ([_vp, _vp, _vp, _i64, _vp, _vp], _i),
    "swcs_mlp_train_step_dev": ([_vp, _vp, _vp, _i64, ctypes.c_float, _vp], _i),
    "swcs_mlp_activations": ([_vp, _vp, _vp, _vp, _i64], _i),
    "swcs_mlp_sync": ([_vp], _i),
    "swcs_mlp_set_option": ([_vp, ctypes.c_char_p, _i64], _i),
    "swcs_log_abs_dev": ([_vp, _i64, _vp, _vp], _i),
    "swcs_pool_features_dev": ([_vp, _vp], _i),
    "swcs_get_sigma": ([_vp, _vp, _vp, _i64, _p64], _i),
    "swcs_sigma_at": ([_vp, _vp, _i64, _vp], _i),
    "swcs_pool_gradients_partial_dev": ([_vp, _i, _i, _vp, _vp], _i),
    "swcs_probe_counts": ([_vp, _vp, _i], _i),
    "swcs_pool_screen_dev": ([_vp, _vp, ctypes.c_double, _vp, _p64], _i),
}

for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class Batch:
    """Many independent instances evaluated by one launch (``swcs_batch``): one
    persistent kernel draining (instance, phase, tile) work items (mode 0), or a
    graph of per-instance kernel branches (mode 1)."""

    def __init__(self, stream=None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        h = _vp()
        r = lib.swcs_batch_create(ctypes.byref(h), _vp(stream))
        if r != 0:
            raise SwcsError(r, "swcs_batch_create failed")
        self._h = h
        self.pool_sizes = []
        self.shapes = []  # (n_so, n_elec, gates, N_keep bucket) of each instance: the tuning cache key

    def _ck(self, r):
        if r != 0:
            raise SwcsError(r, lib.swcs_batch_last_error(self._h).decode())

    def add(self, h, g, n_so, n_elec, ops, theta, n_keep):
        h = _c(h, np.float64)
        g = _c(g, np.float64)
        ops = _c(ops, np.uint8).reshape(-1)
        theta = _c(theta, np.float64)
        idx = ctypes.c_int()
        self._ck(lib.swcs_batch_add(self._h, _ptr(h), _ptr(g), int(n_so), int(n_elec), _ptr(ops), _ptr(theta),
                                    len(theta), int(n_keep), ctypes.byref(idx)))
        n = ctypes.c_int64()
        self._ck(lib.swcs_batch_pool_size(self._h, idx.value, ctypes.byref(n)))
        self.pool_sizes.append(n.value)
        self.shapes.append((int(n_so), int(n_elec), len(theta), int(n_keep).bit_length() if n_keep > 0 else 0))
        return idx.value

    def set_option(self, name, value):
        self._ck(lib.swcs_batch_set_option(self._h, name.encode(), int(value)))

    def set_tuning(self, mode=0, tile=4096, ctas_per_sm=2, hash_factor=2):
        self._ck(lib.swcs_batch_set_tuning(self._h, int(mode), int(tile), int(ctas_per_sm), int(hash_factor)))

    def cache_key(self):
        """The batch's shape: sorted (n_so, n_elec, gates, N_keep bucket) of its instances."""
        import hashlib
        return hashlib.sha256(repr(sorted(self.shapes)).encode()).hexdigest()[:20]

    def build(self, autotune=True, cache_path=None):
        """Sizes buffers and captures the launch.  autotune: time candidate
        settings first.  cache_path: a JSON file of tuned settings keyed by
        the batch's shape -- a hit skips the timing, a miss stores its result."""
        import json
        import os
        key = self.cache_key()
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        if autotune and key in cache:
            t = cache[key]
            self.set_tuning(t["mode"], t["tile"], t["ctas_per_sm"], t["hash_factor"])
            self._ck(lib.swcs_batch_build(self._h, 0))
            self.from_cache = True
            return
        self.from_cache = False
        self._ck(lib.swcs_batch_build(self._h, 1 if autotune else 0))
        if autotune and cache_path:
            t = self.tuning()
            cache[key] = {k: t[k] for k in ("mode", "tile", "ctas_per_sm", "hash_factor", "tuned_ms")}
            d = os.path.dirname(os.path.abspath(cache_path))
            os.makedirs(d, exist_ok=True)
            tmp = cache_path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, cache_path)

    def run(self):
        self._ck(lib.swcs_batch_run(self._h))

    def run_serial(self):
        """Every instance's own kernels back to back on the batch's stream."""
        self._ck(lib.swcs_batch_run_serial(self._h))

    def results(self, i):
        e, n2 = ctypes.c_double(), ctypes.c_double()
        g = np.zeros(self.pool_sizes[i])
        self._ck(lib.swcs_batch_results(self._h, int(i), ctypes.byref(e), ctypes.byref(n2), _ptr(g)))
        return e.value, n2.value, g

    def tuning(self):
        out = np.zeros(8)
        self._ck(lib.swcs_batch_tuning(self._h, _ptr(out)))
        return dict(mode=int(out[0]), tile=int(out[1]), ctas_per_sm=int(out[2]), hash_factor=int(out[3]),
                    tuned_ms=float(out[4]), instances=int(out[5]), share=float(out[6]), cluster=int(out[7]))

    def close(self):
        if getattr(self, "_h", None):
            lib.swcs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """Screening network (``swcs_mlp``); tensors are torch CUDA tensors."""

    def __init__(self, d_in=32, width=256, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = _vp()
        r = lib.swcs_mlp_create(ctypes.byref(h), _vp(stream), int(d_in), int(width))
        if r != 0:
            raise SwcsError(r, "swcs_mlp_create failed")
        self._h = h
        self.d_in, self.width = d_in, width
        n = ctypes.c_int64()
        lib.swcs_mlp_param_count(h, ctypes.byref(n))
        self.n_params = n.value
        self._stream = stream

    def _ck(self, r):
        if r != 0:
            raise SwcsError(r, lib.swcs_mlp_last_error(self._h).decode())

    def layout(self):
        W, D = self.width, self.d_in
        o = {}
        o["W1"] = (0, (W, D))
        o["b1"] = (W * D, (W,))
        o["W2"] = (W * D + W, (W, W))
        o["b2"] = (W * D + W + W * W, (W,))
        o["w3"] = (W * D + 2 * W + W * W, (W,))
        o["b3"] = (W * D + 3 * W + W * W, ())
        return o

    def set_params(self, flat):
        flat = _c(flat, np.float32)
        assert flat.size == self.n_params
        self._ck(lib.swcs_mlp_set_params(self._h, _ptr(flat)))

    def get_params(self):
        out = np.zeros(self.n_params, np.float32)
        self._ck(lib.swcs_mlp_get_params(self._h, _ptr(out)))
        return out

    def forward_dev(self, d_x, d_y):
        self._ck(lib.swcs_mlp_forward_dev(self._h, _tptr(d_x), int(d_x.shape[0]), _tptr(d_y)))

    def predict_dev(self, d_x, d_y):
        """Same y as forward_dev from the fused single-kernel forward (no stored activations)."""
        self._ck(lib.swcs_mlp_predict_dev(self._h, _tptr(d_x), int(d_x.shape[0]), _tptr(d_y)))

    def grad_dev(self, d_x, d_t, d_grad, d_loss):
        self._ck(lib.swcs_mlp_grad_dev(self._h, _tptr(d_x), _tptr(d_t), int(d_x.shape[0]), _tptr(d_grad),
                                       _tptr(d_loss)))

    def train_step_dev(self, d_x, d_t, lr, d_loss):
        self._ck(lib.swcs_mlp_train_step_dev(self._h, _tptr(d_x), _tptr(d_t), int(d_x.shape[0]), float(lr),
                                             _tptr(d_loss)))

    def activations(self, n):
        H1 = np.zeros((n, self.width), np.uint16)
        H2 = np.zeros((n, self.width), np.uint16)
        y = np.zeros(n, np.float32)
        self._ck(lib.swcs_mlp_activations(self._h, _ptr(H1), _ptr(H2), _ptr(y), int(n)))
        return H1, H2, y

    def sync(self):
        self._ck(lib.swcs_mlp_sync(self._h))

    def set_option(self, key, value):
        self._ck(lib.swcs_mlp_set_option(self._h, key.encode(), int(value)))

    def close(self):
        if getattr(self, "_h", None):
            lib.swcs_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def log_abs_dev(d_g, d_t, stream=None):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    r = lib.swcs_log_abs_dev(_tptr(d_g), int(d_g.numel()), _tptr(d_t), _vp(stream))
    if r != 0:
        raise SwcsError(r, "swcs_log_abs_dev failed")


def declared_symbols(header: str = HEADER):
    """Function names declared in include/swcs.h."""
    txt = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(swcs_\w+)\s*\(", txt, re.M)))


class SwcsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _ptr(a):
    return a.ctypes.data_as(_vp) if a is not None else None


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Context:
    """One solver context (``swcs_ctx``) on the current CUDA device and stream."""

    def __init__(self, stream=None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:  # torch missing: legacy default stream
                stream = 0
        h = _vp()
        r = lib.swcs_create(ctypes.byref(h), _vp(stream))
        if r != 0:
            raise SwcsError(r, "swcs_create failed (needs an sm_103 GPU)")
        self._h = h
        self.n_so = None

    def close(self):
        if getattr(self, "_h", None):
            lib.swcs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, r):
        if r != 0:
            raise SwcsError(r, lib.swcs_last_error(self._h).decode())

    # ------------------------------------------------------------------ API
    def load_hamiltonian(self, h, g, n_so, n_elec):
        h = _c(h, np.float64)
        g = _c(g, np.float64)
        assert h.size == n_so * n_so and g.size == n_so ** 4
        self._ck(lib.swcs_load_hamiltonian(self._h, _ptr(h), _ptr(g), int(n_so), int(n_elec)))
        self.n_so = n_so

    def pool_size(self):
        n = ctypes.c_int64()
        self._ck(lib.swcs_pool_size(self._h, ctypes.byref(n)))
        return n.value

    def pool_ops(self):
        out = np.zeros(5 * self.pool_size(), np.uint8)
        self._ck(lib.swcs_pool_ops(self._h, _ptr(out)))
        return out.reshape(-1, 5)

    def mp2_uccsd(self):
        """(ops [M, 5] uint8, theta [M]) of the MP2-ordered UCCSD ansatz."""
        n = ctypes.c_int64()
        self._ck(lib.swcs_mp2_uccsd(self._h, None, None, 0, ctypes.byref(n)))
        ops = np.zeros(5 * n.value, np.uint8)
        theta = np.zeros(n.value)
        self._ck(lib.swcs_mp2_uccsd(self._h, _ptr(ops), _ptr(theta), n.value, ctypes.byref(n)))
        return ops.reshape(-1, 5), theta

    def overlap(self, keys, amps):
        """(<state|given>, <state|state>, <given|given>, infidelity)."""
        keys = _c(keys, np.uint64)
        amps = _c(amps, np.float64)
        out = np.zeros(4)
        self._ck(lib.swcs_overlap(self._h, _ptr(keys), _ptr(amps), len(keys), _ptr(out)))
        return tuple(float(x) for x in out)

    def pool_spin_pairs(self):
        """(partner, sign): the spin flip of kappa_k is sign[k] * kappa_partner[k]."""
        n = self.pool_size()
        partner = np.zeros(n, np.int64)
        sign = np.zeros(n, np.int8)
        self._ck(lib.swcs_pool_spin_pairs(self._h, _ptr(partner), _ptr(sign)))
        return partner, sign

    def apply_ansatz(self, ops, theta, n_keep):
        ops = _c(ops, np.uint8).reshape(-1)
        theta = _c(theta, np.float64)
        self._ck(lib.swcs_apply_ansatz(self._h, _ptr(ops), _ptr(theta), len(theta), int(n_keep)))

    def apply_ansatz_dev(self, d_ops, d_theta, n_keep):
        self._ck(lib.swcs_apply_ansatz_dev(self._h, _tptr(d_ops), _tptr(d_theta), int(d_theta.numel()), int(n_keep)))

    def apply_gates(self, ops, theta, n_keep):
        ops = _c(ops, np.uint8).reshape(-1)
        theta = _c(theta, np.float64)
        self._ck(lib.swcs_apply_gates(self._h, _ptr(ops), _ptr(theta), len(theta), int(n_keep)))

    def truncate(self, n_keep):
        self._ck(lib.swcs_truncate(self._h, int(n_keep)))

    def set_truncation_threshold(self, eps):
        """Magnitude criterion (drop |c| < eps before the size criterion) for
        every later truncation of this context; 0 turns it off."""
        self._ck(lib.swcs_set_truncation_threshold(self._h, float(eps)))

    def energy(self):
        e, n2 = ctypes.c_double(), ctypes.c_double()
        self._ck(lib.swcs_energy(self._h, ctypes.byref(e), ctypes.byref(n2)))
        return e.value, n2.value

    def energy_dev(self, d_out):
        self._ck(lib.swcs_energy_dev(self._h, _tptr(d_out)))

    def pool_gradients(self, subset=None):
        out = np.full(self.pool_size(), np.nan)
        if subset is None:
            self._ck(lib.swcs_pool_gradients(self._h, _ptr(out), None, 0))
        else:
            sub = _c(subset, np.int64)
            self._ck(lib.swcs_pool_gradients(self._h, _ptr(out), _ptr(sub), len(sub)))
        return out

    def pool_gradients_dev(self, d_g, d_subset=None):
        n = 0 if d_subset is None else int(d_subset.numel())
        self._ck(lib.swcs_pool_gradients_dev(self._h, _tptr(d_g), _tptr(d_subset), n))

    def probe_counts(self, reset=False):
        """Hash-probe counts while option count_probes is on: {gate lookups, their slots,
        row-sweep alpha-string lookups, their slots}."""
        out = np.zeros(4, np.int64)
        self._ck(lib.swcs_probe_counts(self._h, _ptr(out), int(bool(reset))))
        return dict(gate_lookups=int(out[0]), gate_slots=int(out[1]), row_lookups=int(out[2]), row_slots=int(out[3]))

    def pool_gradients_partial_dev(self, shard, n_shards, d_graw, d_acc):
        """One shard of the pool sweep: unscaled partial gradient into d_graw and
        (partial energy numerator, <psi|psi>) into d_acc (device tensors)."""
        self._ck(lib.swcs_pool_gradients_partial_dev(self._h, int(shard), int(n_shards), _tptr(d_graw), _tptr(d_acc)))

    def energy_grad(self, ops, theta, n_keep, ckpt_every=20):
        ops = _c(ops, np.uint8).reshape(-1)
        theta = _c(theta, np.float64)
        e = ctypes.c_double()
        d = np.zeros(len(theta))
        self._ck(lib.swcs_energy_grad(self._h, _ptr(ops), _ptr(theta), len(theta), int(n_keep), int(ckpt_every),
                                      ctypes.byref(e), _ptr(d)))
        return e.value, d

    def state_size(self):
        n = ctypes.c_int64()
        self._ck(lib.swcs_state_size(self._h, ctypes.byref(n)))
        return n.value

    def get_state(self):
        n = self.state_size()
        k = np.zeros(max(n, 1), np.uint64)
        a = np.zeros(max(n, 1), np.float64)
        m = ctypes.c_int64()
        self._ck(lib.swcs_get_state(self._h, _ptr(k), _ptr(a), n, ctypes.byref(m)))
        return k[:m.value], a[:m.value]

    def get_sigma(self):
        n = self.state_size()
        k = np.zeros(max(n, 1), np.uint64)
        sg = np.zeros(max(n, 1), np.float64)
        m = ctypes.c_int64()
        self._ck(lib.swcs_get_sigma(self._h, _ptr(k), _ptr(sg), n, ctypes.byref(m)))
        return k[:m.value], sg[:m.value]

    def sigma_at(self, keys):
        """sigma_E = (H psi)_E at the given determinants (in or outside the state)."""
        keys = _c(keys, np.uint64)
        out = np.zeros(max(len(keys), 1), np.float64)
        self._ck(lib.swcs_sigma_at(self._h, _ptr(keys), len(keys), _ptr(out)))
        return out[:len(keys)]

    def set_state(self, keys, amps):
        keys = _c(keys, np.uint64)
        amps = _c(amps, np.float64)
        self._ck(lib.swcs_set_state(self._h, _ptr(keys), _ptr(amps), len(keys)))

    def sweep_energy(self):
        e, n2 = ctypes.c_double(), ctypes.c_double()
        self._ck(lib.swcs_sweep_energy(self._h, ctypes.byref(e), ctypes.byref(n2)))
        return e.value, n2.value

    def pool_features_dev(self, d_x):
        self._ck(lib.swcs_pool_features_dev(self._h, _tptr(d_x)))

    def pool_screen_dev(self, mlp, frac, d_subset):
        n = ctypes.c_int64()
        self._ck(lib.swcs_pool_screen_dev(self._h, mlp._h, float(frac), _tptr(d_subset), ctypes.byref(n)))
        return n.value

    def set_option(self, name, value):
        self._ck(lib.swcs_set_option(self._h, name.encode(), int(value)))

    def energy_noalloc(self, d_keys, d_amps, d_out):
        """Energy of a state in caller-owned device tensors (no device allocation)."""
        self._ck(lib.swcs_energy_noalloc(self._h, _tptr(d_keys), _tptr(d_amps), int(d_keys.numel()), _tptr(d_out)))

    def stats(self):
        out = np.zeros(8, np.int64)
        self._ck(lib.swcs_stats(self._h, _ptr(out)))
        keys = ["gates", "select_passes", "ext_distinct", "ext_buckets", "ext_capacity",
                "kernel_launches", "phi_max", "gate_dets"]
        return dict(zip(keys, out.tolist()))

    KINDS = ("ansatz", "energy", "sigma_scatter", "pool_gather", "table_clear", "other", "row_sweep", "group",
             "adjoint")

    def profile_enable(self, on=True):
        self._ck(lib.swcs_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset=True):
        ms = np.zeros(9)
        n = np.zeros(9, np.int64)
        self._ck(lib.swcs_profile_read(self._h, _ptr(ms), _ptr(n), 1 if reset else 0))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KINDS)}
