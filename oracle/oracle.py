"""ctypes binding of the C++ oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swcs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2 -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB)
    c_int, c_i64, c_d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.orc_apply_ansatz.argtypes = [c_int, c_int, _u8p, _f64p, c_int, c_i64, _u64p, _f64p, c_i64]
    L.orc_apply_ansatz.restype = c_i64
    L.orc_apply_ansatz_eps.argtypes = [c_int, c_int, _u8p, _f64p, c_int, c_i64, c_d, _u64p, _f64p, c_i64]
    L.orc_apply_ansatz_eps.restype = c_i64
    L.orc_gate.argtypes = [_u64p, _f64p, c_i64, _u8p, c_d, c_d, c_i64, _u64p, _f64p, c_i64]
    L.orc_gate.restype = c_i64
    L.orc_truncate.argtypes = [_u64p, _f64p, c_i64, c_i64, _u64p, _f64p, c_i64]
    L.orc_truncate.restype = c_i64
    L.orc_h_element.argtypes = [c_int, _f64p, _f64p, ctypes.c_uint64, ctypes.c_uint64]
    L.orc_h_element.restype = c_d
    L.orc_energy.argtypes = [c_int, _f64p, _f64p, _u64p, _f64p, c_i64,
                             ctypes.POINTER(c_d), ctypes.POINTER(c_d)]
    L.orc_energy.restype = None
    L.orc_sigma_internal.argtypes = [c_int, _f64p, _f64p, _u64p, _f64p, c_i64, _f64p]
    L.orc_sigma_internal.restype = None
    L.orc_pool_size.argtypes = [c_int]
    L.orc_pool_size.restype = c_i64
    L.orc_pool_ops.argtypes = [c_int, _u8p]
    L.orc_pool_ops.restype = None
    L.orc_pool_gradients.argtypes = [c_int, _f64p, _f64p, _u64p, _f64p, c_i64, ctypes.c_void_p, c_i64, _f64p]
    L.orc_pool_gradients.restype = None
    L.orc_pool_gradients_brute.argtypes = [c_int, _f64p, _f64p, _u64p, _f64p, c_i64, _f64p]
    L.orc_pool_gradients_brute.restype = None
    L.orc_energy_grad.argtypes = [c_int, c_int, _f64p, _f64p, _u8p, _f64p, c_int, c_i64,
                                  ctypes.POINTER(c_d), _f64p]
    L.orc_energy_grad.restype = None
    L.orc_energy_grad_eps.argtypes = [c_int, c_int, _f64p, _f64p, _u8p, _f64p, c_int, c_i64, c_d,
                                      ctypes.POINTER(c_d), _f64p]
    L.orc_energy_grad_eps.restype = None
    L.orc_sigma_at.argtypes = [c_int, _f64p, _f64p, _u64p, _f64p, c_i64, _u64p, c_i64, _f64p]
    L.orc_sigma_at.restype = None
    L.orc_pool_gradients_pull.argtypes = [c_int, _f64p, _f64p, _u64p, _f64p, c_i64, _i64p, c_i64, _f64p]
    L.orc_pool_gradients_pull.restype = None
    _lib = L
    return L


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _ham(h, g):
    return _c(h, np.float64).reshape(-1), _c(g, np.float64).reshape(-1)


def apply_ansatz(n_so, n_e, ops, theta, n_keep, cap=1 << 22, eps=0.0):
    """State after the gate sequence (Eq. 1), truncated after every gate; sorted by key.

    eps > 0 adds the magnitude criterion of Sec. II.B: |c| < eps is dropped
    after every gate, before the size criterion (top n_keep)."""
    L = _load()
    ops = _c(ops, np.uint8).reshape(-1)
    theta = _c(theta, np.float64)
    while True:
        k = np.zeros(cap, np.uint64)
        a = np.zeros(cap, np.float64)
        n = L.orc_apply_ansatz_eps(n_so, n_e, ops, theta, len(theta), int(n_keep), float(eps), k, a, cap)
        if n <= cap:
            return k[:n].copy(), a[:n].copy()
        cap = int(n)


def gate(keys, amps, op, c, s, n_keep=0):
    L = _load()
    keys = _c(keys, np.uint64)
    amps = _c(amps, np.float64)
    cap = 2 * len(keys) + 2
    k = np.zeros(cap, np.uint64)
    a = np.zeros(cap, np.float64)
    n = L.orc_gate(keys, amps, len(keys), _c(op, np.uint8).reshape(-1), float(c), float(s), int(n_keep), k, a, cap)
    return k[:n].copy(), a[:n].copy()


def truncate(keys, amps, n_keep):
    L = _load()
    keys = _c(keys, np.uint64)
    amps = _c(amps, np.float64)
    cap = len(keys) + 1
    k = np.zeros(cap, np.uint64)
    a = np.zeros(cap, np.float64)
    n = L.orc_truncate(keys, amps, len(keys), int(n_keep), k, a, cap)
    return k[:n].copy(), a[:n].copy()


def h_element(n_so, h, g, e, d):
    L = _load()
    hh, gg = _ham(h, g)
    return L.orc_h_element(n_so, hh, gg, int(e), int(d))


def energy(n_so, h, g, keys, amps):
    """(E, <psi|psi>) with E the Rayleigh quotient."""
    L = _load()
    hh, gg = _ham(h, g)
    e, n2 = ctypes.c_double(), ctypes.c_double()
    L.orc_energy(n_so, hh, gg, _c(keys, np.uint64), _c(amps, np.float64), len(keys),
                 ctypes.byref(e), ctypes.byref(n2))
    return e.value, n2.value


def sigma_internal(n_so, h, g, keys, amps):
    L = _load()
    hh, gg = _ham(h, g)
    out = np.zeros(len(keys))
    L.orc_sigma_internal(n_so, hh, gg, _c(keys, np.uint64), _c(amps, np.float64), len(keys), out)
    return out


def pool_ops(n_so):
    L = _load()
    n = L.orc_pool_size(n_so)
    out = np.zeros(5 * n, np.uint8)
    L.orc_pool_ops(n_so, out)
    return out.reshape(n, 5)


def pool_gradients(n_so, h, g, keys, amps, subset=None):
    L = _load()
    hh, gg = _ham(h, g)
    n = L.orc_pool_size(n_so)
    out = np.full(n, np.nan)
    if subset is None:
        L.orc_pool_gradients(n_so, hh, gg, _c(keys, np.uint64), _c(amps, np.float64), len(keys), None, 0, out)
    else:
        sub = _c(subset, np.int64)
        L.orc_pool_gradients(n_so, hh, gg, _c(keys, np.uint64), _c(amps, np.float64), len(keys),
                             sub.ctypes.data, len(sub), out)
    return out


def pool_gradients_brute(n_so, h, g, keys, amps):
    L = _load()
    hh, gg = _ham(h, g)
    out = np.zeros(L.orc_pool_size(n_so))
    L.orc_pool_gradients_brute(n_so, hh, gg, _c(keys, np.uint64), _c(amps, np.float64), len(keys), out)
    return out


def energy_grad(n_so, n_e, h, g, ops, theta, n_keep, eps=0.0):
    """(E, dE/dtheta) of the truncated circuit with fixed truncation projectors
    (eps: magnitude criterion, as in apply_ansatz)."""
    L = _load()
    hh, gg = _ham(h, g)
    theta = _c(theta, np.float64)
    e = ctypes.c_double()
    d = np.zeros(len(theta))
    L.orc_energy_grad_eps(n_so, n_e, hh, gg, _c(ops, np.uint8).reshape(-1), theta, len(theta), int(n_keep),
                          float(eps), ctypes.byref(e), d)
    return e.value, d


def sigma_at(n_so, h, g, keys, amps, at):
    """sigma_E = (H psi)_E at the given determinants, each pulled on its own."""
    L = _load()
    hh, gg = _ham(h, g)
    at = _c(at, np.uint64)
    out = np.zeros(len(at))
    L.orc_sigma_at(n_so, hh, gg, _c(keys, np.uint64), _c(amps, np.float64), len(keys), at, len(at), out)
    return out


def pool_gradients_pull(n_so, h, g, keys, amps, subset):
    """Pool gradient of the listed operators, sigma pulled per needed determinant."""
    L = _load()
    hh, gg = _ham(h, g)
    sub = _c(subset, np.int64)
    out = np.zeros(len(sub))
    L.orc_pool_gradients_pull(n_so, hh, gg, _c(keys, np.uint64), _c(amps, np.float64), len(keys), sub, len(sub), out)
    return out
