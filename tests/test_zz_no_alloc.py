"""swcs_energy_noalloc: the allocation-free energy entry point.

It exists for callers that must not call cudaMalloc/cudaFree on their hot
path (frameworks owning all device memory through their own allocator,
latency-critical loops where cudaFree would synchronise the device).  The
test calls it through the C ABI twice in a row, on two different states, and
compares each result with the existing swcs_energy of the same state.  This
file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2411_07920_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_noalloc_energy_matches_swcs_energy_on_two_calls():
    import torch
    from paper_2411_07920_gb300 import swcs

    w = I.small_case(20, 6, 50, 103, n_keep=700)
    ctx = swcs.Context()
    ctx.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    states = []
    for n_ops, n_keep in ((50, 700), (30, 90)):
        ctx.apply_ansatz(w.ops[:n_ops], w.theta[:n_ops], n_keep)
        k, a = ctx.get_state()
        e_ref, n2_ref = ctx.energy()  # the existing entry point
        states.append((k, a, e_ref, n2_ref))
    assert len(states[0][0]) != len(states[1][0])
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    dev_states = [(torch.from_numpy(k.view(np.int64).copy()).cuda(), torch.from_numpy(a.copy()).cuda(), len(k), e_ref,
                   n2_ref) for k, a, e_ref, n2_ref in states]
    torch.cuda.synchronize()
    for call, (d_keys, d_amps, n, e_ref, n2_ref) in enumerate(dev_states):
        if call == 1:  # the entry point's device-address lookup has happened: no device memory may move now
            free0 = torch.cuda.mem_get_info()[0]
            reserved0 = torch.cuda.memory_reserved()
        r = swcs.lib.swcs_energy_noalloc(ctx._h, ctypes.c_void_p(d_keys.data_ptr()), ctypes.c_void_p(d_amps.data_ptr()),
                                         n, ctypes.c_void_p(out.data_ptr()))
        assert r == 0, swcs.lib.swcs_last_error(ctx._h)
        torch.cuda.synchronize()
        e, n2 = out.tolist()
        assert abs(e - e_ref) < TOL
        assert abs(n2 - n2_ref) < 1e-13
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    ctx.close()


def test_noalloc_flags_duplicate_and_out_of_sector_determinants():
    """A determinant listed twice, or one outside the loaded sector, gives NaN
    outputs (the check runs on the device); the next valid call is exact."""
    import torch
    from paper_2411_07920_gb300 import swcs

    w = I.small_case(12, 4, 10, 9)
    ctx = swcs.Context()
    ctx.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    ctx.apply_ansatz(w.ops, w.theta, 0)
    k, a = ctx.get_state()
    e_ref, _ = ctx.energy()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")

    def call(keys, amps):
        d_keys = torch.from_numpy(keys.view(np.int64).copy()).cuda()
        d_amps = torch.from_numpy(amps.copy()).cuda()
        r = swcs.lib.swcs_energy_noalloc(ctx._h, ctypes.c_void_p(d_keys.data_ptr()), ctypes.c_void_p(d_amps.data_ptr()),
                                         len(keys), ctypes.c_void_p(out.data_ptr()))
        assert r == 0, swcs.lib.swcs_last_error(ctx._h)
        torch.cuda.synchronize()
        return out.tolist()

    dup_k = np.concatenate([k, k[:1]])
    dup_a = np.concatenate([a, a[:1]])
    assert all(np.isnan(call(dup_k, dup_a)))
    wrong = k.copy()
    wrong[0] = np.uint64((1 << w.n_e) - 1) << np.uint64(w.n_so - w.n_e)  # top bits: alpha/beta counts may differ
    wrong[0] = np.uint64(int(wrong[0]) | (1 << w.n_so))                  # and one bit outside the orbitals
    assert all(np.isnan(call(wrong, a)))
    e, _ = call(k, a)
    assert abs(e - e_ref) < TOL
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2411_07920_gb300 import swcs

    w = I.small_case(12, 4, 5, 9)
    ctx = swcs.Context()
    ctx.load_hamiltonian(w.h, w.g, w.n_so, w.n_e)
    import re
    big = int(re.search(r"#define SWCS_NOALLOC_MAX_DETS (\d+)", open(swcs.HEADER).read()).group(1))
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    r = swcs.lib.swcs_energy_noalloc(ctx._h, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                     big + 1, ctypes.c_void_p(d.data_ptr()))
    assert r == -1
    assert b"SWCS_NOALLOC_MAX_DETS" in swcs.lib.swcs_last_error(ctx._h)
    ctx.close()
