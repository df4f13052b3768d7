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
    for k, a, e_ref, n2_ref in states:
        d_keys = torch.from_numpy(k.view(np.int64).copy()).cuda()
        d_amps = torch.from_numpy(a.copy()).cuda()
        r = swcs.lib.swcs_energy_noalloc(ctx._h, ctypes.c_void_p(d_keys.data_ptr()), ctypes.c_void_p(d_amps.data_ptr()),
                                         len(k), ctypes.c_void_p(out.data_ptr()))
        assert r == 0, swcs.lib.swcs_last_error(ctx._h)
        torch.cuda.synchronize()
        e, n2 = out.tolist()
        assert abs(e - e_ref) < TOL
        assert abs(n2 - n2_ref) < 1e-13
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
