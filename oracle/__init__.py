"""CPU oracle for the sparse wavefunction circuit solver.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are its only users.  It shares no code with the
CUDA library in ``paper_2411_07920_gb300`` and imports nothing from it.

The arithmetic lives in ``swcs_oracle.cpp`` (plain FP64 C++, built with
``-ffp-contract=off``); this module only compiles and calls it.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  apply_ansatz / gate   dense Jordan-Wigner statevector with scipy expm_multiply,
                        one-gate closed form, norm / particle / S_z invariants,
                        brute-force truncation by lexicographic sort
  energy / sigma        dense Jordan-Wigner Hamiltonian, FCI variational bound,
                        HF closed form, Hermiticity
  pool_gradients        brute-force definition (A_k psi formed explicitly),
                        finite differences of the energy, HF closed form,
                        pool size closed form
  energy_grad           central finite differences of the truncated energy,
                        dense derivative of the untruncated circuit (zero angles too)
  adapt (ADAPT-VQE loop, BFGS-2 / BFGS-2F bootstrap), in tests/test_adapt_oracle.py:
                        two-level ground state of the first iteration, exact
                        one-parameter minimum of BFGS-2's first step, variational
                        bound and monotone energies against dense FCI
  uccsd (MP2-ordered UCCSD guess, overlap and infidelity), in tests/test_uccsd_oracle.py:
                        first-order coefficients and Koopmans orbital energies of the
                        dense Hamiltonian, dense statevector overlaps
  spin (spin-complemented pool), in tests/test_spin_oracle.py: paired gradients
                        on flip-symmetrised states, commuting pairs against the
                        exponential of the summed generator
"""
from .oracle import *  # noqa: F401,F403
