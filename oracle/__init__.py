"""CPU oracle for the noisy neutral-atom MPDO method (arXiv:2309.08572).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference arm may import anything from this package.  The product
(the CUDA library and its binding) never calls it, and it never calls the product.

Plain, slow complex128 NumPy restatement of what the method computes, each function
citing the passage it follows:

  ops.py          local operators, the G0 gate/noise channels, block composition,
                  Choi <-> Kraus (Sec. II Eqs. LME_Hamiltonian..LME, Sec. IV Eqs.
                  HZ_block_representation / HZ_representation, post-promotion Sec. IV.A)
  pulse.py        gate model G1: the Gaussian-pulse CZ integrated from the two-atom
                  Lindbladian (Sec. II Eqs. LME_Hamiltonian, LME_Single_Site, LME; Fig. 1;
                  Sec. III.A), its phase correction and the G1 ZZ block
  qaoa.py         QAOA layer construction on the TFIM (Sec. IV Eqs. tfim_hamiltonian,
                  tfim_model), G0 and G1
  dense.py        exact dense density-matrix simulation (rho in C^{d^N x d^N})
  ppt.py          purity-preserving truncation (Sec. III.D Eqs. xiformula, ppt; App. B)
  mpdo.py         the MPDO two-site update: contract, SVD, truncate, Kraus truncation
                  with PPT (Sec. III, Fig. 2c, Fig. 3)
  observables.py  transfer-matrix energies, success probability, trace, sampling
                  (Sec. III.E, Sec. IV.A)
  philox.py       Philox4x32-10 counter-based generator (Salmon et al., SC'11)
  statevector.py  noiseless qubit statevector QAOA + Lanczos ground state (Table II)

Pins (tests/test_oracle_*.py) tie each part to something other than itself:
closed forms, the paper's printed numbers (Tables I/II), brute force on tiny inputs,
and the exact dense simulation.

Parity unpinned: none of the functions above is without a pin; truncated MPDO runs
(chi/K cut active) are pinned only through invariants (trace, Hermiticity,
positivity, PPT's purity identity) because the paper prints no truncated values.
"""
