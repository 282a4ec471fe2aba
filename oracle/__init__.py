"""Plain FP64 CPU oracle for the MSPCG solve of the even-odd Moebius DWF system.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
It shares no code with the CUDA library; the only common module is the seeded
input generator `paper_1811_08488_gb300.synthetic`, which holds none of the
method's arithmetic.

Everything is written as the definition in numpy, on full-lattice arrays
psi[s][t][z][y][x][spin][colour] (a parity half field is a full array that is
zero on the other parity), in complex128.

Modules
-------
dwf_operator  the operator: Wilson hop, M_phi, M_5, M_5^-1, the 4D-even-odd
              blocks M^4_eo/oe, the Schur complement D_PC and A = D_PC^dag D_PC
              (paper Sec. 2.2, the even-odd system and eq. (dirac_equation),
              eq. (normal_equation)).
solvers       CG, fixed-k inner CG, the Dirichlet block operator A_s with and
              without snake terms, and Algorithm 1 with the multisplitting
              preconditioner (paper Sec. 2.1, 2.3, 2.4, Algorithm 1).
pointwise     the hop at one (site, s), for spot checks on large lattices.
slabs         A = D_PC^dag D_PC on large lattices, evaluated in time slabs
              by worker processes (A couples sites at most four apart).
deflation     low modes of A by Chebyshev-filtered subspace iteration with
              Rayleigh-Ritz, and MSPCG with the deflated start and the
              additive coarse correction V Lambda^-1 V^dag (paper Sec. 1's
              eigen-space methods combined with Algorithm 1).

Parity status: every function is pinned by a CPU test against a closed form,
an invariant, a dense brute-force computation or a library routine (see
tests/test_oracle_*.py). The outer-iteration counts of the paper's Table 1 are
"parity unpinned": the paper's gauge ensembles and action parameters are not
available, so only the trends of Table 1 are tested.
"""
