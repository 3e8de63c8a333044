"""Oracle: a plain, slow FP64 CPU implementation of the OK-action W-form operator and its solver.

TEST INFRASTRUCTURE ONLY. Only the test-suite, the package smoke check and the benchmark's CPU
baseline import this package. The CUDA library never calls it and shares no code with it.

Contents (each function cites the passage of Jang et al., "Optimization of the Oktay-Kronfeld
Action Conjugate Gradient Inverter", PoS LATTICE2013, arXiv:1311.5029, that it follows):

* spin.py    -- Dirac and Pauli matrices in the representation forced by the W formulas (Sec. 2.2).
* gauge.py   -- mean plaquette and tadpole factor u0; clover field strength, E_i and B_i
                (the E-bar^S and B-bar^D fields entering Eqs. shifted_W_first .. shifted_W_last).
* direct.py  -- "O1": the operator assembled directly from the terms of the tree-level,
                tadpole-improved OK action by expanding every term into gauge-link paths.
* wform.py   -- "O2": the precalculation matrices W transcribed from Eqs. shifted_W_first ..
                shifted_W_last, the backward ones from Eqs. conjugate and opp_diag_pre_mat, and the
                operator applied in the form of Eq. minFlopForm (and, as a cross-check, Eq. FinalForm).
* bicgstab.py -- "O3": textbook BiCGStab (van der Vorst 1992), the paper's bi-stabilized CG.
* precond.py -- the learned right preconditioner that the library adds to the paper's solver: a
                gauge-covariant linear network of covariant shifts (the hopping transport of
                Eq. minFlopForm) and learned spin matrices, with its adjoint and its loss gradient.

Everything is complex128 / float64 numpy arithmetic over whole lattice arrays; there is no
blocking, fusion or reordering beyond the definitions.
"""
from . import spin, lattice, gauge, direct, wform, bicgstab, precond  # noqa: F401
