"""CPU oracle for the parameter-dependent MSFV reduced solve and its derivative.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from this
package. The product path (the CUDA library and its Python binding) never
imports it and has no CPU fallback.

* ``msfv_oracle``: plain FP64 implementation of every step of the path, one
  entity (edge / face / dual-cell interior) at a time, following the paper's
  order: basis by local solves (Sec. 3.2, Eq. multiscaleBasis_step3), coarse
  operator and reduced solve (Sec. 3.1, Eq. fwdProbRed / reducedPDE), and the
  adaptive-basis sensitivities (Sec. 4.3, Eq. sensred; local derivative of the
  basis, Sec. 4.5, Eq. reducedDiscreteMSBasisPDE).
* ``bruteforce``: an independent dense formulation of the same forward map for
  tiny meshes, differentiated by complex step; it pins the oracle.

Parity status: every oracle function is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, a library fine-mesh solve, dense brute force and
complex-step derivatives). No function is "parity unpinned".
"""
