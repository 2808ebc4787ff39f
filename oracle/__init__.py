"""CPU FP64 oracle for the Acc-FEM contact hot path (arxiv 2503.06922).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct numpy code written
from the paper: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path (``paper_2503_06922_gb300``) and never
imports it; both sides take their inputs from ``workloads``.

Modules
  rotation  -- SO(3) exponential/logarithm and the spin-to-rotation-vector map
  beam      -- section constants, corotational two-node beam element (Sec. II.B, Eq. 20)
  contact   -- node-vs-triangle closest point and contact detection (Eq. 3-10, Sec. III.C)
  lcp       -- exact solution of the contact LCP / QP (Eq. 12-13, 22-23)
  solver    -- assembly, cable load (Eq. 16-18), Newton loop with step limiter (Eq. 20-29)

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms, invariants or brute force (no function is left unpinned).
"""
