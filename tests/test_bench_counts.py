"""The roofline numerator of the bench: the algorithmic FP64 flops of the block cyclic reduction
(factor + multi-column solve), counted in closed form per level, against an explicit walk of the
reduction over the node indices (which nodes each level eliminates and keeps)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _walk(nf, ncols):
    """An elimination costs a 6x6 inverse and two 6x6 products (3 x 216 FMA), a kept node's update
    three products (3 x 216), its forward step 2 x 36 FMA per column; the root an inverse and 36 per
    column; an eliminated node's back substitution 3 x 36 per column."""
    alive = list(range(nf))
    fma = 0
    eliminated = 0
    while len(alive) > 1:
        kept, gone = alive[0::2], alive[1::2]
        fma += len(gone) * 3 * 216 + len(kept) * (3 * 216 + 72 * ncols)
        eliminated += len(gone)
        alive = kept
    fma += 216 + 36 * ncols + 108 * ncols * eliminated
    return 2.0 * fma


def test_factor_flops_match_the_walk():
    for nf in (1, 2, 3, 4, 5, 7, 8, 17, 100, 129, 300, 513):
        for ncols in (1, 2, 86):
            assert bench.factor_flops(nf, ncols) == _walk(nf, ncols), (nf, ncols)


def test_contact_and_element_counts():
    assert bench.contact_flops(0, 0) == 0.0
    assert bench.contact_flops(10, 3) == 6 * 10 * 3 + 27 + 2 * 10 * 3
    assert bench.ELEMENT_FLOPS == 2 * (216 + 252 + 168 + 546 + 84 + 120)
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9
