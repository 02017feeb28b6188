"""The bench's algorithmic byte model (bench.py: alg_bytes), on the CPU: the relations between the
kernel modes that follow from what each mode moves, and the per-element figures the design notes
quote for N = 4."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("N", [1, 2, 4, 7, 9])
@pytest.mark.parametrize("t", [0, 1, 2, 3])
def test_mode_relations(t, N):
    ab = bench.alg_bytes(t, N)
    n1 = N + 1
    np_ = [n1 ** 3, n1 * n1 * (N + 2) // 2, n1 * (N + 2) * (2 * N + 3) // 6, n1 * (N + 2) * (N + 3) // 6][t]
    state = 16 * np_                                  # one state-sized array, 4 FP32 fields
    # the coarse step writes one more trace set (the half-step traces) than a fine substep
    assert ab["mrc"] - ab["mrf"] == ab["trace_set"]
    # a fine substep moves q in / out and two history slots in, one out: one array more than a stage
    assert ab["mrf"] - ab["stage"] == state
    # a traces-only launch reads the state once and writes one trace set
    assert ab["trace"] >= state + ab["trace_set"]
    assert ab["trace"] < ab["stage"]


def test_documented_n4_figures():
    """Per-element bytes at N = 4 (stage / trace / mrc / mrf) as the design notes list them."""
    want = {0: (10572, 3368, 13772, 12572), 1: (9428, 2760, 11628, 10628),
            2: (7608, 1620, 9168, 8488), 3: (3364, 1088, 4404, 3924)}
    for t, row in want.items():
        ab = bench.alg_bytes(t, 4)
        assert (ab["stage"], ab["trace"], ab["mrc"], ab["mrf"]) == row, t
    # an interior coarse hex (no fine neighbour) writes no half-step traces
    ab = bench.alg_bytes(0, 4)
    assert ab["mrc"] - ab["trace_set"] == 12572
