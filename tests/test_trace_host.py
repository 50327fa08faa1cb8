"""Host-side grouping of kernel trace records into launches (no GPU)."""
import numpy as np

import paper_1010_2592_gb300 as fa


def records(rows):
    r = np.zeros(len(rows), dtype=fa.TRACE_DTYPE)
    for i, (t0, t1, k, grid) in enumerate(rows):
        r[i] = (t0, t1, k, i, 0, grid)
    return r


def test_launch_grouping_and_names():
    F32, DOT = 1 << 8, 1 << 10
    rows = [(0, 5, 9 | F32, 2), (1, 9, 9 | F32, 2),
            (10, 20, 9 | F32 | DOT, 2), (11, 25, 9 | F32 | DOT, 2),
            (30, 40, 4 | F32 | DOT, 1)]
    L = fa.trace_launches(records(rows)[::-1])          # any input order
    assert [x["name"] for x in L] == ["k_hop1<f32>", "k_hop1<f32, dot>", "k_mr<f32, shifts>"]
    assert [x["blocks"] for x in L] == [2, 2, 1]
    assert [(x["start_ns"], x["end_ns"]) for x in L] == [(0, 9), (10, 25), (30, 40)]
    assert [x["tail_ns"] for x in L] == [4, 5, 0]
    assert fa.trace_kernel_name(2 | (2 << 8)) == "k_update_r<df>"
    assert fa.trace_launches(records([])) == []
