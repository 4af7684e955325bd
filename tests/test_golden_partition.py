"""The segment partition the kernels walk (cyq_segment_stages, the same rule
the factor and sweep kernels use) against the paper's worked example of the
Cyqlone ordering, N = 12 on P = 4 processors (tests/golden, Sec. 4.1, eq.
block-matrix-example-4), and against the general rule stated there for
uneven lengths: the segments cover every stage once, segment c >= 1 is a run
of consecutive stages in reverse order, segment 0 starts at stage 0 and wraps
to the end of the horizon."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cyqlone_partition_N12_P4.txt")


def _read_golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    N, P = (int(v) for v in rows[0])
    cols = {int(r[0]): [int(v) for v in r[1:]] for r in rows[1:]}
    return N, P, cols


def test_partition_matches_the_papers_example():
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    N, P, cols = _read_golden()
    assert sorted(cols) == list(range(P))
    for c in range(P):
        assert cyq.segment_stages(N, P, c).tolist() == cols[c], c


@pytest.mark.parametrize("N,P", [(12, 4), (13, 4), (100, 7), (16, 16), (5, 1), (256, 3)])
def test_segments_cover_the_horizon_once(N, P):
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    seen = []
    for c in range(P):
        s = cyq.segment_stages(N, P, c)
        assert len(s) >= 1
        if c == 0:
            assert s[0] == 0 and (len(s) == 1 or s[1] == N - 1)
            tail = s[1:]
        else:
            tail = s
        assert np.all(np.diff(tail) == -1)
        seen += s.tolist()
    assert sorted(seen) == list(range(N))
    # the lengths follow the boundaries floor(c N / P)
    b = [c * N // P for c in range(P)]
    lens = [len(cyq.segment_stages(N, P, c)) for c in range(P)]
    assert lens[1:] == [b[c] - b[c - 1] for c in range(1, P)] and lens[0] == N - b[P - 1]


def test_segment_stages_rejects_bad_arguments():
    import ctypes
    from paper_2512_09058_gb300 import build, cyq
    build.build()
    L = cyq.load()
    n = ctypes.c_int32(0)
    for args in [(0, 1, 0), (4, 0, 0), (4, 5, 0), (4, 2, 2), (4, 2, -1)]:
        assert L.cyq_segment_stages(*args, None, ctypes.byref(n)) == 1, args
    assert L.cyq_segment_stages(4, 2, 0, None, None) == 1
