"""Pins of the Segment Storage Format oracle (no GPU)."""
import os

import numpy as np

from oracle import ssf

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    sections, cur = {}, None
    with open(os.path.join(HERE, "golden", "ssf_5x5.txt")) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# section:"):
                cur = line.split(":", 1)[1].split()[0]
                sections[cur] = []
            elif line and not line.startswith("#"):
                sections[cur].extend(int(x) for x in line.split())
    keyg = np.array(sections["keyg"]).reshape(-1, 4)
    return keyg, np.array(sections["keyv"]), np.array(sections["vals"], dtype=float)


def _golden_dense():
    rows = ["xx..x", ".xxx.", "x.x.x", "...xx", "xxxxx"]
    mask = np.array([[ch == "x" for ch in r] for r in rows])
    vals = np.array([[10 * (r + 1) + (c + 1) for c in range(5)] for r in range(5)], dtype=float)
    return mask, np.where(mask, vals, 0.0)


def test_hand_written_example():
    keyg, keyv, vals = _golden()
    mask, values = _golden_dense()
    g, v, x = ssf.from_dense(mask, values)
    assert np.array_equal(g, keyg) and np.array_equal(v, keyv) and np.array_equal(x, vals)
    m2, v2 = ssf.to_dense(5, keyg, keyv, vals)
    assert np.array_equal(m2, mask) and np.array_equal(v2, values)


def test_round_trip_and_compactness_on_random_patterns():
    rng = np.random.default_rng(4)
    for n, density in ((7, 0.3), (30, 0.1), (40, 0.6)):
        mask = rng.random((n, n)) < density
        values = np.where(mask, rng.normal(size=(n, n)), 0.0)
        keyg, keyv, vals = ssf.from_dense(mask, values)
        m2, v2 = ssf.to_dense(n, keyg, keyv, vals)
        assert np.array_equal(m2, mask) and np.array_equal(v2, values)
        # keyv is redundant: it is the running count of the segment lengths
        lens = keyg[:, 1] - keyg[:, 0] + 1
        assert np.array_equal(keyv, 1 + np.concatenate([[0], np.cumsum(lens)[:-1]]))
        # the format beats CRS (n + nnz descriptors) once segments average more than 4 entries
        nnz = int(mask.sum())
        if nnz / len(keyg) > 4:
            assert ssf.descriptor_count(len(keyg), False) < n + nnz


def test_segments_spanning_rows_are_read_in_row_major_order():
    # one segment from (row 1, col 4) to (row 2, col 2) of a 4x4 matrix
    keyg = np.array([[4, 2, 1, 2]])
    m, v = ssf.to_dense(4, keyg, np.array([1]), np.array([1.0, 2.0, 3.0]))
    want = np.zeros((4, 4), dtype=bool)
    want[0, 3] = want[1, 0] = want[1, 1] = True
    assert np.array_equal(m, want) and v[0, 3] == 1.0 and v[1, 0] == 2.0 and v[1, 1] == 3.0
