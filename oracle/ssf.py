"""Segment Storage Format of a sparse matrix -- TEST INFRASTRUCTURE ONLY.

Sec. "Storage format of the sparse matrices": the nonzero entries are stored in
one array, and the pattern is described by segments of consecutive entries, each
by keyg = (c_s, c_e; r_s, r_e) -- its first and last column and row in dense
coordinates -- and keyv = the position in the value array where it starts.
Readings (the paper does not fix them): indices are 1-based (the Fortran
convention of the descriptors' (2,2,nseg) shape); storage is by rows; a segment
covers the entries from (r_s, c_s) to (r_e, c_e) in row-major order (with
r_s = r_e it is the columns c_s..c_e of one row); the value array lists the
segments in order.  Writing a pattern, each maximal run of consecutive columns
of a row is one segment (segments never span rows).

Plain loops over dense boolean masks (small sizes only).
"""

from __future__ import annotations

import numpy as np


def from_dense(mask: np.ndarray, values: np.ndarray):
    """(keyg int[nseg,4] as (c_s, c_e, r_s, r_e), keyv int[nseg], vals) of the
    pattern `mask` (n x n booleans) with the entries of `values` on it."""
    n = mask.shape[0]
    keyg, keyv, vals = [], [], []
    for r in range(n):
        c = 0
        while c < n:
            if not mask[r, c]:
                c += 1
                continue
            c0 = c
            while c < n and mask[r, c]:
                c += 1
            keyg.append((c0 + 1, c, r + 1, r + 1))
            keyv.append(len(vals) + 1)
            vals.extend(values[r, c0:c].tolist())
    return np.array(keyg, dtype=np.int64).reshape(-1, 4), np.array(keyv, dtype=np.int64), np.array(vals)


def to_dense(n: int, keyg: np.ndarray, keyv: np.ndarray, vals: np.ndarray):
    """(mask, values) of the n x n matrix the descriptors describe: segment s
    holds the entries from (r_s, c_s) to (r_e, c_e) in row-major order, its
    values from vals[keyv_s - 1] on."""
    mask = np.zeros((n, n), dtype=bool)
    values = np.zeros((n, n))
    for (cs, ce, rs, re), kv in zip(keyg, keyv):
        start, end = (rs - 1) * n + (cs - 1), (re - 1) * n + (ce - 1)
        for j, lin in enumerate(range(start, end + 1)):
            r, c = divmod(lin, n)
            mask[r, c] = True
            values[r, c] = vals[kv - 1 + j]
    return mask, values


def descriptor_count(nseg: int, with_keyv: bool = True) -> int:
    """Elements describing the pattern: 4 per segment for keyg, 1 more for keyv."""
    return (5 if with_keyv else 4) * nseg
