"""Segment Storage Format import and export through the C ABI against the
oracle's plain definition: bit-exact descriptors and values."""
import numpy as np
import pytest
import torch

import synth
from oracle import pipelines, ssf

pytestmark = pytest.mark.gpu

cg = pytest.importorskip("paper_1704_00512_gb300")

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
if DEV is None:
    pytest.skip("no CUDA device", allow_module_level=True)


def dbsr(A):
    return cg.Bsr(torch.as_tensor(A.row_ptr, device=DEV), torch.as_tensor(A.col_idx, device=DEV),
                  torch.as_tensor(np.ascontiguousarray(A.vals), device=DEV))


def block_mask(A):
    n = 4 * A.nbr
    m = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(A.nbr), np.diff(A.row_ptr))
    for I, J in zip(rows, A.col_idx):
        m[4 * I:4 * I + 4, 4 * J:4 * J + 4] = True
    return m


@pytest.mark.parametrize("n_atoms,r_c,seed", [(10, 3.0, 1), (60, 4.0, 2), (200, 5.0, 3)])
def test_export_matches_the_definition(n_atoms, r_c, seed):
    s = synth.make_system(n_atoms, r_c, seed)
    S, H, P_out = pipelines.system_mats(s, 1.0)
    keyg, keyv, vals = cg.ssf_export(dbsr(H))
    want_g, want_v, want_x = ssf.from_dense(block_mask(H), H.dense())
    assert np.array_equal(keyg.cpu().numpy().astype(np.int64), want_g)
    assert np.array_equal(keyv.cpu().numpy(), want_v)
    assert np.array_equal(vals.cpu().numpy(), want_x)


def test_import_of_a_scalar_pattern_and_round_trip():
    rng = np.random.default_rng(7)
    n = 4 * 37
    mask = rng.random((n, n)) < 0.08
    values = np.where(mask, rng.normal(size=(n, n)), 0.0)
    keyg, keyv, vals = ssf.from_dense(mask, values)
    A = cg.ssf_import(n, keyg, torch.as_tensor(keyv, device=DEV), torch.as_tensor(vals, device=DEV))
    # block pattern: every block holding an entry, plus the diagonal blocks
    blocks = mask.reshape(n // 4, 4, n // 4, 4).any(axis=(1, 3)) | np.eye(n // 4, dtype=bool)
    rp, ci = A.row_ptr.cpu().numpy(), A.col_idx.cpu().numpy()
    got_blocks = np.zeros_like(blocks)
    got_blocks[np.repeat(np.arange(n // 4), np.diff(rp)), ci] = True
    assert np.array_equal(got_blocks, blocks)
    assert np.all(np.diff(ci)[np.diff(np.repeat(np.arange(n // 4), np.diff(rp))) == 0] > 0)  # sorted rows
    dense = np.zeros((n, n))
    V = A.vals.cpu().numpy()
    for I in range(n // 4):
        for p in range(rp[I], rp[I + 1]):
            dense[4 * I:4 * I + 4, 4 * ci[p]:4 * ci[p] + 4] = V[p]
    assert np.array_equal(dense, values)
    # segments that span rows are read in row-major order
    kg2 = np.array([[n - 1, 2, 3, 4]])  # from (row 3, col n-1) to (row 4, col 2)
    B = cg.ssf_import(n, kg2, torch.tensor([1], device=DEV), torch.tensor([1.0, 2.0, 3.0, 4.0], device=DEV))
    mB, vB = ssf.to_dense(n, kg2, np.array([1]), np.array([1.0, 2.0, 3.0, 4.0]))
    rpB, ciB, VB = B.row_ptr.cpu().numpy(), B.col_idx.cpu().numpy(), B.vals.cpu().numpy()
    dB = np.zeros((n, n))
    for I in range(n // 4):
        for p in range(rpB[I], rpB[I + 1]):
            dB[4 * I:4 * I + 4, 4 * ciB[p]:4 * ciB[p] + 4] = VB[p]
    assert np.array_equal(dB, vB)


def test_import_rejects_segments_outside_the_matrix():
    n = 8
    with pytest.raises(cg.ChebError):
        cg.ssf_import(n, np.array([[1, 9, 1, 1]]), torch.tensor([1], device=DEV), torch.zeros(9, device=DEV,
                                                                                                dtype=torch.float64))
    with pytest.raises(cg.ChebError):  # values run past the value array
        cg.ssf_import(n, np.array([[1, 4, 1, 1]]), torch.tensor([1], device=DEV), torch.zeros(3, device=DEV,
                                                                                                dtype=torch.float64))
