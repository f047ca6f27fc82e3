"""Locality relabelling of a system (a library addition, not in the paper).

The atoms are put in Hilbert-curve order (cheb_locality_order), the patterns
are built from the reordered atoms, values move between the labellings by a
position map, and the solve runs in the new labelling.  Checked here:
  * the device order equals a plain restatement of Skilling's Hilbert index
    (AIP Conf. Proc. 707, 381 (2004)) sorted with ties by atom index, bit for bit;
  * the position map sends every block (I', J') to (perm I', perm J'), and
    gather then scatter is the identity;
  * an FP64 FOE solved in the new labelling and returned in the caller's
    matches the FP64 oracle (F to 1e-10, identical mu decision bits);
  * the mixed-precision 4-mu solve gives the same F in both labellings (FP32
    products: 1e-6).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import pipelines

pytestmark = pytest.mark.gpu

cg = pytest.importorskip("paper_1704_00512_gb300")
from paper_1704_00512_gb300 import _lib as L  # noqa: E402
from paper_1704_00512_gb300 import solve  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
if DEV is None:
    pytest.skip("no CUDA device", allow_module_level=True)

from hilbert_ref import order_ref  # noqa: E402


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (1000, 2), (3000, 3)])
def test_locality_order_is_the_hilbert_order(n, seed):
    if n >= 1000:
        xyz, box = synth.place_atoms(n, seed)
    else:
        box = 12.0
        xyz = np.random.default_rng(seed).uniform(-box, 2 * box, (n, 3))  # images outside the box too
    got = L.locality_order(torch.as_tensor(xyz, device=DEV), box).cpu().numpy()
    assert np.array_equal(got, order_ref(xyz, box))
    assert np.array_equal(np.sort(got), np.arange(n))


def _relabelled(n_atoms, r_cut, seed):
    xyz, box = synth.place_atoms(n_atoms, seed)
    dx = torch.as_tensor(xyz, device=DEV)
    perm = L.locality_order(dx, box)
    dxp = L.gather_rows(dx.reshape(-1), perm, 3).view(-1, 3)
    old = cg.Bsr(*L.pattern_build(dx, box, r_cut))
    new = cg.Bsr(*L.pattern_build(dxp, box, r_cut))
    return perm, old, new


def test_position_map_relabels_every_block_and_round_trips():
    perm, old, new = _relabelled(400, 7.0, 5)
    m = L.position_map(new, old, perm)
    p = perm.cpu().numpy()
    rp_o, ci_o = old.row_ptr.cpu().numpy(), old.col_idx.cpu().numpy()
    rp_n, ci_n = new.row_ptr.cpu().numpy(), new.col_idx.cpu().numpy()
    rows_n = np.repeat(np.arange(len(rp_n) - 1), np.diff(rp_n))
    rows_o = np.repeat(np.arange(len(rp_o) - 1), np.diff(rp_o))
    mh = m.cpu().numpy()
    assert np.array_equal(np.sort(mh), np.arange(old.nnzb))  # a bijection of the blocks
    assert np.array_equal(rows_o[mh], p[rows_n])
    assert np.array_equal(ci_o[mh], p[ci_n])
    vals = torch.randn(old.nnzb * 16, dtype=torch.float64, device=DEV)
    moved = L.gather_rows(vals, m, 16)
    back = L.scatter_rows(moved, m, 16, torch.zeros_like(vals))
    assert torch.equal(back, vals)


def test_position_map_refuses_a_foreign_pattern():
    perm, old, new = _relabelled(200, 6.0, 6)
    shuffled = perm[torch.randperm(perm.numel(), device=DEV)]
    with pytest.raises(cg.ChebError):
        L.position_map(new, old, shuffled)


def test_fp64_foe_in_hilbert_order_matches_the_oracle():
    s = synth.make_system(120, 4.0, 12)
    S, H, P_out = pipelines.system_mats(s, 2.0)
    N_e = float(s.n_rows // 2)
    out = solve.foe_solve(s, 2.0, kT=0.08, N_e=N_e, tol=1e-9, device=DEV, order="hilbert")
    assert out["problem"].perm is not None
    orc = pipelines.foe(S, H, P_out, 0.08, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e)
    r = out["mu_result"]
    assert r["converged"] and orc["mu"].converged
    assert r["bits"] == orc["mu"].bits and r["iters"] == orc["mu"].iters
    assert abs(out["mu"] - orc["mu"].mu) < 1e-12
    F = out["F_host"]  # the caller's labelling
    assert np.linalg.norm(F - orc["F"].vals) / np.linalg.norm(orc["F"].vals) < 1e-10
    assert abs(out["trace_FS"] - N_e) < 1e-6


def test_mixed_solve_gives_the_same_density_matrix_in_both_labellings():
    s = synth.make_system(700, 6.0, 13)
    N_e = float(s.n_rows // 2)
    kw = dict(kT=0.05, N_e=N_e, tol=1e-7, precision=L.F32, device=DEV, form="mu4", n_mu=4, tol_S=1e-10,
              tol_N=1e-9 * N_e)
    a = solve.foe_solve(s, 3.0, **kw)
    b = solve.foe_solve(s, 3.0, order="hilbert", **kw)
    assert b["problem"].perm is not None and a["problem"].perm is None
    assert abs(a["mu"] - b["mu"]) < 1e-8
    assert np.linalg.norm(a["F_host"] - b["F_host"]) / np.linalg.norm(a["F_host"]) < 1e-6
    assert abs(b["trace_FS"] - N_e) < 1e-6 * N_e
    ea = L.plan_col_info(a["problem"].planX)[2]
    eb = L.plan_col_info(b["problem"].planX)[2]
    print(f"column-kernel entries per step: generator order {ea}, Hilbert order {eb}")
