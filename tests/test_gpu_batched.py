"""Batched density matrices (many uneven systems in one launch per pass) against
the oracle, one system at a time, through the C ABI."""

import numpy as np
import pytest
import torch

import synth
from oracle import pipelines, ref

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1704_00512_gb300 as cg  # noqa: E402
from paper_1704_00512_gb300 import batched  # noqa: E402

DEV = torch.device("cuda:0")
SIZES = ((40, 11), (90, 12), (25, 13), (60, 14))
R_C, R_BUF, KT = 4.0, 2.0, 0.1


def relF(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _systems():
    return [synth.make_system(na, R_C, seed) for na, seed in SIZES]


def test_block_diag_matches_concatenation():
    systems = _systems()
    parts, want_rp, want_ci, want_v = [], [0], [], []
    off = boff = 0
    for s in systems:
        parts.append(cg.Bsr(torch.as_tensor(s.row_ptr, device=DEV), torch.as_tensor(s.col_idx, device=DEV),
                            torch.as_tensor(s.S, device=DEV)))
        want_rp += list(s.row_ptr[1:] + boff)
        want_ci += list(s.col_idx + off)
        want_v.append(s.S)
        off += s.n_atoms
        boff += s.nnzb
    out = cg.block_diag(parts)
    assert out.row_ptr.cpu().tolist() == want_rp
    assert out.col_idx.cpu().tolist() == want_ci
    assert torch.equal(out.vals.cpu(), torch.as_tensor(np.concatenate(want_v)))


@pytest.mark.parametrize("prec", [cg.F64, cg.F32])
def test_batched_foe_matches_per_system_oracle_and_replays(prec):
    systems = _systems()
    N_e = [2.0 * s.n_atoms for s in systems]
    bp = batched.BatchedProblem(systems, R_BUF, DEV, precision=prec)
    tolN = [(1e-9 if prec == cg.F64 else 1e-6) * n for n in N_e]
    out = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, tol_N=tolN)
    assert out["captured"]
    # the autotuner picked a shape of the table for both batched launches
    assert set(bp.tiles) == {cg.F64, prec} or set(bp.tiles) == {cg.F64}
    F = out["F"].cpu().numpy()
    for i, s in enumerate(systems):
        S, H, P_out = pipelines.system_mats(s, R_BUF)
        orc = pipelines.foe(S, H, P_out, KT, N_e[i], out["bounds_S"][i], out["n_S"][i], out["bounds_H"][i],
                            out["n_terms"][i], tol_N=tolN[i])
        Fi = F[bp.ooff[i]:bp.ooff[i + 1]]
        r = out["mu_result"][i]
        assert r["converged"]
        assert abs(out["trace_FS"][i] - N_e[i]) < 1e-5 * N_e[i]
        if prec == cg.F64:
            assert relF(Fi, orc["F"].vals) < 1e-10
            assert r["bits"] == orc["mu"].bits and r["iters"] == orc["mu"].iters
            assert abs(out["mu"][i] - orc["mu"].mu) < 1e-12
        else:
            assert relF(Fi, orc["F"].vals) < 1e-5
    # a second solve of the same batch replays the captured passes: same results
    again = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, tol_N=tolN)
    assert not again["captured"]
    assert torch.equal(again["F"], out["F"])
    assert again["mu"] == out["mu"]
    # and so does the eager sequence without graphs
    eager = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, tol_N=tolN, use_graphs=False)
    assert torch.equal(eager["F"], out["F"])
    # a new Hamiltonian in place (every system's H scaled by 1.0003: new bounds,
    # coefficients and mu, the same term counts): the replayed graphs read the
    # new values and agree with the eager sequence and with the oracle
    fac = 1.0003
    bp.H.vals.mul_(fac)
    new = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, tol_N=tolN)
    assert not new["captured"] and new["n_terms"] == out["n_terms"]
    assert new["mu"] != out["mu"]
    eager2 = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, tol_N=tolN, use_graphs=False)
    assert torch.equal(eager2["F"], new["F"]) and eager2["mu"] == new["mu"]
    assert [r["bits"] for r in eager2["mu_result"]] == [r["bits"] for r in new["mu_result"]]
    if prec == cg.F64:
        F2 = new["F"].cpu().numpy()
        for i, s in enumerate(systems):
            S, H, P_out = pipelines.system_mats(s, R_BUF)
            H = H.with_vals(H.vals * fac)
            orc = pipelines.foe(S, H, P_out, KT, N_e[i], new["bounds_S"][i], new["n_S"][i], new["bounds_H"][i],
                                new["n_terms"][i], tol_N=tolN[i])
            assert relF(F2[bp.ooff[i]:bp.ooff[i + 1]], orc["F"].vals) < 1e-10
            assert new["mu_result"][i]["bits"] == orc["mu"].bits


def test_autotune_caches_a_valid_tile():
    systems = _systems()
    bp = batched.BatchedProblem(systems, R_BUF, DEV, precision=cg.F32)
    Ht = bp.H.with_vals(torch.empty_like(bp.H.vals))
    for i, s in enumerate(systems):
        Hi = cg.Bsr(bp.PH[i].row_ptr, bp.PH[i].col_idx, bp.H.vals[bp.hoff[i]:bp.hoff[i + 1]])
        cg.scale(Hi, -3.0, 3.0, out=Ht.vals[bp.hoff[i]:bp.hoff[i + 1]])
    t = batched.autotune_tile(bp.P_out, bp.starts, cg.F32, Ht)
    assert 0 <= t < len(cg.tile_shapes(cg.F32))
    assert batched.autotune_tile(bp.P_out, bp.starts, cg.F32, Ht) == t


def test_batched_penalty_flags_the_system_whose_bound_is_shrunk():
    # Eq. 5 on every system's own traces from pass 1: Lanczos bounds pass; a
    # shrunk upper bound of system 2 (given as a warm start) is reported as
    # CHEB_ERR_BOUNDS naming that system and bound
    systems = _systems()
    N_e = [2.0 * s.n_atoms for s in systems]
    bp = batched.BatchedProblem(systems, R_BUF, DEV, precision=cg.F64)
    out = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, use_graphs=False)
    bH = list(out["bounds_H"])
    e0, e1 = bH[2]
    bH[2] = (e0, e1 - 0.02 * (e1 - e0))
    with pytest.raises(cg.ChebError) as e:
        batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, use_graphs=False, bounds_H=bH)
    assert e.value.code == batched.L.ERR_BOUNDS and "system 2" in str(e.value) and "upper" in str(e.value)
    # the warm start with the Lanczos bounds themselves solves as before
    again = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, use_graphs=False, bounds_H=out["bounds_H"])
    assert relF(again["F"].cpu().numpy(), out["F"].cpu().numpy()) < 1e-12


def test_batched_foe_in_the_double_float_mode():
    # CHEB_F64X through the batched resident kernel (per-system term counts):
    # the FP64 bar against the oracle, the same bisection decisions
    systems = _systems()
    N_e = [2.0 * s.n_atoms for s in systems]
    bp = batched.BatchedProblem(systems, R_BUF, DEV, precision=cg.F64X)
    tolN = [1e-9 * n for n in N_e]
    out = batched.foe_batched(bp, KT, N_e, tol=1e-9, tol_S=1e-10, tol_N=tolN, use_graphs=False)
    F = out["F"].cpu().numpy()
    for i, s in enumerate(systems):
        S, H, P_out = pipelines.system_mats(s, R_BUF)
        orc = pipelines.foe(S, H, P_out, KT, N_e[i], out["bounds_S"][i], out["n_S"][i], out["bounds_H"][i],
                            out["n_terms"][i], tol_N=tolN[i])
        assert relF(F[bp.ooff[i]:bp.ooff[i + 1]], orc["F"].vals) < 1e-10
        assert out["mu_result"][i]["bits"] == orc["mu"].bits
