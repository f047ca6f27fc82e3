"""GPU tests of the FOE solve sequence: the penalty check of Eq. 5 on the solve
path, and the form that accumulates 4 mu of a bracket in one pass against the
two-pass form and the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import pipelines, ref

pytestmark = pytest.mark.gpu

cg = pytest.importorskip("paper_1704_00512_gb300")
from paper_1704_00512_gb300 import _lib as L  # noqa: E402
from paper_1704_00512_gb300 import solve  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
if DEV is None:
    pytest.skip("no CUDA device", allow_module_level=True)


def relF(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def small():
    s = synth.make_system(120, 5.0, 31)
    pb = solve.problem_from_system(s, 2.5, DEV, cg.F64)
    ov = solve.overlap_setup(pb, 1e-10)
    return s, pb, ov


def test_penalty_silent_on_lanczos_bounds(small):
    s, pb, ov = small
    N_e = float(s.n_rows // 2)
    out = solve.foe(pb, 0.05, N_e, tol=1e-9, overlap=ov)
    assert len(out["penalty"]) == 1 and out["penalty"][0][0] == 0
    assert abs(out["penalty"][0][1]) < 1.0


@pytest.mark.parametrize("side", ["lower", "upper"])
def test_penalty_fires_on_shrunk_bounds_and_the_widened_retry_succeeds(small, side):
    s, pb, ov = small
    N_e = float(s.n_rows // 2)
    good = solve.foe(pb, 0.05, N_e, tol=1e-9, overlap=ov)
    e0, e1 = good["bounds_H"]
    w = e1 - e0
    shrunk = (e0 + 0.02 * w, e1) if side == "lower" else (e0, e1 - 0.02 * w)
    out = solve.foe(pb, 0.05, N_e, tol=1e-9, overlap=ov, bounds_H=shrunk, penalty_widen=0.05)
    verdicts = [p[0] for p in out["penalty"]]
    assert verdicts == [-1 if side == "lower" else 1, 0], out["penalty"]
    lo, hi = out["bounds_H"]
    if side == "lower":
        assert lo < shrunk[0] and hi == shrunk[1]
    else:
        assert hi > shrunk[1] and lo == shrunk[0]
    # the widened solve agrees with the one on Lanczos bounds to the fit tolerance
    assert abs(out["mu"] - good["mu"]) < 1e-6
    assert relF(out["F"].cpu().numpy(), good["F"].cpu().numpy()) < 1e-6


def test_penalty_reports_bounds_error_when_the_retry_fails(small):
    s, pb, ov = small
    N_e = float(s.n_rows // 2)
    good = solve.foe(pb, 0.05, N_e, tol=1e-9, overlap=ov)
    e0, e1 = good["bounds_H"]
    with pytest.raises(cg.ChebError) as e:
        solve.foe(pb, 0.05, N_e, tol=1e-9, overlap=ov, bounds_H=(e0 + 0.02 * (e1 - e0), e1), penalty_widen=0.0)
    assert e.value.code == L.ERR_BOUNDS


@pytest.mark.parametrize("prec,tol_F", [(0, 1e-9), (1, 1e-6)])
def test_four_mu_form_matches_two_pass_form(prec, tol_F):
    # the half-length moment pass brackets mu*, one pass accumulates 4 mu, the
    # bisection on all moments gives the two-pass mu*, F(mu*) interpolated
    s = synth.make_system(300, 6.0, 37)
    N_e = float(s.n_rows // 2)
    pb = solve.problem_from_system(s, 3.0, DEV, prec)
    ov = solve.overlap_setup(pb, 1e-10)
    two = solve.foe(pb, 0.02, N_e, tol=1e-8, overlap=ov, form="twopass")
    four = solve.foe(pb, 0.02, N_e, tol=1e-8, overlap=ov, form="mu4", bounds_H=two["bounds_H"],
                     n_H=two["n_terms"])
    assert four["passes"] == 2 and four["n_pass1"] == two["n_terms"] // 2
    assert abs(four["mu_half"]["mu"] - four["mu"]) < 0.1 * 0.02
    assert four["mu_result"]["bits"] == two["mu_result"]["bits"]
    assert abs(four["mu"] - two["mu"]) < 1e-12 * max(1.0, abs(two["mu"]))
    assert relF(four["F"].cpu().numpy(), two["F"].cpu().numpy()) < tol_F
    assert abs(four["trace_FS"].item() - N_e) < (1e-7 if prec == 0 else 1e-5) * N_e


def test_four_mu_form_fp64_against_the_oracle():
    s = synth.make_system(64, 4.0, 41)
    N_e = float(s.n_rows // 2)
    kT = 0.05
    pb = solve.problem_from_system(s, 2.0, DEV, cg.F64)
    out = solve.foe(pb, kT, N_e, tol=1e-9, form="mu4", mu_half_kT=0.02)
    S, H, P_out = pipelines.system_mats(s, 2.0)
    orc = pipelines.foe(S, H, P_out, kT, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e)
    assert abs(out["mu"] - orc["mu"].mu) < 1e-9
    assert relF(out["F"].cpu().numpy(), orc["F"].vals) < 1e-9


def test_energy_moments_and_energy_pair_fp64_against_the_oracle():
    s = synth.make_system(64, 4.0, 41)
    N_e = float(s.n_rows // 2)
    kT = 0.05
    pb = solve.problem_from_system(s, 2.0, DEV, cg.F64)
    out = solve.foe(pb, kT, N_e, tol=1e-9, energy=True)
    S, H, P_out = pipelines.system_mats(s, 2.0)
    orc = pipelines.foe(S, H, P_out, kT, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e, energy=True)
    e = out["emoments"].cpu().numpy()
    assert np.max(np.abs(e - orc["emoments"])) < 1e-10 * np.max(np.abs(orc["emoments"]))
    ep = solve.energy_pair(pb, out, 1.25 * kT)
    op = pipelines.energy_pair(orc, 1.25 * kT)
    E, Ep = float(ep["E"].item()), float(ep["E_prime"].item())
    assert abs(E - op["E"]) < 1e-10 * max(1.0, abs(op["E"]))
    assert abs(Ep - op["E_prime"]) < 1e-10 * max(1.0, abs(op["E_prime"]))
    assert abs(ep["mu_prime"] - op["mu_prime"].mu) < 1e-9
    # the energy functional is the adjoint of post-processing: the re-summed E
    # is Tr(F H) of the kernel the solve returned
    trFH = float(L.trace(pb.P_out.with_vals(out["F"]), pb.H).item())
    assert abs(trFH - E) < 1e-9 * max(1.0, abs(E))


def test_energy_moments_fp32_column_path_against_the_oracle():
    s = synth.make_system(120, 5.0, 31)
    N_e = float(s.n_rows // 2)
    kT = 0.05
    pb = solve.problem_from_system(s, 2.5, DEV, cg.F32)
    assert cg.plan_col_info(pb.planX)[0] > 0  # the column kernel runs the passes
    out = solve.foe(pb, kT, N_e, tol=1e-8, energy=True)
    S, H, P_out = pipelines.system_mats(s, 2.5)
    orc = pipelines.foe(S, H, P_out, kT, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e, energy=True)
    e = out["emoments"].cpu().numpy()
    # each raw moment within the FP32 recursion's perturbation bound: a rounding
    # at step j grows through U_{k-j} (at most k+1), summed over the k steps,
    # against |<dT_k, G_H>| <= ||dT_k|| ||G_H||
    k = np.arange(len(e))
    bound = 8 * 2.0 ** -24 * (k + 1) ** 2 * np.linalg.norm(orc["G_H"].vals) * np.sqrt(4 * H.nbr)
    assert np.all(np.abs(e - orc["emoments"]) < bound)
    # the energies the smearing check compares, at the reduced-precision bar
    ep = solve.energy_pair(pb, out, 1.25 * kT)
    op = pipelines.energy_pair(orc, 1.25 * kT)
    assert abs(float(ep["E"].item()) - op["E"]) < 1e-6 * abs(op["E"])
    assert abs(float(ep["E_prime"].item()) - op["E_prime"]) < 1e-6 * abs(op["E_prime"])


def test_auto_kT_fp64_against_the_oracle():
    s = synth.make_system(64, 4.0, 43)
    N_e = float(s.n_rows // 2)
    pb = solve.problem_from_system(s, 2.0, DEV, cg.F64)
    ov = solve.overlap_setup(pb, 1e-10)
    kT0, widen, shrink = 0.2, 1.25, 0.5
    probe = solve.foe_auto_kT(pb, kT0, N_e, 1e-300, widen, shrink, max_rounds=3, tol=1e-9, overlap=ov)
    dE = [abs(r[2] - r[3]) for r in probe["rounds"]]
    assert len(dE) == 3 and not probe["accepted"] and dE[0] > dE[1] > dE[2]
    dE_tol = float(np.sqrt(dE[1] * dE[2]))
    out = solve.foe_auto_kT(pb, kT0, N_e, dE_tol, widen, shrink, tol=1e-9, overlap=ov)
    S, H, P_out = pipelines.system_mats(s, 2.0)
    orc = pipelines.foe_auto_kT(S, H, P_out, kT0, N_e, dE_tol, ov["bounds_S"], ov["n_S"], out["bounds_H"], 1e-9,
                                16384, 1e-9 * N_e, widen=widen, shrink=shrink)
    assert [r[:2] for r in out["rounds"]] == [r[:2] for r in orc["rounds"]]
    assert [r[4] for r in out["rounds"]] == [r[4] for r in orc["rounds"]] == [False, False, True]
    for a, b in zip(out["rounds"], orc["rounds"]):
        assert abs(a[2] - b[2]) < 1e-10 * abs(b[2]) and abs(a[3] - b[3]) < 1e-10 * abs(b[3])
    assert out["kT"] == kT0 * shrink ** 2 and abs(out["mu"] - orc["mu"].mu) < 1e-9
    assert relF(out["F"].cpu().numpy(), orc["F"].vals) < 1e-9
