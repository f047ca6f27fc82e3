"""GPU parity: every C-ABI call against the FP64 CPU oracle on the same seeded inputs.

Tolerances: integer work (patterns, mu decisions, degrees) must be identical;
FP64 values must match to relative Frobenius 1e-10 (rounding-order differences
only); the FP32 recursion is compared against FP64 with the bound derived in
test_expand_fp32_error_bound.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import pipelines, ref

pytestmark = pytest.mark.gpu

cg = pytest.importorskip("paper_1704_00512_gb300")
from paper_1704_00512_gb300 import solve  # noqa: E402

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
if DEV is None:
    pytest.skip("no CUDA device", allow_module_level=True)


def relF(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dbsr(row_ptr, col_idx, vals=None):
    return cg.Bsr(torch.as_tensor(row_ptr, dtype=torch.int64, device=DEV),
                  torch.as_tensor(col_idx, dtype=torch.int32, device=DEV),
                  None if vals is None else torch.as_tensor(np.ascontiguousarray(vals), dtype=torch.float64,
                                                           device=DEV))


def setup(n_atoms, r_c, r_buf, seed):
    s = synth.make_system(n_atoms, r_c, seed)
    S, H, P_out = pipelines.system_mats(s, r_buf)
    return s, S, H, P_out


# --------------------------------------------------------------------------
# A1 patterns: bit-exact
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n_atoms,r", [(1, 5.0), (7, 3.0), (200, 8.0), (200, 12.0), (1000, 10.0), (3000, 14.0)])
def test_pattern_build_exact(n_atoms, r):
    xyz, L = synth.place_atoms(n_atoms, seed=n_atoms)
    rp, ci = cg.pattern_build(torch.as_tensor(xyz, device=DEV), L, r)
    orp, oci = ref.pattern(xyz, L, r)
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(ci.cpu().numpy(), oci)


def test_pattern_build_boundary_distances_exact():
    # atoms at exactly representable distances on the cutoff
    xyz = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 2.0, 0.0], [9.0, 9.0, 9.0], [1.0, 1.0, 1.0]])
    for r in (2.0, np.sqrt(3.0), 1.9999999999999998):
        rp, ci = cg.pattern_build(torch.as_tensor(xyz, device=DEV), 10.0, float(r))
        orp, oci = ref.pattern(xyz, 10.0, float(r))
        assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(ci.cpu().numpy(), oci)


# --------------------------------------------------------------------------
# elementwise helpers
# --------------------------------------------------------------------------

def test_scale_transpose_restrict_trace():
    s, S, H, P_out = setup(60, 4.0, 2.0, 1)
    dH = dbsr(s.row_ptr, s.col_idx, s.H)
    got = cg.scale(dH, -3.0, 2.5).cpu().numpy()
    want = ref.scale(H, -3.0, 2.5).vals
    assert np.max(np.abs(got - want)) == 0.0
    rng = np.random.default_rng(0)
    X = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
    dP = dbsr(P_out.row_ptr, P_out.col_idx, X.vals)
    plan = cg.Plan(dP, cg.F64)
    assert np.array_equal(cg.transpose(plan, dP.vals).cpu().numpy(), ref.transpose(X).vals)
    dS = dbsr(s.row_ptr, s.col_idx, s.S)
    r = cg.restrict(dP, dS).cpu().numpy()
    assert np.array_equal(r, ref.restrict(X, S).vals)
    tr = cg.trace(dP, dS).item()
    assert abs(tr - ref.trace_product(X, S)) < 1e-12 * abs(tr) + 1e-12


# --------------------------------------------------------------------------
# masked products: several panels, ragged tail, both left patterns
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n_atoms,r_c,r_buf", [(33, 3.0, 1.5), (150, 5.0, 3.0), (600, 8.0, 4.0)])
def test_masked_product_fp64(n_atoms, r_c, r_buf):
    s, S, H, P_out = setup(n_atoms, r_c, r_buf, n_atoms)
    rng = np.random.default_rng(n_atoms)
    R = rng.normal(size=(P_out.nnzb, 4, 4))
    D = rng.normal(size=(P_out.nnzb, 4, 4))
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    plan = cg.Plan(dP, cg.F64)
    npan, width, mu = plan.info()
    assert width == 2 and npan >= (n_atoms + 1) // 2
    dR = torch.as_tensor(R, device=DEV)
    dD = torch.as_tensor(D, device=DEV)
    for Lm in (H, P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))):
        dL = dbsr(Lm.row_ptr, Lm.col_idx, Lm.vals)
        C = torch.empty_like(dR)
        cg.masked_product(plan, dL, dR, C, alpha=2.0, D=dD, beta=-1.0)
        want = 2.0 * ref.masked_product(Lm, P_out.with_vals(R), P_out.row_ptr, P_out.col_idx) - D
        assert relF(C.cpu().numpy(), want) < 1e-13


# --------------------------------------------------------------------------
# the fused recursion
# --------------------------------------------------------------------------

def _expand_case(n_atoms, r_c, r_buf, seed, n, nf):
    s, S, H, P_out = setup(n_atoms, r_c, r_buf, seed)
    w = np.linalg.eigvalsh(H.dense()) if n_atoms <= 300 else None
    e0, e1 = (w[0] - 0.05, w[-1] + 0.05) if w is not None else (-12.0, 12.0)
    Ht = ref.scale(H, e0, e1)
    rng = np.random.default_rng(seed)
    coeffs = rng.normal(size=(nf, n)) / (1.0 + np.arange(n)) ** 1.5
    G = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
    return s, H, P_out, e0, e1, Ht, coeffs, G


@pytest.mark.parametrize("n_atoms,r_c,r_buf,n,nf", [(33, 3.0, 1.5, 40, 1), (120, 4.0, 2.0, 64, 3),
                                                     (400, 6.0, 3.0, 30, 8)])
def test_expand_fp64_parity(n_atoms, r_c, r_buf, n, nf):
    s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(n_atoms, r_c, r_buf, n_atoms + 1, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    plan = cg.Plan(dP, cg.F64)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    t = torch.zeros(n, dtype=torch.float64, device=DEV)
    g = torch.zeros(n, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, moments=t,
              G=torch.as_tensor(G.vals, device=DEV), gmoments=g, precision=cg.F64)
    for j in range(nf):
        assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < 1e-10
    assert relF(t.cpu().numpy(), ex.t) < 1e-10
    assert relF(g.cpu().numpy(), ex.g) < 1e-10


def test_expand_deterministic_and_moments_only():
    s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(120, 4.0, 2.0, 5, 50, 2)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    plan = cg.Plan(dP, cg.F64)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    dG = torch.as_tensor(G.vals, device=DEV)
    outs = []
    for _ in range(2):
        acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(2)]
        g = torch.zeros(50, dtype=torch.float64, device=DEV)
        cg.expand(plan, dHt, 50, torch.as_tensor(coeffs, device=DEV), acc, G=dG, gmoments=g)
        outs.append((acc[0].cpu().numpy(), g.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    g2 = torch.zeros(50, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, 50, None, [], G=dG, gmoments=g2)
    assert np.array_equal(g2.cpu().numpy(), outs[0][1])


def test_expand_fp32_error_bound():
    # FP32 T_k: each step adds a rounding of relative size u = 2^-24 to a term
    # whose norm stays O(1) in the scaled spectrum; a perturbation at step j
    # reaches T_k through U_{k-j} (|U_m| <= m+1), so the accumulated error of
    # sum c_k T_k is below u * sum_k |c_k| * k^2 (up to a modest constant).
    n, nf = 64, 2
    s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(150, 4.0, 2.0, 9, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    plan = cg.Plan(dP, cg.F32)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    g = torch.zeros(n, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, G=torch.as_tensor(G.vals, device=DEV),
              gmoments=g, precision=cg.F32)
    u = 2.0 ** -24
    k = np.arange(n)
    for j in range(nf):
        bound = 8 * u * np.sum(np.abs(coeffs[j]) * (1 + k) ** 2) * np.sqrt(P_out.nnzb * 16)
        err = np.linalg.norm(acc[j].cpu().numpy() - ex.acc[j].vals)
        assert err < bound, (err, bound)
        assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < 1e-4


def test_expand_bf16_error_bound():
    # BF16 mode: M~ and every stored T_k rounded to bfloat16 (u = 2^-8), block
    # products summed in FP32, accumulators and moments in FP64.  The same
    # perturbation argument as for FP32 bounds the error with u = 2^-8.
    n, nf = 64, 2
    s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(150, 4.0, 2.0, 9, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    plan = cg.Plan(dP, cg.BF16)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    g = torch.zeros(n, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, G=torch.as_tensor(G.vals, device=DEV),
              gmoments=g, precision=cg.BF16, stepwise=True)
    u = 2.0 ** -8
    k = np.arange(n)
    errs = []
    for j in range(nf):
        bound = 8 * u * np.sum(np.abs(coeffs[j]) * (1 + k) ** 2) * np.sqrt(P_out.nnzb * 16)
        err = np.linalg.norm(acc[j].cpu().numpy() - ex.acc[j].vals)
        errs.append(relF(acc[j].cpu().numpy(), ex.acc[j].vals))
        assert err < bound, (err, bound)
    print(f"BF16 recursion, {n} terms: relative Frobenius error of the accumulators {max(errs):.2e}")
    # bfloat16 really is coarser than FP32 here, and still a usable approximation
    assert 1e-5 < max(errs) < 5e-2


# --------------------------------------------------------------------------
# coefficients and degree (Eq. 4, Eq. 6)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("func,emin,emax,tol,rel", [
    ({"kind": 0, "mu": 0.1, "kT": 0.05}, -2.0, 3.0, 1e-10, False),
    ({"kind": 1, "mu": -0.3, "kT": 0.1}, -2.0, 3.0, 1e-9, False),
    ({"kind": 2, "a": -1.0}, 0.05, 3.0, 1e-10, True),
    ({"kind": 2, "a": 0.5}, 0.05, 3.0, 1e-10, True),
    ({"kind": 2, "a": -0.5}, 0.05, 3.0, 1e-10, True),
    ({"kind": 3, "lo": -0.5, "hi": 0.7, "kT": 0.05}, -2.0, 3.0, 1e-8, False),
])
def test_coeffs_and_degree_parity(func, emin, emax, tol, rel):
    n, c = cg.coeffs([func], emin, emax, tol, 4096, rel=rel, device=DEV)
    f = ref.Func(func["kind"], mu=func.get("mu", 0.0), kT=func.get("kT", 0.0), a=func.get("a", 0.0),
                 lo=func.get("lo", 0.0), hi=func.get("hi", 0.0))
    assert n == ref.choose_degree(f, emin, emax, tol, 4096, rel=rel)
    want = ref.cheb_coeffs(f, n, emin, emax)
    got = c.cpu().numpy()[0]
    assert np.max(np.abs(got[:n] - want)) < 1e-13 * max(1.0, np.max(np.abs(want)))
    assert np.all(got[n:] == 0)


def test_coeffs_several_functions_take_largest_degree():
    fs = [{"kind": 0, "mu": 0.0, "kT": 0.2}, {"kind": 0, "mu": 0.0, "kT": 0.05}]
    n, c = cg.coeffs(fs, -2.0, 2.0, 1e-10, 8192, device=DEV)
    n2 = max(ref.choose_degree(ref.Func(0, mu=0.0, kT=f["kT"]), -2.0, 2.0, 1e-10, 8192) for f in fs)
    assert n == n2
    with pytest.raises(cg.ChebError) as e:
        cg.coeffs([{"kind": 0, "mu": 0.0, "kT": 1e-4}], -2.0, 2.0, 1e-10, 64, device=DEV)
    assert e.value.code == 5


def test_penalty_trace_parity():
    rng = np.random.default_rng(3)
    t = rng.normal(size=300)
    got = cg.penalty_trace(torch.as_tensor(t, device=DEV), 300, -100.0).item()
    want = ref.penalty_trace(t, -100.0, -1.0, 1.0)
    assert abs(got - want) < 1e-12 * max(1.0, abs(want))


# --------------------------------------------------------------------------
# Lanczos bounds
# --------------------------------------------------------------------------

def test_bounds_parity_and_containment():
    s, S, H, P_out = setup(300, 6.0, 3.0, 4)
    for M in (S, H):
        dM = dbsr(M.row_ptr, M.col_idx, M.vals)
        e0, e1, th = cg.bounds(dM, 40)
        a, b = ref.lanczos(M, pipelines.lanczos_start(4 * 300), 40)
        o0, o1, oth0, oth1 = ref.ritz_bounds(a, b)
        w = np.linalg.eigvalsh(M.dense())
        width = w[-1] - w[0]
        assert e0 <= w[0] and e1 >= w[-1]
        assert abs(th[0] - oth0) < 1e-9 * width and abs(th[1] - oth1) < 1e-9 * width
        # margins depend on tiny Ritz residuals; agree to the 1e-6 of the width
        assert abs(e0 - o0) < 1e-6 * width and abs(e1 - o1) < 1e-6 * width


def test_bounds_warm_start_hull():
    s, S, H, P_out = setup(300, 6.0, 3.0, 4)
    dH = dbsr(H.row_ptr, H.col_idx, H.vals)
    e0, e1, th = cg.bounds(dH, 8)
    w = np.linalg.eigvalsh(H.dense())
    assert th[0] >= w[0] - 1e-12 and th[1] <= w[-1] + 1e-12  # Ritz values lie inside the spectrum
    # a warm interval that contains the Lanczos interval is kept as it is
    wide = (e0 - 0.3, e1 + 0.2)
    assert cg.bounds_warm(dH, wide, 8)[:2] == wide
    # a warm interval that misses it on either side is widened to it there
    narrow = (0.5 * (e0 + e1) - 0.1, 0.5 * (e0 + e1) + 0.1)
    assert cg.bounds_warm(dH, narrow, 8)[:2] == (e0, e1)
    assert cg.bounds_warm(dH, (e0 + 0.05, e1 + 0.5), 8)[:2] == (e0, e1 + 0.5)
    with pytest.raises(cg.ChebError):
        cg.bounds_warm(dH, (1.0, 1.0), 8)


# --------------------------------------------------------------------------
# mu search, Newton-Schulz, whole solves
# --------------------------------------------------------------------------

def test_mu_search_decisions_match():
    s, S, H, P_out = setup(40, 3.0, 1.5, 6)
    w = np.linalg.eigvalsh(H.dense())
    e0, e1 = w[0] - 0.1, w[-1] + 0.1
    n = 400
    Ht = ref.scale(H, e0, e1)
    ex = ref.chebyshev_expand(Ht, P_out, np.zeros((1, n)), G=ref.identity(P_out))
    N_e = 80.0
    for kind in (0, 1):
        want = ref.mu_bisect(ex.g, kind, 0.05, e0, e1, N_e, 1e-9 * N_e)
        res = cg.decode_mu_result(cg.mu_search(torch.as_tensor(ex.g, device=DEV), n, e0, e1, kind, 0.05, N_e,
                                               1e-9 * N_e))
        assert res["converged"] == want.converged and res["iters"] == want.iters
        assert res["bits"] == want.bits
        assert abs(res["mu"] - want.mu) <= 1e-15 * max(1.0, abs(want.mu))


def test_newton_schulz_parity():
    s, S, H, P_out = setup(150, 5.0, 3.0, 7)
    rng = np.random.default_rng(1)
    X0 = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)) * 0.1)
    want = ref.newton_schulz(S, X0, P_out).vals
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    plan = cg.Plan(dP, cg.F64)
    dX0 = torch.as_tensor(X0.vals, device=DEV)
    X1, tmp = torch.empty_like(dX0), torch.empty_like(dX0)
    cg.newton_schulz(plan, dbsr(s.row_ptr, s.col_idx, s.S), dX0, X1, tmp)
    assert relF(X1.cpu().numpy(), want) < 1e-12


def test_powers_solve_parity():
    s, S, H, P_out = setup(300, 6.0, 3.0, 8)
    pb = solve.problem_from_system(s, 3.0, DEV)
    out = solve.powers(pb, exponents=(-1.0, 0.5, -0.5), tol=1e-10, n_max=512, newton_schulz=True)
    orc = pipelines.powers(S, P_out, (-1.0, 0.5, -0.5), out["bounds"], out["n_terms"], newton_schulz=True)
    for j in range(3):
        assert relF(out["acc"][j].cpu().numpy(), orc["acc"][j].vals) < 1e-10
    assert relF(out["inv_ns"].cpu().numpy(), orc["inv_ns"].vals) < 1e-10


@pytest.mark.parametrize("kind", [0, 1])
def test_foe_solve_parity(kind):
    s, S, H, P_out = setup(48, 3.5, 1.5, 10)
    N_e = float(s.n_rows // 2)
    out = solve.foe_solve(s, 1.5, kT=0.08, N_e=N_e, tol=1e-9, kind=kind, device=DEV)
    orc = pipelines.foe(S, H, P_out, 0.08, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e, kind=kind)
    r = out["mu_result"]
    assert r["converged"] and orc["mu"].converged
    assert r["bits"] == orc["mu"].bits and r["iters"] == orc["mu"].iters
    assert abs(out["mu"] - orc["mu"].mu) < 1e-12
    assert relF(out["gmoments"].cpu().numpy(), orc["gmoments"]) < 1e-10
    assert relF(out["F_host"], orc["F"].vals) < 1e-10
    assert abs(out["trace_FS"] - N_e) < 1e-6


def test_invalid_pattern_and_workspace_errors():
    rp = torch.tensor([0, 1, 2], dtype=torch.int64, device=DEV)
    ci = torch.tensor([1, 1], dtype=torch.int32, device=DEV)  # row 0 misses its diagonal
    with pytest.raises(cg.ChebError) as e:
        cg.Plan(cg.Bsr(rp, ci), cg.F64)
    assert e.value.code == 1
    ci2 = torch.tensor([0, 1, 1], dtype=torch.int32, device=DEV)
    rp2 = torch.tensor([0, 2, 3], dtype=torch.int64, device=DEV)  # (0,1) present, (1,0) missing
    with pytest.raises(cg.ChebError) as e:
        cg.Plan(cg.Bsr(rp2, ci2), cg.F64)
    assert "symmetric" in str(e.value)


@pytest.mark.parametrize("prec", [0, 1])
def test_every_tile_shape_matches(prec):
    n, nf = 40, 2
    s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(150, 5.0, 3.0, 21, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    tol = 1e-10 if prec == cg.F64 else 1e-5
    for tile in range(len(cg.tile_shapes(prec))):
        plan = cg.Plan(dP, prec, tile)
        acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
        g = torch.zeros(n, dtype=torch.float64, device=DEV)
        cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, G=torch.as_tensor(G.vals, device=DEV),
                  gmoments=g, precision=prec)
        for j in range(nf):
            assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < tol, (tile, j)
        assert relF(g.cpu().numpy(), ex.g) < tol


def test_resident_and_stepwise_expansions_agree_with_oracle():
    n, nf = 48, 3
    s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(180, 5.0, 3.0, 31, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    for prec, tol in ((cg.F64, 1e-10), (cg.F32, 1e-5)):
        plan = cg.Plan(dP, prec)
        outs = {}
        for stepwise in (False, True):
            acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
            t = torch.zeros(n, dtype=torch.float64, device=DEV)
            g = torch.zeros(n, dtype=torch.float64, device=DEV)
            cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, moments=t,
                      G=torch.as_tensor(G.vals, device=DEV), gmoments=g, precision=prec, stepwise=stepwise)
            for j in range(nf):
                assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < tol
            assert relF(t.cpu().numpy(), ex.t) < tol and relF(g.cpu().numpy(), ex.g) < tol
            outs[stepwise] = acc[0].cpu().numpy()
        # two independent kernels, same arithmetic up to summation order
        assert relF(outs[False], outs[True]) < (1e-12 if prec == cg.F64 else 1e-5)


def _block_diag(systems, r_buf):
    """Concatenate systems block-diagonally: (P_H, S, H, P_out, row starts)."""
    rps, cis, Ss, Hs, orps, ocis, starts = [], [], [], [], [], [], [0]
    off = 0
    boff = 0
    oboff = 0
    for s in systems:
        rp, ci = ref.pattern(s.xyz, s.L, s.r_cut + r_buf)
        rps.append(s.row_ptr[:-1] + boff)
        cis.append(s.col_idx + off)
        Ss.append(s.S)
        Hs.append(s.H)
        orps.append(rp[:-1] + oboff)
        ocis.append(ci + off)
        off += s.n_atoms
        boff += s.nnzb
        oboff += len(ci)
        starts.append(off)
    rp = np.concatenate(rps + [[boff]]).astype(np.int64)
    orp = np.concatenate(orps + [[oboff]]).astype(np.int64)
    return (rp, np.concatenate(cis).astype(np.int32), np.concatenate(Ss), np.concatenate(Hs), orp,
            np.concatenate(ocis).astype(np.int32), starts)


@pytest.mark.parametrize("prec", [1, 0])
def test_batched_expansion_matches_per_system_oracle(prec):
    systems = [synth.make_system(na, 4.0, seed) for na, seed in ((40, 1), (90, 2), (25, 3))]
    rp, ci, S, H, orp, oci, starts = _block_diag(systems, 2.0)
    rng = np.random.default_rng(4)
    ns = [30, 45, 20]
    nf = 2
    kmax = max(ns)
    bounds, Hts = [], []
    for s in systems:
        w = np.linalg.eigvalsh(synth.to_dense(s.row_ptr, s.col_idx, s.H))
        bounds.append((w[0] - 0.1, w[-1] + 0.1))
    # scale each system's block range of H with its own bounds
    Ht_vals = np.empty_like(H)
    bo = 0
    for s, (e0, e1) in zip(systems, bounds):
        Ht_vals[bo:bo + s.nnzb] = ref.scale(ref.Bsr(s.row_ptr, s.col_idx, s.H), e0, e1).vals
        bo += s.nnzb
    coeffs = np.zeros((len(systems), nf, kmax))
    for i, n in enumerate(ns):
        coeffs[i, :, :n] = rng.normal(size=(nf, n)) / (1.0 + np.arange(n)) ** 1.5
    Gv = rng.normal(size=(len(oci), 4, 4))
    dP = dbsr(orp, oci)
    plan = cg.BatchedPlan(dP, starts, prec)
    assert cg.plan_resident_info(plan)[0] >= len(systems)
    dHt = dbsr(rp, ci, Ht_vals)
    acc = [torch.zeros((len(oci), 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    t = torch.zeros((len(systems), kmax), dtype=torch.float64, device=DEV)
    g = torch.zeros((len(systems), kmax), dtype=torch.float64, device=DEV)
    cg.expand_batched(plan, dHt, kmax, torch.tensor(ns, dtype=torch.int32, device=DEV),
                      torch.as_tensor(coeffs.reshape(-1), device=DEV),
                      torch.tensor([i * nf * kmax for i in range(len(systems))], dtype=torch.int64, device=DEV),
                      kmax, acc, moments=t, G=torch.as_tensor(Gv, device=DEV), gmoments=g, moment_stride=kmax,
                      precision=prec)
    tol = 1e-10 if prec == cg.F64 else 1e-5
    ob = 0
    for i, s in enumerate(systems):
        rpo, cio = ref.pattern(s.xyz, s.L, s.r_cut + 2.0)
        Po = ref.Bsr(rpo, cio, None)
        Hti = ref.Bsr(s.row_ptr, s.col_idx, Ht_vals[sum(x.nnzb for x in systems[:i]):][:s.nnzb])
        Gi = Po.with_vals(Gv[ob:ob + len(cio)])
        ex = ref.chebyshev_expand(Hti, Po, coeffs[i, :, :ns[i]], G=Gi)
        for j in range(nf):
            assert relF(acc[j][ob:ob + len(cio)].cpu().numpy(), ex.acc[j].vals) < tol
        assert relF(t[i, :ns[i]].cpu().numpy(), ex.t) < tol
        assert relF(g[i, :ns[i]].cpu().numpy(), ex.g) < tol
        ob += len(cio)


def test_newton_schulz_isqrt_parity():
    s, S, H, P_out = setup(150, 5.0, 3.0, 17)
    rng = np.random.default_rng(5)
    Z0 = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)) * 0.1)
    want = ref.newton_schulz_isqrt(S, Z0, P_out).vals
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    plan = cg.Plan(dP, cg.F64)
    dZ0 = torch.as_tensor(Z0.vals, device=DEV)
    Z1, t1, t2 = torch.empty_like(dZ0), torch.empty_like(dZ0), torch.empty_like(dZ0)
    cg.newton_schulz_isqrt(plan, dbsr(s.row_ptr, s.col_idx, s.S), dZ0, Z1, t1, t2)
    assert relF(Z1.cpu().numpy(), want) < 1e-12


def test_mixed_precision_foe_error_vs_fp64():
    # The FP32 recursion (FP64 accumulators, FP64 S^-1/2) against the all-FP64
    # solve with the same bounds and term count must stay within the 1e-6
    # relative Frobenius target.  The alternative S^-1/2 from an FP32 expansion
    # plus one FP64 Newton-Schulz step converges to the in-pattern fixed point
    # of that iteration, which differs from the truncated Chebyshev S^-1/2 by
    # the truncation error of the pattern (reported, loose bound).
    s = synth.make_system(400, 6.0, 18)
    N_e = float(s.n_rows // 2)
    ref64 = solve.foe_solve(s, 3.0, kT=0.04, N_e=N_e, tol=1e-9, device=DEV)
    F64 = ref64["F_host"]
    errs = {}
    for mode in ("f64", "f32ns"):
        out = solve.foe_solve(s, 3.0, kT=0.04, N_e=N_e, tol=1e-9, precision=cg.F32, device=DEV,
                              bounds_S=ref64["bounds_S"], n_S=ref64["n_S"], bounds_H=ref64["bounds_H"],
                              n_H=ref64["n_terms"], isqrt=mode)
        errs[mode] = relF(out["F_host"], F64)
        print(f"isqrt={mode}: n_terms={out['n_terms']} relF(F32 vs F64) = {errs[mode]:.3e}, "
              f"Tr(FS)-N_e = {out['trace_FS'] - N_e:.2e}")
        assert abs(out["trace_FS"] - N_e) < 1e-5 * N_e
    assert errs["f64"] < 1e-6
    assert errs["f32ns"] < 1e-3


def test_mixed_precision_error_at_the_bench_degree():
    # Same kT (0.005 Ha) and fit tolerance (1e-7) as the 40,000-row bench solve,
    # hence about the same number of terms (~9e3), on a 2,000-row system: the
    # FP32-recursion F against the all-FP64 F.
    s = synth.make_system(500, 10.0, 19)
    N_e = float(s.n_rows // 2)
    ref64 = solve.foe_solve(s, 4.0, kT=0.005, N_e=N_e, tol=1e-7, tol_S=1e-10, device=DEV)
    out = solve.foe_solve(s, 4.0, kT=0.005, N_e=N_e, tol=1e-7, tol_S=1e-10, precision=cg.F32, device=DEV,
                          bounds_S=ref64["bounds_S"], n_S=ref64["n_S"], bounds_H=ref64["bounds_H"],
                          n_H=ref64["n_terms"])
    err = relF(out["F_host"], ref64["F_host"])
    print(f"bench degree: n_terms={out['n_terms']} relF(F32 vs F64) = {err:.3e}, "
          f"|mu32 - mu64| = {abs(out['mu'] - ref64['mu']):.2e}")
    assert out["n_terms"] >= 7000
    assert err < 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_operator_row_lists_match_oracle_and_ranking_path(prec):
    n, nf = 40, 2
    for n_atoms, r_c, r_buf in ((33, 3.0, 1.5), (300, 6.0, 3.0)):
        s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(n_atoms, r_c, r_buf, 51 + n_atoms, n, nf)
        ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
        dP = dbsr(P_out.row_ptr, P_out.col_idx)
        dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
        dc = torch.as_tensor(coeffs, device=DEV)
        dG = torch.as_tensor(G.vals, device=DEV)

        def run(plan):
            acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
            g = torch.zeros(n, dtype=torch.float64, device=DEV)
            cg.expand(plan, dHt, n, dc, acc, G=dG, gmoments=g, precision=prec, stepwise=True)
            return acc, g

        acc_rank, g_rank = run(cg.Plan(dP, prec))
        acc, g = run(cg.Plan(dP, prec).attach_operator(dHt))
        tol = 1e-10 if prec == cg.F64 else 1e-5
        for j in range(nf):
            assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < tol
            if prec == cg.F64:
                # same blocks multiplied in the same order as the ranking path
                assert torch.equal(acc[j], acc_rank[j])
            else:
                # FP32 plans with lists run the column-order kernel, which
                # sums each block product in another order
                assert relF(acc[j].cpu().numpy(), acc_rank[j].cpu().numpy()) < tol
        assert relF(g.cpu().numpy(), ex.g) < tol
        if prec == cg.F64:
            assert torch.equal(g, g_rank)


@pytest.mark.parametrize("n_atoms,r_c,r_buf", [(33, 3.0, 1.5), (150, 5.0, 3.0), (600, 8.0, 4.0)])
def test_masked_product_row_lists(n_atoms, r_c, r_buf):
    """Masked products through the row lists, including an operator whose rows
    have no block inside some panels' unions, and an operator of another
    pattern on the same plan (ranking path)."""
    s, S, H, P_out = setup(n_atoms, r_c, r_buf, n_atoms)
    rng = np.random.default_rng(n_atoms + 7)
    R = torch.as_tensor(rng.normal(size=(P_out.nnzb, 4, 4)), device=DEV)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    # a sparse operator on P_H: only blocks with (I + K) % 3 == 0 kept, so some
    # rows have none in a panel's union
    keep_rows = [[k for k in range(H.row_ptr[i], H.row_ptr[i + 1]) if (i + H.col_idx[k]) % 3 == 0]
                 for i in range(H.nbr)]
    rp = np.zeros(H.nbr + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in keep_rows])
    ks = np.array([k for r in keep_rows for k in r], dtype=np.int64)
    Ls = ref.Bsr(rp, H.col_idx[ks], rng.normal(size=(len(ks), 4, 4)))
    for Lm in (H, Ls):
        dL = dbsr(Lm.row_ptr, Lm.col_idx, Lm.vals)
        plan = cg.Plan(dP, cg.F64).attach_operator(dL)
        C = torch.empty_like(R)
        cg.masked_product(plan, dL, R, C)
        want = ref.masked_product(Lm, P_out.with_vals(R.cpu().numpy()), P_out.row_ptr, P_out.col_idx)
        assert relF(C.cpu().numpy(), want) < 1e-13
        # another operator pattern on the same plan takes the ranking path
        dO = dbsr(P_out.row_ptr, P_out.col_idx, rng.normal(size=(P_out.nnzb, 4, 4)))
        C2 = torch.empty_like(R)
        cg.masked_product(plan, dO, R, C2)
        want2 = ref.masked_product(ref.Bsr(P_out.row_ptr, P_out.col_idx, dO.vals.cpu().numpy()),
                                   P_out.with_vals(R.cpu().numpy()), P_out.row_ptr, P_out.col_idx)
        assert relF(C2.cpu().numpy(), want2) < 1e-13


def test_selected_eigenvalues_counts_and_levels():
    # Sec. "Extraction of selected eigenvalues" on a 40-row system whose
    # patterns are dense: the interval projector counts the generalised
    # eigenvalues in (lo, hi), the bisection to N - 1/2 lands on eps_N, and the
    # GPU sequence matches the oracle's step by step.
    import scipy.linalg as sla
    s = synth.make_system(10, 30.0, 13)
    S, H, P_out = pipelines.system_mats(s, 4.0)
    eps = sla.eigh(H.dense(), S.dense(), eigvals_only=True)
    kT = 0.01
    gaps = np.diff(eps)
    i = int(np.argmax(gaps[: len(gaps) // 2]))
    j = len(gaps) // 2 + int(np.argmax(gaps[len(gaps) // 2:]))
    lo, hi = 0.5 * (eps[i] + eps[i + 1]), 0.5 * (eps[j] + eps[j + 1])
    N = 7
    pb = solve.problem_from_system(s, 4.0, DEV, cg.F64)
    out = solve.selected_eigenvalues(pb, kT, intervals=[(lo, hi)], levels=[N], tol=1e-9)
    want = int(np.sum((eps > lo) & (eps < hi)))
    assert abs(out["counts"][0] - want) < 1e-4, (out["counts"], want)
    assert abs(out["eigenvalues"][0] - eps[N - 1]) < 3 * kT
    # the oracle's steps with the same bounds and degrees
    e0, e1 = out["bounds_H"]
    A = pipelines.powers(S, P_out, (-0.5,), out["bounds_S"], out["n_S"])["acc"][0]
    Hp = ref.orthogonalise(H, A, P_out)
    G = ref.trace_functional_matrix(A, S, P_out)
    c = ref.cheb_coeffs(ref.Func(ref.KIND_INTERVAL, kT=kT, lo=lo, hi=hi), out["n_terms"], e0, e1)
    ex = ref.chebyshev_expand(ref.scale(Hp, e0, e1), P_out, c[None], G=G)
    count = ref.trace_product(ref.postprocess(ex.acc[0], A, P_out), S)
    assert abs(out["counts"][0] - count) < 1e-9 * max(1.0, abs(count))
    assert relF(out["gmoments"].cpu().numpy(), ex.g) < 1e-10
    r = ref.mu_bisect(ex.g, ref.KIND_FERMI, kT, e0, e1, N - 0.5, 1e-10, 128)
    assert abs(out["eigenvalues"][0] - r.mu) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_resident_row_lists_bit_identical_to_ranking(prec):
    # the one-launch (resident) expansion reads its in-union operator blocks
    # from the plan's row lists when they are attached: same blocks, same
    # order, so the same bits as ranking them at every step
    n, nf = 40, 2
    s, H, P_out, e0, e1, Ht, coeffs, G = _expand_case(120, 4.0, 2.0, 77, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)

    def run(plan):
        assert cg.plan_resident_info(plan)[0] > 0
        acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
        g = torch.zeros(n, dtype=torch.float64, device=DEV)
        cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, G=torch.as_tensor(G.vals, device=DEV),
                  gmoments=g, precision=prec)
        return acc, g

    acc0, g0 = run(cg.Plan(dP, prec))
    acc1, g1 = run(cg.Plan(dP, prec).attach_operator(dHt))
    tol = 1e-10 if prec == cg.F64 else 1e-5
    for j in range(nf):
        assert torch.equal(acc1[j], acc0[j])
        assert relF(acc1[j].cpu().numpy(), ex.acc[j].vals) < tol
    assert torch.equal(g1, g0)
