"""GPU parity of the FP64-accurate double-float mode (CHEB_F64X: T_k, the
operator and every block product as hi + lo float pairs on the FP32 pipe)
against the FP64 oracle, at the FP64 bar: relative Frobenius error below 1e-10
for accumulators and moments, the same mu decisions as the oracle."""
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


def case(n_atoms, r_c, r_buf, seed, n, nf):
    s = synth.make_system(n_atoms, r_c, seed)
    S, H, P_out = pipelines.system_mats(s, r_buf)
    w = np.linalg.eigvalsh(H.dense()) if n_atoms <= 200 else None
    e0, e1 = (w[0] - 0.05, w[-1] + 0.05) if w is not None else (-12.0, 12.0)
    Ht = ref.scale(H, e0, e1)
    rng = np.random.default_rng(seed)
    coeffs = rng.normal(size=(nf, n)) / (1.0 + np.arange(n)) ** 1.5
    G = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
    return Ht, P_out, coeffs, G


def run(plan, dHt, n, coeffs, G, nnzb, stepwise):
    nf = coeffs.shape[0]
    acc = [torch.zeros((nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    t = torch.zeros(n, dtype=torch.float64, device=DEV)
    g = torch.zeros(n, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, moments=t,
              G=torch.as_tensor(G.vals, device=DEV), gmoments=g, precision=cg.F64X, stepwise=stepwise)
    return acc, t, g


@pytest.mark.parametrize("n_atoms,r_c,r_buf,n,nf", [
    (40, 3.0, 1.5, 60, 1),     # one or two panels
    (200, 5.0, 2.5, 200, 3),   # many panels, a ragged last one, a long recursion
    (500, 6.0, 3.0, 40, 8),    # every accumulator
])
@pytest.mark.parametrize("stepwise", [True, False])
def test_f64x_expansion_parity(n_atoms, r_c, r_buf, n, nf, stepwise):
    Ht, P_out, coeffs, G = case(n_atoms, r_c, r_buf, 300 + n_atoms, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    plan = cg.Plan(dP, cg.F64X).attach_operator(dHt)
    acc, t, g = run(plan, dHt, n, coeffs, G, P_out.nnzb, stepwise)
    for j in range(nf):
        assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < 1e-10, j
    assert relF(t.cpu().numpy(), ex.t) < 1e-10
    assert relF(g.cpu().numpy(), ex.g) < 1e-10
    # far more accurate than FP32 products on the same case
    acc32 = [torch.zeros_like(acc[0])]
    cg.expand(cg.Plan(dP, cg.F32), dHt, n, torch.as_tensor(coeffs[:1], device=DEV), acc32, precision=cg.F32,
              stepwise=True)
    e64x = relF(acc[0].cpu().numpy(), ex.acc[0].vals)
    e32 = relF(acc32[0].cpu().numpy(), ex.acc[0].vals)
    assert e64x < 1e-3 * e32, (e64x, e32)


def test_f64x_every_tile_shape():
    n, nf = 40, 2
    Ht, P_out, coeffs, G = case(150, 5.0, 3.0, 21, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    assert cg.tile_shapes(cg.F64X) == cg.tile_shapes(cg.F64)
    for tile in range(len(cg.tile_shapes(cg.F64X))):
        acc, t, g = run(cg.Plan(dP, cg.F64X, tile), dHt, n, coeffs, G, P_out.nnzb, True)
        for j in range(nf):
            assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < 1e-10, (tile, j)
        assert relF(g.cpu().numpy(), ex.g) < 1e-10


def test_f64x_foe_and_powers_against_the_oracle():
    s = synth.make_system(64, 4.0, 41)
    N_e = float(s.n_rows // 2)
    kT = 0.05
    pb = solve.problem_from_system(s, 2.0, DEV, cg.F64X)
    out = solve.foe(pb, kT, N_e, tol=1e-9)
    S, H, P_out = pipelines.system_mats(s, 2.0)
    orc = pipelines.foe(S, H, P_out, kT, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e)
    assert out["mu_result"]["bits"] == orc["mu"].bits
    assert abs(out["mu"] - orc["mu"].mu) < 1e-12
    assert relF(out["F"].cpu().numpy(), orc["F"].vals) < 1e-10
    pw = solve.powers(pb, exponents=(-1.0, 0.5, -0.5), tol=1e-10, n_max=512, precision=cg.F64X)
    opw = pipelines.powers(S, P_out, (-1.0, 0.5, -0.5), pw["bounds"], pw["n_terms"])
    for j in range(3):
        assert relF(pw["acc"][j].cpu().numpy(), opw["acc"][j].vals) < 1e-10
