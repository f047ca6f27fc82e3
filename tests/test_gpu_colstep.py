"""GPU parity of the column-order FP32/BF16 step kernel (cheb_expand_stepwise on
a reduced-precision plan with the operator's lists attached) against the FP64
oracle, and against the ranking step kernel on the same plan without lists.

Bars: the FP32 recursion within the perturbation bound u * sum_k |c_k| (k+1)^2
(u = 2^-24, the growth of a rounding at step j through U_{k-j}) and a relative
Frobenius error below 1e-5 on these short expansions; BF16 within the same
bound at u = 2^-8; runs bitwise repeatable.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import pipelines, ref

pytestmark = pytest.mark.gpu

cg = pytest.importorskip("paper_1704_00512_gb300")

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
    Ht = ref.scale(H, -12.0, 12.0)
    rng = np.random.default_rng(seed)
    coeffs = rng.normal(size=(max(nf, 1), n)) / (1.0 + np.arange(n)) ** 1.5
    G = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
    return Ht, P_out, coeffs, G


def run(plan, dHt, n, coeffs, nf, G, nnzb, prec):
    acc = [torch.zeros((nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    t = torch.zeros(n, dtype=torch.float64, device=DEV)
    g = torch.zeros(n, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, n, torch.as_tensor(coeffs[:max(nf, 1)], device=DEV) if nf else None, acc, moments=t,
              G=torch.as_tensor(G.vals, device=DEV), gmoments=g, precision=prec, stepwise=True)
    return acc, t, g


@pytest.mark.parametrize("n_atoms,r_c,r_buf,n,nf", [
    (33, 3.0, 1.5, 40, 1),     # one or two panels
    (300, 6.0, 3.0, 48, 3),    # several panels, a ragged last panel
    (1000, 8.0, 4.0, 24, 8),   # many panels, accumulators beyond the prefetched ones
    (400, 6.0, 3.0, 30, 0),    # moments only
    (250, 5.0, 2.0, 30, 2),
])
def test_col_kernel_fp32_parity(n_atoms, r_c, r_buf, n, nf):
    Ht, P_out, coeffs, G = case(n_atoms, r_c, r_buf, 100 + n_atoms, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs[:max(nf, 1)], G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    plan = cg.Plan(dP, cg.F32).attach_operator(dHt)
    npan, mu, nent = cg.plan_col_info(plan)
    assert npan >= 1 and mu >= 1 and nent >= P_out.nbr
    acc, t, g = run(plan, dHt, n, coeffs, nf, G, P_out.nnzb, cg.F32)
    u = 2.0 ** -24
    k = np.arange(n)
    for j in range(nf):
        bound = 8 * u * np.sum(np.abs(coeffs[j]) * (1 + k) ** 2) * np.sqrt(P_out.nnzb * 16)
        err = np.linalg.norm(acc[j].cpu().numpy() - ex.acc[j].vals)
        assert err < bound, (err, bound)
        assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < 1e-5
    assert relF(t.cpu().numpy(), ex.t) < 1e-5
    assert relF(g.cpu().numpy(), ex.g) < 1e-5
    # the ranking kernel (same plan without lists) agrees to FP32 rounding
    acc_r, t_r, g_r = run(cg.Plan(dP, cg.F32), dHt, n, coeffs, nf, G, P_out.nnzb, cg.F32)
    for j in range(nf):
        assert relF(acc[j].cpu().numpy(), acc_r[j].cpu().numpy()) < 1e-5
    assert relF(g.cpu().numpy(), g_r.cpu().numpy()) < 1e-5
    # bitwise repeatable
    acc2, t2, g2 = run(plan, dHt, n, coeffs, nf, G, P_out.nnzb, cg.F32)
    for j in range(nf):
        assert torch.equal(acc[j], acc2[j])
    assert torch.equal(t, t2) and torch.equal(g, g2)


def test_col_kernel_bf16_within_bound():
    n, nf = 48, 2
    Ht, P_out, coeffs, G = case(200, 5.0, 2.5, 7, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    plan = cg.Plan(dP, cg.BF16).attach_operator(dHt)
    assert cg.plan_col_info(plan)[0] >= 1
    acc, t, g = run(plan, dHt, n, coeffs, nf, G, P_out.nnzb, cg.BF16)
    u = 2.0 ** -8
    k = np.arange(n)
    for j in range(nf):
        bound = 8 * u * np.sum(np.abs(coeffs[j]) * (1 + k) ** 2) * np.sqrt(P_out.nnzb * 16)
        err = np.linalg.norm(acc[j].cpu().numpy() - ex.acc[j].vals)
        assert err < bound, (err, bound)
    # the same bfloat16 roundings as the ranking kernel up to FP32 summation order
    acc_r, _, _ = run(cg.Plan(dP, cg.BF16), dHt, n, coeffs, nf, G, P_out.nnzb, cg.BF16)
    assert relF(acc[0].cpu().numpy(), acc_r[0].cpu().numpy()) < 5e-2


def test_col_kernel_sparse_operator_rows():
    # an operator on P_H with only the blocks (I, K), (I + K) % 3 == 0: some
    # union rows have no operator block in a panel's union (empty rows still
    # produce T_{k+1} = -T_{k-1} on their blocks)
    n, nf = 20, 1
    s = synth.make_system(300, 6.0, 5)
    S, H, P_out = pipelines.system_mats(s, 3.0)
    keep = [[k for k in range(H.row_ptr[i], H.row_ptr[i + 1]) if (i + H.col_idx[k]) % 3 == 0 or H.col_idx[k] == i]
            for i in range(H.nbr)]
    rp = np.zeros(H.nbr + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in keep])
    ks = np.array([k for r in keep for k in r], dtype=np.int64)
    rng = np.random.default_rng(9)
    Ls = ref.Bsr(rp, H.col_idx[ks], 0.05 * rng.normal(size=(len(ks), 4, 4)))
    coeffs = rng.normal(size=(nf, n))
    G = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
    ex = ref.chebyshev_expand(Ls, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dL = dbsr(Ls.row_ptr, Ls.col_idx, Ls.vals)
    plan = cg.Plan(dP, cg.F32).attach_operator(dL)
    assert cg.plan_col_info(plan)[0] >= 1
    acc, t, g = run(plan, dL, n, coeffs, nf, G, P_out.nnzb, cg.F32)
    assert relF(acc[0].cpu().numpy(), ex.acc[0].vals) < 1e-5
    assert relF(g.cpu().numpy(), ex.g) < 1e-5


def test_resident_expansion_bf16_within_bound():
    # cheb_expand (one launch, panels resident in shared memory) on a CHEB_BF16
    # plan: Mt and every stored T_k rounded to bfloat16, products summed in FP32
    n, nf = 48, 2
    Ht, P_out, coeffs, G = case(200, 5.0, 2.5, 7, n, nf)
    ex = ref.chebyshev_expand(Ht, P_out, coeffs, G=G)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    plan = cg.Plan(dP, cg.BF16)
    acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    t = torch.zeros(n, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, moments=t, precision=cg.BF16, stepwise=False)
    u = 2.0 ** -8
    k = np.arange(n)
    for j in range(nf):
        bound = 8 * u * np.sum(np.abs(coeffs[j]) * (1 + k) ** 2) * np.sqrt(P_out.nnzb * 16)
        err = np.linalg.norm(acc[j].cpu().numpy() - ex.acc[j].vals)
        assert err < bound, (err, bound)
    # rounding really happens: farther from the oracle than the FP32 resident run
    acc32 = [torch.zeros_like(acc[0])]
    cg.expand(cg.Plan(dP, cg.F32), dHt, n, torch.as_tensor(coeffs[:1], device=DEV), acc32, precision=cg.F32,
              stepwise=False)
    e16 = relF(acc[0].cpu().numpy(), ex.acc[0].vals)
    e32 = relF(acc32[0].cpu().numpy(), ex.acc[0].vals)
    assert e32 < 1e-5 and e16 > 10 * e32
    # and the same roundings as the stepwise BF16 form up to FP32 summation order
    acc_s, _, _ = run(plan, dHt, n, coeffs, nf, G, P_out.nnzb, cg.BF16)
    assert relF(acc[0].cpu().numpy(), acc_s[0].cpu().numpy()) < 5e-2
