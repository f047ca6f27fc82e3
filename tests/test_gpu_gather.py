"""The gather plan of the column-order step kernel built by the device kernels
(the default) against the host builder: the same panels, warp streams, row
words, entry words and slots, bit for bit, on patterns from one panel to unions
near the shared-memory cap; and the expansion through the device-built plan
against the oracle."""
import time

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


def dbsr(row_ptr, col_idx, vals=None):
    return cg.Bsr(torch.as_tensor(row_ptr, dtype=torch.int64, device=DEV),
                  torch.as_tensor(col_idx, dtype=torch.int32, device=DEV),
                  None if vals is None else torch.as_tensor(np.ascontiguousarray(vals), dtype=torch.float64,
                                                           device=DEV))


def sparse_operator(H, keep_mod=3):
    keep = [[k for k in range(H.row_ptr[i], H.row_ptr[i + 1]) if (i + H.col_idx[k]) % keep_mod == 0
             or H.col_idx[k] == i] for i in range(H.nbr)]
    rp = np.zeros(H.nbr + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in keep])
    ks = np.array([k for r in keep for k in r], dtype=np.int64)
    return ref.Bsr(rp, H.col_idx[ks], H.vals[ks])


@pytest.mark.parametrize("n_atoms,r_c,r_buf,seed,sparse", [
    (33, 3.0, 1.5, 1, False),     # one or two panels
    (300, 6.0, 3.0, 2, False),    # several panels, a ragged last one
    (300, 6.0, 3.0, 5, True),     # union rows without operator entries in the union
    (1000, 8.0, 4.0, 3, False),
    (3000, 10.0, 4.0, 4, False),  # the bench's cutoffs: unions near the 1023-row cap
])
def test_device_gather_plan_bit_identical_to_host(n_atoms, r_c, r_buf, seed, sparse):
    s = synth.make_system(n_atoms, r_c, seed)
    S, H, P_out = pipelines.system_mats(s, r_buf)
    L = sparse_operator(H) if sparse else H
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dL = dbsr(L.row_ptr, L.col_idx, L.vals)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dev = cg.Plan(dP, cg.F32).attach_operator(dL)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    host = cg.Plan(dP, cg.F32).attach_operator(dL, gather="host")
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    print(f"\n{n_atoms} atoms: plan + operator lists {t1 - t0:.3f} s (device gather plan), "
          f"{t2 - t1:.3f} s (host builder)")
    assert cg.plan_col_info(dev) == cg.plan_col_info(host)
    assert cg.plan_col_info(dev)[0] >= 1
    for which, (a, b) in enumerate(zip(cg.plan_col_lists(dev), cg.plan_col_lists(host))):
        assert a.numel() == b.numel() and torch.equal(a, b), which


def test_expansion_through_the_device_gather_plan():
    n, nf = 30, 2
    s = synth.make_system(300, 6.0, 9)
    S, H, P_out = pipelines.system_mats(s, 3.0)
    Ht = ref.scale(H, -12.0, 12.0)
    rng = np.random.default_rng(9)
    coeffs = rng.normal(size=(nf, n)) / (1.0 + np.arange(n)) ** 1.5
    ex = ref.chebyshev_expand(Ht, P_out, coeffs)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dHt = dbsr(Ht.row_ptr, Ht.col_idx, Ht.vals)
    plan = cg.Plan(dP, cg.F32).attach_operator(dHt)
    acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(nf)]
    cg.expand(plan, dHt, n, torch.as_tensor(coeffs, device=DEV), acc, precision=cg.F32, stepwise=True)
    for j in range(nf):
        a, b = acc[j].cpu().numpy(), ex.acc[j].vals
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5


def _plan(dP, prec, dL, builder, sys_starts=None):
    cg.set_plan_builder(builder)
    try:
        if sys_starts is None:
            plan = cg.Plan(dP, prec)
        else:
            plan = cg.BatchedPlan(dP, sys_starts, precision=prec)
        return plan.attach_operator(dL)
    finally:
        cg.set_plan_builder("device")


@pytest.mark.parametrize("prec", [cg.F64, cg.F32, cg.F64X])
@pytest.mark.parametrize("n_atoms,r_c,r_buf,seed", [(33, 3.0, 1.5, 1), (300, 6.0, 3.0, 2), (1000, 8.0, 4.0, 3)])
def test_device_plan_bit_identical_to_host(prec, n_atoms, r_c, r_buf, seed):
    # cheb_plan_create + attach with no host copy of the patterns: checks,
    # transposition map, step and resident panels, both row-list sets and the
    # column kernel's lists, against the host builders
    s = synth.make_system(n_atoms, r_c, seed)
    S, H, P_out = pipelines.system_mats(s, r_buf)
    dP = dbsr(P_out.row_ptr, P_out.col_idx)
    dL = dbsr(H.row_ptr, H.col_idx, H.vals)
    dev = _plan(dP, prec, dL, "device")
    host = _plan(dP, prec, dL, "host")
    assert dev.info() == host.info() and cg.plan_resident_info(dev) == cg.plan_resident_info(host)
    which = list(range(6, 17)) + (list(range(6)) if prec == cg.F32 else [])
    for w, a, b in zip(which, cg.plan_lists(dev, which), cg.plan_lists(host, which)):
        assert a.numel() == b.numel() and torch.equal(a, b), w


def test_device_batched_plan_bit_identical_to_host():
    systems = [synth.make_system(n, 4.0, 20 + i) for i, n in enumerate((40, 90, 25, 60))]
    Ps = [pipelines.system_mats(x, 2.0) for x in systems]
    bd = cg.block_diag([dbsr(P.row_ptr, P.col_idx, np.zeros((P.nnzb, 4, 4))) for _, _, P in Ps])
    Hd = cg.block_diag([dbsr(H.row_ptr, H.col_idx, H.vals) for _, H, _ in Ps])
    starts = np.concatenate([[0], np.cumsum([x.n_atoms for x in systems])]).tolist()
    dP = cg.Bsr(bd.row_ptr, bd.col_idx)
    dev = _plan(dP, cg.F64, Hd, "device", starts)
    host = _plan(dP, cg.F64, Hd, "host", starts)
    which = list(range(6, 17))
    for w, a, b in zip(which, cg.plan_lists(dev, which), cg.plan_lists(host, which)):
        assert a.numel() == b.numel() and torch.equal(a, b), w
