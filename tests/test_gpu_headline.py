"""The headline configuration's accuracy against the FP64 oracle, column-sampled.

By Eq. 3's column independence (Sec. "Expansion in Chebyshev polynomials") the
oracle advances only the sampled block columns, which is exact, so the GPU
expansion is checked element by element on those columns at full size:
  * FP32 block products (the column-order kernel) on the 10,000-atom bench
    system (r_c 10, r_buf 4 bohr) with a 9,216-term Fermi expansion (the
    bench's kT = 0.005 Ha scaled to this operator's spectral width): relative
    Frobenius error of the accumulator over 64 sampled columns below 1e-6;
    the BF16 mode's error on the same columns (reported; bounded by the FP32
    error times the ratio of unit roundoffs);
  * FP64 products at the same term count on a 1,000-atom system (32 sampled
    columns): below 1e-10;
  * unions near the shared-memory cap (3,000 atoms, 14 bohr output cutoff),
    FP64 and FP32, 96 terms.
Operator and coefficients come from the generator and the oracle only.
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

BENCH_KT, BENCH_WIDTH = 0.005, 17.0  # Ha; spectral width of the bench's H'


def relF_cols(got_full, want_cols, P_out, cols):
    got = ref.column_blocks(got_full, P_out, cols)
    num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, want_cols))
    den = sum(np.linalg.norm(b) ** 2 for b in want_cols)
    return float(np.sqrt(num / den))


def case(n_atoms, r_c, r_buf, seed):
    s = synth.make_system(n_atoms, r_c, seed)
    S, H, P_out = pipelines.system_mats(s, r_buf)
    alpha, beta = ref.lanczos(H, pipelines.lanczos_start(4 * H.nbr), 40)
    lo, hi, _, _ = ref.ritz_bounds(alpha, beta, 0.01)
    return s, H, P_out, lo, hi


def gpu_expand(H, P_out, lo, hi, coeffs, prec):
    dP = cg.Bsr(torch.as_tensor(P_out.row_ptr, device=DEV), torch.as_tensor(P_out.col_idx, device=DEV))
    Ht = ref.scale(H, lo, hi)
    dHt = cg.Bsr(torch.as_tensor(Ht.row_ptr, device=DEV), torch.as_tensor(Ht.col_idx, device=DEV),
                 torch.as_tensor(Ht.vals, device=DEV))
    plan = cg.Plan(dP, prec).attach_operator(dHt)
    if prec != cg.F64:
        assert cg.plan_col_info(plan)[0] > 0
    acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(len(coeffs))]
    cg.expand(plan, dHt, coeffs.shape[1], torch.as_tensor(coeffs, device=DEV), acc, precision=prec, stepwise=True)
    return Ht, [a.cpu().numpy() for a in acc]


def fermi_coeffs(lo, hi, n):
    kT = BENCH_KT * (hi - lo) / BENCH_WIDTH
    f = ref.Func(ref.KIND_FERMI, mu=0.5 * (lo + hi) + 0.05 * (hi - lo), kT=kT)
    return ref.cheb_coeffs(f, n, lo, hi)[None]


def sampled(P_out, n, seed):
    return sorted(np.random.default_rng(seed).choice(P_out.nbr, n, replace=False).tolist())


def test_fp32_expansion_at_the_bench_configuration():
    s, H, P_out, lo, hi = case(10000, 10.0, 4.0, 0)
    c = fermi_coeffs(lo, hi, 9216)
    Ht, acc = gpu_expand(H, P_out, lo, hi, c, cg.F32)
    cols = sampled(P_out, 64, 1)
    want = ref.column_expand(Ht, P_out, cols, c)
    err = relF_cols(acc[0], want[0], P_out, cols)
    print(f"FP32, 9216 terms, 40,000 rows: relative Frobenius error over 64 sampled columns {err:.3e}")
    assert err < 1e-6
    # BF16 mode on the same operator and columns: every stored T_k rounded to
    # bfloat16 (unit roundoff 2^-8 instead of 2^-24).  Its error is reported;
    # the bar is the FP32 error scaled by the ratio of unit roundoffs (x 4).
    _, acc16 = gpu_expand(H, P_out, lo, hi, c, cg.BF16)
    err16 = relF_cols(acc16[0], want[0], P_out, cols)
    print(f"BF16, 9216 terms, 40,000 rows: relative Frobenius error over 64 sampled columns {err16:.3e}")
    assert err < err16 < 4 * 2.0 ** 16 * err


def test_fp64_expansion_at_the_bench_term_count():
    s, H, P_out, lo, hi = case(1000, 10.0, 4.0, 2)
    c = fermi_coeffs(lo, hi, 9216)
    Ht, acc = gpu_expand(H, P_out, lo, hi, c, cg.F64)
    cols = sampled(P_out, 32, 3)
    want = ref.column_expand(Ht, P_out, cols, c)
    err = relF_cols(acc[0], want[0], P_out, cols)
    print(f"FP64, 9216 terms, 4,000 rows: relative Frobenius error over 32 sampled columns {err:.3e}")
    assert err < 1e-10


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_expansion_with_unions_near_the_shared_memory_cap(prec, tol):
    s, H, P_out, lo, hi = case(3000, 10.0, 4.0, 4)
    rng = np.random.default_rng(5)
    n = 96
    c = rng.normal(size=(2, n)) / (1.0 + np.arange(n)) ** 1.5
    Ht, acc = gpu_expand(H, P_out, lo, hi, c, prec)
    cols = sampled(P_out, 64, 6)
    want = ref.column_expand(Ht, P_out, cols, c)
    for j in range(2):
        err = relF_cols(acc[j], want[j], P_out, cols)
        assert err < tol, (j, err)
