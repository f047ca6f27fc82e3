"""Edge and degenerate cases of the method through the C ABI, against dense
definitions or the oracle: an orthogonal basis (S = I), a single atom, the
smallest expansion (two terms), a degenerate spectrum (H = c S: every
generalised eigenvalue equal), and an output pattern equal to the operator's
(no buffer)."""
import numpy as np
import pytest
import scipy.linalg as sla
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
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fermi(x):
    return 0.5 * (1.0 - np.tanh(0.5 * x))


def dense_F(pb, F):
    P = ref.Bsr(pb.P_out.row_ptr.cpu().numpy(), pb.P_out.col_idx.cpu().numpy(), F.cpu().numpy())
    return P.dense()


def system_with(s, S_vals=None, H_vals=None):
    return synth.System(xyz=s.xyz, L=s.L, r_cut=s.r_cut, row_ptr=s.row_ptr, col_idx=s.col_idx,
                        S=s.S if S_vals is None else S_vals, H=s.H if H_vals is None else H_vals, seed=s.seed)


def test_orthogonal_basis():
    # S = I: S^-1/2 = I (its bounds come from a Lanczos breakdown and the
    # minimum interval width), and F = f(H) on a dense pattern
    s = synth.make_system(12, 30.0, 3)
    I_blocks = np.where((np.repeat(np.arange(s.n_atoms), np.diff(s.row_ptr)) == s.col_idx)[:, None, None],
                        np.eye(4)[None], 0.0)
    so = system_with(s, S_vals=I_blocks)
    pb = solve.problem_from_system(so, 2.0, DEV, cg.F64)
    N_e = float(so.n_rows // 2)
    kT = 0.05
    out = solve.foe(pb, kT, N_e, tol=1e-10)
    A = out["A"].cpu().numpy()
    diag = np.repeat(np.arange(pb.P_out.nbr), np.diff(pb.P_out.row_ptr.cpu().numpy())) == \
        pb.P_out.col_idx.cpu().numpy()
    assert np.max(np.abs(A[diag] - np.eye(4))) < 1e-10 and np.max(np.abs(A[~diag])) < 1e-10
    Hd = synth.to_dense(so.row_ptr, so.col_idx, so.H)
    w, U = np.linalg.eigh(Hd)
    F_ex = (U * fermi((w - out["mu"]) / kT)) @ U.T
    assert relF(dense_F(pb, out["F"]), F_ex) < 1e-8
    assert abs(out["trace_FS"].item() - N_e) < 1e-8 * N_e


@pytest.mark.parametrize("prec,tol", [(cg.F64, 1e-9), (cg.F32, 1e-5), (cg.F64X, 1e-9)])
def test_single_atom(prec, tol):
    # (cutoffs below the box edge: no periodic image inside them)
    s = synth.make_system(1, 1.0, 4)
    assert s.L > 2.0
    pb = solve.problem_from_system(s, 1.0, DEV, prec)
    assert pb.P_out.nbr == 1 and pb.P_out.nnzb == 1
    kT = 0.05
    out = solve.foe(pb, kT, 2.0, tol=1e-9)
    Sd = synth.to_dense(s.row_ptr, s.col_idx, s.S)
    Hd = synth.to_dense(s.row_ptr, s.col_idx, s.H)
    F_ex = ref.dense_function(Hd, lambda e: fermi((e - out["mu"]) / kT), Sd)
    assert relF(dense_F(pb, out["F"]), F_ex) < tol
    assert abs(out["trace_FS"].item() - 2.0) < 10 * tol * 2.0


@pytest.mark.parametrize("prec", [cg.F64, cg.F32, cg.F64X])
@pytest.mark.parametrize("stepwise", [True, False])
def test_two_term_expansion(prec, stepwise):
    # n = 2: acc = c_0/2 I + c_1 M~ on P_out, moments Tr I and Tr M~
    s = synth.make_system(60, 4.0, 5)
    S, H, P_out = pipelines.system_mats(s, 2.0)
    Ht = ref.scale(H, -12.0, 12.0)
    c = np.array([[0.7, -0.3], [1.1, 0.4]])
    ex = ref.chebyshev_expand(Ht, P_out, c)
    dP = cg.Bsr(torch.as_tensor(P_out.row_ptr, device=DEV), torch.as_tensor(P_out.col_idx, device=DEV))
    dHt = cg.Bsr(torch.as_tensor(Ht.row_ptr, device=DEV), torch.as_tensor(Ht.col_idx, device=DEV),
                 torch.as_tensor(Ht.vals, device=DEV))
    plan = cg.Plan(dP, prec).attach_operator(dHt)
    acc = [torch.zeros((P_out.nnzb, 4, 4), dtype=torch.float64, device=DEV) for _ in range(2)]
    t = torch.zeros(2, dtype=torch.float64, device=DEV)
    cg.expand(plan, dHt, 2, torch.as_tensor(c, device=DEV), acc, moments=t, precision=prec, stepwise=stepwise)
    tol = {cg.F64: 1e-15, cg.F64X: 1e-13, cg.F32: 1e-7}[prec]
    for j in range(2):
        assert relF(acc[j].cpu().numpy(), ex.acc[j].vals) < tol
    assert relF(t.cpu().numpy(), ex.t) < tol


def test_degenerate_spectrum_H_proportional_to_S():
    # H = c S: every generalised eigenvalue is c, so mu* = c for half filling
    # and F = f(0) S^-1 = S^-1 / 2
    s = synth.make_system(24, 5.0, 6)
    c = -0.4
    sd = system_with(s, H_vals=c * s.S)
    pb = solve.problem_from_system(sd, 2.0, DEV, cg.F64)
    N_e = float(sd.n_rows // 2)
    out = solve.foe(pb, 0.05, N_e, tol=1e-9)
    assert abs(out["mu"] - c) < 1e-6
    e0, e1 = out["bounds_H"]
    assert e0 < c < e1
    S, H, P_out = pipelines.system_mats(sd, 2.0)
    orc = pipelines.foe(S, H, P_out, 0.05, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e)
    assert relF(out["F"].cpu().numpy(), orc["F"].vals) < 1e-9
    assert abs(out["trace_FS"].item() - N_e) < 1e-6 * N_e


def test_output_pattern_equal_to_operator_pattern():
    # r_buf = 0: P_out = P_H, every product truncated to the operator's own pattern
    s = synth.make_system(80, 5.0, 7)
    pb = solve.problem_from_system(s, 0.0, DEV, cg.F64)
    assert pb.P_out.nnzb == pb.P_H.nnzb
    N_e = float(s.n_rows // 2)
    out = solve.foe(pb, 0.05, N_e, tol=1e-9)
    S, H, P_out = pipelines.system_mats(s, 0.0)
    orc = pipelines.foe(S, H, P_out, 0.05, N_e, out["bounds_S"], out["n_S"], out["bounds_H"], out["n_terms"],
                        tol_N=1e-9 * N_e)
    assert out["mu_result"]["bits"] == orc["mu"].bits
    assert relF(out["F"].cpu().numpy(), orc["F"].vals) < 1e-10


def test_columns_beyond_the_column_kernel_capacity():
    # a dense 700-row block pattern: every column has 700 rows, more than a
    # column-kernel panel holds (about 670), so the column kernel's lists are
    # not built and the per-step products run on the ranking kernel; a tile
    # whose shared memory cannot hold one column is refused with NOSPACE
    nb = 700
    rng = np.random.default_rng(11)
    rp = np.arange(nb + 1, dtype=np.int64) * nb
    ci = np.tile(np.arange(nb, dtype=np.int32), nb)
    B = rng.normal(size=(4 * nb, 4 * nb))
    Md = (B + B.T) / (4.0 * np.sqrt(4 * nb))  # spectrum inside [-1, 1]
    vals = Md.reshape(nb, 4, nb, 4).transpose(0, 2, 1, 3).reshape(nb * nb, 4, 4)
    Mt = ref.Bsr(rp, ci, vals)
    assert np.max(np.abs(np.linalg.eigvalsh(Md))) < 1.0
    n = 8
    c = np.random.default_rng(12).normal(size=(1, n))
    cols = [0, 351, 699]
    want = ref.column_expand(Mt, Mt, cols, c)
    dP = cg.Bsr(torch.as_tensor(rp, device=DEV), torch.as_tensor(ci, device=DEV))
    dM = cg.Bsr(torch.as_tensor(rp, device=DEV), torch.as_tensor(ci, device=DEV), torch.as_tensor(vals, device=DEV))
    for prec, tol in ((cg.F32, 1e-5), (cg.F64, 1e-12)):
        built = 0
        for tile in range(len(cg.tile_shapes(prec))):
            try:
                plan = cg.Plan(dP, prec, tile)
            except cg.ChebError as e:
                assert e.code == 7 and "does not fit" in str(e)  # CHEB_ERR_NOSPACE
                continue
            plan.attach_operator(dM)
            assert cg.plan_col_info(plan)[0] == 0  # no column-kernel lists for these columns
            acc = [torch.zeros((nb * nb, 4, 4), dtype=torch.float64, device=DEV)]
            cg.expand(plan, dM, n, torch.as_tensor(c, device=DEV), acc, precision=prec, stepwise=True)
            got = ref.column_blocks(acc[0].cpu().numpy(), Mt, cols)
            num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, want[0]))
            den = sum(np.linalg.norm(b) ** 2 for b in want[0])
            assert np.sqrt(num / den) < tol, (prec, tile)
            built += 1
        # a 1-column FP32 tile holds these columns; FP64 tiles may all refuse
        assert built >= 1 or prec == cg.F64, prec
