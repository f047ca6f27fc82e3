"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a
hand-derived golden fixture, a closed form, a library routine computing the
same quantity a different way, dense linear algebra, or brute force on tiny
inputs.  No GPU is needed.
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.fft import dct
from scipy.optimize import brentq
from scipy.spatial import cKDTree
from scipy.special import iv

import synth
from oracle import pipelines, ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers (test-only): small symmetric block matrices
# --------------------------------------------------------------------------

def _bsr_from_dense(A, row_ptr, col_idx):
    nbr = len(row_ptr) - 1
    rows = np.repeat(np.arange(nbr), np.diff(row_ptr))
    vals = np.stack([A[4 * I:4 * I + 4, 4 * J:4 * J + 4] for I, J in zip(rows, col_idx)])
    return ref.Bsr(row_ptr, col_idx, vals)


def _small_system(n_atoms=24, r_c=4.0, r_out=6.5, seed=3):
    s = synth.make_system(n_atoms, r_c, seed)
    P_H = ref.Bsr(s.row_ptr, s.col_idx, None)
    rp, ci = ref.pattern(s.xyz, s.L, r_out)
    P_out = ref.Bsr(rp, ci, None)
    return s, ref.Bsr(s.row_ptr, s.col_idx, s.S), ref.Bsr(s.row_ptr, s.col_idx, s.H), P_H, P_out


def _dense_pattern(n_atoms):
    rp = np.arange(0, n_atoms * n_atoms + 1, n_atoms, dtype=np.int64)
    ci = np.tile(np.arange(n_atoms, dtype=np.int32), n_atoms)
    return ref.Bsr(rp, ci, None)


# --------------------------------------------------------------------------
# A1 patterns
# --------------------------------------------------------------------------

def test_pattern_golden_line():
    lines = open(os.path.join(GOLDEN, "pattern_line.txt")).read().splitlines()
    kv = {}
    rows = {}
    for ln in lines:
        if not ln.strip() or ln.startswith("#"):
            continue
        if ln.startswith("row"):
            h, v = ln.split(":")
            rows[int(h.split()[1])] = [int(x) for x in v.split()]
        else:
            k, *v = ln.split()
            kv[k] = [float(x) for x in v]
    xs = np.array(kv["atoms"])
    xyz = np.stack([xs, np.ones_like(xs), np.ones_like(xs)], axis=1)
    rp, ci = ref.pattern(xyz, kv["L"][0], kv["r"][0])
    for I, cols in rows.items():
        assert list(ci[rp[I]:rp[I + 1]]) == cols
    rp2, ci2 = ref.pattern_python(xyz, kv["L"][0], kv["r"][0])
    assert (rp2 == rp).all() and (ci2 == ci).all()


@pytest.mark.parametrize("n_atoms,r", [(60, 5.0), (200, 8.0), (200, 12.0)])
def test_pattern_matches_periodic_kdtree(n_atoms, r):
    xyz, L = synth.place_atoms(n_atoms, seed=1)
    rp, ci = ref.pattern(xyz, L, r)
    tree = cKDTree(np.mod(xyz, L), boxsize=L)
    pairs = tree.query_pairs(r, output_type="ndarray")
    want = set(map(tuple, pairs.tolist())) | {(j, i) for i, j in pairs.tolist()} | {(i, i) for i in range(n_atoms)}
    rows = np.repeat(np.arange(n_atoms), np.diff(rp))
    got = set(zip(rows.tolist(), ci.tolist()))
    assert got == want
    for I in range(n_atoms):  # sorted, symmetric
        row = ci[rp[I]:rp[I + 1]]
        assert (np.diff(row) > 0).all()


def test_pattern_equals_generator_pattern():
    s = synth.make_system(150, 7.0, seed=5)
    rp, ci = ref.pattern(s.xyz, s.L, 7.0)
    assert (rp == s.row_ptr).all() and (ci == s.col_idx).all()


def test_generator_properties():
    s = synth.make_system(120, 8.0, seed=2)
    L = s.L
    assert abs(L - 18.0 * (120 / 200) ** (1 / 3)) < 1e-12
    d = synth.min_image(s.xyz[:, None, :] - s.xyz[None, :, :], L)
    r = np.sqrt((d * d).sum(-1)) + np.eye(len(s.xyz)) * 1e9
    assert r.min() >= 2.0
    S = synth.to_dense(s.row_ptr, s.col_idx, s.S)
    H = synth.to_dense(s.row_ptr, s.col_idx, s.H)
    assert np.allclose(S, S.T, atol=0) and np.allclose(H, H.T, atol=0)
    assert np.linalg.eigvalsh(S)[0] > 0
    assert np.allclose(np.diag(S), 1.0)
    # diagonal of H uniform in [-1.2, 0.3]
    assert np.diag(H).min() >= -1.2 and np.diag(H).max() <= 0.3


# --------------------------------------------------------------------------
# Eq. 4 coefficients, Eq. 1 evaluation, Eq. 6 degree
# --------------------------------------------------------------------------

class _Scaled:
    """A function of the scaled variable wrapped as an unscaled ref.Func-like callable."""

    def __init__(self, g, emin, emax):
        self.g, self.s, self.t = g, *ref.sigma_tau(emin, emax)

    def __call__(self, x, emin=None, emax=None):
        return self.g(self.s * (np.asarray(x) - self.t))


def test_coeffs_of_chebyshev_polynomial_are_kronecker():
    emin, emax = -3.0, 5.0
    for m in (0, 1, 5, 17):
        f = _Scaled(lambda x, m=m: np.cos(m * np.arccos(np.clip(x, -1, 1))), emin, emax)
        c = ref.cheb_coeffs(f, 32, emin, emax)
        want = np.zeros(32)
        want[m] = 2.0 if m == 0 else 1.0
        assert np.max(np.abs(c - want)) < 1e-13


def test_coeffs_of_exponential_are_bessel():
    a = 1.7
    f = _Scaled(lambda x: np.exp(a * x), -1.0, 1.0)
    c = ref.cheb_coeffs(f, 40, -1.0, 1.0)
    want = 2.0 * iv(np.arange(40), a)
    assert np.max(np.abs(c - want)) < 1e-14


def test_coeffs_of_resolvent_are_geometric():
    z = 1.3
    rho = z + np.sqrt(z * z - 1)
    f = _Scaled(lambda x: 1.0 / (z - x), -1.0, 1.0)
    n = 200
    c = ref.cheb_coeffs(f, n, -1.0, 1.0)
    want = 2.0 / np.sqrt(z * z - 1) * rho ** (-np.arange(n, dtype=float))
    assert np.max(np.abs(c - want)) < 1e-13


def test_coeffs_match_library_dct2():
    f = ref.Func(ref.KIND_FERMI, mu=0.3, kT=0.2)
    emin, emax = -2.0, 3.0
    n = 97
    s, t = ref.sigma_tau(emin, emax)
    xk = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    want = dct(f(xk / s + t), type=2) / n
    assert np.max(np.abs(ref.cheb_coeffs(f, n, emin, emax) - want)) < 1e-14


def test_cheb_eval_closed_form():
    x = np.linspace(-1, 1, 101)
    for j in (0, 1, 2, 7, 40):
        c = np.zeros(j + 1)
        c[j] = 2.0 if j == 0 else 1.0
        assert np.max(np.abs(ref.cheb_eval(c, x) - np.cos(j * np.arccos(x)))) < 1e-12


def test_degree_rule_against_geometric_tail():
    # For 1/(z - x) the truncation error of the first n terms is the tail
    # sum_{j>=n} c_j T_j, bounded by c_n / (1 - 1/rho), attained at x = 1.
    z = 1.2
    rho = z + np.sqrt(z * z - 1)
    f = _Scaled(lambda x: 1.0 / (z - x), -1.0, 1.0)
    tol = 1e-9
    n = ref.choose_degree(f, -1.0, 1.0, tol, 4096)
    tail = lambda n: 2.0 / np.sqrt(z * z - 1) * rho ** (-n) / (1 - 1 / rho)
    lad = ref.degree_ladder(4096)
    assert tail(n) < tol * 1.001
    prev = lad[lad.index(n) - 1]
    assert tail(prev) > tol * 0.999


def test_degree_ladder():
    lad = ref.degree_ladder(300)
    assert lad[:10] == [16, 18, 20, 22, 24, 26, 28, 30, 32, 36]
    assert lad[-1] == 288 and all(b > a for a, b in zip(lad, lad[1:]))


# --------------------------------------------------------------------------
# Eq. 3 recursion: closed forms, dense case, brute force
# --------------------------------------------------------------------------

def test_recursion_diagonal_matrix_closed_form():
    nb = 6
    rp = np.arange(nb + 1, dtype=np.int64)
    ci = np.arange(nb, dtype=np.int32)
    rng = np.random.default_rng(0)
    h = rng.uniform(-0.95, 0.95, size=(nb, 4))
    vals = np.zeros((nb, 4, 4))
    for b in range(nb):
        vals[b] = np.diag(h[b])
    M = ref.Bsr(rp, ci, vals)
    n = 50
    coeffs = rng.normal(size=(2, n))
    ex = ref.chebyshev_expand(M, M, coeffs)
    th = np.arccos(h.reshape(-1))
    Tk = np.cos(np.outer(np.arange(n), th))  # [n, rows]
    for j in range(2):
        want = 0.5 * coeffs[j, 0] + coeffs[j, 1:] @ Tk[1:]
        got = np.concatenate([np.diag(ex.acc[j].vals[b]) for b in range(nb)])
        assert np.max(np.abs(got - want)) < 1e-13
    assert np.max(np.abs(ex.t - Tk.sum(axis=1))) < 1e-12


def test_recursion_dense_pattern_is_polynomial_of_matrix():
    s = synth.make_system(10, 20.0, seed=4)  # 10 atoms, all pairs within cutoff
    P = _dense_pattern(10)
    assert len(s.col_idx) == 100
    S = ref.Bsr(s.row_ptr, s.col_idx, s.S)
    Sd = S.dense()
    w = np.linalg.eigvalsh(Sd)
    emin, emax = 0.9 * w[0], 1.1 * w[-1]
    St = ref.scale(S, emin, emax)
    f = ref.Func(ref.KIND_POWER, a=-1.0)
    n = ref.choose_degree(f, emin, emax, 1e-10, 2048, rel=True)
    assert n > 0
    c = ref.cheb_coeffs(f, n, emin, emax)
    ex = ref.chebyshev_expand(St, P, c[None])
    got = ex.acc[0].dense()
    wd, U = np.linalg.eigh(Sd)
    s_, t_ = ref.sigma_tau(emin, emax)
    poly = (U * ref.cheb_eval(c, s_ * (wd - t_))) @ U.T
    assert ref.rel_frobenius(got, poly) < 1e-12
    inv = np.linalg.inv(Sd)
    # relative fit tolerance 1e-10 of max|f| bounds the matrix error
    assert np.max(np.abs(got - inv)) < 1e-10 * (1.0 / emin) * 1.01
    # moments are sums of T_k over the eigenvalues
    for k in (0, 1, 2, 9):
        Tk = np.cos(k * np.arccos(s_ * (wd - t_)))
        assert abs(ex.t[k] - Tk.sum()) < 1e-10 * max(1.0, abs(Tk.sum()))


def test_recursion_masked_matches_dense_brute_force():
    s, S, H, P_H, P_out = _small_system(n_atoms=40, r_c=3.0, r_out=4.5, seed=7)
    Hd = H.dense()
    nat = P_out.nbr
    mask_blk = np.zeros((nat, nat), bool)
    rows = np.repeat(np.arange(nat), np.diff(P_out.row_ptr))
    mask_blk[rows, P_out.col_idx] = True
    mask = np.kron(mask_blk, np.ones((4, 4), bool))
    assert 0.1 < mask_blk.mean() < 0.95
    w = sla.eigvalsh(Hd)
    emin, emax = w[0] - 0.1, w[-1] + 0.1
    Ht = ref.scale(H, emin, emax)
    Htd = Ht.dense()
    n = 40
    rng = np.random.default_rng(1)
    c = rng.normal(size=(3, n)) / (1 + np.arange(n))
    G = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
    ex = ref.chebyshev_expand(Ht, P_out, c, G=G)
    # brute force: dense matrices, elementwise mask after each product
    T0 = np.eye(4 * nat) * mask
    T1 = Htd * mask
    Ts = [T0, T1]
    for k in range(1, n - 1):
        Ts.append(2.0 * (Htd @ Ts[-1]) * mask - Ts[-2])
    Gd = G.dense()
    for j in range(3):
        want = 0.5 * c[j, 0] * Ts[0] + sum(c[j, k] * Ts[k] for k in range(1, n))
        assert np.max(np.abs(ex.acc[j].dense() - want)) < 1e-11
    for k in range(n):
        assert abs(ex.t[k] - np.trace(Ts[k])) < 1e-10
        assert abs(ex.g[k] - np.sum(Ts[k] * Gd)) < 1e-10


def test_recursion_column_subset_equals_full():
    s, S, H, P_H, P_out = _small_system(n_atoms=20, r_c=4.0, r_out=6.0, seed=8)
    w = sla.eigvalsh(H.dense())
    Ht = ref.scale(H, w[0] - 0.1, w[-1] + 0.1)
    n = 30
    c = np.random.default_rng(2).normal(size=(1, n))
    full = ref.chebyshev_expand(Ht, P_out, c)
    cols = np.zeros(20, bool)
    cols[[0, 7, 19]] = True
    part = ref.chebyshev_expand(Ht, P_out, c, colmask=cols)
    sel = cols[P_out.col_idx]
    assert np.array_equal(part.acc[0].vals[sel], full.acc[0].vals[sel])
    assert np.all(part.acc[0].vals[~sel] == 0)


# --------------------------------------------------------------------------
# Lanczos bounds, penalty check
# --------------------------------------------------------------------------

def test_lanczos_bounds_contain_spectrum():
    s, S, H, P_H, P_out = _small_system(n_atoms=40, r_c=5.0, r_out=7.0, seed=9)
    v0 = np.random.default_rng(12345).uniform(-1, 1, size=4 * 40)
    for A in (S, H):
        w = np.linalg.eigvalsh(A.dense())
        a, b = ref.lanczos(A, v0, 40)
        lo, hi, thlo, thhi = ref.ritz_bounds(a, b)
        assert lo <= w[0] and hi >= w[-1]
        width = w[-1] - w[0]
        assert w[0] - lo <= 0.05 * width and hi - w[-1] <= 0.05 * width
        assert thlo >= w[0] - 1e-9 and thhi <= w[-1] + 1e-9


def test_lanczos_full_steps_on_diagonal_gives_exact_extremes():
    nb = 5
    d = np.linspace(-2.0, 3.0, 20)
    vals = np.zeros((nb, 4, 4))
    for b in range(nb):
        vals[b] = np.diag(d[4 * b:4 * b + 4])
    A = ref.Bsr(np.arange(nb + 1, dtype=np.int64), np.arange(nb, dtype=np.int32), vals)
    a, b = ref.lanczos(A, np.ones(20), 20)
    lo, hi, thlo, thhi = ref.ritz_bounds(a, b)
    assert abs(thlo - d[0]) < 1e-10 and abs(thhi - d[-1]) < 1e-10


def test_penalty_fires_only_on_bad_bounds():
    s, S, H, P_H, P_out = _small_system(n_atoms=20, r_c=4.0, r_out=6.0, seed=10)
    w = np.linalg.eigvalsh(S.dense())
    n = 200
    wd = w[-1] - w[0]
    for (emin, emax, fires) in [(w[0] - 0.05 * wd, w[-1] + 0.05 * wd, False),
                                (w[0] + 0.3 * wd, w[-1] + 0.05 * wd, True),
                                (w[0] - 0.05 * wd, w[-1] - 0.3 * wd, True)]:
        St = ref.scale(S, emin, emax)
        ex = ref.chebyshev_expand(St, P_out, np.zeros((1, n)))
        tr = ref.penalty_trace(ex.t, -100.0, emin, emax)
        assert (abs(tr) >= 1.0) == fires, (emin, emax, tr)


# --------------------------------------------------------------------------
# FOE on a dense pattern: electron count, mu, idempotency, eigenvalue counts
# --------------------------------------------------------------------------

def _dense_foe_case(kT=0.05, n_atoms=12, seed=11):
    s = synth.make_system(n_atoms, 30.0, seed=seed)
    P = _dense_pattern(n_atoms)
    S = ref.Bsr(s.row_ptr, s.col_idx, s.S)
    H = ref.Bsr(s.row_ptr, s.col_idx, s.H)
    return s, S, H, P


def test_foe_dense_matches_generalised_eigh():
    s, S, H, P = _dense_foe_case()
    Sd, Hd = S.dense(), H.dense()
    ws = np.linalg.eigvalsh(Sd)
    # S^-1/2 by the method itself (matrix power expansion), checked against eigh
    se0, se1 = 0.95 * ws[0], 1.05 * ws[-1]
    fpow = ref.Func(ref.KIND_POWER, a=-0.5)
    n_s = ref.choose_degree(fpow, se0, se1, 1e-13, 4096, rel=True)
    A = ref.chebyshev_expand(ref.scale(S, se0, se1), P, ref.cheb_coeffs(fpow, n_s, se0, se1)[None]).acc[0]
    wd, U = np.linalg.eigh(Sd)
    Aex = (U * wd ** -0.5) @ U.T
    assert ref.rel_frobenius(A.dense(), Aex) < 1e-11
    Hp = ref.orthogonalise(H, A, P)
    assert ref.rel_frobenius(Hp.dense(), Aex @ Hd @ Aex) < 1e-11
    eps = sla.eigh(Hd, Sd, eigvals_only=True)
    e0, e1 = eps[0] - 0.1, eps[-1] + 0.1
    kT = 0.05
    N_e = float(len(eps) // 2)
    f_mid = ref.Func(ref.KIND_FERMI, mu=0.5 * (e0 + e1), kT=kT)
    n = ref.choose_degree(f_mid, e0, e1, 1e-10, 8192)
    assert n > 0
    G = ref.trace_functional_matrix(A, S, P)
    ex0 = ref.chebyshev_expand(ref.scale(Hp, e0, e1), P, np.zeros((1, n)), G=G)
    res = ref.mu_bisect(ex0.g, ref.KIND_FERMI, kT, e0, e1, N_e, 1e-9 * N_e)
    assert res.converged
    # exact count root (brute force on the generalised eigenvalues)
    mu_ex = brentq(lambda m: np.sum(1 / (1 + np.exp((eps - m) / kT))) - N_e, e0, e1, xtol=1e-14)
    assert abs(res.mu - mu_ex) < 1e-6
    f = ref.Func(ref.KIND_FERMI, mu=res.mu, kT=kT)
    ex = ref.chebyshev_expand(ref.scale(Hp, e0, e1), P, ref.cheb_coeffs(f, n, e0, e1)[None])
    F = ref.postprocess(ex.acc[0], A, P)
    Fex = ref.dense_function(Hd, f, Sd)
    assert ref.rel_frobenius(F.dense(), Fex) < 1e-8
    assert abs(ref.trace_product(F, S) - N_e) < 1e-7


def _dense_isqrt_case(n_atoms=12, seed=11):
    s, S, H, P = _dense_foe_case(n_atoms=n_atoms, seed=seed)
    Sd, Hd = S.dense(), H.dense()
    ws = np.linalg.eigvalsh(Sd)
    se0, se1 = 0.95 * ws[0], 1.05 * ws[-1]
    fpow = ref.Func(ref.KIND_POWER, a=-0.5)
    n_s = ref.choose_degree(fpow, se0, se1, 1e-13, 4096, rel=True)
    A = ref.chebyshev_expand(ref.scale(S, se0, se1), P, ref.cheb_coeffs(fpow, n_s, se0, se1)[None]).acc[0]
    eps = sla.eigh(Hd, Sd, eigvals_only=True)
    return s, S, H, P, A, eps, ((se0, se1), n_s)


def _fermi(x):
    return 0.5 * (1.0 - np.tanh(0.5 * x))


@pytest.mark.parametrize("kind", [ref.KIND_FERMI, ref.KIND_ERFC])
def test_energy_moments_resum_to_the_eigenvalue_sum(kind):
    # E = Tr(K H) = sum_i f(eps_i) eps_i over the generalised eigenvalues (K
    # built from c_i with c^T S c = 1): the energy moments re-summed with the
    # coefficients of any (mu, kT) -- a second kernel costs no new products.
    s, S, H, P, A, eps, _ = _dense_isqrt_case()
    Hp = ref.orthogonalise(H, A, P)
    e0, e1 = eps[0] - 0.1, eps[-1] + 0.1
    GH = ref.trace_functional_matrix(A, H, P)
    n = ref.choose_degree(ref.Func(kind, mu=0.5 * (e0 + e1), kT=0.02), e0, e1, 1e-12, 16384)
    e = ref.chebyshev_expand(ref.scale(Hp, e0, e1), P, np.zeros((1, n)), G=GH).g
    occ = _fermi if kind == ref.KIND_FERMI else (lambda x: 0.5 * erfc_vec(x))
    for mu, kT in ((float(np.median(eps)), 0.02), (float(eps[10]), 0.05), (float(eps[30]), 0.03)):
        E = ref.energy(e, ref.Func(kind, mu=mu, kT=kT), e0, e1)
        want = float(np.sum(occ((eps - mu) / kT) * eps))
        assert abs(E - want) < 1e-8 * max(1.0, abs(want)), (mu, kT, E, want)
    # the electron-count functional on the same moments is a different number
    G = ref.trace_functional_matrix(A, S, P)
    g = ref.chebyshev_expand(ref.scale(Hp, e0, e1), P, np.zeros((1, n)), G=G).g
    assert abs(ref.energy(g, ref.Func(kind, mu=float(np.median(eps)), kT=0.02), e0, e1) - want) > 1e-3


def erfc_vec(x):
    return np.array([math.erfc(v) for v in np.ravel(x)]).reshape(np.shape(x))


def test_auto_kT_matches_brute_force_on_eigenvalues():
    # The oracle's smearing loop against the same loop run on the generalised
    # eigenvalues: mu(kT) from sum f = N_e, E = sum f eps, the same rule.
    s, S, H, P, A, eps, (bS, n_S) = _dense_isqrt_case()
    N_e = float(len(eps) // 2)
    e0, e1 = eps[0] - 0.1, eps[-1] + 0.1
    kT0, widen, shrink = 0.2, 1.25, 0.5

    def exact(kT):
        mu = brentq(lambda m: np.sum(_fermi((eps - m) / kT)) - N_e, e0, e1, xtol=1e-14)
        return float(np.sum(_fermi((eps - mu) / kT) * eps))

    dE = [abs(exact(kT0 * shrink ** r) - exact(widen * kT0 * shrink ** r)) for r in range(4)]
    assert dE[0] > dE[1] > dE[2]  # the difference shrinks with the smearing
    dE_tol = float(np.sqrt(dE[1] * dE[2]))  # accept in the third round, far from the edge
    out = pipelines.foe_auto_kT(S, H, P, kT0, N_e, dE_tol, bS, n_S, (e0, e1), 1e-11, 16384, 1e-10 * N_e,
                                widen=widen, shrink=shrink)
    assert [r[0] for r in out["rounds"]] == [kT0, kT0 * shrink, kT0 * shrink ** 2]
    assert [r[4] for r in out["rounds"]] == [False, False, True] and out["accepted"]
    for r, k in zip(out["rounds"], range(3)):
        kT = kT0 * shrink ** k
        assert abs(r[2] - exact(kT)) < 1e-7 * N_e and abs(r[3] - exact(widen * kT)) < 1e-7 * N_e
    assert abs(out["trace_FS"] - N_e) < 1e-7 * N_e


def test_trace_functional_is_adjoint_of_postprocessing():
    s, S, H, P_H, P_out = _small_system(n_atoms=20, r_c=4.0, r_out=6.0, seed=12)
    rng = np.random.default_rng(3)
    A = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))  # not symmetric on purpose
    G = ref.trace_functional_matrix(A, S, P_out)
    for _ in range(3):
        X = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
        lhs = float(np.sum(X.vals * G.vals))
        rhs = ref.trace_product(ref.postprocess(X, A, P_out), S)
        assert abs(lhs - rhs) < 1e-10 * max(1, abs(rhs))
    # and against dense matrices with explicit masks
    mask_blk = np.zeros((20, 20), bool)
    rows = np.repeat(np.arange(20), np.diff(P_out.row_ptr))
    mask_blk[rows, P_out.col_idx] = True
    mask = np.kron(mask_blk, np.ones((4, 4), bool))
    Ad, Sd, Xd = A.dense(), S.dense(), X.dense()
    want = np.sum((Ad @ ((Xd @ Ad) * mask)) * mask * Sd)
    assert abs(lhs - want) < 1e-10 * max(1, abs(want))


def test_idempotency_at_low_temperature_with_gap():
    # Orthogonal basis, gapped spectrum: F = f(H) tends to a projector as kT -> 0.
    nb = 8
    rng = np.random.default_rng(5)
    d = np.where(np.arange(4 * nb) % 2 == 0, -1.0, 1.0) + 0.05 * rng.normal(size=4 * nb)
    B = 0.02 * rng.normal(size=(4 * nb, 4 * nb))
    Hd = np.diag(d) + (B + B.T)
    P = _dense_pattern(nb)
    H = _bsr_from_dense(Hd, P.row_ptr, P.col_idx)
    w = np.linalg.eigvalsh(Hd)
    e0, e1 = w[0] - 0.05, w[-1] + 0.05
    errs = []
    for kT in (0.1, 0.03, 0.01):
        f = ref.Func(ref.KIND_FERMI, mu=0.0, kT=kT)
        n = ref.choose_degree(f, e0, e1, 1e-11, 8192)
        F = ref.chebyshev_expand(ref.scale(H, e0, e1), P, ref.cheb_coeffs(f, n, e0, e1)[None]).acc[0].dense()
        errs.append(np.linalg.norm(F @ F - F) / np.linalg.norm(F))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-10


def test_interval_count_matches_brute_force():
    s, S, H, P = _dense_foe_case(n_atoms=10, seed=13)
    Sd, Hd = S.dense(), H.dense()
    ws = np.linalg.eigvalsh(Sd)
    se0, se1 = 0.95 * ws[0], 1.05 * ws[-1]
    fpow = ref.Func(ref.KIND_POWER, a=-0.5)
    n_s = ref.choose_degree(fpow, se0, se1, 1e-13, 4096, rel=True)
    A = ref.chebyshev_expand(ref.scale(S, se0, se1), P, ref.cheb_coeffs(fpow, n_s, se0, se1)[None]).acc[0]
    Hp = ref.orthogonalise(H, A, P)
    eps = sla.eigh(Hd, Sd, eigvals_only=True)
    e0, e1 = eps[0] - 0.1, eps[-1] + 0.1
    kT = 0.01
    gaps = np.diff(eps)
    i = int(np.argmax(gaps[: len(gaps) // 2]))
    j = len(gaps) // 2 + int(np.argmax(gaps[len(gaps) // 2:]))
    lo, hi = 0.5 * (eps[i] + eps[i + 1]), 0.5 * (eps[j] + eps[j + 1])
    assert min(np.abs(eps - lo).min(), np.abs(eps - hi).min()) >= 10 * kT
    f = ref.Func(ref.KIND_INTERVAL, kT=kT, lo=lo, hi=hi)
    n = ref.choose_degree(f, e0, e1, 1e-9, 16384)
    G = ref.trace_functional_matrix(A, S, P)
    ex = ref.chebyshev_expand(ref.scale(Hp, e0, e1), P, ref.cheb_coeffs(f, n, e0, e1)[None], G=G)
    count = 0.5 * ex.acc[0].vals.size and ref.trace_product(ref.postprocess(ex.acc[0], A, P), S)
    want = int(np.sum((eps > lo) & (eps < hi)))
    assert abs(count - want) < 1e-4
    # selected eigenvalue by half occupation (N - 1/2) lands on eps_N
    g = ex.g if ex.g is not None else None
    ex0 = ref.chebyshev_expand(ref.scale(Hp, e0, e1), P, np.zeros((1, n)), G=G)
    N = 7
    res = ref.mu_bisect(ex0.g, ref.KIND_FERMI, kT, e0, e1, N - 0.5, 1e-10)
    assert abs(res.mu - eps[N - 1]) < 3 * kT


# --------------------------------------------------------------------------
# Newton-Schulz, transposes, error metrics
# --------------------------------------------------------------------------

def test_newton_schulz_squares_the_error():
    s, S, H, P = _dense_foe_case(n_atoms=8, seed=14)
    Sd = S.dense()
    inv = np.linalg.inv(Sd)
    rng = np.random.default_rng(6)
    E = rng.normal(size=inv.shape)
    E = 0.5 * (E + E.T)
    for eps in (1e-3, 1e-5):
        X0 = _bsr_from_dense(inv + eps * E / np.linalg.norm(E), P.row_ptr, P.col_idx)
        X1 = ref.newton_schulz(S, X0, P).dense()
        e0 = np.linalg.norm(X0.dense() - inv)
        e1 = np.linalg.norm(X1 - inv)
        assert e1 < 10 * np.linalg.norm(Sd) * e0 ** 2
    X1 = ref.newton_schulz(S, _bsr_from_dense(inv, P.row_ptr, P.col_idx), P).dense()
    assert ref.rel_frobenius(X1, inv) < 1e-13


def test_transpose_and_error_metrics():
    s, S, H, P_H, P_out = _small_system(n_atoms=16, r_c=4.0, r_out=6.0, seed=15)
    rng = np.random.default_rng(7)
    X = P_out.with_vals(rng.normal(size=(P_out.nnzb, 4, 4)))
    assert np.array_equal(ref.transpose(X).dense(), X.dense().T)
    assert np.array_equal(ref.transpose(ref.transpose(X)).vals, X.vals)
    M = np.eye(3)
    mask = np.ones((3, 3), bool)
    assert ref.error_eq9(M + 0.3, M, mask) == pytest.approx(np.sqrt(9 * 0.09) / 9)
    assert ref.error_eq8(M, M, mask) == 0.0


def test_newton_schulz_isqrt_squares_the_error():
    s, S, H, P = _dense_foe_case(n_atoms=8, seed=16)
    Sd = S.dense()
    w, U = np.linalg.eigh(Sd)
    Z = (U * w ** -0.5) @ U.T
    for eps in (1e-3, 1e-5):
        # a perturbation that commutes with S: Z0 = Z (1 + eps D), D diagonal in S's eigenbasis
        D = (U * np.linspace(-1, 1, len(w))) @ U.T
        Z0 = _bsr_from_dense(Z @ (np.eye(len(w)) + eps * D), P.row_ptr, P.col_idx)
        Z1 = ref.newton_schulz_isqrt(S, Z0, P).dense()
        e0 = np.linalg.norm(Z0.dense() - Z) / np.linalg.norm(Z)
        e1 = np.linalg.norm(Z1 - Z) / np.linalg.norm(Z)
        assert e1 < 3 * e0 ** 2
    Z1 = ref.newton_schulz_isqrt(S, _bsr_from_dense(Z, P.row_ptr, P.col_idx), P).dense()
    assert ref.rel_frobenius(Z1, Z) < 1e-13


# --------------------------------------------------------------------------
# column-sampled expansion, erfc occupations, penalty side
# --------------------------------------------------------------------------

def test_column_expand_matches_masked_dense_brute_force():
    # the C column recursion against dense matrices masked after each product
    s, S, H, P_H, P_out = _small_system(n_atoms=40, r_c=3.0, r_out=4.5, seed=17)
    Hd = H.dense()
    nat = P_out.nbr
    mask_blk = np.zeros((nat, nat), bool)
    rows = np.repeat(np.arange(nat), np.diff(P_out.row_ptr))
    mask_blk[rows, P_out.col_idx] = True
    mask = np.kron(mask_blk, np.ones((4, 4), bool))
    w = sla.eigvalsh(Hd)
    emin, emax = w[0] - 0.1, w[-1] + 0.1
    Ht = ref.scale(H, emin, emax)
    Htd = Ht.dense()
    n = 35
    c = np.random.default_rng(5).normal(size=(2, n)) / (1 + np.arange(n))
    Ts = [np.eye(4 * nat) * mask, Htd * mask]
    for k in range(1, n - 1):
        Ts.append(2.0 * (Htd @ Ts[-1]) * mask - Ts[-2])
    cols = [0, 3, 17, 39]
    got = ref.column_expand(Ht, P_out, cols, c)
    for j in range(2):
        want = 0.5 * c[j, 0] * Ts[0] + sum(c[j, k] * Ts[k] for k in range(1, n))
        for ci, J in enumerate(cols):
            I = P_out.col_idx[P_out.row_ptr[J]:P_out.row_ptr[J + 1]]
            wb = np.stack([want[4 * i:4 * i + 4, 4 * J:4 * J + 4] for i in I])
            assert np.max(np.abs(got[j][ci] - wb)) < 1e-11


def test_erfc_occupations_count_brute_force_levels():
    # Eq. 9 with beta = 1/kT: on a diagonal operator the re-summed count
    # sum_k c_k(mu) g_k (g_k = sum_i T_k(x~_i)) equals sum_i erfc((e_i - mu)/kT)/2
    # computed level by level with the standard library's erfc
    import math
    rng = np.random.default_rng(23)
    eps = np.sort(rng.uniform(-1.0, 1.5, 60))
    emin, emax = -1.2, 1.7
    s_, t_ = ref.sigma_tau(emin, emax)
    x = s_ * (eps - t_)
    n = 1024
    g = np.array([np.sum(np.cos(k * np.arccos(x))) for k in range(n)])
    kT, mu = 0.04, 0.3
    got = ref.electron_count(g, ref.Func(ref.KIND_ERFC, mu=mu, kT=kT), emin, emax)
    want = sum(0.5 * math.erfc((e - mu) / kT) for e in eps)
    assert abs(got - want) < 1e-9 * len(eps)
    # occupied below mu, empty above, one half at mu, and the two tails of one
    # width add to one (erfc(-y) = 2 - erfc(y))
    f = ref.Func(ref.KIND_ERFC, mu=mu, kT=kT)
    assert f(mu - 5 * kT) > 1 - 1e-10 and f(mu + 5 * kT) < 1e-10 and f(mu) == 0.5
    for d in (0.3 * kT, kT, 2.5 * kT):
        assert abs(f(mu - d) + f(mu + d) - 1.0) < 1e-15
    assert abs(f(mu + kT) - 0.5 * math.erfc(1.0)) < 1e-15


def test_penalty_side_shows_in_the_sign_pattern_of_the_moments():
    # a level below -1 makes T_k(x) = (-1)^k cosh(k acosh|x|) dominate the
    # moments (alternating signs); a level above +1 gives one sign
    s, S, H, P_H, P_out = _small_system(n_atoms=20, r_c=4.0, r_out=6.0, seed=10)
    w = np.linalg.eigvalsh(S.dense())
    wd = w[-1] - w[0]
    n = 120
    for emin, emax, side in [(w[0] + 0.1 * wd, w[-1] + 0.05 * wd, -1), (w[0] - 0.05 * wd, w[-1] - 0.1 * wd, 1)]:
        ex = ref.chebyshev_expand(ref.scale(S, emin, emax), P_out, np.zeros((1, n)))
        assert abs(ref.penalty_trace(ex.t, -40.0, emin, emax)) >= 1.0
        assert (-1 if ex.t[-1] * ex.t[-2] < 0 else 1) == side


def test_lanczos_bounds_of_a_multiple_of_the_identity():
    # a degenerate spectrum: Lanczos breaks down after one step (the Krylov
    # space of c I is invariant), theta = c exactly, and the interval is widened
    # to 1e-3 |c| around c, so that it still contains the spectrum
    n = 6
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    for c in (1.0, -2.5, 0.0):
        A = ref.Bsr(rp, ci, np.stack([c * np.eye(4)] * n))
        alpha, beta = ref.lanczos(A, np.ones(4 * n), 40)
        assert len(alpha) == 1 and alpha[0] == pytest.approx(c, abs=1e-15)
        e0, e1, t0, t1 = ref.ritz_bounds(alpha, beta, 0.01)
        w = 1e-3 * (abs(c) if c != 0.0 else 1.0)
        assert e0 < c < e1 and e1 - e0 == pytest.approx(w, rel=1e-12)
    # a spectrum of normal width is untouched by the floor
    Ad = np.diag(np.linspace(-1.0, 2.0, 4 * n))
    A = ref.Bsr(rp, ci, np.stack([Ad[4 * i:4 * i + 4, 4 * i:4 * i + 4] for i in range(n)]))
    alpha, beta = ref.lanczos(A, np.ones(4 * n), 40)
    e0, e1, t0, t1 = ref.ritz_bounds(alpha, beta, 0.01)
    assert e0 <= -1.0 and e1 >= 2.0 and e1 - e0 < 3.2


def test_lanczos_start_vector_sees_every_eigenvalue_of_one_atoms_overlap():
    # the overlap of one atom's four Gaussians: the all-ones vector lies in a
    # two-dimensional invariant subspace (Lanczos stops there and misses the
    # smallest eigenvalue); the default start vector does not
    s = synth.make_system(1, 1.0, 4)
    S = ref.Bsr(s.row_ptr, s.col_idx, s.S)
    w = np.linalg.eigvalsh(S.dense())
    a1, b1 = ref.lanczos(S, np.ones(4), 40)
    assert len(a1) == 2 and ref.ritz_bounds(a1, b1)[0] > w[0]
    a2, b2 = ref.lanczos(S, pipelines.lanczos_start(4), 40)
    e0, e1, t0, t1 = ref.ritz_bounds(a2, b2)
    assert len(a2) == 4 and e0 <= w[0] and e1 >= w[-1]
    assert abs(t0 - w[0]) < 1e-12 and abs(t1 - w[-1]) < 1e-12
    v = pipelines.lanczos_start(1000)
    assert v.min() >= 1.0 and v.max() < 1.5 and abs(v.mean() - 1.25) < 0.02
