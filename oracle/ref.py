"""FP64 CPU oracle of the Chebyshev sparse-matrix-function method -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this module.  It shares no code with the CUDA library
(``paper_1704_00512_gb300``) and never imports it; the only module both sides use
is the seeded input generator ``synth``.

Every function restates one step of the paper (Mohr et al., "Efficient
computation of sparse matrix functions for large scale electronic structure
calculations: The CheSS library") in plain float64 numpy, or calls the plain C
loops of ``liboracle.c`` (compiled with -ffp-contract=off).  Readings taken where
the paper is silent or garbled are stated at each function.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
closed forms, brute force or dense linear algebra, except the penalty-function
threshold (Eq. 5), whose pass/fail rule has no closed form to check against:
parity unpinned beyond "silent on valid bounds, fires on shrunk bounds".
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np
import scipy.linalg as sla
from scipy.special import erfc as _erfc

BS = 4
_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build() -> str:
    """Compile liboracle.c into liboracle.so next to it (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "liboracle.c")
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared",
           "-fPIC", src, "-o", _LIB_PATH]
    subprocess.run(cmd, check=True)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH) or (
                os.path.getmtime(_LIB_PATH) < os.path.getmtime(os.path.join(_HERE, "liboracle.c"))):
            build()
        lib = ctypes.CDLL(_LIB_PATH)
        p = ctypes.c_void_p
        lib.oracle_masked_product.argtypes = [ctypes.c_int64] + [p] * 9 + [p]
        lib.oracle_masked_product.restype = None
        lib.oracle_spmv.argtypes = [ctypes.c_int64, p, p, p, p, p]
        lib.oracle_spmv.restype = None
        lib.oracle_pattern.argtypes = [ctypes.c_int64, p, ctypes.c_double, ctypes.c_double, p, p]
        lib.oracle_column_expand.argtypes = [ctypes.c_int64, p, p, p, p, p, ctypes.c_int64, p, ctypes.c_int64,
                                             ctypes.c_int64, p, p]
        lib.oracle_column_expand.restype = None
        lib.oracle_pattern.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# Block-CSR container
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Bsr:
    """4x4 block-CSR matrix: row_ptr int64[nbr+1], col_idx int32, vals float64[nnzb,4,4]."""

    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray

    @property
    def nbr(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnzb(self) -> int:
        return len(self.col_idx)

    def with_vals(self, vals: np.ndarray) -> "Bsr":
        return Bsr(self.row_ptr, self.col_idx, vals)

    def zeros(self) -> "Bsr":
        return self.with_vals(np.zeros((self.nnzb, BS, BS)))

    def dense(self) -> np.ndarray:
        n = BS * self.nbr
        A = np.zeros((n, n))
        rows = np.repeat(np.arange(self.nbr), np.diff(self.row_ptr))
        for b in range(self.nnzb):
            I, J = rows[b], int(self.col_idx[b])
            A[BS * I:BS * I + BS, BS * J:BS * J + BS] = self.vals[b]
        return A


def block_rows(row_ptr: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))


def find_blocks(P: Bsr, I: np.ndarray, J: np.ndarray) -> np.ndarray:
    """Index of each block (I[k], J[k]) in pattern P, or -1 (vectorised binary search)."""
    out = np.full(len(I), -1, dtype=np.int64)
    for k in range(len(I)):
        lo, hi = P.row_ptr[I[k]], P.row_ptr[I[k] + 1]
        pos = lo + np.searchsorted(P.col_idx[lo:hi], J[k])
        if pos < hi and P.col_idx[pos] == J[k]:
            out[k] = pos
    return out


def embed(A: Bsr, P: Bsr) -> Bsr:
    """Place A (pattern contained in P) into pattern P, zero elsewhere."""
    out = P.zeros()
    idx = find_blocks(P, block_rows(A.row_ptr), A.col_idx)
    if np.any(idx < 0):
        raise ValueError("pattern of A is not contained in P")
    out.vals[idx] = A.vals
    return out


def restrict(A: Bsr, P: Bsr) -> Bsr:
    """Keep only the blocks of A that lie in pattern P (P contained in A's pattern)."""
    idx = find_blocks(A, block_rows(P.row_ptr), P.col_idx)
    if np.any(idx < 0):
        raise ValueError("P is not contained in the pattern of A")
    return P.with_vals(A.vals[idx].copy())


def identity(P: Bsr) -> Bsr:
    out = P.zeros()
    rows = block_rows(P.row_ptr)
    d = rows == P.col_idx
    out.vals[d] = np.eye(BS)
    return out


def transpose(A: Bsr) -> Bsr:
    """A^T on a symmetric pattern: block (I,J) <- block (J,I) transposed."""
    rows = block_rows(A.row_ptr)
    idx = find_blocks(A, A.col_idx.astype(np.int64), rows)
    if np.any(idx < 0):
        raise ValueError("pattern is not symmetric")
    return A.with_vals(np.ascontiguousarray(A.vals[idx].transpose(0, 2, 1)))


# ----------------------------------------------------------------------------
# A1: sparsity patterns (Sec. "Sparsity and truncation": fixed pattern with buffers)
# ----------------------------------------------------------------------------

def pattern(xyz: np.ndarray, L: float, r: float) -> tuple[np.ndarray, np.ndarray]:
    """Brute-force block pattern {(I,J): minimum-image distance <= r}, diagonal always in.

    The paper works with a fixed sparsity pattern whose output pattern is a
    slightly larger "buffer" pattern (Sec. "Sparsity and truncation"); both are
    defined here geometrically by a distance cutoff, as the paper's own tests do
    (Sec. "Performance", opening paragraph).
    """
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = len(xyz)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    lib.oracle_pattern(n, _ptr(xyz), float(L), float(r), _ptr(row_ptr), None)
    row_ptr = np.concatenate([[0], np.cumsum(row_ptr[1:])]).astype(np.int64)
    col_idx = np.zeros(int(row_ptr[-1]), dtype=np.int32)
    lib.oracle_pattern(n, _ptr(xyz), float(L), float(r), _ptr(row_ptr), _ptr(col_idx))
    return row_ptr, col_idx


def pattern_python(xyz: np.ndarray, L: float, r: float):
    """Same definition as :func:`pattern`, pure Python double loop (tiny inputs only)."""
    n = len(xyz)
    rows = []
    for I in range(n):
        row = []
        for J in range(n):
            d = []
            for ax in range(3):
                t = float(xyz[J, ax]) - float(xyz[I, ax])
                if t > 0.5 * L:
                    t = t - L
                elif t < -0.5 * L:
                    t = t + L
                d.append(t)
            if (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] <= r * r or I == J:
                row.append(J)
        rows.append(row)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(x) for x in rows])
    return row_ptr, np.array([j for x in rows for j in x], dtype=np.int32)


# ----------------------------------------------------------------------------
# Masked products (Eq. 3 restricted to a fixed pattern)
# ----------------------------------------------------------------------------

def masked_product(L: Bsr, R: Bsr, C_row_ptr: np.ndarray, C_col_idx: np.ndarray,
                   colmask: np.ndarray | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """Values of P_C(L R) on the pattern (C_row_ptr, C_col_idx); plain triple loop in C."""
    lib = _load()
    nnzc = len(C_col_idx)
    if out is None:
        out = np.zeros((nnzc, BS, BS))
    Lv = np.ascontiguousarray(L.vals, dtype=np.float64)
    Rv = np.ascontiguousarray(R.vals, dtype=np.float64)
    cm = None if colmask is None else np.ascontiguousarray(colmask, dtype=np.uint8)
    lib.oracle_masked_product(L.nbr, _ptr(L.row_ptr), _ptr(L.col_idx), _ptr(Lv),
                              _ptr(R.row_ptr), _ptr(R.col_idx), _ptr(Rv),
                              _ptr(C_row_ptr), _ptr(C_col_idx), _ptr(out), _ptr(cm))
    return out


def mp(L: Bsr, R: Bsr, P: Bsr, colmask=None) -> Bsr:
    """P(L R) as a Bsr on pattern P."""
    return P.with_vals(masked_product(L, R, P.row_ptr, P.col_idx, colmask))


def spmv(A: Bsr, x: np.ndarray) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    lib.oracle_spmv(A.nbr, _ptr(A.row_ptr), _ptr(A.col_idx),
                    _ptr(np.ascontiguousarray(A.vals)), _ptr(x), _ptr(y))
    return y


# ----------------------------------------------------------------------------
# Eq. 2: spectrum scaling
# ----------------------------------------------------------------------------

def sigma_tau(emin: float, emax: float) -> tuple[float, float]:
    """sigma = 2/(emax-emin), tau = (emin+emax)/2 (Eq. 2)."""
    return 2.0 / (emax - emin), (emin + emax) / 2.0


def scale(A: Bsr, emin: float, emax: float) -> Bsr:
    """A~ = sigma (A - tau I) on A's pattern (Eq. 2); the diagonal blocks must be present."""
    s, t = sigma_tau(emin, emax)
    v = A.vals.copy()
    rows = block_rows(A.row_ptr)
    d = rows == A.col_idx
    if d.sum() != A.nbr:
        raise ValueError("every diagonal block must be in the pattern")
    v[d] = v[d] - t * np.eye(BS)
    return A.with_vals(s * v)


# ----------------------------------------------------------------------------
# Functions to expand (Sec. "Available operations")
# ----------------------------------------------------------------------------

KIND_FERMI, KIND_ERFC, KIND_POWER, KIND_INTERVAL, KIND_PENALTY = 0, 1, 2, 3, 4


@dataclasses.dataclass
class Func:
    """A scalar function f(x) of the unscaled variable x.

    kind FERMI: 1/(1+exp((x-mu)/kT))                     (Eq. 7, beta = 1/kT)
    kind ERFC:  0.5*erfc((x-mu)/kT)                       (Eq. 9, beta = 1/kT)
    kind POWER: x**a                                      (Sec. "Matrix powers")
    kind INTERVAL: Fermi(x; mu=hi) - Fermi(x; mu=lo)      (Sec. "Extraction of
        selected eigenvalues": a projector counting states between lo and hi)
    kind PENALTY: Eq. 5 in the scaled variable x~ in [-1, 1]:
        exp(-|a|(x~+1)) - exp(|a|(x~-1))  with a = alpha
    """

    kind: int
    mu: float = 0.0
    kT: float = 0.01
    a: float = 0.0
    lo: float = 0.0
    hi: float = 0.0

    def __call__(self, x: np.ndarray, emin: float | None = None, emax: float | None = None):
        x = np.asarray(x, dtype=np.float64)
        if self.kind == KIND_FERMI:
            with np.errstate(over="ignore"):
                return 1.0 / (1.0 + np.exp((x - self.mu) / self.kT))
        if self.kind == KIND_ERFC:
            return 0.5 * _erfc((x - self.mu) / self.kT)
        if self.kind == KIND_POWER:
            return np.power(x, self.a)
        if self.kind == KIND_INTERVAL:
            with np.errstate(over="ignore"):
                return (1.0 / (1.0 + np.exp((x - self.hi) / self.kT))
                        - 1.0 / (1.0 + np.exp((x - self.lo) / self.kT)))
        if self.kind == KIND_PENALTY:
            s, t = sigma_tau(emin, emax)
            xs = s * (x - t)
            al = abs(self.a)
            return np.exp(-al * (xs + 1.0)) - np.exp(al * (xs - 1.0))
        raise ValueError(self.kind)


# ----------------------------------------------------------------------------
# Eq. 4: Chebyshev coefficients;  Eq. 6: degree
# ----------------------------------------------------------------------------

def cheb_coeffs(f: Func, n: int, emin: float, emax: float) -> np.ndarray:
    """c_j, j = 0..n-1, from Eq. 4 with its garbled parenthesis read as

        c_j = (2/n) sum_{k=0}^{n-1} f(cos(pi (k+1/2)/n) / sigma + tau) cos(pi j (k+1/2)/n),

    i.e. f sampled at the n Chebyshev nodes mapped back to the unscaled interval
    (Eq. 2).  The expansion uses these n coefficients with c_0 halved (Eq. 1).
    The cosine argument pi j (2k+1)/(2n) is reduced exactly (integer j(2k+1)
    modulo 4n) before the cosine, so large j k lose no precision.
    """
    s, t = sigma_tau(emin, emax)
    k = np.arange(n, dtype=np.float64)
    xk = np.cos(np.pi * (k + 0.5) / n)
    fk = f(xk / s + t, emin, emax)
    c = np.empty(n)
    k2 = 2 * np.arange(n, dtype=np.int64) + 1
    step = max(1, 4_000_000 // max(n, 1))
    for j0 in range(0, n, step):
        j = np.arange(j0, min(n, j0 + step), dtype=np.int64)
        idx = np.outer(j, k2) % (4 * n)
        c[j0:j0 + len(j)] = (2.0 / n) * (np.cos(np.pi * idx / (2 * n)) @ fk)
    return c


def cheb_eval(c: np.ndarray, x: np.ndarray) -> np.ndarray:
    """p(x) = c_0/2 + sum_{j>=1} c_j T_j(x), with T_j from the three-term recursion (Eq. 3, scalar)."""
    x = np.asarray(x, dtype=np.float64)
    Tm, T = np.ones_like(x), x.copy()
    p = 0.5 * c[0] * Tm
    if len(c) > 1:
        p = p + c[1] * T
    for j in range(2, len(c)):
        Tm, T = T, 2.0 * x * T - Tm
        p = p + c[j] * T
    return p


def degree_ladder(n_max: int) -> list[int]:
    """Candidate term counts: m * 2**e for m in 8..15, e >= 1, between 16 and n_max.

    The paper tries "various degrees" without naming them (Eq. 6); this ladder
    has a step of 1/8 octave or less.
    """
    out = set()
    e = 1
    while 8 * 2 ** e <= n_max:
        for m in range(8, 16):
            v = m * 2 ** e
            if 16 <= v <= n_max:
                out.add(v)
        e += 1
    return sorted(out)


def degree_grid(n: int) -> np.ndarray:
    """Error grid in the scaled variable: 8193 uniform points on [-1,1] plus the
    2n+1 extrema cos(pi i/(2n)) of T_{2n}."""
    u = np.linspace(-1.0, 1.0, 8193)
    e = np.cos(np.pi * np.arange(2 * n + 1) / (2 * n))
    return np.concatenate([u, e])


def max_fit_error(f: Func, n: int, emin: float, emax: float, rel: bool = False) -> float:
    s, t = sigma_tau(emin, emax)
    c = cheb_coeffs(f, n, emin, emax)
    xs = degree_grid(n)
    fx = f(xs / s + t, emin, emax)
    err = float(np.max(np.abs(cheb_eval(c, xs) - fx)))
    if rel:
        err = err / float(np.max(np.abs(fx)))
    return err


def choose_degree(f: Func, emin: float, emax: float, tol: float, n_max: int,
                  rel: bool = False) -> int:
    """Eq. 6: the smallest ladder entry n whose fit error max|p_n - f| < tol.

    ``rel`` divides the error by max|f| on the grid (used for matrix powers).
    Returns -1 when no ladder entry up to n_max reaches tol.
    """
    for n in degree_ladder(n_max):
        if max_fit_error(f, n, emin, emax, rel) < tol:
            return n
    return -1


# ----------------------------------------------------------------------------
# Eq. 1 + Eq. 3: the masked Chebyshev recursion with accumulators and moments
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Expansion:
    acc: list[Bsr]           # p_j(M~) on P_out, one per coefficient vector
    t: np.ndarray            # moments Tr T_k, k = 0..n-1
    g: np.ndarray | None     # functional <T_k, G>, k = 0..n-1


def chebyshev_expand(Mt: Bsr, P_out: Bsr, coeffs: np.ndarray, G: Bsr | None = None,
                     colmask: np.ndarray | None = None, keep_T: bool = False):
    """Accumulate p_j = c_j0/2 I + sum_{k=1}^{n-1} c_jk T_k for every row j of ``coeffs``.

    T_0 = I, T_1 = M~, T_{k+1} = 2 P_out(M~ T_k) - T_{k-1} (Eq. 3), each
    product truncated to the fixed output pattern P_out (Sec. "Sparsity and
    truncation"), left multiplication, no symmetrisation.  The coefficients of
    several functions are summed over the same T_k, so no product is repeated
    when the coefficients change (Sec. "Expansion in Chebyshev polynomials").
    Moments t_k = Tr T_k (feeding the penalty check, Eq. 5) and, when G is
    given, g_k = <T_k, G> = sum of elementwise products over P_out.
    With ``colmask`` only the selected block columns are advanced (columns are
    independent under Eq. 3); moments are then partial and returned as NaN.
    """
    coeffs = np.atleast_2d(np.asarray(coeffs, dtype=np.float64))
    nf, n = coeffs.shape
    T0 = identity(P_out)
    T1 = embed(Mt, P_out)
    if colmask is not None:
        cols = np.asarray(colmask, dtype=bool)[P_out.col_idx]
        T1.vals[~cols] = 0.0
        T0.vals[~cols] = 0.0
    acc = [P_out.with_vals(0.5 * coeffs[j, 0] * T0.vals) for j in range(nf)]
    t = np.zeros(n)
    g = np.zeros(n) if G is not None else None
    diag = block_rows(P_out.row_ptr) == P_out.col_idx

    def moments(k, T):
        t[k] = float(np.trace(T.vals[diag], axis1=1, axis2=2).sum())
        if G is not None:
            g[k] = float(np.sum(T.vals * G.vals))

    moments(0, T0)
    if n > 1:
        for j in range(nf):
            acc[j].vals += coeffs[j, 1] * T1.vals
        moments(1, T1)
    Ts = [T0, T1] if keep_T else None
    Tm, T = T0, T1
    for k in range(1, n - 1):
        prod = masked_product(Mt, T, P_out.row_ptr, P_out.col_idx, colmask)
        Tn = P_out.with_vals(2.0 * prod - Tm.vals)
        if colmask is not None:
            Tn.vals[~cols] = 0.0
        for j in range(nf):
            acc[j].vals += coeffs[j, k + 1] * Tn.vals
        moments(k + 1, Tn)
        if keep_T:
            Ts.append(Tn)
        Tm, T = T, Tn
    if colmask is not None:
        t[:] = np.nan
        if g is not None:
            g[:] = np.nan
    ex = Expansion(acc=acc, t=t, g=g)
    return (ex, Ts) if keep_T else ex


def column_expand(Mt: Bsr, P_out: Bsr, cols, coeffs: np.ndarray) -> list[list[np.ndarray]]:
    """The accumulators of Eq. 1 on the sampled block columns only (by Eq. 3's
    column independence, Sec. "Expansion in Chebyshev polynomials"): result
    [f][c] = array [rows of column cols[c], 4, 4], the blocks (I, cols[c]) of
    acc_f in ascending I (the column list of row cols[c] of the symmetric
    P_out).  Same recursion as chebyshev_expand, run in liboracle.c per column."""
    coeffs = np.ascontiguousarray(np.atleast_2d(np.asarray(coeffs, dtype=np.float64)))
    nf, n = coeffs.shape
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int32))
    lens = [int(P_out.row_ptr[j + 1] - P_out.row_ptr[j]) for j in cols]
    total = int(sum(lens))
    out = np.zeros((nf, total, 4, 4))
    lib = _load()
    lib.oracle_column_expand(Mt.nbr, _ptr(np.ascontiguousarray(Mt.row_ptr, dtype=np.int64)),
                             _ptr(np.ascontiguousarray(Mt.col_idx, dtype=np.int32)),
                             _ptr(np.ascontiguousarray(Mt.vals, dtype=np.float64)),
                             _ptr(np.ascontiguousarray(P_out.row_ptr, dtype=np.int64)),
                             _ptr(np.ascontiguousarray(P_out.col_idx, dtype=np.int32)), len(cols), _ptr(cols), n, nf,
                             _ptr(coeffs), _ptr(out))
    res, off = [], np.concatenate([[0], np.cumsum(lens)])
    for f in range(nf):
        res.append([out[f, off[c]:off[c + 1]] for c in range(len(cols))])
    return res


def column_blocks(A: np.ndarray, P_out: Bsr, cols) -> list[np.ndarray]:
    """The blocks (I, J) of a P_out-valued array A (BCSR order) for each J in
    cols, in ascending I: the layout of column_expand's result."""
    out = []
    for J in cols:
        rows = P_out.col_idx[P_out.row_ptr[J]:P_out.row_ptr[J + 1]]
        idx = [P_out.row_ptr[I] + int(np.searchsorted(P_out.col_idx[P_out.row_ptr[I]:P_out.row_ptr[I + 1]], J))
               for I in rows]
        out.append(np.asarray(A)[idx])
    return out


# ----------------------------------------------------------------------------
# A3: spectral bounds by Lanczos (Sec. "Determination of the eigenvalue bounds")
# ----------------------------------------------------------------------------

def lanczos(A: Bsr, v0: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """k steps of plain Lanczos (no reorthogonalisation) from v0.

    Returns alpha[0..k-1] and beta[0..k-1], where beta[j] couples steps j and
    j+1 (beta[k-1] is the residual norm after the last step).  The paper only
    says "a few steps of a Lanczos method" give a starting interval.
    """
    v = v0 / np.linalg.norm(v0)
    vm = np.zeros_like(v)
    b = 0.0
    alpha = np.zeros(k)
    beta = np.zeros(k)
    for j in range(k):
        w = spmv(A, v) - b * vm
        a = float(np.dot(w, v))
        w = w - a * v
        b = float(np.linalg.norm(w))
        alpha[j], beta[j] = a, b
        # breakdown (reading: beta at rounding level of the step's scale, 1e-12
        # of |alpha_j| + beta_{j-1}): the Krylov space is invariant
        if b == 0.0 or b <= 1e-12 * (abs(a) + (beta[j - 1] if j > 0 else 0.0)):
            return alpha[:j + 1], beta[:j + 1]
        vm, v = v, w / b
    return alpha, beta


def ritz_bounds(alpha: np.ndarray, beta: np.ndarray, margin_frac: float = 0.01):
    """Interval [theta_min - m_lo, theta_max + m_hi] from the Lanczos tridiagonal.

    theta are the extreme eigenvalues of the tridiagonal (alpha, beta[:-1]); the
    residual of Ritz pair i is beta[-1] |s_i| (s_i = last eigenvector
    component); each margin is max(2 residual, margin_frac * (theta_max - theta_min)).
    """
    k = len(alpha)
    if k == 1:
        th = np.array([alpha[0]])
        s = np.ones((1, 1))
    else:
        th, s = sla.eigh_tridiagonal(alpha, beta[:k - 1])
    res_lo = abs(beta[-1] * s[-1, 0])
    res_hi = abs(beta[-1] * s[-1, -1])
    width = th[-1] - th[0]
    m_lo = max(2.0 * res_lo, margin_frac * width)
    m_hi = max(2.0 * res_hi, margin_frac * width)
    e0, e1 = th[0] - m_lo, th[-1] + m_hi
    # reading for a degenerate spectrum (the paper gives none): the interval is
    # at least 1e-3 of the Ritz values' magnitude wide (1e-3 around zero),
    # centred on them, so that there is a scaling (Eq. 2)
    mag = max(abs(th[0]), abs(th[-1]))
    wmin = 1e-3 * (mag if mag > 0.0 else 1.0)
    if e1 - e0 < wmin:
        c = 0.5 * (th[0] + th[-1])
        e0, e1 = min(e0, c - 0.5 * wmin), max(e1, c + 0.5 * wmin)
    return e0, e1, th[0], th[-1]


# ----------------------------------------------------------------------------
# A10: penalty check (Eq. 5)
# ----------------------------------------------------------------------------

def penalty_trace(t: np.ndarray, alpha: float, emin: float, emax: float) -> float:
    """Tr W^p = c^p_0/2 t_0 + sum_k c^p_k t_k with c^p from Eq. 4 for Eq. 5's
    penalty function in the scaled variable (reading: x~min = -1, x~max = +1)."""
    n = len(t)
    c = cheb_coeffs(Func(KIND_PENALTY, a=alpha), n, emin, emax)
    return 0.5 * c[0] * t[0] + float(np.dot(c[1:], t[1:]))


# ----------------------------------------------------------------------------
# A11: mu search on the trace functional (Sec. "Fermi Operator Expansion")
# ----------------------------------------------------------------------------

def electron_count(g: np.ndarray, f: Func, emin: float, emax: float) -> float:
    """N(mu) = Tr(F(mu) S) = c_0/2 g_0 + sum_k c_k g_k: the trace is linear in the
    expansion coefficients, so re-summing needs no new products."""
    c = cheb_coeffs(f, len(g), emin, emax)
    return 0.5 * c[0] * g[0] + float(np.dot(c[1:], g[1:]))


def energy(e: np.ndarray, f: Func, emin: float, emax: float) -> float:
    """E = Tr(K H) = c_0/2 e_0 + sum_k c_k e_k, with the energy moments
    e_k = <T_k, G_H> (G_H = trace_functional_matrix(A, H, P_out)).  The energy
    is linear in the coefficients like the electron count, so the energy of a
    second kernel K' of the same polynomials (another smearing, another mu) is
    a re-sum as well (Sec. "Fermi Operator Expansion", the choice of beta)."""
    c = cheb_coeffs(f, len(e), emin, emax)
    return 0.5 * c[0] * e[0] + float(np.dot(c[1:], e[1:]))


@dataclasses.dataclass
class MuSearch:
    mu: float
    iters: int
    bits: list[int]
    counts: list[float]
    converged: bool


def mu_bisect(g: np.ndarray, kind: int, kT: float, emin: float, emax: float,
              N_e: float, tol_N: float, max_iter: int = 100,
              bracket: tuple[float, float] | None = None) -> MuSearch:
    """Bisection for Tr(F(mu) S) = N_e (the paper adjusts mu "until this condition is
    satisfied" without naming the method).  Bracket [emin, emax] unless given;
    midpoint in float64; bit = [N(mid) > N_e] (then hi = mid, else lo = mid);
    stop when |N(mid) - N_e| <= tol_N."""
    lo, hi = (emin, emax) if bracket is None else bracket
    bits, counts = [], []
    for it in range(1, max_iter + 1):
        mid = 0.5 * (lo + hi)
        N = electron_count(g, Func(kind, mu=mid, kT=kT), emin, emax)
        counts.append(N)
        if abs(N - N_e) <= tol_N:
            return MuSearch(mid, it, bits, counts, True)
        if N > N_e:
            bits.append(1)
            hi = mid
        else:
            bits.append(0)
            lo = mid
    return MuSearch(0.5 * (lo + hi), max_iter, bits, counts, False)


# ----------------------------------------------------------------------------
# A8/A9/A12: Newton-Schulz, orthogonalisation, post-processing, traces
# ----------------------------------------------------------------------------

def newton_schulz(S: Bsr, X0: Bsr, P_out: Bsr) -> Bsr:
    """One in-pattern Newton-Schulz step for S^-1: X1 = 2 X0 - P(X0 P(S X0))."""
    Y = mp(S, X0, P_out)
    Z = mp(X0, Y, P_out)
    return P_out.with_vals(2.0 * X0.vals - Z.vals)


def newton_schulz_isqrt(S: Bsr, Z0: Bsr, P_out: Bsr) -> Bsr:
    """One in-pattern Newton-Schulz step for S^-1/2: Z1 = 1.5 Z0 - 0.5 P(Z0 P(S P(Z0 Z0)))."""
    Y = mp(Z0, Z0, P_out)
    W = mp(S, Y, P_out)
    V = mp(Z0, W, P_out)
    return P_out.with_vals(1.5 * Z0.vals - 0.5 * V.vals)


def orthogonalise(H: Bsr, A: Bsr, P_out: Bsr) -> Bsr:
    """M' = P_H(A P_out(H A)) with A = S^-1/2 (Sec. "Fermi Operator Expansion":
    the input matrix is replaced by S^-1/2 M S^-1/2); the result keeps H's pattern."""
    Y = mp(H, A, P_out)
    Z = mp(A, Y, P_out)
    return restrict(Z, H)


def postprocess(p: Bsr, A: Bsr, P_out: Bsr) -> Bsr:
    """F = P_out(A P_out(p A)) (the output of the expansion is post-processed as
    S^-1/2 p S^-1/2, Sec. "Fermi Operator Expansion")."""
    Y = mp(p, A, P_out)
    return mp(A, Y, P_out)


def trace_functional_matrix(A: Bsr, S: Bsr, P_out: Bsr) -> Bsr:
    """G with <X, G> = Tr(postprocess(X) S) for every X on P_out.

    <P(A P(X A)), S> = <X, P(P(A^T S) A^T)> (S within P_out); with S symmetric
    this is the transpose of P(A P(S A)).
    """
    Y = mp(S, A, P_out)
    Z = mp(A, Y, P_out)
    return transpose(Z)


def trace_product(F: Bsr, S: Bsr) -> float:
    """sum over (i,j) in P_S of F_ij S_ij (= Tr(F S) for symmetric S)."""
    idx = find_blocks(F, block_rows(S.row_ptr), S.col_idx)
    if np.any(idx < 0):
        raise ValueError("P_S is not contained in F's pattern")
    return float(np.sum(F.vals[idx] * S.vals))


# ----------------------------------------------------------------------------
# Exact definitions (dense, small sizes) and error metrics
# ----------------------------------------------------------------------------

def dense_function(Hd: np.ndarray, f, Sd: np.ndarray | None = None) -> np.ndarray:
    """Density-kernel definition K = sum_i f(eps_i) c_i c_i^T with H c = eps S c and
    c^T S c = 1 (Sec. "Fermi Operator Expansion"); S = I gives U f(Lambda) U^T."""
    if Sd is None:
        w, U = np.linalg.eigh(Hd)
    else:
        w, U = sla.eigh(Hd, Sd)
    return (U * f(w)) @ U.T


def rel_frobenius(X: np.ndarray, Y: np.ndarray) -> float:
    """||X - Y||_F / ||Y||_F."""
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def error_eq8(approx_inv_of_f: np.ndarray, M: np.ndarray, mask: np.ndarray) -> float:
    """Eq. 8: RMS over the output pattern of f^-1(f(M)) - M, divided as printed
    by the element count |f(M)| outside the square root."""
    d = (approx_inv_of_f - M)[mask]
    return float(np.sqrt(np.sum(d * d)) / mask.sum())


def error_eq9(f_sparse: np.ndarray, f_exact: np.ndarray, mask: np.ndarray) -> float:
    """Eq. 9: sqrt(sum over pattern of (f_sparse - f_exact)^2) / |pattern|."""
    d = (f_sparse - f_exact)[mask]
    return float(np.sqrt(np.sum(d * d)) / mask.sum())
