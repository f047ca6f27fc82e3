"""Seeded synthetic inputs: atom-centred overlap (S) and Hamiltonian (H) matrices.

This module only *generates inputs*.  It holds none of the Chebyshev method's
arithmetic (no scaling, no recursion, no coefficients, no bounds, no traces) and
is imported by both the CUDA path's tests/bench and the CPU oracle, which never
import each other.

The paper fills sparsity patterns taken from BigDFT water droplets with random
numbers chosen to give the desired spectral properties (Sec. "Performance",
opening paragraph).  Those matrices are not available, so this generator stands
in for them with the recipe below (all lengths in bohr, energies in Ha):

* Atoms: random sequential addition, uniform in a periodic cube of edge
  ``L = 18 * (n_atoms / 200) ** (1/3)`` (the density of 200 atoms in an 18 bohr
  cube), rejecting a candidate whose minimum-image distance to an accepted atom
  is below ``d_min = 2.0``.  Positions come from ``numpy.random.default_rng(seed)``
  three uniforms per attempt.  Accepted atoms are then emitted in Morton
  (Z-curve) order of their position, the spatially local ordering a
  linear-scaling code would hand over.
* Basis: 4 normalised s-type Gaussians per atom with exponents ``EXPONENTS``.
  Their overlap at distance r is
  ``(2 sqrt(a b) / (a + b)) ** 1.5 * exp(-a b / (a + b) * r**2)``, which is
  ``exp(-0.3 r**2)`` for a = b = 0.6.  S is a Gram matrix, hence SPD; the
  exponents were tuned once so that kappa(S) is about 50 at the 3000-atom,
  10 bohr configuration.  Periodic images within the cutoff are summed.
* Block pattern P_H: atom pairs whose minimum-image distance is <= r_c
  (inclusive), always including the diagonal.
* H_ij = -0.5 * S_ij * (1 + 0.1 * z_ij) off the diagonal, z_ij standard normal,
  symmetric; H_ii ~ U[-1.2, 0.3].  Diagonal draws come from the same rng after
  the positions; z_ij comes from a counter-based generator keyed by
  (seed, min(i, j), max(i, j)) so that it does not depend on enumeration order.

Blocks are 4x4, row-major, in block-CSR: ``row_ptr`` int64 [nbr+1], ``col_idx``
int32 sorted ascending within each row, ``vals`` float64 [nnzb, 4, 4].
"""

from __future__ import annotations

import dataclasses

import numpy as np

BS = 4
RHO_REF_ATOMS = 200
RHO_REF_EDGE = 18.0
D_MIN = 2.0
# Four s-Gaussian exponents 0.6 * 4**m: the most diffuse one gives exp(-0.3 r**2)
# between atoms; the spread was tuned for kappa(S) ~ 50 (see module doc).
EXPONENTS = 0.6 * 4.0 ** np.arange(4)


def box_length(n_atoms: int) -> float:
    """Edge of the periodic cube that keeps the 200-atoms-per-18-bohr density."""
    return RHO_REF_EDGE * (n_atoms / RHO_REF_ATOMS) ** (1.0 / 3.0)


def min_image(d: np.ndarray, L: float) -> np.ndarray:
    """Wrap coordinate differences of points inside [0, L) into [-L/2, L/2]."""
    d = np.where(d > 0.5 * L, d - L, d)
    return np.where(d < -0.5 * L, d + L, d)


def _morton_key(xyz: np.ndarray, L: float, bits: int = 10) -> np.ndarray:
    q = np.clip((xyz / L * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1)
    key = np.zeros(len(xyz), dtype=np.int64)
    for b in range(bits):
        for ax in range(3):
            key |= ((q[:, ax] >> b) & 1) << (3 * b + ax)
    return key


def place_atoms(n_atoms: int, seed: int, d_min: float = D_MIN,
                max_attempts_per_atom: int = 10_000) -> tuple[np.ndarray, float]:
    """Random sequential addition in a periodic cube; Morton-sorted positions."""
    L = box_length(n_atoms)
    rng = np.random.default_rng(seed)
    nc = max(1, int(L // d_min))
    cw = L / nc
    cells: dict[tuple[int, int, int], list[int]] = {}
    pos = np.empty((n_atoms, 3))
    n = 0
    d2min = d_min * d_min
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    attempts = 0
    while n < n_atoms:
        attempts += 1
        if attempts > max_attempts_per_atom * n_atoms:
            raise RuntimeError("random sequential addition did not converge")
        p = rng.random(3) * L
        c = tuple(int(v) % nc for v in (p // cw))
        ok = True
        seen = set()
        for o in offs:
            cc = ((c[0] + o[0]) % nc, (c[1] + o[1]) % nc, (c[2] + o[2]) % nc)
            if cc in seen:
                continue
            seen.add(cc)
            lst = cells.get(cc)
            if not lst:
                continue
            d = min_image(pos[lst] - p, L)
            if np.any((d * d).sum(axis=1) < d2min):
                ok = False
                break
        if ok:
            pos[n] = p
            cells.setdefault(c, []).append(n)
            n += 1
    order = np.argsort(_morton_key(pos, L), kind="stable")
    return pos[order].copy(), L


def neighbour_pattern(xyz: np.ndarray, L: float, r_cut: float):
    """Block pattern {(I, J): minimum-image distance <= r_cut} as block-CSR.

    The distance test is ``(dx*dx + dy*dy) + dz*dz <= r_cut*r_cut`` in float64
    with ``dx`` wrapped by a single +/- L.  This is input construction (the
    paper leaves the pattern to the caller, Sec. "Introduction"); the solver
    library builds its own patterns independently.
    """
    n = len(xyz)
    rows = []
    r2 = r_cut * r_cut
    chunk = 512
    for s in range(0, n, chunk):
        blk = xyz[s:s + chunk]
        dx = min_image(xyz[None, :, 0] - blk[:, None, 0], L)
        dy = min_image(xyz[None, :, 1] - blk[:, None, 1], L)
        dz = min_image(xyz[None, :, 2] - blk[:, None, 2], L)
        d2 = (dx * dx + dy * dy) + dz * dz
        m = d2 <= r2
        for i in range(len(blk)):
            m[i, s + i] = True
            rows.append(np.nonzero(m[i])[0].astype(np.int32))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col_idx = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    return row_ptr, col_idx


def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def pair_normal(seed: int, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """Standard normal z(i, j) = z(j, i) from a counter-based hash (splitmix64 + Box-Muller)."""
    lo = np.minimum(i, j).astype(np.uint64)
    hi = np.maximum(i, j).astype(np.uint64)
    with np.errstate(over="ignore"):
        ctr = (lo << np.uint64(32)) ^ hi ^ (np.uint64(seed) * np.uint64(0xD1B54A32D192ED03))
    a = _splitmix64(ctr)
    b = _splitmix64(a)
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    u2 = (b >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _overlap_blocks(xyz, L, I, J, r_cut, exps):
    a = exps[:, None]
    b = exps[None, :]
    pref = (2.0 * np.sqrt(a * b) / (a + b)) ** 1.5
    red = a * b / (a + b)
    d = xyz[J] - xyz[I]
    d = min_image(d, L)
    out = np.zeros((len(I), BS, BS))
    rc2 = r_cut * r_cut
    if L > 2.0 * r_cut:
        # every other periodic image is farther than L - L/2 > r_cut
        r2 = (d * d).sum(axis=1)
        use = r2 <= rc2
        out[use] = pref[None] * np.exp(-red[None] * r2[use, None, None])
        return out
    # Sum over periodic images with distance <= r_cut (only the minimum image
    # unless L < 2 r_cut).
    for nx in (-1, 0, 1):
        for ny in (-1, 0, 1):
            for nz in (-1, 0, 1):
                v = d + L * np.array([nx, ny, nz], dtype=np.float64)
                r2 = (v * v).sum(axis=1)
                use = r2 <= rc2
                if not np.any(use):
                    continue
                out[use] += pref[None] * np.exp(-red[None] * r2[use, None, None])
    return out


@dataclasses.dataclass
class System:
    """One synthetic system: atoms, box and S/H on the block pattern P_H."""

    xyz: np.ndarray
    L: float
    r_cut: float
    row_ptr: np.ndarray
    col_idx: np.ndarray
    S: np.ndarray
    H: np.ndarray
    seed: int

    @property
    def n_atoms(self) -> int:
        return len(self.xyz)

    @property
    def n_rows(self) -> int:
        return BS * len(self.xyz)

    @property
    def nnzb(self) -> int:
        return len(self.col_idx)


def make_system(n_atoms: int, r_cut: float, seed: int = 0,
                exps: np.ndarray | None = None) -> System:
    """Generate atoms and S, H on P_H (the ``r_cut`` block pattern)."""
    exps = EXPONENTS if exps is None else np.asarray(exps, dtype=np.float64)
    xyz, L = place_atoms(n_atoms, seed)
    # The diagonal of H comes from a second stream keyed by (seed, 1), so the
    # positions never depend on how many diagonal values are drawn.
    rng_diag = np.random.default_rng([seed, 1])
    diag = rng_diag.uniform(-1.2, 0.3, size=BS * n_atoms)
    row_ptr, col_idx = neighbour_pattern(xyz, L, r_cut)
    nbr = n_atoms
    I = np.repeat(np.arange(nbr), np.diff(row_ptr))
    J = col_idx.astype(np.int64)
    S = _overlap_blocks(xyz, L, I, J, r_cut, exps)
    gi = (BS * I[:, None, None] + np.arange(BS)[None, :, None]) * np.ones((1, 1, BS), np.int64)
    gj = (BS * J[:, None, None] + np.arange(BS)[None, None, :]) * np.ones((1, BS, 1), np.int64)
    z = pair_normal(seed, gi, gj)
    H = -0.5 * S * (1.0 + 0.1 * z)
    dmask = I == J
    for m in range(BS):
        H[dmask, m, m] = diag[BS * I[dmask] + m]
    return System(xyz=xyz, L=L, r_cut=r_cut, row_ptr=row_ptr, col_idx=col_idx,
                  S=S, H=H, seed=seed)


def to_dense(row_ptr: np.ndarray, col_idx: np.ndarray, vals: np.ndarray) -> np.ndarray:
    """Expand a 4x4 block-CSR matrix to dense (small sizes only)."""
    nbr = len(row_ptr) - 1
    A = np.zeros((BS * nbr, BS * nbr), dtype=vals.dtype)
    for I in range(nbr):
        for p in range(row_ptr[I], row_ptr[I + 1]):
            J = int(col_idx[p])
            A[BS * I:BS * I + BS, BS * J:BS * J + BS] = vals[p]
    return A
