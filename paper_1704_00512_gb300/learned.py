"""Learned mu proposal: training data from the method, training with the library's
MLP kernels, and the one-pass solve it enables.  (Not in the paper.)

The plain FOE (solve.foe) needs two expansions: one to collect the trace
functional g_k for the bisection on Tr(F(mu) S) = N_e, and one to accumulate
F at the mu it finds.  A proposal (mu_hat, h) lets one expansion carry both:
g_k plus n_mu accumulators at the Chebyshev nodes mu_i of [mu_hat - h,
mu_hat + h].  The bisection on g stays the judge; if its mu* lies inside the
bracket, F(mu*) is the Lagrange interpolant of the n_mu accumulators (F is
analytic in mu with its nearest singularities about pi*kT from the real axis,
so for h well below kT the interpolation error is ~(h / (2 pi kT))^n_mu);
otherwise a second expansion at mu* is run (the fallback).

Every numerical step runs in libcheb.so; this module sequences calls.
"""

from __future__ import annotations

import dataclasses
import os

import numpy as np
import torch

from . import _lib as L
from . import solve

N_IN = 35
N_MOM = 32
N_PARAMS_EXPECTED = 35 * 128 + 128 + 128 * 128 + 128 + 2 * 128 + 2


@dataclasses.dataclass
class Instance:
    features: np.ndarray  # [35]
    xstar: float          # sigma (mu* - tau), the scaled Fermi level
    scale: float          # sigma * kT
    kT: float
    bounds: tuple[float, float]
    mu: float
    n_terms: int


def prepare(pb: solve.Problem, tol_S: float = 1e-10, lanczos_k: int = 40):
    """S^-1/2, H', bounds of H', scaled H~', the trace functional G (as in
    solve.foe) and H' itself (to rescale if the penalty check moves a bound)."""
    pw = solve.powers(pb, exponents=(-0.5,), tol=tol_S, precision=L.F64)
    A = pw["acc"][0]
    Hp = solve.orthogonalise(pb, A)
    e0, e1, _ = L.bounds(Hp, lanczos_k)
    Hpt = Hp.with_vals(L.scale(Hp, e0, e1))
    G = solve.trace_functional(pb, A)
    return A, Hpt, (e0, e1), G, Hp


def moments32(pb: solve.Problem, Hpt: L.Bsr, stepwise: bool = False) -> torch.Tensor:
    """t_k = Tr T_k for k < 32 (a 32-term expansion with no accumulators)."""
    t = torch.zeros(N_MOM, dtype=torch.float64, device=pb.device)
    L.expand(pb.planX, Hpt, N_MOM, None, [], moments=t, precision=pb.precision, stepwise=stepwise)
    return t


def features(pb: solve.Problem, t32: torch.Tensor, bounds, N_e: float) -> torch.Tensor:
    f = torch.empty(N_IN, dtype=torch.float32, device=pb.device)
    return L.mlp_features(t32, pb.n_rows, bounds[0], bounds[1], N_e, f)


def label_instance(sysm, r_buf: float, kT: float, N_e: float, device, tol: float = 1e-6,
                   precision: int = L.F32) -> Instance:
    """Features and the bisection's mu* (the label) for one generated system."""
    pb = solve.problem_from_system(sysm, r_buf, device, precision)
    A, Hpt, (e0, e1), G, _ = prepare(pb)
    n, _ = L.coeffs([{"kind": L.FERMI, "mu": 0.5 * (e0 + e1), "kT": kT}], e0, e1, tol, 16384, device=pb.device)
    t = torch.zeros(n, dtype=torch.float64, device=pb.device)
    g = torch.zeros(n, dtype=torch.float64, device=pb.device)
    L.expand(pb.planX, Hpt, n, None, [], moments=t, G=G, gmoments=g, precision=precision)
    r = L.decode_mu_result(L.mu_search(g, n, e0, e1, L.FERMI, kT, N_e, 1e-6 * N_e))
    f = features(pb, t[:N_MOM].contiguous(), (e0, e1), N_e).cpu().numpy()
    sigma, tau = 2.0 / (e1 - e0), 0.5 * (e0 + e1)
    return Instance(f, sigma * (r["mu"] - tau), sigma * kT, kT, (e0, e1), r["mu"], n)


def label_batch(systems, kTs, r_buf: float, device, tol: float = 1e-7, precision: int = L.F32):
    """Features, scaled mu* and scale sigma*kT of many instances from one batched
    moment pass (each instance half filled, N_e = rows/2)."""
    from . import batched
    bp = batched.BatchedProblem(systems, r_buf, device, precision=precision, tune=False)
    N_e = [2.0 * s.n_atoms for s in systems]
    mp = batched.moment_pass_batched(bp, list(kTs), N_e, n_moments=N_MOM, tol=tol)
    X = torch.empty((len(systems), N_IN), dtype=torch.float32, device=bp.device)
    xstar, scale = np.zeros(len(systems)), np.zeros(len(systems))
    for i, s in enumerate(systems):
        e0, e1 = mp["bounds_H"][i]
        L.mlp_features(mp["t"][i], s.n_rows, e0, e1, N_e[i], X[i])
        sigma, tau = 2.0 / (e1 - e0), 0.5 * (e0 + e1)
        xstar[i] = sigma * (mp["mu"][i] - tau)
        scale[i] = sigma * kTs[i]
    conv = all(r["converged"] for r in mp["mu_result"])
    return X.cpu().numpy(), xstar, scale, {"mu": mp["mu"], "n_terms": mp["n_terms"], "converged": conv}


class Proposal:
    """The network's parameters on the device plus training state."""

    def __init__(self, theta0: np.ndarray, device):
        self.device = torch.device(device)
        self.theta = torch.as_tensor(theta0, dtype=torch.float32, device=self.device).contiguous()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.t = 0

    @staticmethod
    def xavier(seed: int, device) -> torch.Tensor:
        """Xavier-uniform weights, zero biases (cheb_mlp_init on the device)."""
        return L.mlp_init(seed, device)

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        act = torch.empty(X.shape[0] * 256, dtype=torch.float32, device=self.device)
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=self.device)
        L.mlp_forward(self.theta, X, act, out)
        return out

    def train(self, X: np.ndarray, xstar: np.ndarray, scale: np.ndarray, iters: int = 2000, lr: float = 1e-3,
              log_every: int = 0) -> list[float]:
        X = torch.as_tensor(X, dtype=torch.float32, device=self.device).contiguous()
        xs = torch.as_tensor(xstar, dtype=torch.float32, device=self.device).contiguous()
        sc = torch.as_tensor(scale, dtype=torch.float32, device=self.device).contiguous()
        B = X.shape[0]
        act = torch.empty(B * 256, dtype=torch.float32, device=self.device)
        out = torch.empty((B, 2), dtype=torch.float32, device=self.device)
        dout = torch.empty_like(out)
        grad = torch.empty_like(self.theta)
        ws = torch.empty(B * 256, dtype=torch.float32, device=self.device)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        hist = []
        for it in range(iters):
            L.mlp_forward(self.theta, X, act, out)
            L.mlp_loss(out, xs, sc, dout, loss)
            L.mlp_backward(self.theta, X, act, dout, grad, ws)
            self.t += 1
            L.mlp_adam(self.theta, grad, self.m, self.v, self.t, lr)
            if log_every and (it % log_every == 0 or it == iters - 1):
                hist.append(float(loss.item()))
        return hist


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "mu_proposal.npz")


def load_proposal(device, path: str = WEIGHTS) -> Proposal:
    """The trained proposal written by train_mu.py."""
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} missing: train it with python -m paper_1704_00512_gb300.train_mu")
    with np.load(path) as d:
        theta = d["theta"]
    if theta.shape != (N_PARAMS_EXPECTED,):
        raise ValueError(f"{path}: {theta.shape[0]} parameters, expected {N_PARAMS_EXPECTED}")
    return Proposal(theta, device)


def foe_learned(pb: solve.Problem, prop: Proposal, kT: float, N_e: float, tol: float = 1e-7, n_mu: int = 8,
                min_half_kT: float = 0.05, max_half_kT: float = 1.0, tol_N: float | None = None,
                prepared=None, bracket: tuple[float, float] | None = None, stepwise: bool = True,
                penalty_alpha: float = -200.0, penalty_threshold: float = 1.0, penalty_widen: float = 0.05,
                penalty_terms: int = 512, timings: dict | None = None, _checks=None) -> dict:
    """One-expansion FOE with the learned bracket; bisection judges, fallback on a miss.

    With n_mu = 8 Chebyshev nodes the interpolation error of the Fermi function
    in mu stays below 4e-7 for a half-width of one kT and below 2e-9 for half a
    kT.  bracket: (mu_hat, half) to use instead of the network's (tests).
    prepared: (A, H~', bounds, G[, H']) from prepare().  The pass also collects
    Tr T_k for the penalty check of Eq. 5: a failing bound is widened by
    penalty_widen of the interval and the solve repeated once (this needs H'
    in prepared); a second failure raises ChebError(ERR_BOUNDS)."""
    tm = {} if timings is None else timings
    checks = [] if _checks is None else _checks
    prepared = prepare(pb) if prepared is None else prepared
    A, Hpt, (e0, e1), G = prepared[:4]
    Hp = prepared[4] if len(prepared) > 4 else None
    tau = 0.5 * (e0 + e1)  # the degree is chosen at the interval centre
    if bracket is None:
        t32 = moments32(pb, Hpt, stepwise=stepwise)
        X = features(pb, t32, (e0, e1), N_e).view(1, N_IN)
        o = prop.forward(X).cpu().numpy()[0]
        mu_hat, half = L.mlp_bracket(o, e0, e1, kT, min_half_kT, max_half_kT)
    else:
        mu_hat, half = bracket
    mus = L.mu_nodes(mu_hat, half, n_mu)
    # same term count as the plain solve (degree chosen at the interval centre)
    n, _ = L.coeffs([{"kind": L.FERMI, "mu": tau, "kT": kT}], e0, e1, tol, 16384, device=pb.device)
    _, c = L.coeffs([{"kind": L.FERMI, "mu": m, "kT": kT} for m in mus], e0, e1, 0.0, n, device=pb.device)
    accs = [pb.zeros_out() for _ in mus]
    g = torch.zeros(n, dtype=torch.float64, device=pb.device)
    t = torch.zeros(n, dtype=torch.float64, device=pb.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    ws = L.expand(pb.planX, Hpt, n, c, accs, moments=t, G=G, gmoments=g, precision=pb.precision,
                  stepwise=stepwise)
    ev[1].record()
    verdict, value = solve.penalty(t, n, penalty_alpha, penalty_threshold, penalty_terms)
    checks.append((verdict, value, (e0, e1)))
    if verdict != 0:
        if len(checks) > 1 or Hp is None:
            raise L.ChebError(L.ERR_BOUNDS, f"penalty check (Eq. 5) failed: trace {value:g} on [{e0}, {e1}]")
        b = solve.widen((e0, e1), verdict, penalty_widen)
        return foe_learned(pb, prop, kT, N_e, tol, n_mu, min_half_kT, max_half_kT, tol_N,
                           (A, Hp.with_vals(L.scale(Hp, *b)), b, G, Hp), bracket, stepwise, penalty_alpha,
                           penalty_threshold, penalty_widen, penalty_terms, timings, checks)
    if tol_N is None:
        tol_N = 1e-6 * N_e
    r = L.decode_mu_result(L.mu_search(g, n, e0, e1, L.FERMI, kT, N_e, tol_N))
    mu = r["mu"]
    passes = 1
    p = pb.zeros_out()
    ev[2].record()
    if abs(mu - mu_hat) <= half:
        L.lincomb(L.lagrange_weights(mus, mu), accs, p)
    else:
        _, c2 = L.coeffs([{"kind": L.FERMI, "mu": mu, "kT": kT}], e0, e1, 0.0, n, device=pb.device)
        L.expand(pb.planX, Hpt, n, c2, [p], precision=pb.precision, ws=ws, stepwise=stepwise)
        passes = 2
    ev[3].record()
    F = solve.postprocess(pb, A, p)
    trFS = L.trace(pb.P_out.with_vals(F), pb.S)
    tm["events"] = ev
    return {"F": F, "p": p, "mu": mu, "mu_hat": mu_hat, "half": half, "passes": passes + len(checks) - 1,
            "n_terms": n, "mu_result": r, "trace_FS": trFS, "bounds_H": (e0, e1), "n_mu": n_mu, "penalty": checks}
