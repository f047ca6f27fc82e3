"""Train the learned mu proposal on instances the method generates.

    python -m paper_1704_00512_gb300.train_mu --batches 6 --out paper_1704_00512_gb300/weights/mu_proposal.npz

Each batch draws per_batch synthetic systems (atoms uniform in
[atoms_lo, atoms_hi], 10 bohr cutoff, kT log-uniform in [kT_lo, kT_hi] Ha, half
filling, seeds from --seed), labels them with one batched moment pass and the
bisection (learned.label_batch), and the network is trained on the library's
MLP kernels (forward, loss, backward, Adam).  A held-out tenth of the
instances reports how far the proposal lands from mu* in units of kT and how
often its bracket holds mu*.  The weights, the training curve and those
statistics are written to one .npz file.
"""

from __future__ import annotations

import argparse
import math
import time

import numpy as np
import torch

import synth

from . import learned


def make_instances(n_batches: int, per_batch: int, atoms_lo: int, atoms_hi: int, kT_lo: float, kT_hi: float,
                   seed: int, r_c: float, r_buf: float, device, log=None):
    log = log or (lambda m: print(m, flush=True))
    rng = np.random.default_rng(seed)
    Xs, xs, sc, meta = [], [], [], []
    for b in range(n_batches):
        t0 = time.time()
        sizes = rng.integers(atoms_lo, atoms_hi + 1, per_batch)
        kTs = np.exp(rng.uniform(math.log(kT_lo), math.log(kT_hi), per_batch))
        seeds = [seed + b * per_batch + i for i in range(per_batch)]
        systems = [synth.make_system(int(n), r_c, sd) for n, sd in zip(sizes, seeds)]
        X, xstar, scale, m = learned.label_batch(systems, kTs, r_buf, device)
        if not m["converged"]:
            raise RuntimeError(f"batch {b}: a bisection did not converge")
        Xs.append(X)
        xs.append(xstar)
        sc.append(scale)
        meta += [(float(n), float(k), float(sd), float(mu)) for n, k, sd, mu in zip(sizes, kTs, seeds, m["mu"])]
        log(f"batch {b}: {per_batch} instances, {int(sizes.sum())} atoms, terms {min(m['n_terms'])}.."
            f"{max(m['n_terms'])}, {time.time() - t0:.1f}s")
    return np.concatenate(Xs), np.concatenate(xs), np.concatenate(sc), meta


def evaluate(prop: learned.Proposal, X: np.ndarray, xstar: np.ndarray, scale: np.ndarray,
             min_half_kT: float = 0.05, max_half_kT: float = 1.0) -> dict:
    """Distance of the proposal from mu* in kT and the fraction of (clamped) brackets holding mu*."""
    out = prop.forward(torch.as_tensor(X, dtype=torch.float32, device=prop.device).contiguous()).cpu().numpy()
    d = np.abs(out[:, 0] - xstar) / scale
    w = np.clip(np.exp(out[:, 1]) / scale, min_half_kT, max_half_kT)
    return {"median_abs_err_kT": float(np.median(d)), "p90_abs_err_kT": float(np.percentile(d, 90)),
            "max_abs_err_kT": float(np.max(d)), "coverage": float(np.mean(d <= w)),
            "median_half_kT": float(np.median(w))}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--batches", type=int, default=6)
    ap.add_argument("--per-batch", type=int, default=64)
    ap.add_argument("--atoms-lo", type=int, default=500)
    ap.add_argument("--atoms-hi", type=int, default=1000)
    ap.add_argument("--kT-lo", type=float, default=0.004)
    ap.add_argument("--kT-hi", type=float, default=0.02)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--r-cut", type=float, default=10.0)
    ap.add_argument("--r-buf", type=float, default=4.0)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="paper_1704_00512_gb300/weights/mu_proposal.npz")
    args = ap.parse_args(argv)
    dev = torch.device("cuda:0")
    X, xstar, scale, meta = make_instances(args.batches, args.per_batch, args.atoms_lo, args.atoms_hi, args.kT_lo,
                                           args.kT_hi, args.seed, args.r_cut, args.r_buf, dev)
    n = len(xstar)
    perm = np.random.default_rng(args.seed + 1).permutation(n)
    n_hold = max(1, n // 10)
    hold, train = perm[:n_hold], perm[n_hold:]
    prop = learned.Proposal(learned.Proposal.xavier(args.seed + 2, dev), dev)
    t0 = time.time()
    hist = prop.train(X[train], xstar[train], scale[train], iters=args.iters, lr=args.lr,
                      log_every=max(1, args.iters // 20))
    ev_train = evaluate(prop, X[train], xstar[train], scale[train])
    ev_hold = evaluate(prop, X[hold], xstar[hold], scale[hold])
    print(f"trained {len(train)} instances in {time.time() - t0:.1f}s; loss {hist[0]:.3g} -> {hist[-1]:.3g}")
    print(f"train: {ev_train}")
    print(f"held out ({n_hold}): {ev_hold}", flush=True)
    np.savez(args.out, theta=prop.theta.cpu().numpy(), loss=np.array(hist), n_train=len(train), n_hold=n_hold,
             hold_median_abs_err_kT=ev_hold["median_abs_err_kT"], hold_max_abs_err_kT=ev_hold["max_abs_err_kT"],
             hold_coverage=ev_hold["coverage"], train_coverage=ev_train["coverage"],
             instances=np.array(meta, dtype=np.float64), features=X, xstar=xstar, scale=scale,
             recipe=np.array(f"atoms U[{args.atoms_lo},{args.atoms_hi}], r_c {args.r_cut}, r_buf {args.r_buf}, "
                             f"kT logU[{args.kT_lo},{args.kT_hi}], half filling, seeds from {args.seed}, "
                             f"{args.iters} Adam steps lr {args.lr}"))
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
