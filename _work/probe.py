"""One short per-step expansion on a synthetic system, for profilers.

    python -m paper_1704_00512_gb300.probe --atoms 4000 --precision f32 --acc 4
    python -m paper_1704_00512_gb300.probe --atoms 4000 --precision f32 --acc 0 --moments

Builds the seeded atom-centred system (r_c = 10, r_buf = 4 bohr by default), its
patterns and plan with the operator row lists, and runs --terms terms of the
recursion on the scaled H with --acc FP64 accumulators (or, with --moments,
the moment pass: Tr T_k and <T_k, G>).  Each term after the first two is one
k_step launch, so `ncu -k regex:k_step -s 2 -c 1` captures a steady-state step.
"""

from __future__ import annotations

import argparse

import torch

import synth

from . import _lib as L
from . import solve


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--atoms", type=int, default=4000)
    ap.add_argument("--r-cut", type=float, default=10.0)
    ap.add_argument("--r-buf", type=float, default=4.0)
    ap.add_argument("--precision", choices=["f64", "f32", "bf16"], default="f32")
    ap.add_argument("--acc", type=int, default=4)
    ap.add_argument("--moments", action="store_true")
    ap.add_argument("--terms", type=int, default=8)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-lists", action="store_true")
    args = ap.parse_args(argv)
    prec = {"f64": L.F64, "f32": L.F32, "bf16": L.BF16}[args.precision]
    dev = torch.device("cuda:0")
    sysm = synth.make_system(args.atoms, args.r_cut, 0)
    pb = solve.problem_from_system(sysm, args.r_buf, dev, L.F64, op_lists=False)
    plan = L.Plan(pb.P_out, prec, args.tile)
    Ht = pb.H.with_vals(L.scale(pb.H, -9.0, 9.0))
    if not args.no_lists:
        plan.attach_operator(Ht)
    n = args.terms
    gen = torch.Generator(device="cpu").manual_seed(1)
    c = (torch.rand((max(args.acc, 1), n), generator=gen, dtype=torch.float64) * 1e-3).to(dev)
    accs = [pb.zeros_out() for _ in range(args.acc)]
    kw = {}
    if args.moments:
        kw = dict(moments=torch.zeros(n, dtype=torch.float64, device=dev), G=pb.zeros_out() + 1e-3,
                  gmoments=torch.zeros(n, dtype=torch.float64, device=dev))
    L.expand(plan, Ht, n, c if args.acc else None, accs, precision=prec, stepwise=True, **kw)
    torch.cuda.synchronize()
    print("ok", pb.P_out.nnzb, plan.info(), flush=True)


if __name__ == "__main__":
    main()
