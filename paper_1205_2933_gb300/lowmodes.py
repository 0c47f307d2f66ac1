"""The low-mode diagnostic of the paper's Fig. 1 on a heatbath lattice.

Host-side control only (every computation runs in libdwfmg.so): the
smallest eigenpairs of D^+ D (`dwf_lowest_modes`, with the multigrid of a
full adaptive setup), then the share |P^+ v|^2 / |v|^2 of each mode inside
the coarse spaces of several setups: the full adaptive setup, random start
vectors, random vectors relaxed 25 and 100 iterations, and the committed
proposal network's vectors relaxed 25 iterations.

  python -m paper_1205_2933_gb300.lowmodes [--dims 8 8 8 8] [--k 16] [--seed 1035]
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import pathlib
import time

from . import dwfmg as G
from . import learned as Lm


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[8, 8, 8, 8])
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--seed", type=int, default=1035)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-6)
    args = ap.parse_args(argv)
    import torch
    dims, k = tuple(args.dims), args.k
    ctx = Lm.lattice(dims, 16, args.seed)
    nvec, block = 24, (4, 4, 4, 4)
    G.mg_setup(ctx.h, 2, [nvec], [block], Lm.solve_params())
    vecs = torch.empty(k * ctx.field_elems, dtype=torch.complex128, device="cuda")
    t0 = time.time()
    ev, res, its = G.dwf_lowest_modes(ctx.h, k, vecs, max_iters=args.iters, tol=args.tol)
    out = {"dims": dims, "k": k, "seed": args.seed, "evals": ev, "resid": res, "iters": its,
           "eig_s": round(time.time() - t0, 1), "adaptive": G.mg_coarse_overlap(ctx.h, 0, vecs, k)}
    for name, iters in (("random", 0), ("relax25", 25), ("relax100", 100)):
        G.mg_setup(ctx.h, 2, [nvec], [block], Lm.solve_params(iters))
        out[name] = G.mg_coarse_overlap(ctx.h, 0, vecs, k)
    shape, params, _ = Lm.load(pathlib.Path(Lm.__file__).parent / "weights" / "near_null_8x8x8x8_Ls16.npz")
    net = Lm.make_net(ctx, shape, params)
    G.mg_setup_learned(ctx.h, net, 3, 2, [nvec], [block], Lm.solve_params(25))
    out["learned25"] = G.mg_coarse_overlap(ctx.h, 0, vecs, k)
    G.net_destroy(net)
    ctx.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
