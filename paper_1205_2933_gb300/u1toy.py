"""The paper's 2D U(1) toy (Sec. 3, Fig. 2) on the library: the 20^2 x 8
lattice embedded in four dimensions as X x 1 x 1 x Y, the U(1) angles on
diagonal SU(3) links of charges (1, 1, -2) (so the embedded operator holds,
per colour, two copies of the 2D domain-wall operator for links e^{i q theta}),
then for each mass CG on the normal equations and the multigrid solve, with
their fine-operator applications to |r|/|b| <= tol.

Host-side control only (every computation runs in libdwfmg.so).

  python -m paper_1205_2933_gb300.u1toy [--coarsen squared] [--beta 6] [--masses 0.1 0.01]
prints one JSON line per mass.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import dwfmg as G
from . import inputs as I


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--dims", type=int, nargs=2, default=[20, 20])
    ap.add_argument("--Ls", type=int, default=8)
    ap.add_argument("--M5", type=float, default=1.0)
    ap.add_argument("--beta", type=float, default=6.0)
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--masses", type=float, nargs="+", default=[0.10, 0.05, 0.03, 0.02, 0.01])
    ap.add_argument("--nvec", type=int, default=24)
    ap.add_argument("--coarsen", choices=["unsquared", "squared"], default="squared")
    ap.add_argument("--tol", type=float, default=1e-10)
    args = ap.parse_args(argv)
    import torch
    dims2 = tuple(args.dims)
    theta = I.u1_links_2d(dims2, args.beta, args.sweeps, args.seed)
    U, dims4 = I.embed_u1_2d(theta)
    links = torch.from_numpy(U).cuda()
    src = torch.from_numpy(np.ascontiguousarray(I.gaussian_source(dims4, args.Ls, args.seed + 1))).cuda()
    for mf in args.masses:
        ctx = G.Context(dims4, args.Ls, args.M5, mf, links)
        b = torch.empty(ctx.field_elems, dtype=torch.complex128, device="cuda")
        G.dwf_pack(ctx.h, b, src, G.DWF_F64, 1)
        x = torch.zeros_like(b)
        cg = G.dwf_cg_solve(ctx.h, b, x, args.tol, 100000, 1, G.DWF_F64, check=False)
        p = G.mg_default_params()
        p.coarsen = 1 if args.coarsen == "squared" else 0
        p.nu_post = 4
        p.setup_iters0 = 200
        p.coarsest_tol = 0.05
        p.coarsest_maxiter = 200
        p.coarse_restart = 32
        p.outer_maxiter = 300
        t0 = time.time()
        G.mg_setup(ctx.h, 2, [args.nvec], [(4, 1, 1, 4)], p)
        x.zero_()
        st = G.mg_solve(ctx.h, b, x, args.tol, 1, check=False)
        torch.cuda.synchronize()
        print(json.dumps({"mf": mf, "coarsen": args.coarsen, "cg_status": cg.status, "cg_iters": cg.iters,
                          "cg_applies": cg.fine_applies_f64, "mg_status": st.status, "mg_iters": st.iters,
                          "mg_applies": st.fine_applies_f64 + st.fine_applies_f32, "true_res": st.true_res,
                          "setup_and_solve_s": round(time.time() - t0, 3)}), flush=True)
        ctx.close()


if __name__ == "__main__":
    main()
