"""The two coarse operators side by side on one heatbath lattice: R D P
(9-point, the unsquared operator) and P^+ D^+ D P (33-point, the squared
operator that Sec. 4 coarsens), each with the same adaptive setup, FP32
V-cycle and FP64 outer GCR, for one Gaussian right-hand side.

Host-side control only (every computation runs in libdwfmg.so).

  python -m paper_1205_2933_gb300.coarsen_compare [--dims 16 16 16 32] [--seed 100]
prints one JSON line per configuration: setup and solve seconds, status
(0 = converged, -4 = not within --max-iters outer iterations), outer
iterations, FP64 true residual, FP32 fine applications.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import dwfmg as G
from . import inputs as I
from . import learned as Lm

# name, coarsening, coarse link precision, coarsest tolerance, its iteration cap, its restart
CONFIGS = (
    ("unsquared-bf16", 0, G.DWF_BF16, 0.03, 128, 16),
    ("squared-f32-0.03/128", 1, G.DWF_F32, 0.03, 128, 16),
    ("squared-f32-0.01/512", 1, G.DWF_F32, 0.01, 512, 32),
    ("squared-bf16-0.01/512", 1, G.DWF_BF16, 0.01, 512, 32),
)


def params(coarsen, coarse_prec, coarsest_tol, coarsest_maxiter, restart, max_iters):
    """The benchmark's mixed-precision solver (16 CGNR post-smoothing steps,
    600 setup relaxation iterations) with the given coarse operator."""
    p = Lm.solve_params(600)
    p.nu_post = 16
    p.coarsen = coarsen
    p.coarse_prec[0] = coarse_prec
    p.coarsest_tol = coarsest_tol
    p.coarsest_maxiter = coarsest_maxiter
    p.coarse_restart = restart
    p.outer_maxiter = max_iters
    return p


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--Ls", type=int, default=16)
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--source-seed", type=int, default=101)
    ap.add_argument("--max-iters", type=int, default=250)
    args = ap.parse_args(argv)
    import torch
    dims = tuple(args.dims)
    ctx = Lm.lattice(dims, args.Ls, args.seed)
    b = torch.empty(ctx.field_elems, dtype=torch.complex128, device="cuda")
    src = np.ascontiguousarray(I.gaussian_source(dims, args.Ls, args.source_seed))
    G.dwf_pack(ctx.h, b, torch.from_numpy(src).cuda(), G.DWF_F64, 1)
    for name, co, cp, ct, cm, cr in CONFIGS:
        p = params(co, cp, ct, cm, cr, args.max_iters)
        torch.cuda.synchronize()
        t0 = time.time()
        G.mg_setup(ctx.h, 2, [24], [(4, 4, 4, 4)], p)
        torch.cuda.synchronize()
        t1 = time.time()
        x = torch.zeros_like(b)
        st = G.mg_solve(ctx.h, b, x, 1e-10, 1, check=False)
        torch.cuda.synchronize()
        t2 = time.time()
        print(json.dumps({"cfg": name, "dims": dims, "setup_s": round(t1 - t0, 3), "solve_s": round(t2 - t1, 3),
                          "status": st.status, "iters": st.iters, "true_res": st.true_res,
                          "f32_applies": st.fine_applies_f32}), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
