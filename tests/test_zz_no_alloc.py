"""mg_coarse_solve_static: the coarsest-level solve without any device
allocation, for callers that cannot allocate device memory while they solve.

It must give the same result as mg_coarse_solve (which uses context-owned
workspaces), twice in a row through the shared static scratch.  This file
sorts last so that a run stopping at the first failure has run every other
test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("sp", [0, 1], ids=["f64", "f32"])
def test_static_scratch_coarse_solve_matches(sp):
    from paper_1205_2933_gb300 import dwfmg as G
    dims, Ls = (4, 4, 4, 4), 8
    U = I.epsilon_links(dims, 0.3, 1)
    ctx = G.Context(dims, Ls, 1.8, 0.1, torch.from_numpy(U).cuda())
    p = G.mg_default_params()
    p.smoother_prec = sp
    p.setup_iters0 = 10
    p.setup_sweeps = 0
    p.coarsest_tol = 1e-6
    p.coarsest_maxiter = 200
    start = torch.from_numpy(I.random_vectors(4, dims, Ls, 3)).cuda()
    G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p, start)
    d, n = G.mg_level_info(ctx.h, 1)
    dt = torch.complex128 if sp == 0 else torch.complex64
    tol = 1e-12 if sp == 0 else 1e-6
    for seed in (41, 42):  # two calls in a row share the static scratch
        b = torch.from_numpy(I.gauss_complex((int(np.prod(d)) * n,), seed, 50)).to(dt).cuda()
        x_ref = torch.empty_like(b)
        G.mg_coarse_solve(ctx.h, 1, x_ref, b)
        x = torch.full_like(b, float("nan"))
        G.mg_coarse_solve_static(ctx.h, 1, x, b)
        err = ((x - x_ref).abs().max() / x_ref.abs().max()).item()
        assert err <= tol, err
    ctx.close()


def test_static_scratch_rejects_oversize():
    from paper_1205_2933_gb300 import dwfmg as G
    dims, Ls = (4, 4, 4, 4), 4
    U = I.epsilon_links(dims, 0.3, 1)
    ctx = G.Context(dims, Ls, 1.8, 0.1, torch.from_numpy(U).cuda())
    p = G.mg_default_params()
    p.setup_iters0 = 5
    p.setup_sweeps = 0
    p.coarse_restart = 24  # beyond the static solver's restart limit of 16
    G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p)
    d, n = G.mg_level_info(ctx.h, 1)
    b = torch.ones(int(np.prod(d)) * n, dtype=torch.complex128, device="cuda")
    x = torch.empty_like(b)
    assert G.lib().mg_coarse_solve_static(ctx.h, 1, G._ptr(x), G._ptr(b)) == G.DWF_EINVAL
    ctx.close()
