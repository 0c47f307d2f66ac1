"""mg_coarse_solve_static: the coarsest-level solve without any device
allocation, for callers that cannot allocate device memory while they solve.

It must give the same result as mg_coarse_solve (which uses context-owned
workspaces), twice in a row through the shared static scratch, on the
9-point R D P stencil and on the squared operator's 33-point stencil.  It
must refuse requests beyond its fixed 8 MiB array (by restart length and by
bytes) and an in-place call whose x and b overlap.  This file sorts last so
that a run stopping at the first failure has run every other test first; it
also passes alone in a fresh process.
"""
import numpy as np
import pytest

import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCRATCH = 8 << 20


def _setup(G, dims, Ls, nvec, block, **kw):
    U = I.epsilon_links(dims, 0.3, 1)
    ctx = G.Context(dims, Ls, 1.8, 0.1, torch.from_numpy(U).cuda())
    p = G.mg_default_params()
    p.setup_iters0 = 5
    p.setup_sweeps = 0
    for k, v in kw.items():
        setattr(p, k, v)
    start = torch.from_numpy(I.random_vectors(nvec // 2, dims, Ls, 3)).cuda()
    G.mg_setup(ctx.h, 2, [nvec], [block], p, start)
    d, n = G.mg_level_info(ctx.h, 1)
    return ctx, int(np.prod(d)) * n


@pytest.mark.parametrize("sq", [0, 1], ids=["rdp", "squared"])
@pytest.mark.parametrize("sp", [0, 1], ids=["f64", "f32"])
def test_static_scratch_coarse_solve_matches(sp, sq):
    from paper_1205_2933_gb300 import dwfmg as G
    dims = (4, 6, 4, 4) if sq else (4, 4, 4, 4)
    ctx, N = _setup(G, dims, 4 if sq else 8, 8, (2, 2, 2, 2), smoother_prec=sp, coarsen=sq,
                    setup_iters0=10, coarsest_tol=1e-6, coarsest_maxiter=200)
    dt = torch.complex128 if sp == 0 else torch.complex64
    tol = 1e-12 if sp == 0 else 1e-6
    for seed in (41, 42):  # two calls in a row share the static scratch
        b = torch.from_numpy(I.gauss_complex((N,), seed, 50)).to(dt).cuda()
        x_ref = torch.empty_like(b)
        G.mg_coarse_solve(ctx.h, 1, x_ref, b)
        x = torch.full_like(b, float("nan"))
        G.mg_coarse_solve_static(ctx.h, 1, x, b)
        err = ((x - x_ref).abs().max() / x_ref.abs().max()).item()
        assert err <= tol, err
    ctx.close()


def test_static_scratch_rejects_long_restart():
    from paper_1205_2933_gb300 import dwfmg as G
    ctx, N = _setup(G, (4, 4, 4, 4), 4, 8, (2, 2, 2, 2), coarse_restart=24)  # the static limit is 16
    b = torch.ones(N, dtype=torch.complex128, device="cuda")
    x = torch.empty_like(b)
    assert G.lib().mg_coarse_solve_static(ctx.h, 1, G._ptr(x), G._ptr(b)) == G.DWF_EINVAL
    ctx.close()


def test_static_scratch_byte_limit():
    """A coarse level of 512 sites x 32 components in FP64 (256 KiB per
    vector): the largest restart whose vectors and partial sums fit in the
    8 MiB array is accepted and matches mg_coarse_solve; one more is refused."""
    from paper_1205_2933_gb300 import dwfmg as G
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    off = 256 + (1632 * sms + 255) // 256 * 256
    vec = 512 * 32 * 16
    fit = ((SCRATCH - off) // vec - 1) // 2
    assert 1 <= fit < 16, fit  # the byte branch, not the restart branch, decides at fit + 1
    for restart, ok in ((fit, True), (fit + 1, False)):
        ctx, N = _setup(G, (16, 8, 8, 8), 4, 32, (2, 2, 2, 2), coarse_restart=restart, coarsest_tol=1e-4,
                        coarsest_maxiter=60)
        assert N * 16 == vec
        b = torch.from_numpy(I.gauss_complex((N,), 43, 50)).cuda()
        x = torch.full_like(b, float("nan"))
        st = G.lib().mg_coarse_solve_static(ctx.h, 1, G._ptr(x), G._ptr(b))
        if ok:
            assert st == G.DWF_OK
            x_ref = torch.empty_like(b)
            G.mg_coarse_solve(ctx.h, 1, x_ref, b)
            assert ((x - x_ref).abs().max() / x_ref.abs().max()).item() <= 1e-12
        else:
            assert st == G.DWF_EINVAL
        ctx.close()


def test_static_scratch_rejects_aliasing():
    """The solver writes x = 0 before it reads b, so an in-place call is refused."""
    from paper_1205_2933_gb300 import dwfmg as G
    ctx, N = _setup(G, (4, 4, 4, 4), 4, 8, (2, 2, 2, 2))
    b = torch.from_numpy(I.gauss_complex((N + 1,), 44, 50)).cuda()
    assert G.lib().mg_coarse_solve_static(ctx.h, 1, G._ptr(b), G._ptr(b)) == G.DWF_EINVAL
    # partial overlap: x starts one element into b
    xo = b[1:]
    assert G.lib().mg_coarse_solve_static(ctx.h, 1, G._ptr(xo), G._ptr(b)) == G.DWF_EINVAL
    ctx.close()
