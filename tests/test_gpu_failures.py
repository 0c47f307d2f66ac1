"""Failure paths of the solve, made without a GPU fault: a NaN in a
source must come back as DWF_ENAN with the context still usable, an
iteration limit that is too small must come back as DWF_ENOCONV with x
holding the best iterate (its true residual is the one reported), and a
bounded device-side wait that runs out must come back as DWF_ETIMEOUT."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS, LS, MF = (4, 4, 4, 4), 8, 0.1


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


def _ctx(G, **kw):
    from gpu_util import ctx_for
    U = I.epsilon_links(DIMS, 0.3, 1)
    ctx = ctx_for(U, DIMS, LS, 1.8, MF)
    p = G.mg_default_params()
    p.setup_iters0 = 20
    for k, v in kw.items():
        setattr(p, k, v)
    G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p)
    return ctx, U


@pytest.mark.parametrize("sp,nrhs", [(0, 1), (1, 3)], ids=["f64-1rhs", "f32-batched3"])
def test_nan_source_returns_enan(G, sp, nrhs):
    from gpu_util import to_internal
    ctx, _ = _ctx(G, smoother_prec=sp)
    bs = np.stack([I.gaussian_source(DIMS, LS, 60 + i) for i in range(nrhs)])
    bs[nrhs - 1].reshape(-1)[123] = np.nan
    bt = to_internal(ctx, bs, nrhs=nrhs)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(ctx.h, bt, xt, 1e-10, nrhs=nrhs, check=False)
    assert st.status == G.DWF_ENAN
    # the context stays usable: a clean source solves
    b1 = to_internal(ctx, I.gaussian_source(DIMS, LS, 70))
    x1 = torch.zeros_like(b1)
    st = G.mg_solve(ctx.h, b1, x1, 1e-10)
    assert st.status == G.DWF_OK and st.true_res <= 1e-10
    ctx.close()


def test_iteration_limit_returns_enoconv_with_best_iterate(G):
    from gpu_util import to_internal, to_canonical
    ctx, U = _ctx(G, outer_maxiter=2, outer_restart=2)
    b = I.gaussian_source(DIMS, LS, 71)
    bt = to_internal(ctx, b)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(ctx.h, bt, xt, 1e-10, check=False)
    assert st.status == G.DWF_ENOCONV
    assert st.iters == 2
    x = to_canonical(ctx, xt, b.shape)
    # the reported residual is that of the returned iterate, recomputed by the oracle's operator
    r = b - oracle.DWF(U, DIMS, LS, 1.8, MF).D(x)
    res = np.linalg.norm(r) / np.linalg.norm(b)
    assert 1e-10 < st.true_res < 1.0
    assert abs(res - st.true_res) <= 1e-9 * st.true_res + 1e-14
    ctx.close()


def test_expired_wait_returns_etimeout():
    """The tensor-core coarsest solver bounds each of its waits (about one
    second).  DWF_TC_FORCE_WAIT=1 makes its first launch begin with a wait on
    a barrier that nothing completes: the wait runs out, every CTA stops at the
    next reduction, and the solve returns DWF_ETIMEOUT; the next solve on the
    same context (no forced wait left) converges.  Run in a child process so
    that the environment variable is read fresh."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = textwrap.dedent(f"""
        import sys, time
        sys.path[:0] = [{root!r}, {os.path.join(root, "tests")!r}]
        import numpy as np, torch
        from paper_1205_2933_gb300 import dwfmg as G
        import paper_1205_2933_gb300.inputs as I
        from gpu_util import ctx_for, to_internal
        dims, Ls = (4, 4, 4, 4), 8
        ctx = ctx_for(I.epsilon_links(dims, 0.3, 1), dims, Ls, 1.8, 0.1)
        p = G.mg_default_params()
        p.setup_iters0 = 20
        p.smoother_prec = G.DWF_F32
        p.coarse_prec[0] = G.DWF_BF16
        G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p)
        bs = np.stack([I.gaussian_source(dims, Ls, 80 + i) for i in range(3)])
        bt = to_internal(ctx, bs, nrhs=3)
        xt = torch.zeros_like(bt)
        t0 = time.time()
        st = G.mg_solve(ctx.h, bt, xt, 1e-10, nrhs=3, check=False)
        print("first", st.status, round(time.time() - t0, 2))
        xt.zero_()
        st = G.mg_solve(ctx.h, bt, xt, 1e-10, nrhs=3, check=False)
        print("second", st.status, st.true_res)
        ctx.close()
    """)
    env = dict(os.environ, DWF_TC_FORCE_WAIT="1")
    out = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = dict(l.split(" ", 1) for l in out.stdout.strip().splitlines())
    from paper_1205_2933_gb300 import dwfmg as G
    first = lines["first"].split()
    assert int(first[0]) == G.DWF_ETIMEOUT
    assert float(first[1]) >= 0.9  # the wait ran for its full bound
    second = lines["second"].split()
    assert int(second[0]) == G.DWF_OK and float(second[1]) <= 1e-10
