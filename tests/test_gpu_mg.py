"""GPU parity of the multigrid steps (block Gram-Schmidt, R/P, the 9-point
coarse operator, coarse stencil, V-cycle) and of whole solves, against the
FP64 oracle on identical seeded inputs, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import mg as OM
import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


def _params(G, **kw):
    p = G.mg_default_params()
    for k, v in kw.items():
        if k == "coarse_prec":
            for i, x in enumerate(v):
                p.coarse_prec[i] = x
        else:
            setattr(p, k, v)
    return p


def _oracle_params(nvec, block, gpu_params):
    """Oracle parameters equal to the GPU's, field by field."""
    keys = ("nu_pre", "nu_post", "coarse_tol", "coarse_maxiter", "coarsest_tol", "coarsest_maxiter",
            "coarse_restart", "setup_iters0", "setup_tol0", "setup_sweeps", "setup_sweep_iters",
            "setup_sweep_tol", "split")
    return OM.MGParams(nvec=tuple(nvec), block=tuple(tuple(b) for b in block),
                       cycle="W" if gpu_params.cycle == 1 else "K",
                       coarsen="squared" if gpu_params.coarsen == 1 else "unsquared",
                       **{k: getattr(gpu_params, k) for k in keys})


class Case:
    """One lattice, its oracle, a GPU context and matching MG setups."""

    def __init__(self, G, dims, Ls, mf, nvec, block, seed=1, eps=0.3, hb=False, hb_sweeps=20, **kw):
        from gpu_util import ctx_for, to_internal
        self.G, self.dims, self.Ls, self.nvec, self.block = G, dims, Ls, nvec, block
        self.U = I.heatbath_links(dims, 6.0, hb_sweeps, seed) if hb else I.epsilon_links(dims, eps, seed)
        self.dwf = oracle.DWF(self.U, dims, Ls, 1.8, mf)
        self.op = OM.FineOp(self.dwf)
        self.ctx = ctx_for(self.U, dims, Ls, 1.8, mf)
        na = nvec[0] // 2
        self.start = I.random_vectors(na, dims, Ls, 3)
        self.p = _params(G, **kw)
        G.mg_setup(self.ctx.h, len(nvec) + 1, nvec, block, self.p, torch.from_numpy(self.start).cuda())
        rv = [self.start.reshape((na,) + self.op.shape)]
        for l in range(1, len(nvec)):
            d, n = G.mg_level_info(self.ctx.h, l)
            Vc = int(np.prod(d))
            rv.append(I.gauss_complex((nvec[l] // 2, Vc * n), self.p.seed + l, I.STREAM_NULLVEC)
                      .reshape(nvec[l] // 2, 1, d[3], d[2], d[1], d[0], n))
        self.mg = OM.adaptive_setup(self.op, _oracle_params(nvec, block, self.p), rv)

    def close(self):
        self.ctx.close()


SMALL = dict(dims=(4, 4, 4, 4), Ls=8, mf=0.1, nvec=[8], block=[(2, 2, 2, 2)])          # plain-method workload
RAGGED = dict(dims=(4, 2, 6, 4), Ls=3, mf=0.05, nvec=[6], block=[(2, 2, 3, 2)])        # coarse 2x1x2x2


@pytest.mark.parametrize("cfg", [SMALL, RAGGED], ids=["4^4xLs8", "ragged"])
def test_basis_and_coarse_operator(G, cfg):
    """No setup iterations: the GPU's block Gram-Schmidt of the same start
    vectors and its 9-point R D P must equal the oracle's."""
    c = Case(G, **cfg, setup_iters0=0, setup_sweeps=0)
    from gpu_util import to_canonical, rel_max
    nv = cfg["nvec"][0]
    q = torch.empty(c.ctx.field_elems * nv, dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(c.ctx.h, 0, q)
    got = to_canonical(c.ctx, q, (nv,) + c.op.shape, nrhs=nv)
    T = c.mg.levels[0].transfer
    ref = np.stack([T.vector(k) for k in range(nv)])
    assert rel_max(got, ref) < 1e-12
    d, n = G.mg_level_info(c.ctx.h, 1)
    Vc = int(np.prod(d))
    Y = torch.empty(Vc * 9 * n * n, dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_links(c.ctx.h, 1, Y)
    Yref = c.mg.levels[1].op.Y.reshape(Vc, 9, n, n)
    assert rel_max(Y.cpu().numpy().reshape(Vc, 9, n, n), Yref) < 1e-12
    c.close()


def test_device_philox_start_vectors(G):
    """Without given start vectors the GPU draws them from its own Philox:
    they must equal the host generator's (same counters) to rounding."""
    from gpu_util import ctx_for, to_canonical, rel_max
    dims, Ls = (4, 4, 4, 4), 4
    U = I.epsilon_links(dims, 0.3, 1)
    ctx = ctx_for(U, dims, Ls, 1.8, 0.1)
    p = _params(G, setup_iters0=0, setup_sweeps=0, seed=9)
    G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p)
    op = OM.FineOp(oracle.DWF(U, dims, Ls, 1.8, 0.1))
    rv = I.random_vectors(4, dims, Ls, 9).reshape((4,) + op.shape)
    mg = OM.adaptive_setup(op, _oracle_params([8], [(2, 2, 2, 2)], p), [rv])
    q = torch.empty(ctx.field_elems * 8, dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(ctx.h, 0, q)
    got = to_canonical(ctx, q, (8,) + op.shape, nrhs=8)
    ref = np.stack([mg.levels[0].transfer.vector(k) for k in range(8)])
    assert rel_max(got, ref) < 1e-12
    ctx.close()


def test_restrict_prolong_and_coarse_stencil(G):
    c = Case(G, **SMALL, setup_iters0=5, setup_sweeps=0)
    from gpu_util import to_internal, rel_max
    T = c.mg.levels[0].transfer
    A = c.mg.levels[1].op
    d, n = G.mg_level_info(c.ctx.h, 1)
    Vc = int(np.prod(d))
    f = I.gaussian_source(c.dims, c.Ls, 21)
    ft = to_internal(c.ctx, f)
    co = torch.empty(Vc * n, dtype=torch.complex128, device="cuda")
    G.mg_restrict(c.ctx.h, 0, co, ft)
    ref = T.restrict(f.reshape(c.op.shape)).reshape(Vc, n)
    assert rel_max(co.cpu().numpy().reshape(Vc, n), ref) < 1e-12
    cin = I.gauss_complex((Vc * n,), 22, 50)
    ct = torch.from_numpy(cin).cuda()
    fo = torch.empty(c.ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.mg_prolong(c.ctx.h, 0, fo, ct)
    from gpu_util import to_canonical
    got = to_canonical(c.ctx, fo, f.shape)
    assert rel_max(got, T.prolong(cin.reshape(T.cshape)).reshape(f.shape)) < 1e-13
    for dag in (False, True):
        yo = torch.empty_like(ct)
        G.mg_coarse_apply(c.ctx.h, 1, yo, ct, dag, G.DWF_F64)
        ref = (A.apply_dag if dag else A.apply)(cin.reshape(A.shape)).ravel()
        assert rel_max(yo.cpu().numpy(), ref) < 1e-12
    c.close()


@pytest.mark.parametrize("lp,tol", [(1, 1e-6), (2, 1e-2), (3, 2e-3)], ids=["f32", "bf16", "f16"])
def test_reduced_precision_coarse_stencil(G, lp, tol):
    c = Case(G, **SMALL, setup_iters0=5, setup_sweeps=0, coarse_prec=[lp])
    A = c.mg.levels[1].op
    d, n = G.mg_level_info(c.ctx.h, 1)
    cin = I.gauss_complex((int(np.prod(d)) * n,), 23, 50)
    ct = torch.from_numpy(cin.astype(np.complex64)).cuda()
    yo = torch.empty_like(ct)
    G.mg_coarse_apply(c.ctx.h, 1, yo, ct, False, G.DWF_F32)
    ref = A.apply(cin.reshape(A.shape)).ravel()
    got = yo.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    c.close()


@pytest.mark.parametrize("sp", [0, 1], ids=["f64", "f32"])
def test_coarse_solve_parity(G, sp):
    """S2 on the coarsest level (the fused GCR) against the oracle's GCR on R D P."""
    c = Case(G, **SMALL, setup_iters0=10, setup_sweeps=0, smoother_prec=sp, coarsest_tol=1e-6,
             coarsest_maxiter=200)
    A = c.mg.levels[1].op
    d, n = G.mg_level_info(c.ctx.h, 1)
    bc = I.gauss_complex((int(np.prod(d)) * n,), 33, 50)
    dt = torch.complex128 if sp == 0 else torch.complex64
    bt = torch.from_numpy(bc).to(dt).cuda()
    xt = torch.empty_like(bt)
    G.mg_coarse_solve(c.ctx.h, 1, xt, bt)
    x = xt.cpu().numpy().astype(np.complex128).reshape(A.shape)
    # the solution meets the tolerance on the oracle's coarse operator
    res = OM.norm(bc.reshape(A.shape) - A.apply(x)) / OM.norm(bc)
    assert res < (2e-6 if sp == 0 else 2e-5), res
    xo, info = OM.gcr(A.apply, bc.reshape(A.shape), tol=1e-6, maxiter=200, restart=c.p.coarse_restart)
    if sp == 0:
        assert OM.norm(x - xo) / OM.norm(xo) < 1e-3  # both meet 1e-6 on an operator of modest condition
    c.close()


def test_vcycle_parity(G):
    c = Case(G, **SMALL, setup_iters0=10, setup_sweeps=0)
    from gpu_util import to_internal, to_canonical, rel_norm
    b = I.gaussian_source(c.dims, c.Ls, 31)
    bt = to_internal(c.ctx, b)
    xt = torch.empty_like(bt)
    G.mg_vcycle(c.ctx.h, xt, bt)
    got = to_canonical(c.ctx, xt, b.shape)
    ref = c.mg.vcycle(0, b.reshape(c.op.shape)).reshape(b.shape)
    assert rel_norm(got, ref) < 1e-9
    c.close()


@pytest.mark.parametrize("cfg,nu,hist", [(SMALL, 4, 1), (RAGGED, 4, 1), (SMALL, 5, 1), (SMALL, 1, 1), (SMALL, 8, 1),
                                         (SMALL, 1, 0), (SMALL, 5, 0), (SMALL, 8, 0), (RAGGED, 4, 0)],
                         ids=["4^4xLs8", "ragged", "4^4xLs8-nu5", "4^4xLs8-nu1", "4^4xLs8-nu8",
                              "4^4xLs8-nu1-p", "4^4xLs8-nu5-p", "4^4xLs8-nu8-p", "ragged-p"])
def test_vcycle_batch_parity(G, cfg, nu, hist, monkeypatch):
    """The batched FP32 V-cycle (three right-hand sides together) against the
    oracle's V-cycle of each and against the one-at-a-time GPU V-cycle.  A
    fixed number of coarsest GCR iterations (tolerance 0) keeps both sides on
    the same Krylov step count, so the comparison is one of rounding only.
    The batched smoother has two forms.  With its residuals kept (hist = 1)
    it carries w = D p by recursion and forms x once from the stored z.  With
    a direction p (hist = 0, DWF_SMOOTHER_HISTORY=0) it defers the solution
    updates of up to three iterations and adds them in one pass: nu = 1
    defers none, nu = 5 ends with three deferred steps, and nu = 8 also
    flushes three in its middle."""
    if not hist:
        monkeypatch.setenv("DWF_SMOOTHER_HISTORY", "0")
    c = Case(G, **cfg, setup_iters0=10, setup_sweeps=0, smoother_prec=G.DWF_F32,
             coarse_prec=[G.DWF_F32], coarsest_tol=0.0, coarsest_maxiter=8, nu_post=nu)
    from gpu_util import to_internal, to_canonical, rel_norm
    nr = 3
    bs = [I.gaussian_source(c.dims, c.Ls, 40 + r) for r in range(nr)]
    bt = torch.cat([to_internal(c.ctx, b) for b in bs])
    xb = torch.empty_like(bt)
    G.mg_vcycle_batch(c.ctx.h, xb, bt, nr)
    n = c.ctx.field_elems
    for r in range(nr):
        x1 = torch.empty(n, dtype=torch.complex128, device="cuda")
        G.mg_vcycle(c.ctx.h, x1, bt[r * n:(r + 1) * n].contiguous())
        e1 = (xb[r * n:(r + 1) * n] - x1).norm().item() / x1.norm().item()
        assert e1 < 1e-4, (r, e1)
        got = to_canonical(c.ctx, xb[r * n:(r + 1) * n].contiguous(), bs[r].shape)
        ref = c.mg.vcycle(0, bs[r].reshape(c.op.shape)).reshape(bs[r].shape)
        eo = rel_norm(got, ref)
        assert eo < 1e-4, (r, eo)
    c.close()


@pytest.mark.parametrize("hist", [1, 0], ids=["chunks", "direction"])
def test_fp32_batched_relaxation_stops_with_the_oracle(G, hist, monkeypatch):
    """The FP32 setup relaxes the start vectors in one batched CGNR whose
    residual test (every 8 iterations) forms |D x| explicitly.  On this lattice
    the oracle's relaxation of each vector passes |D x| <= 4e-3 |D x0| first at
    iteration 24 (about 7e-3 at 16, 2.1e-3 to 2.4e-3 at 24), so both sides stop
    there and the bases agree to FP32 rounding; had the GPU run on to the
    100-iteration cap, or stopped at 16, they would differ by order one (0.85 and 1.4
    in this measure, oracle against oracle).  Both forms of the batched CGNR run:
    chunks of 8 iterations that keep their residuals (hist = 1) and the form with
    a direction vector (hist = 0, DWF_SMOOTHER_HISTORY=0)."""
    if not hist:
        monkeypatch.setenv("DWF_SMOOTHER_HISTORY", "0")
    c = Case(G, **SMALL, setup_iters0=100, setup_tol0=4e-3, setup_sweeps=0, smoother_prec=G.DWF_F32,
             coarse_prec=[G.DWF_F32])
    from gpu_util import to_canonical, rel_max
    nv = SMALL["nvec"][0]
    q = torch.empty(c.ctx.field_elems * nv, dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(c.ctx.h, 0, q)
    got = to_canonical(c.ctx, q, (nv,) + c.op.shape, nrhs=nv)
    ref = np.stack([c.mg.levels[0].transfer.vector(k) for k in range(nv)])
    assert rel_max(got, ref) < 1e-4
    c.close()


def test_vcycle_galerkin_orthogonality(G):
    """nu1 = nu3 = 0 and a tight coarse solve: R (b - D x) = 0 on the GPU."""
    c = Case(G, **SMALL, setup_iters0=10, setup_sweeps=0, nu_post=0, coarsest_tol=1e-12,
             coarsest_maxiter=500, coarse_restart=32)
    from gpu_util import to_internal
    b = I.gaussian_source(c.dims, c.Ls, 32)
    bt = to_internal(c.ctx, b)
    xt = torch.empty_like(bt)
    G.mg_vcycle(c.ctx.h, xt, bt)
    Dx = torch.empty_like(bt)
    G.dwf_apply(c.ctx.h, Dx, xt)
    d, n = G.mg_level_info(c.ctx.h, 1)
    r1 = torch.empty(int(np.prod(d)) * n, dtype=torch.complex128, device="cuda")
    r0 = torch.empty_like(r1)
    G.mg_restrict(c.ctx.h, 0, r1, (bt - Dx).contiguous())
    G.mg_restrict(c.ctx.h, 0, r0, bt)
    assert (r1.abs().max() / r0.abs().max()).item() < 1e-10
    c.close()


def _oracle_solution(c, b):
    x, info = OM.cgnr(c.op.apply, c.op.apply_dag, b.reshape(c.op.shape), tol=1e-13, maxiter=50000)
    assert info.converged
    return x.reshape(b.shape)


def test_solve_fp64_matches_oracle(G):
    """Plain FP64 method: same setup and solve as the oracle; solution within
    1e-8, FP64 true residual <= 1e-10, outer iterations within 2."""
    c = Case(G, **SMALL, setup_sweeps=1)
    from gpu_util import to_internal, to_canonical, rel_norm
    b = I.gaussian_source(c.dims, c.Ls, 2)
    bt = to_internal(c.ctx, b)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10)
    x = to_canonical(c.ctx, xt, b.shape)
    xo, info = OM.mg_solve(c.mg, b.reshape(c.op.shape), tol=1e-10, restart=c.p.outer_restart)
    assert st.true_res <= 1e-10
    assert rel_norm(x, _oracle_solution(c, b)) < 1e-8
    assert abs(st.iters - info.iters) <= max(2, info.iters // 20), (st.iters, info.iters)
    tr = OM.norm(b.reshape(c.op.shape) - c.op.apply(x.reshape(c.op.shape))) / OM.norm(b)
    assert tr <= 1e-10
    c.close()


@pytest.mark.parametrize("cp,bp", [(1, 1), (2, 1), (3, 1), (2, 3)], ids=["f32", "bf16", "f16", "bf16-f16basis"])
def test_solve_mixed_precision(G, cp, bp):
    """FP32 V-cycle with reduced-precision coarse stencil (and optionally an
    FP16 basis for the transfers), FP64 outer GCR with reliable updates:
    still |r|/|b| <= 1e-10 and the oracle's solution."""
    c = Case(G, **SMALL, setup_sweeps=1, smoother_prec=G.DWF_F32, coarse_prec=[cp], basis_prec=bp)
    from gpu_util import to_internal, to_canonical, rel_norm
    b = I.gaussian_source(c.dims, c.Ls, 2)
    bt = to_internal(c.ctx, b)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10)
    x = to_canonical(c.ctx, xt, b.shape)
    assert st.true_res <= 1e-10 and st.fine_applies_f32 > st.fine_applies_f64
    assert rel_norm(x, _oracle_solution(c, b)) < 1e-8
    c.close()


def test_solve_host_buffers_and_multi_rhs(G):
    """mg_solve with host (numpy) buffers, two right-hand sides."""
    c = Case(G, **SMALL, setup_sweeps=0)
    from gpu_util import to_internal
    bs = np.stack([I.gaussian_source(c.dims, c.Ls, 40 + i) for i in range(2)])
    bt = to_internal(c.ctx, bs, nrhs=2)
    bh = bt.cpu().numpy()
    xh = np.zeros_like(bh)
    st = G.mg_solve(c.ctx.h, bh, xh, 1e-10, nrhs=2)
    assert st.true_res <= 1e-10 and np.abs(xh).max() > 0
    xd = torch.zeros_like(bt)
    G.mg_solve(c.ctx.h, bt, xd, 1e-10, nrhs=2)
    assert np.linalg.norm(xd.cpu().numpy() - xh) / np.linalg.norm(xh) < 1e-9
    c.close()


def test_three_level_solve(G):
    """Recursion (Sec. 2): S2 is a V-cycle of the second coarse level."""
    c = Case(G, dims=(4, 4, 4, 8), Ls=4, mf=0.1, nvec=[8, 8], block=[(2, 2, 2, 2), (2, 2, 2, 2)],
             setup_sweeps=1, setup_iters0=20, setup_tol0=0.0)
    from gpu_util import to_internal, to_canonical, rel_norm
    b = I.gaussian_source(c.dims, c.Ls, 2)
    bt = to_internal(c.ctx, b)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10)
    assert st.true_res <= 1e-10 and st.coarse_applies[2] > 0
    x = to_canonical(c.ctx, xt, b.shape)
    assert rel_norm(x, _oracle_solution(c, b)) < 1e-8
    d, n = G.mg_level_info(c.ctx.h, 2)
    Y = torch.empty(int(np.prod(d)) * 9 * n * n, dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_links(c.ctx.h, 2, Y)
    Yref = c.mg.levels[2].op.Y.reshape(-1)
    assert np.linalg.norm(Y.cpu().numpy() - Yref) / np.linalg.norm(Yref) < 1e-6
    c.close()


def test_three_level_w_cycle(G):
    """The W-cycle of Sec. 2 (S2 on the intermediate level = two V-cycles):
    the GPU solve reaches the oracle's solution."""
    c = Case(G, dims=(4, 4, 4, 8), Ls=4, mf=0.1, nvec=[8, 8], block=[(2, 2, 2, 2), (2, 2, 2, 2)],
             setup_sweeps=0, setup_iters0=20, setup_tol0=0.0, cycle=1)
    from gpu_util import to_internal, to_canonical, rel_norm
    b = I.gaussian_source(c.dims, c.Ls, 3)
    bt = to_internal(c.ctx, b)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10)
    assert st.true_res <= 1e-10 and st.coarse_applies[2] > 0
    x = to_canonical(c.ctx, xt, b.shape)
    assert rel_norm(x, _oracle_solution(c, b)) < 1e-8
    # the oracle's W-cycle solve takes a similar number of outer iterations
    xo, info = OM.mg_solve(c.mg, b.reshape(c.op.shape), tol=1e-10)
    assert abs(info.iters - st.iters) <= max(2, info.iters // 10), (info.iters, st.iters)
    c.close()


def test_zero_source_and_bad_setup(G):
    c = Case(G, **SMALL, setup_sweeps=0)
    bt = torch.zeros(c.ctx.field_elems, dtype=torch.complex128, device="cuda")
    xt = torch.ones_like(bt)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10)
    assert st.true_res == 0.0 and xt.abs().max().item() == 0.0
    # a block that does not divide the lattice, an odd split Nvec
    with pytest.raises(G.DWFError):
        G.mg_setup(c.ctx.h, 2, [8], [(3, 2, 2, 2)])
    with pytest.raises(G.DWFError):
        G.mg_setup(c.ctx.h, 2, [6 + 1], [(2, 2, 2, 2)])
    c.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_cg_normal_equations_matches_oracle(G, prec):
    """The paper's comparison solver (CG on the squared operator) on the GPU."""
    from gpu_util import ctx_for, to_internal, to_canonical, rel_norm
    dims, Ls = (4, 4, 4, 4), 8
    U = I.epsilon_links(dims, 0.3, 1)
    ctx = ctx_for(U, dims, Ls, 1.8, 0.1)
    op = OM.FineOp(oracle.DWF(U, dims, Ls, 1.8, 0.1))
    b = I.gaussian_source(dims, Ls, 2)
    bt = to_internal(ctx, b)
    xt = torch.zeros_like(bt)
    st = G.dwf_cg_solve(ctx.h, bt, xt, 1e-10, 5000, 1, prec)
    assert st.true_res <= 1e-10
    xo, info = OM.cgnr(op.apply, op.apply_dag, b.reshape(op.shape), tol=1e-13, maxiter=50000)
    assert rel_norm(to_canonical(ctx, xt, b.shape), xo.reshape(b.shape)) < 1e-8
    if prec == 0:
        _, info10 = OM.cgnr(op.apply, op.apply_dag, b.reshape(op.shape), tol=1e-10, maxiter=50000)
        assert abs(st.iters - info10.iters) <= 16, (st.iters, info10.iters)  # GPU tests every 16
    ctx.close()


@pytest.mark.parametrize("nrhs", [3, 13])
def test_batched_solve_matches_oracle(G, nrhs):
    """Right-hand sides solved together (batched fine-level kernels, per-RHS
    GCR coefficients): each solution equals the oracle's, true residual <= 1e-10."""
    c = Case(G, **SMALL, setup_sweeps=0, smoother_prec=G.DWF_F32, coarse_prec=[G.DWF_BF16])
    from gpu_util import to_internal, to_canonical, rel_norm
    bs = np.stack([I.gaussian_source(c.dims, c.Ls, 60 + i) for i in range(nrhs)])
    bt = to_internal(c.ctx, bs, nrhs=nrhs)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10, nrhs=nrhs)
    assert st.true_res <= 1e-10
    x = to_canonical(c.ctx, xt, bs.shape, nrhs=nrhs)
    for i in (0, nrhs - 1):
        assert rel_norm(x[i], _oracle_solution(c, bs[i])) < 1e-8
    c.close()


def test_batched_solve_zero_member_and_guess(G):
    """A zero right-hand side inside a batch gets x = 0 whatever the initial
    guess; the others start from the guess and still reach the oracle's
    solutions (members leave the batch as they converge)."""
    c = Case(G, **SMALL, setup_sweeps=0, smoother_prec=G.DWF_F32, coarse_prec=[G.DWF_BF16])
    from gpu_util import to_internal, to_canonical, rel_norm
    bs = np.stack([I.gaussian_source(c.dims, c.Ls, 70 + i) for i in range(3)])
    bs[1] = 0.0
    bt = to_internal(c.ctx, bs, nrhs=3)
    xt = torch.full_like(bt, 0.25)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10, nrhs=3)
    assert st.true_res <= 1e-10
    x = to_canonical(c.ctx, xt, bs.shape, nrhs=3)
    assert np.abs(x[1]).max() == 0.0
    for i in (0, 2):
        assert rel_norm(x[i], _oracle_solution(c, bs[i])) < 1e-8
    c.close()


def test_full_size_batched_solve_sampled_residual(G):
    """16^3 x 32, Ls = 16, m_f = 0.001 with the benchmark's solver parameters
    (epsilon links instead of the heatbath ensemble, to keep host time short;
    two right-hand sides in the batched path): the FP64 true residual meets
    1e-10, and the oracle's own operator, applied to the GPU solution at 202
    sampled 5D sites (both lattice corners among them), reproduces the source
    there within that bound."""
    from gpu_util import ctx_for, to_internal
    import bench
    dims, Ls, mf = (16, 16, 16, 32), 16, 0.001
    U = I.epsilon_links(dims, 0.5, 17)
    ctx = ctx_for(U, dims, Ls, 1.8, mf)
    G.mg_setup(ctx.h, 2, [24], [(4, 4, 4, 4)], bench.mixed_params(G))
    bs = np.stack([I.gaussian_source(dims, Ls, 18 + i) for i in range(2)])
    bt = to_internal(ctx, bs, nrhs=2)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(ctx.h, bt, xt, 1e-10, nrhs=2)
    assert st.status == G.DWF_OK and st.true_res <= 1e-10
    n = ctx.field_elems
    canon = torch.empty(n, dtype=torch.complex128, device="cuda")
    G.dwf_unpack(ctx.h, canon, xt[:n].contiguous())
    torch.cuda.synchronize()
    x0 = canon.cpu().numpy().reshape(bs[0].shape)
    V = int(np.prod(dims))
    rng = np.random.default_rng(1)
    idx5 = np.concatenate([rng.integers(0, V * Ls, 200), [0, V * Ls - 1]])
    dx = oracle.DWF(U, dims, Ls, 1.8, mf).D_sites(x0, idx5).reshape(len(idx5), 12)
    b0 = bs[0].reshape(Ls * V, 12)[idx5]
    assert np.abs(dx - b0).max() <= 2e-10 * np.linalg.norm(bs[0])
    ctx.close()


# ---- the coarsened squared operator P^+ D^+ D P (Sec. 4) ------------------

SQ = dict(dims=(4, 6, 4, 4), Ls=4, mf=0.05, nvec=[8], block=[(2, 2, 2, 2)])        # coarse 2x3x2x2
SQ_ANISO = dict(dims=(4, 4, 6, 4), Ls=3, mf=0.05, nvec=[6], block=[(2, 2, 3, 2)])  # coarse 2^4


@pytest.mark.parametrize("cfg", [SQ, SQ_ANISO], ids=["2x3x2x2", "aniso"])
@pytest.mark.parametrize("sp", [0, 1], ids=["f64", "f32"])
def test_squared_coarse_operator_parity(G, cfg, sp):
    """The GPU's 33-point P^+ D^+ D P from the same start vectors equals the
    oracle's (FP64 build to rounding; FP32 products with FP64 sums to 1e-5)."""
    c = Case(G, **cfg, setup_iters0=0, setup_sweeps=0, coarsen=1, smoother_prec=sp)
    from gpu_util import rel_max
    d, n = G.mg_level_info(c.ctx.h, 1)
    Vc = int(np.prod(d))
    Y = torch.empty(Vc * 33 * n * n, dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_links(c.ctx.h, 1, Y)
    Yref = c.mg.levels[1].op.Y.reshape(Vc, 33, n, n)
    assert rel_max(Y.cpu().numpy().reshape(Vc, 33, n, n), Yref) < (1e-12 if sp == 0 else 1e-5)
    c.close()


def test_squared_coarse_apply_solve_and_vcycle(G):
    """FP64: the 33-point stencil apply (dagger ignored: Hermitian), the fused
    coarsest GCR on it and one V-cycle, each against the oracle."""
    c = Case(G, **SQ, setup_iters0=10, setup_sweeps=0, coarsen=1, coarsest_tol=1e-8, coarsest_maxiter=400,
             coarse_restart=32)
    from gpu_util import to_internal, to_canonical, rel_norm
    A = c.mg.levels[1].op
    d, n = G.mg_level_info(c.ctx.h, 1)
    cv = I.gauss_complex((int(np.prod(d)) * n,), 34, 50)
    ct = torch.from_numpy(cv).cuda()
    for dag in (0, 1):
        yt = torch.empty_like(ct)
        G.mg_coarse_apply(c.ctx.h, 1, yt, ct, dag, G.DWF_F64)
        ref = A.apply(cv.reshape(A.shape)).ravel()
        assert np.abs(yt.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    xt = torch.empty_like(ct)
    G.mg_coarse_solve(c.ctx.h, 1, xt, ct)
    res = OM.norm(cv.reshape(A.shape) - A.apply(xt.cpu().numpy().reshape(A.shape))) / OM.norm(cv)
    assert res < 2e-8, res
    b = I.gaussian_source(c.dims, c.Ls, 35)
    bt = to_internal(c.ctx, b)
    xv = torch.empty_like(bt)
    G.mg_vcycle(c.ctx.h, xv, bt)
    got = to_canonical(c.ctx, xv, b.shape)
    ref = c.mg.vcycle(0, b.reshape(c.op.shape)).reshape(b.shape)
    assert rel_norm(got, ref) < 1e-7
    c.close()


@pytest.mark.parametrize("sp,cp", [(0, 0), (1, 2)], ids=["f64", "f32-bf16"])
def test_squared_solve_matches_oracle(G, sp, cp):
    """Whole solves with the squared coarsening: FP64 (and FP32 V-cycle with
    BF16 coarse links, two right-hand sides one after another) reach the
    oracle's solution with true residual <= 1e-10."""
    c = Case(G, **SQ, setup_sweeps=0, coarsen=1, smoother_prec=sp, coarse_prec=[cp])
    from gpu_util import to_internal, to_canonical, rel_norm
    bs = np.stack([I.gaussian_source(c.dims, c.Ls, 80 + i) for i in range(2)])
    bt = to_internal(c.ctx, bs, nrhs=2)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(c.ctx.h, bt, xt, 1e-10, nrhs=2)
    assert st.true_res <= 1e-10
    x = to_canonical(c.ctx, xt, bs.shape, nrhs=2)
    for i in range(2):
        assert rel_norm(x[i], _oracle_solution(c, bs[i])) < 1e-8
    if sp == 0:
        xo, info = OM.mg_solve(c.mg, bs[0].reshape(c.op.shape), tol=1e-10, restart=c.p.outer_restart)
        assert info.converged
    c.close()


def test_squared_setup_rejects_unsupported(G):
    """Three levels, or a block of extent 1, are refused with the squared coarsening."""
    from gpu_util import ctx_for
    dims, Ls = (4, 4, 4, 4), 4
    ctx = ctx_for(I.epsilon_links(dims, 0.3, 1), dims, Ls, 1.8, 0.1)
    p = _params(G, setup_iters0=0, coarsen=1)
    with pytest.raises(G.DWFError):
        G.mg_setup(ctx.h, 3, [8, 8], [(2, 2, 2, 2), (2, 1, 1, 1)], p)
    with pytest.raises(G.DWFError):
        G.mg_setup(ctx.h, 2, [8], [(1, 2, 2, 2)], p)
    ctx.close()


def test_batched_vcycle_graphs_and_profiler(G):
    """The batched V-cycle replayed as CUDA graphs gives the solution of the
    kernel-by-kernel path, and the event profiler and application counters
    see the replayed launches: with the profiler on, both paths report the
    same fine applications, and the profiler's FP32 Dslash units (plain and
    fused-residual launches) match them."""
    from gpu_util import to_internal, to_canonical, rel_norm
    res = {}
    for graph in (0, 1):
        c = Case(G, **SMALL, setup_iters0=20, setup_sweeps=0, smoother_prec=G.DWF_F32,
                 coarse_prec=[G.DWF_BF16], graph=graph)
        bs = np.stack([I.gaussian_source(c.dims, c.Ls, 90 + i) for i in range(3)])
        bt = to_internal(c.ctx, bs, nrhs=3)
        xt = torch.zeros_like(bt)
        G.dwf_profile(c.ctx.h, True)
        st = G.mg_solve(c.ctx.h, bt, xt, 1e-10, nrhs=3)
        n32, ms32 = G.dwf_profile_read(c.ctx.h, G.K_DSLASH_F32)
        u32 = G.dwf_profile_units(c.ctx.h, G.K_DSLASH_F32)
        nz, msz = G.dwf_profile_read(c.ctx.h, G.K_DSLASH_F32_Z)
        uz = G.dwf_profile_units(c.ctx.h, G.K_DSLASH_F32_Z)
        G.dwf_profile(c.ctx.h, False)
        assert st.true_res <= 1e-10 and n32 > 0 and ms32 > 0 and nz > 0 and msz > 0
        assert u32 + uz == st.fine_applies_f32
        res[graph] = (to_canonical(c.ctx, xt, bs.shape, nrhs=3), st.iters, st.fine_applies_f32)
        c.close()
    assert rel_norm(res[1][0], res[0][0]) < 1e-8
    assert abs(res[1][1] - res[0][1]) <= 1 and abs(res[1][2] - res[0][2]) <= 2 * 20 * 3
