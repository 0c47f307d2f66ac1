"""A batch of independent lattices of uneven size behind one context
(dwf_create with nlat > 1): fields hold the lattices one after another, the
fine operator, the layout conversions, the setup and the solve run over all
of them in one call, and every lattice's result must equal the oracle's
(and that of a context holding the lattice alone)."""
import numpy as np
import pytest

import oracle
from oracle import mg as OM
import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

M5 = 1.8


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


def _batch(G, dims_list, Ls, mf, links):
    return G.BatchContext(dims_list, Ls, M5, mf, [torch.from_numpy(u).cuda() for u in links])


def _pack(G, bc, fields, prec=0):
    """canonical numpy fields (one per lattice, each shape (nrhs, ...)) -> batch internal tensor"""
    canon = torch.from_numpy(np.concatenate([f.reshape(-1) for f in fields])).cuda()
    dt = torch.complex128 if prec == 0 else torch.complex64
    nrhs = fields[0].shape[0]
    out = torch.empty(bc.field_elems() * nrhs, dtype=dt, device="cuda")
    G.dwf_pack(bc.h, out, canon, prec, nrhs)
    return out


def _unpack(G, bc, t, nrhs):
    out = torch.empty(bc.field_elems() * nrhs, dtype=torch.complex128, device="cuda")
    G.dwf_unpack(bc.h, out, t, 0, nrhs)
    torch.cuda.synchronize()
    a = out.cpu().numpy()
    res, o = [], 0
    for i, d in enumerate(bc.dims):
        n = bc.field_elems(i) * nrhs
        res.append(a[o:o + n].reshape((nrhs, bc.Ls, d[3], d[2], d[1], d[0], 4, 3)))
        o += n
    return res


DIMS3 = [(4, 4, 4, 4), (4, 4, 4, 8), (8, 4, 4, 4)]


def test_batch_apply_and_layout(G):
    Ls, mf = 8, 0.1
    links = [I.epsilon_links(d, 0.3, 11 + i) for i, d in enumerate(DIMS3)]
    bc = _batch(G, DIMS3, Ls, mf, links)
    nrhs = 2
    fs = [np.stack([I.gaussian_source(d, Ls, 20 + 2 * i + r) for r in range(nrhs)]) for i, d in enumerate(DIMS3)]
    t = _pack(G, bc, fs)
    back = _unpack(G, bc, t, nrhs)
    for i in range(3):
        assert np.array_equal(back[i], fs[i])
    out = torch.empty_like(t)
    G.dwf_apply(bc.h, out, t, G.DWF_F64, False, nrhs)
    got = _unpack(G, bc, out, nrhs)
    for i, d in enumerate(DIMS3):
        D = oracle.DWF(links[i], d, Ls, M5, mf)
        for r in range(nrhs):
            ref = D.D(fs[i][r])
            assert np.abs(got[i][r] - ref).max() <= 1e-13 * np.abs(ref).max()
    # per-lattice calls go through dwf_lattice; batch-wide component calls are refused
    h1 = bc.lattice(1)
    assert G.lib().mg_level_info(bc.h, 0, (G.ctypes.c_int * 4)(), G.ctypes.byref(G.ctypes.c_int())) == G.DWF_EINVAL
    with pytest.raises(G.DWFError):
        bc.lattice(3)
    assert h1.value is not None
    bc.close()


@pytest.mark.parametrize("sp,cp", [(0, 0), (1, 2)], ids=["f64", "f32-bf16"])
def test_batch_solve_matches_oracle_and_single(G, sp, cp):
    """Three uneven lattices, two right-hand sides each, in one mg_setup and
    one mg_solve: every solution equals the oracle's to 1e-8 (true residual
    <= 1e-10) and, to the same bound, the solution of the lattice solved in a
    context of its own (FP64: to 1e-10; with the FP32 V-cycle the two contexts
    may time their tensor-core coarse solvers onto different grids, whose
    reduction orders differ in rounding)."""
    from gpu_util import ctx_for, to_internal, to_canonical, rel_norm
    Ls, mf, nrhs = 8, 0.1, 2
    links = [I.epsilon_links(d, 0.3, 11 + i) for i, d in enumerate(DIMS3)]
    bc = _batch(G, DIMS3, Ls, mf, links)
    p = G.mg_default_params()
    p.smoother_prec = sp
    p.coarse_prec[0] = cp
    p.setup_iters0 = 50
    G.mg_setup(bc.h, 2, [8], [(2, 2, 2, 2)], p)
    bs = [np.stack([I.gaussian_source(d, Ls, 40 + 2 * i + r) for r in range(nrhs)]) for i, d in enumerate(DIMS3)]
    bt = _pack(G, bc, bs)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(bc.h, bt, xt, 1e-10, nrhs=nrhs)
    assert st.status == G.DWF_OK and st.true_res <= 1e-10
    xs = _unpack(G, bc, xt, nrhs)
    for i, d in enumerate(DIMS3):
        op = OM.FineOp(oracle.DWF(links[i], d, Ls, M5, mf))
        ctx = ctx_for(links[i], d, Ls, M5, mf)
        G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p)
        b1 = to_internal(ctx, bs[i], nrhs=nrhs)
        x1 = torch.zeros_like(b1)
        G.mg_solve(ctx.h, b1, x1, 1e-10, nrhs=nrhs)
        x1c = to_canonical(ctx, x1, bs[i].shape, nrhs=nrhs)
        for r in range(nrhs):
            xo, info = OM.cgnr(op.apply, op.apply_dag, bs[i][r].reshape(op.shape), tol=1e-13, maxiter=50000)
            assert rel_norm(xs[i][r], xo.reshape(bs[i][r].shape)) < 1e-8
            assert rel_norm(xs[i][r], x1c[r]) < (1e-10 if sp == 0 else 1e-8)
        ctx.close()
    bc.close()


def test_batch_uneven_heatbath_ls16(G):
    """8^4 and 12^3 x 24 at Ls = 16, m_f = 0.002, heatbath beta = 5.9 (20
    sweeps), mixed precision with the bench's Nvec = 24 and 4^4 blocks, one
    right-hand side per lattice in one call: the oracle's FP64 operator
    applied to each returned solution reproduces its source to 1e-10."""
    import bench
    Ls, mf = 16, 0.002
    dims = [(8, 8, 8, 8), (12, 12, 12, 24)]
    links = [I.heatbath_links(d, 5.9, 20, 300 + i) for i, d in enumerate(dims)]
    bc = _batch(G, dims, Ls, mf, links)
    p = bench.mixed_params(G)
    p.setup_iters0 = 300
    G.mg_setup(bc.h, 2, [24], [(4, 4, 4, 4)], p)
    bs = [I.gaussian_source(d, Ls, 310 + i)[None] for i, d in enumerate(dims)]
    bt = _pack(G, bc, bs)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(bc.h, bt, xt, 1e-10, nrhs=1)
    assert st.status == G.DWF_OK and st.true_res <= 1e-10
    xs = _unpack(G, bc, xt, 1)
    for i, d in enumerate(dims):
        D = oracle.DWF(links[i], d, Ls, M5, mf)
        res = np.linalg.norm(bs[i][0] - D.D(xs[i][0])) / np.linalg.norm(bs[i][0])
        assert res <= 1.0001e-10, (i, res)
    bc.close()
