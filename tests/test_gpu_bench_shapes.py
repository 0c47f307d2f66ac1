"""GPU parity at the benchmark's multigrid shapes: Nvec = 24 (12 adaptive
vectors, Gamma-split), 4^4 blocks collapsing Ls = 16, BF16 coarse links,
FP32 V-cycle, 12 right-hand sides in the batched path (the instantiations the
benchmark times), on an 8^4 heatbath lattice (beta = 6.0, 200 sweeps) with
the benchmark's m_f = 0.001, so that the coarse lattice is 2^4.

The BF16 coarse stencil is compared twice: with the FP64 oracle (within the
BF16 rounding of the links, 1e-2) and with the oracle run on the same links
rounded the way the library stores them (FP64 -> FP32 -> BF16, both steps
round-to-nearest-even), where only FP32 vector arithmetic separates the two."""
import numpy as np
import pytest

import oracle
from oracle import mg as OM
import paper_1205_2933_gb300.inputs as I
import test_gpu_mg as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HB8 = dict(dims=(8, 8, 8, 8), Ls=16, mf=0.001, nvec=[24], block=[(4, 4, 4, 4)], hb=True, hb_sweeps=200,
           seed=5)


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


def bf16_round(a):
    """Complex128 -> FP32 -> BF16 (round to nearest even at each step), back to complex128."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).astype(np.complex64)).view(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).view(np.complex64).astype(np.complex128).reshape(np.shape(a))


def test_bf16_round_helper():
    # exact halfway cases go to even; FP32 rounding happens first
    x = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -30], dtype=np.float64)
    got = bf16_round(x + 0j).real
    assert got[0] == 1.0 and got[1] == 1.0 + 2 * 2.0 ** -7 and got[2] == 1.0  # 2^-30 lost in FP32
    assert bf16_round(np.array([-1.5 + 0.25j]))[0] == -1.5 + 0.25j


@pytest.fixture(scope="module")
def case(G):
    c = M.Case(G, **HB8, setup_iters0=0, setup_sweeps=0, smoother_prec=G.DWF_F32,
               coarse_prec=[G.DWF_BF16], coarsest_tol=0.0, coarsest_maxiter=8)
    yield c
    c.close()


def test_basis_and_coarse_links_nvec24(G, case):
    c = case
    from gpu_util import to_canonical, rel_max
    nv = 24
    q = torch.empty(c.ctx.field_elems * nv, dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(c.ctx.h, 0, q)
    got = to_canonical(c.ctx, q, (nv,) + c.op.shape, nrhs=nv)
    T = c.mg.levels[0].transfer
    ref = np.stack([T.vector(k) for k in range(nv)])
    # the FP32 V-cycle's setup orthonormalises FP32 copies of the vectors (FP64 sums)
    assert rel_max(got, ref) < 1e-6
    del q, got
    d, n = G.mg_level_info(c.ctx.h, 1)
    assert tuple(d) == (2, 2, 2, 2) and n == 24
    Y = torch.empty(16 * 9 * n * n, dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_links(c.ctx.h, 1, Y)
    Yref = c.mg.levels[1].op.Y.reshape(16, 9, n, n)
    # FP32 products with FP64 sums (FP32 V-cycle setup)
    assert rel_max(Y.cpu().numpy().reshape(16, 9, n, n), Yref) < 1e-5


def _rounded_coarse_op(c):
    A = c.mg.levels[1].op
    return OM.CoarseOp(bf16_round(A.Y), A.dims)


def test_bf16_coarse_apply_nvec24(G, case):
    c = case
    A = c.mg.levels[1].op
    Ab = _rounded_coarse_op(c)
    cin = I.gauss_complex((16 * 24,), 23, 50)
    ct = torch.from_numpy(cin.astype(np.complex64)).cuda()
    for dag in (False, True):
        yo = torch.empty_like(ct)
        G.mg_coarse_apply(c.ctx.h, 1, yo, ct, dag, G.DWF_F32)
        got = yo.cpu().numpy().astype(np.complex128)
        x32 = cin.astype(np.complex64).astype(np.complex128).reshape(A.shape)
        refb = (Ab.apply_dag if dag else Ab.apply)(x32).ravel()
        ref = (A.apply_dag if dag else A.apply)(cin.reshape(A.shape)).ravel()
        assert np.linalg.norm(got - refb) / np.linalg.norm(refb) < 1e-5
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-2


@pytest.mark.parametrize("nu_post", [0, 4])
def test_vcycle_batch_12_rhs_nvec24(G, case, nu_post):
    """The batched V-cycle of 12 right-hand sides (batched restriction and
    prolongation with Nvec = 24, the batched BF16 coarsest GCR with 8 fixed
    iterations, nu_post CGNR post-smoothing steps) against the oracle's
    V-cycle of each right-hand side on the BF16-rounded coarse operator."""
    c = case
    from gpu_util import to_internal, to_canonical, rel_norm
    import dataclasses
    G.mg_setup(c.ctx.h, 2, [24], [(4, 4, 4, 4)], M._params(G, setup_iters0=0, setup_sweeps=0,
               smoother_prec=G.DWF_F32, coarse_prec=[G.DWF_BF16], coarsest_tol=0.0, coarsest_maxiter=8,
               nu_post=nu_post), torch.from_numpy(c.start).cuda())
    mg = c.mg
    mg.p = dataclasses.replace(mg.p, nu_post=nu_post, coarsest_tol=0.0, coarsest_maxiter=8)
    saved = mg.levels[1].op
    mg.levels[1].op = _rounded_coarse_op(c)
    try:
        nr = 12
        bs = np.stack([I.gaussian_source(c.dims, c.Ls, 500 + r) for r in range(nr)])
        bt = to_internal(c.ctx, bs, nrhs=nr)
        xb = torch.empty_like(bt)
        G.mg_vcycle_batch(c.ctx.h, xb, bt, nr)
        got = to_canonical(c.ctx, xb, bs.shape, nrhs=nr)
        # The tensor-core stencil multiplies the BF16 links by the FP32 vectors split
        # into two BF16 parts, exact to 2^-16 relatively per apply; 8 FP32 GCR
        # iterations on the coarse level carry that to ~1e-4 in the coarse solution,
        # which the V-cycle returns as it is when nothing smooths after it.
        tol = 1e-3 if nu_post == 0 else 1e-4
        for r in range(nr):
            ref = mg.vcycle(0, bs[r].reshape(c.op.shape)).reshape(bs[r].shape)
            e = rel_norm(got[r], ref)
            assert e < tol, (r, e)
    finally:
        mg.levels[1].op = saved


def test_batched_solve_12_rhs_bench_parameters(G):
    """The benchmark's solver parameters (600 setup iterations, 16 CGNR
    post-smoothing steps, coarsest GCR to 0.03, BF16 links) on the 8^4 x 16
    heatbath lattice with 12 right-hand sides: the oracle's FP64 operator
    applied to every returned solution reproduces its source to 1e-10."""
    import bench
    from gpu_util import ctx_for, to_internal, to_canonical
    dims, Ls, mf = (8, 8, 8, 8), 16, 0.001
    U = I.heatbath_links(dims, 6.0, 200, 5)
    ctx = ctx_for(U, dims, Ls, 1.8, mf)
    G.mg_setup(ctx.h, 2, [24], [(4, 4, 4, 4)], bench.mixed_params(G))
    nr = 12
    bs = np.stack([I.gaussian_source(dims, Ls, 600 + r) for r in range(nr)])
    bt = to_internal(ctx, bs, nrhs=nr)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(ctx.h, bt, xt, 1e-10, nrhs=nr)
    assert st.status == G.DWF_OK and st.true_res <= 1e-10
    x = to_canonical(ctx, xt, bs.shape, nrhs=nr)
    D = oracle.DWF(U, dims, Ls, 1.8, mf)
    for r in range(nr):
        res = np.linalg.norm(bs[r] - D.D(x[r])) / np.linalg.norm(bs[r])
        assert res <= 1.0001e-10, (r, res)
    ctx.close()


@pytest.mark.parametrize("nvec", [16, 32])
def test_vcycle_batch_tensor_core_other_nvec(G, nvec):
    """The tensor-core coarsest solver's other instantiations (Nvec 16 and 32,
    one and two 8-row groups more than Nvec 8 and 24): the batched V-cycle of
    five right-hand sides (padded to eight tensor-core columns per part)
    against the oracle's V-cycle on the BF16-rounded coarse operator."""
    from gpu_util import to_internal, to_canonical, rel_norm
    c = M.Case(G, dims=(4, 4, 4, 4), Ls=8, mf=0.1, nvec=[nvec], block=[(2, 2, 2, 2)], setup_iters0=10,
               setup_sweeps=0, smoother_prec=G.DWF_F32, coarse_prec=[G.DWF_BF16], coarsest_tol=0.0,
               coarsest_maxiter=8, nu_post=4)
    mg = c.mg
    mg.levels[1].op = _rounded_coarse_op(c)  # the oracle's operator with the library's BF16 rounding
    nr = 5
    bs = np.stack([I.gaussian_source(c.dims, c.Ls, 700 + r) for r in range(nr)])
    bt = to_internal(c.ctx, bs, nrhs=nr)
    xb = torch.empty_like(bt)
    G.mg_vcycle_batch(c.ctx.h, xb, bt, nr)
    got = to_canonical(c.ctx, xb, bs.shape, nrhs=nr)
    for r in range(nr):
        ref = mg.vcycle(0, bs[r].reshape(c.op.shape)).reshape(bs[r].shape)
        e = rel_norm(got[r], ref)
        assert e < 1e-4, (r, e)
    c.close()
