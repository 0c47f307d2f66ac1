"""The 2D U(1) toy of Sec. 3 on the GPU through the library's 4D operator:
X x 1 x 1 x Y lattices carrying the U(1) angles on diagonal SU(3) links of
charges (1, 1, -2) (the embedding pinned on the CPU against the 2D operator).
The coarse operators of both coarsenings (R D P and the squared operator's
P^+ D^+ D P, whose construction treats the hops along the two extent-1
directions as block-internal) must equal the oracle's, and whole solves on
the paper's 20^2 x 8 lattice must reach the oracle's solution."""
import numpy as np
import pytest

import oracle
from oracle import mg as OM
import paper_1205_2933_gb300.inputs as I
import test_gpu_mg as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

M5 = 1.0  # the toy's domain-wall height (3 - M5 on the 2D diagonal)


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


def _embedded(dims2, beta, sweeps, seed):
    U, dims4 = I.embed_u1_2d(I.u1_links_2d(dims2, beta, sweeps, seed))
    assert dims4 == (dims2[0], 1, 1, dims2[1])
    return U, dims4


@pytest.mark.parametrize("sp", [0, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("coarsen", [0, 1], ids=["rdp", "squared"])
def test_embedded_coarse_operator_parity(G, coarsen, sp):
    """FP64 construction to rounding; with the FP32 V-cycle (FP32 products,
    FP64 sums) to 1e-5, as on the 4D lattices."""
    from gpu_util import ctx_for, rel_max
    U, dims4 = _embedded((8, 8), 3.0, 20, 31)
    Ls, mf, nvec, block = 4, 0.05, 8, (4, 1, 1, 4)
    ctx = ctx_for(U, dims4, Ls, M5, mf)
    op = OM.FineOp(oracle.DWF(U, dims4, Ls, M5, mf))
    rv = I.random_vectors(nvec // 2, dims4, Ls, 32)
    p = M._params(G, setup_iters0=0, setup_sweeps=0, coarsen=coarsen, smoother_prec=sp)
    G.mg_setup(ctx.h, 2, [nvec], [block], p, torch.from_numpy(rv).cuda())
    mg = OM.adaptive_setup(op, M._oracle_params([nvec], [block], p), [rv.reshape((nvec // 2,) + op.shape)])
    d, n = G.mg_level_info(ctx.h, 1)
    assert tuple(d) == (2, 1, 1, 2)
    npts = 33 if coarsen else 9
    Y = torch.empty(4 * npts * n * n, dtype=torch.complex128, device="cuda")
    G.mg_get_coarse_links(ctx.h, 1, Y)
    Yref = mg.levels[1].op.Y.reshape(4, npts, n, n)
    assert rel_max(Y.cpu().numpy().reshape(4, npts, n, n), Yref) < (1e-12 if sp == 0 else 1e-5)
    ctx.close()


@pytest.mark.parametrize("coarsen,seed", [(0, 31), (1, 11)], ids=["rdp-Q0", "squared-Q-6"])
def test_embedded_20x20_solve_matches_oracle(G, coarsen, seed):
    """The paper's 20^2 x 8 lattice (beta = 6, 200 Metropolis sweeps), m_f =
    0.1, 24 coarse components on 4 x 1 x 1 x 4 blocks (4^2 x 8 in the toy's
    own coordinates), FP64: the GPU solution equals the oracle's to 1e-8 with
    true residual <= 1e-10.  The squared coarsening runs on the field of
    topological charge -6 (seed 11); the unsquared one, which the near-zero
    modes of that field defeat, on the charge-0 field of seed 31."""
    from gpu_util import ctx_for, to_internal, to_canonical, rel_norm
    U, dims4 = _embedded((20, 20), 6.0, 200, seed)
    Ls, mf = 8, 0.10
    ctx = ctx_for(U, dims4, Ls, M5, mf)
    p = M._params(G, coarsen=coarsen, nu_post=4, setup_iters0=200, coarsest_tol=0.05, coarsest_maxiter=200,
                  coarse_restart=32, outer_maxiter=1000)
    G.mg_setup(ctx.h, 2, [24], [(4, 1, 1, 4)], p)
    b = I.gaussian_source(dims4, Ls, 12)
    bt = to_internal(ctx, b)
    xt = torch.zeros_like(bt)
    st = G.mg_solve(ctx.h, bt, xt, 1e-10)
    assert st.status == G.DWF_OK and st.true_res <= 1e-10
    op = OM.FineOp(oracle.DWF(U, dims4, Ls, M5, mf))
    xo, info = OM.cgnr(op.apply, op.apply_dag, b.reshape(op.shape), tol=1e-13, maxiter=50000)
    assert info.converged
    assert rel_norm(to_canonical(ctx, xt, b.shape), xo.reshape(b.shape)) < 1e-8
    ctx.close()
