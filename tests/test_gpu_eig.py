"""GPU low-mode diagnostic (dwf_lowest_modes, mg_coarse_overlap) against the
oracle's dense eigensolver and its coarse-space projector on a tiny lattice."""
import numpy as np
import pytest

import oracle
from oracle import eig as E
from oracle import mg as OM
import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


def test_lowest_modes_and_overlap_match_oracle(G):
    from gpu_util import ctx_for, to_canonical
    # k + 4 vectors are iterated (oversampling speeds up the lowest k)
    dims, Ls, mf, k, ko = (2, 2, 2, 4), 4, 0.01, 4, 8
    U = I.epsilon_links(dims, 0.4, 21)
    ctx = ctx_for(U, dims, Ls, 1.8, mf)
    p = G.mg_default_params()
    p.setup_iters0 = 50
    G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p)
    vecs = torch.empty(ko * ctx.field_elems, dtype=torch.complex128, device="cuda")
    ev, res, its = G.dwf_lowest_modes(ctx.h, ko, vecs, max_iters=80, tol=1e-8)
    ev, res = ev[:k], res[:k]
    op = OM.FineOp(oracle.DWF(U, dims, Ls, 1.8, mf))
    w, V = E.lowest_modes(op, k)
    assert max(res) <= 1e-7, (res, its)
    assert np.abs(np.array(ev) - w).max() < 1e-8 * w.max(), (ev, w)
    # each GPU eigenvector is an eigenvector of the oracle's D^+ D
    got = to_canonical(ctx, vecs, (ko,) + op.shape, nrhs=ko)[:k]
    for j in range(k):
        r = op.apply_dag(op.apply(got[j])) - ev[j] * got[j]
        assert OM.norm(r) < 2e-7 * ev[j]
    # overlaps with the GPU's coarse space, recomputed by the oracle's projector
    ov = G.mg_coarse_overlap(ctx.h, 0, vecs, k)
    nv = 8
    q = torch.empty(nv * ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(ctx.h, 0, q)
    Q = to_canonical(ctx, q, (nv,) + op.shape, nrhs=nv)
    T = OM.Transfer(Q, dims, (2, 2, 2, 2))
    for j in range(k):
        assert abs(ov[j] - E.coarse_overlap(T, got[j])) < 1e-10
    assert all(0.0 <= o <= 1.0 + 1e-12 for o in ov)
    ctx.close()
