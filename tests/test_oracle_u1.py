"""Pins of the 2D U(1) toy model (Sec. 3): the Metropolis gauge fields against
the exact plaquette of 2D U(1) gauge theory, the 2D domain-wall operator
(oracle/dwf2d.py) against momentum-space and Wilson-limit closed forms,
adjointness and gauge covariance, whole multigrid solves against dense LU,
and the paper's Fig. 2 claim on a 20^2 x 8 lattice."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment
from scipy.special import iv

from oracle import mg as M
from oracle.dwf2d import DWF2D, momentum_matrix
import paper_1205_2933_gb300.inputs as I


def _match(a, b):
    """Largest distance after pairing two multisets of complex numbers optimally."""
    d = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(d)
    return d[r, c].max()


def test_u1_plaquette_matches_exact_value():
    """2D U(1) with the Wilson action is exactly solvable: <cos theta_P> =
    I_1(beta) / I_0(beta) (up to exponentially small finite-volume terms)."""
    tr = []
    I.u1_links_2d((20, 20), 2.0, 600, 5, trace=tr)
    a = np.array(tr[100:])
    assert abs(a.mean() - iv(1, 2.0) / iv(0, 2.0)) < 0.005


@pytest.mark.parametrize("ap", [True, False])
def test_free_spectrum_from_momentum_space(ap):
    """U = 1: the eigenvalues of D are the union over momenta of those of the
    (2 Ls) x (2 Ls) momentum-space matrix."""
    dims2, Ls, M5, mf = (4, 6), 4, 1.0, 0.1
    op = DWF2D(np.zeros((2, 6, 4)), dims2, Ls, M5, mf, antiperiodic_y=ap)
    ev = np.linalg.eigvals(M.dense_matrix(op.apply, op.shape))
    shift = 0.5 if ap else 0.0
    ref = np.concatenate([np.linalg.eigvals(momentum_matrix((2 * np.pi * nx / 4, 2 * np.pi * (ny + shift) / 6),
                                                            Ls, M5, mf))
                          for nx in range(4) for ny in range(6)])
    assert _match(ev, ref) < 1e-10


def test_ls1_is_the_wilson_operator():
    """Ls = 1: D is the 2D Wilson operator with mass 1 - M5 + m_f, free-field
    eigenvalues m + sum_mu (1 - cos p_mu) +- i |sin p| (textbook)."""
    M5, mf = 0.7, 0.05
    op = DWF2D(np.zeros((2, 4, 4)), (4, 4), 1, M5, mf, antiperiodic_y=False)
    ev = np.linalg.eigvals(M.dense_matrix(op.apply, op.shape))
    ref = []
    for nx in range(4):
        for ny in range(4):
            p = (2 * np.pi * nx / 4, 2 * np.pi * ny / 4)
            re = 1 - M5 + mf + (1 - np.cos(p[0])) + (1 - np.cos(p[1]))
            im = np.sqrt(np.sin(p[0]) ** 2 + np.sin(p[1]) ** 2)
            ref += [re + 1j * im, re - 1j * im]
    assert _match(ev, np.array(ref)) < 1e-12


def test_adjoint_gauge_covariance_and_walls():
    dims2, Ls = (4, 6), 4
    th = I.u1_links_2d(dims2, 1.0, 5, 3)
    op = DWF2D(th, dims2, Ls, 1.0, 0.05)
    D = M.dense_matrix(op.apply, op.shape)
    Dd = M.dense_matrix(op.apply_dag, op.shape)
    assert np.abs(Dd - D.conj().T).max() < 1e-14             # Gamma D Gamma = D^+
    # gauge covariance: theta'_mu(x) = theta_mu(x) + a(x) - a(x + mu), psi' = e^{i a} psi
    a = 2 * np.pi * I.uniform(24, 9, I.STREAM_GAUGE_TRANSFORM).reshape(6, 4)
    th2 = np.stack([th[0] + a - np.roll(a, -1, axis=1), th[1] + a - np.roll(a, -1, axis=0)])
    op2 = DWF2D(th2, dims2, Ls, 1.0, 0.05)
    psi = I.u1_gauss_field(dims2, Ls, 1, 4)[0]
    g = np.exp(1j * a)[None, None, None, :, :, None]
    assert np.abs(op2.apply(g * psi) - g * op.apply(psi)).max() < 1e-13
    # m_f is affine and lives on the walls s = 0, Ls - 1
    d = op.apply(psi) - DWF2D(th, dims2, Ls, 1.0, 0.3).apply(psi)
    assert np.abs(d[1:Ls - 1]).max() == 0 and np.abs(d[0]).max() > 0 and np.abs(d[Ls - 1]).max() > 0


@pytest.mark.parametrize("coarsen", ["unsquared", "squared"])
def test_mg_solve_matches_dense_lu(coarsen):
    dims2, Ls = (8, 8), 4
    op = DWF2D(I.u1_links_2d(dims2, 3.0, 20, 6), dims2, Ls, 1.0, 0.05)
    b = I.u1_gauss_field(dims2, Ls, 1, 7)[0]
    rv = I.u1_gauss_field(dims2, Ls, 4, 8, I.STREAM_NULLVEC)
    mg = M.adaptive_setup(op, M.MGParams(nvec=(8,), block=((4, 4, 1, 1),), coarsen=coarsen), [rv])
    x, info = M.mg_solve(mg, b, tol=1e-10)
    xs = np.linalg.solve(M.dense_matrix(op.apply, op.shape), b.ravel()).reshape(b.shape)
    assert info.converged and M.norm(b - op.apply(x)) / M.norm(b) <= 1e-10
    assert M.norm(x - xs) / M.norm(xs) < 1e-8


def test_fig2_mass_independence():
    """Sec. 3, Fig. 2: on a 20^2 x 8 quenched U(1) lattice with 16 near-null
    vectors and 4^2 x 8 blocks, CG on the normal equations slows down as the
    mass falls while the multigrid (the paper's squared-operator coarsening)
    needs about the same number of fine applications at every mass, while the
    coarse operator itself becomes ill-conditioned as the mass falls.  Lattice:
    beta = 6, 200 Metropolis sweeps (topological charge -6), M5 = 1,
    antiperiodic in y; masses 0.10 and 0.01."""
    dims2, Ls = (20, 20), 8
    th = I.u1_links_2d(dims2, 6.0, 200, 11)
    b = I.u1_gauss_field(dims2, Ls, 1, 12)[0]
    rv = I.u1_gauss_field(dims2, Ls, 8, 13, I.STREAM_NULLVEC)
    cg, mgc, lmin = {}, {}, {}
    for mf in (0.10, 0.01):
        op = DWF2D(th, dims2, Ls, 1.0, mf)
        _, info = M.cgnr(op.apply, op.apply_dag, b, tol=1e-10, maxiter=20000)
        assert info.converged
        cg[mf] = op.count
        p = M.MGParams(nvec=(16,), block=((4, 4, 1, 1),), nu_post=4, setup_iters0=200, coarsest_tol=0.05,
                       coarsest_maxiter=200, coarse_restart=32, coarsen="squared")
        mg = M.adaptive_setup(op, p, [rv])
        op.count = 0
        x, info = M.mg_solve(mg, b, tol=1e-10, maxiter=300)
        assert info.converged and M.norm(b - op.apply(x)) / M.norm(b) <= 1e-10
        mgc[mf] = op.count - 1
        # Fig. 2 (right): the coarse level does slow down; its smallest eigenvalue falls like m_f^2
        A = mg.levels[1].op
        lmin[mf] = np.linalg.eigvalsh(M.dense_matrix(A.apply, A.shape))[0]
    assert cg[0.01] >= 1.3 * cg[0.10], cg
    assert lmin[0.01] < 0.02 * lmin[0.10], lmin
    assert mgc[0.01] <= 1.3 * mgc[0.10], mgc
    assert mgc[0.01] < 0.6 * cg[0.01], (mgc, cg)


def test_4d_embedding_reproduces_the_2d_operator():
    """The 2D toy on the four-dimensional operator: on X x 1 x 1 x Y with the
    U(1) angles on diagonal SU(3) links of charges (1, 1, -2) and unit links in
    the two extent-1 directions, those directions' hops add -2 to the
    diagonal (5 - M5 -> 3 - M5) and the 4D spectrum is, per colour, twice the
    2D spectrum for links e^{i q theta} (gamma_x, gamma_t and gamma_5 act on
    two copies of the 2D spin space, the second with sigma_3 -> -sigma_3,
    which R_5 maps back)."""
    import oracle
    dims2, Ls, M5, mf = (4, 4), 2, 1.0, 0.1
    th = I.u1_links_2d(dims2, 1.0, 5, 21)
    U, dims4 = I.embed_u1_2d(th)
    d4 = oracle.DWF(U, dims4, Ls, M5, mf)
    ev4 = np.linalg.eigvals(M.dense_matrix(d4.D, d4.shape))
    ref = []
    for q in (1, 1, -2):
        op = DWF2D(q * th, dims2, Ls, M5, mf)
        e = np.linalg.eigvals(M.dense_matrix(op.apply, op.shape))
        ref += [e, e]
    assert _match(ev4, np.concatenate(ref)) < 1e-10


def test_squared_coarsening_of_the_embedded_toy():
    """On the embedded lattice X x 1 x 1 x Y the hops along the extent-1
    directions stay on the site: the squared coarse stencil (blocks of extent
    1 there) still equals (D P)^+ (D P) by brute force, and the multigrid
    with it reaches the dense-LU solution."""
    import oracle
    dims2, Ls = (8, 8), 2
    U, dims4 = I.embed_u1_2d(I.u1_links_2d(dims2, 3.0, 20, 31))
    op = M.FineOp(oracle.DWF(U, dims4, Ls, 1.0, 0.05))
    rv = I.random_vectors(2, dims4, Ls, 32).reshape((2,) + op.shape)
    vecs = np.stack([h for v in rv for h in M.gamma_halves(op, v)])
    T = M.Transfer(vecs, op.dims, (4, 1, 1, 4))
    C = M.squared_coarse_operator(op, T)
    dense = M.squared_coarse_bruteforce(op, T)
    assert np.abs(M.dense_matrix(C.apply, T.cshape) - dense).max() < 1e-13 * np.abs(dense).max()
    b = I.gaussian_source(dims4, Ls, 33).reshape(op.shape)
    mg = M.adaptive_setup(op, M.MGParams(nvec=(8,), block=((4, 1, 1, 4),), coarsen="squared"),
                          [I.random_vectors(4, dims4, Ls, 34).reshape((4,) + op.shape)])
    x, info = M.mg_solve(mg, b, tol=1e-10)
    xs = np.linalg.solve(M.dense_matrix(op.apply, op.shape), b.ravel()).reshape(b.shape)
    assert info.converged and M.norm(x - xs) / M.norm(xs) < 1e-8
