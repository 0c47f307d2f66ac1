"""Pins of the oracle's multigrid pieces: block Gram-Schmidt, R/P, the Galerkin
coarse operator, the Krylov solvers, the V-cycle and the whole solve."""
import os

import numpy as np
import pytest

import oracle
from oracle import mg as M
import paper_1205_2933_gb300.inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _op(dims=(4, 4, 4, 4), Ls=4, mf=0.1, eps=0.3, seed=1):
    return M.FineOp(oracle.DWF(I.epsilon_links(dims, eps, seed), dims, Ls, 1.8, mf))


def _vectors(op, n, seed=3):
    return I.random_vectors(n, op.dims, op.S, seed).reshape((n,) + op.shape)


def test_block_orthonormalise_against_qr():
    """Q = V R^-1 with R upper triangular, positive diagonal: equals numpy's QR
    after fixing its phases, and spans the same space."""
    rng = np.random.default_rng(0)
    Vb = rng.normal(size=(6, 5, 40)) + 1j * rng.normal(size=(6, 5, 40))
    Q = M.block_orthonormalise(Vb)
    for b in range(5):
        A = Vb[:, b, :].T                       # (40, 6) columns = vectors
        q, r = np.linalg.qr(A)
        ph = np.diag(r) / np.abs(np.diag(r))
        q = q * ph[None, :]
        assert np.abs(Q[:, b, :].T - q).max() < 1e-13
        G = Q[:, b, :].conj() @ Q[:, b, :].T
        assert np.abs(G - np.eye(6)).max() < 1e-14
        R = Q[:, b, :].conj() @ Vb[:, b, :].T      # Q^+ V, must be upper triangular
        assert np.abs(np.tril(R, -1)).max() < 1e-13
        assert np.all(np.diag(R).real > 0)


def test_block_orthonormalise_breakdown():
    Vb = np.ones((2, 3, 10), complex)
    with pytest.raises(FloatingPointError):
        M.block_orthonormalise(Vb)


def test_blocks_roundtrip_and_cover_fifth_dimension():
    op = _op((4, 4, 2, 4), 3)
    f = I.gauss_complex(op.shape, 7, 50)
    b = M.to_blocks(f, op.dims, (2, 2, 2, 2))
    assert b.shape == (2 * 2 * 1 * 2, 3 * 16 * 12)   # every block holds all Ls
    assert np.array_equal(M.from_blocks(b, 3, 12, op.dims, (2, 2, 2, 2)), f)
    # the block of site (x,y,z,t) = (3,1,0,2) is coarse site (1,0,0,1)
    g = np.zeros(op.shape, complex)
    g[1, 2, 0, 1, 3, 5] = 1.0
    hit = np.nonzero(np.abs(M.to_blocks(g, op.dims, (2, 2, 2, 2))).sum(1))[0]
    assert list(hit) == [((1 * 1 + 0) * 2 + 0) * 2 + 1]


def test_restrict_prolong_adjoint_and_RP_identity():
    """R = P^+ and R P = 1_c (Sec. 1)."""
    op = _op((4, 4, 4, 4), 4)
    T = M.Transfer(_vectors(op, 6), op.dims, (2, 2, 2, 2))
    c = I.gauss_complex(T.cshape, 8, 50)
    psi = I.gauss_complex(op.shape, 9, 50)
    assert abs(np.vdot(c, T.restrict(psi)) - np.vdot(T.prolong(c), psi)) < 1e-12 * abs(np.vdot(c, T.restrict(psi)))
    assert np.abs(T.restrict(T.prolong(c)) - c).max() < 1e-13


@pytest.mark.parametrize("dims,block,Ls,nv", [
    ((2, 2, 2, 4), (2, 2, 2, 2), 4, 4),     # coarse 1x1x1x2: +-mu reach the same site
    ((4, 4, 4, 4), (2, 2, 2, 2), 2, 4),     # coarse 2^4
    ((4, 2, 6, 4), (2, 2, 3, 2), 3, 6),     # anisotropic blocks, coarse 2x1x2x2
])
def test_coarse_operator_equals_bruteforce(dims, block, Ls, nv):
    """The 9-point stencil Y equals the dense P^+ D P built column by column."""
    op = _op(dims, Ls, 0.05, 0.5, 2)
    T = M.Transfer(_vectors(op, nv), op.dims, block)
    C = M.coarse_operator(op, T)
    dense = M.coarse_operator_bruteforce(op, T)
    Ac = M.dense_matrix(C.apply, T.cshape)
    assert np.abs(Ac - dense).max() < 1e-13 * np.abs(dense).max()
    Acd = M.dense_matrix(C.apply_dag, T.cshape)
    assert np.abs(Acd - Ac.conj().T).max() < 1e-13 * np.abs(dense).max()


def test_coarse_stencil_is_nine_point():
    expected = {}
    for line in open(os.path.join(GOLDEN, "stencil_sizes.txt")):
        if not line.startswith("#"):
            k, v = line.split()
            expected[k] = int(v)
    op = _op((8, 8, 8, 8), 2, 0.1, 0.3, 4)
    T = M.Transfer(_vectors(op, 4), op.dims, (2, 2, 2, 2))
    C = M.coarse_operator(op, T)
    c = np.zeros(T.cshape, complex)
    c[0, 1, 2, 1, 2, :] = 1.0
    out = np.abs(C.apply(c)).sum(axis=(0, -1))
    assert np.count_nonzero(out > 1e-14) == expected["coarse_sites"]


def test_split_coarse_operator_gamma_hermitian():
    """With Gamma-split vectors the coarse space is Gamma-invariant, so
    R D P inherits the gamma5-R5 hermiticity: Gc Ac Gc = Ac^+."""
    op = _op((4, 4, 4, 4), 4, 0.05, 0.5, 2)
    vecs = np.stack([h for v in _vectors(op, 3) for h in M.gamma_halves(op, v)])
    T = M.Transfer(vecs, op.dims, (2, 2, 2, 2))
    Ac = M.dense_matrix(M.coarse_operator(op, T).apply, T.cshape)
    g = np.tile(np.array([1.0, -1.0]), Ac.shape[0] // 2)
    assert np.abs(g[:, None] * Ac * g[None, :] - Ac.conj().T).max() < 1e-13 * np.abs(Ac).max()


def _dense_solution(op, b):
    D = M.dense_matrix(op.dwf.D, op.dwf.shape)
    return np.linalg.solve(D, b.ravel()).reshape(b.shape)


def test_gcr_and_cgnr_match_dense_lu():
    op = _op((2, 2, 2, 4), 4, 0.1, 0.3, 1)
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    xs = _dense_solution(op, b)
    x, info = M.gcr(op.apply, b, tol=1e-12, maxiter=3000, restart=40)
    assert info.converged and np.abs(x - xs).max() < 1e-9 * np.abs(xs).max()
    hist = np.array(info.history)
    x2, info2 = M.cgnr(op.apply, op.apply_dag, b, tol=1e-12, maxiter=5000)
    assert info2.converged and np.abs(x2 - xs).max() < 1e-9 * np.abs(xs).max()


def test_gcr_residual_monotone_within_cycle():
    op = _op((2, 2, 2, 4), 4, 0.1, 0.3, 1)
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    _, info = M.gcr(op.apply, b, tol=1e-8, maxiter=2000, restart=1000)
    h = np.array(info.history)
    assert np.all(np.diff(h) <= 1e-14)


def test_vcycle_galerkin_orthogonality():
    """nu1 = nu3 = 0 and an exact coarse solve: the V-cycle output x satisfies
    R (b - D x) = 0 (the coarse-grid correction is a Galerkin projection)."""
    op = _op((4, 4, 4, 4), 4, 0.1, 0.3, 1)
    p = M.MGParams(nvec=(8,), block=((2, 2, 2, 2),), nu_pre=0, nu_post=0, coarsest_tol=1e-14,
                   coarsest_maxiter=2000, coarse_restart=200)
    mg = M.MG(op, p)
    mg.build_from_vectors(0, _vectors(op, 4))
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    x = mg.vcycle(0, b)
    T = mg.levels[0].transfer
    assert np.abs(T.restrict(b - op.apply(x))).max() < 1e-11 * np.abs(T.restrict(b)).max()


def test_mg_solve_matches_dense_lu():
    op = _op((2, 2, 2, 4), 4, 0.1, 0.3, 1)
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    p = M.MGParams(nvec=(8,), block=((2, 2, 2, 2),), setup_sweeps=1)
    mg = M.adaptive_setup(op, p, [_vectors(op, 4)])
    x, info = M.mg_solve(mg, b, tol=1e-10)
    xs = _dense_solution(op, b)
    true_res = M.norm(b - op.apply(x)) / M.norm(b)
    assert info.converged and true_res <= 1e-10
    assert M.norm(x - xs) / M.norm(xs) < 1e-8


def test_adaptive_setup_finds_near_null_vectors():
    """Sec. 2 adaptive setup: Krylov iterations on A x = 0 leave near-null
    vectors (Rayleigh quotients |D v| / |v| far below those of the random
    start vectors); inverse-iteration sweeps with the current multigrid keep
    an orthonormal set, and the rebuilt solver converges."""
    op = _op((4, 4, 4, 4), 4, 0.05, 0.3, 1)
    rv = _vectors(op, 3)
    rq = lambda v: M.norm(op.apply(v)) / M.norm(v)
    r0 = np.mean([rq(v) for v in rv])
    p = M.MGParams(nvec=(6,), block=((2, 2, 2, 2),), setup_sweeps=0)
    v1 = M.initial_vectors(op, 3, rv, p)
    assert np.mean([rq(v) for v in v1]) < 0.25 * r0
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    p = M.MGParams(nvec=(6,), block=((2, 2, 2, 2),), setup_sweeps=2)
    mg = M.adaptive_setup(op, p, [rv])
    assert len(mg.vectors[0]) == 3
    G = np.array([[M.vdot(a, b) for b in mg.vectors[0]] for a in mg.vectors[0]])
    assert np.abs(G - np.eye(3)).max() < 1e-12
    # still a near-null set after the sweep
    assert np.mean([rq(v) for v in mg.vectors[0]]) < 0.35 * r0
    _, info = M.mg_solve(mg, b, tol=1e-8)
    assert info.converged


def test_three_level_solve():
    """Recursion (Sec. 2): S2 is itself a V-cycle on the second coarse level."""
    op = _op((4, 4, 4, 4), 4, 0.1, 0.3, 1)
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    p = M.MGParams(nvec=(8, 8), block=((2, 2, 2, 2), (2, 2, 2, 2)), setup_sweeps=1)
    rv1 = I.random_vectors(4, (2, 2, 2, 2), 1, 5).reshape(4, 1, 2, 2, 2, 2, 12)[..., :8]
    mg = M.adaptive_setup(op, p, [_vectors(op, 4), np.ascontiguousarray(rv1)])
    assert mg.nlevels == 3
    x, info = M.mg_solve(mg, b, tol=1e-10)
    assert info.converged and M.norm(b - op.apply(x)) / M.norm(b) <= 1e-10


def test_w_cycle():
    """Sec. 2: S2 replaced by two V-cycles (W-cycle).  With two levels there is
    no intermediate level and the option changes nothing; with three levels
    the W-cycle-preconditioned solve reaches the dense-LU solution."""
    op = _op((4, 4, 2, 2), 4, 0.1, 0.3, 1)
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    rv = _vectors(op, 4)
    outs = []
    for cyc in ("K", "W"):
        mg = M.adaptive_setup(op, M.MGParams(nvec=(8,), block=((2, 2, 2, 2),), cycle=cyc), [rv])
        outs.append(mg.vcycle(0, b))
    assert np.array_equal(outs[0], outs[1])
    p = M.MGParams(nvec=(8, 8), block=((2, 2, 2, 2), (2, 2, 1, 1)), cycle="W")
    rv1 = I.random_vectors(4, (2, 2, 1, 1), 1, 5).reshape(4, 1, 1, 1, 2, 2, 12)[..., :8]
    mg = M.adaptive_setup(op, p, [rv, np.ascontiguousarray(rv1)])
    assert mg.nlevels == 3
    x, info = M.mg_solve(mg, b, tol=1e-10)
    xs = _dense_solution(op, b)
    assert info.converged and M.norm(b - op.apply(x)) / M.norm(b) <= 1e-10
    assert M.norm(x - xs) / M.norm(xs) < 1e-8


# ---- the coarsened squared operator (Sec. 4) ------------------------------

@pytest.mark.parametrize("dims,block,Ls,nv", [
    ((4, 6, 4, 4), (2, 2, 2, 2), 2, 4),     # coarse 2x3x2x2: +-mu meet on the extent-2 axes
    ((8, 4, 4, 4), (2, 2, 2, 2), 2, 2),     # coarse 4x2x2x2: room for an offset of 2 in x
    ((4, 4, 6, 4), (2, 2, 3, 2), 3, 4),     # anisotropic blocks
])
def test_squared_coarse_operator_equals_bruteforce(dims, block, Ls, nv):
    """The 33-point stencil equals (D P)^+ (D P) built column by column; the
    coarse matrix is Hermitian positive definite."""
    op = _op(dims, Ls, 0.05, 0.5, 2)
    T = M.Transfer(_vectors(op, nv), op.dims, block)
    C = M.squared_coarse_operator(op, T)
    dense = M.squared_coarse_bruteforce(op, T)
    Ac = M.dense_matrix(C.apply, T.cshape)
    assert np.abs(Ac - dense).max() < 1e-13 * np.abs(dense).max()
    assert np.abs(M.dense_matrix(C.apply_dag, T.cshape) - Ac).max() < 1e-13 * np.abs(dense).max()
    assert np.linalg.eigvalsh(0.5 * (dense + dense.conj().T)).min() > 0


def test_squared_coarse_stencil_reach():
    """Sec. 4 states that the squared operator's coarse stencil reaches two
    hops.  With 2^4 blocks a coarse site couples to every site whose offset has
    components in {-1, 0, 1} with at most two of them nonzero (33 sites) and to
    no other: on a 6^4 coarse lattice exactly 33 coarse sites respond to a
    point source, and no coupling reaches an offset of 2 in any direction."""
    op = _op((12, 12, 12, 12), 1, 0.1, 0.3, 4)
    T = M.Transfer(_vectors(op, 2), op.dims, (2, 2, 2, 2))
    C = M.squared_coarse_operator(op, T)
    c = np.zeros(T.cshape, complex)
    c[0, 3, 3, 3, 3, :] = 1.0
    out = np.abs(C.apply(c)).sum(axis=(0, -1))
    hit = np.argwhere(out > 1e-14)
    assert len(hit) == 33
    d = np.abs(hit - 3)
    assert d.max() == 1 and (d > 0).sum(axis=1).max() == 2
    # brute force on a lattice with room for offset 2 along x
    op2 = _op((8, 4, 4, 4), 2, 0.1, 0.5, 5)
    T2 = M.Transfer(_vectors(op2, 2), op2.dims, (2, 2, 2, 2))
    dense = M.squared_coarse_bruteforce(op2, T2).reshape(2, 2, 2, 4, 2, 2, 2, 2, 4, 2)
    for x in range(4):
        assert np.all(dense[:, :, :, x, :, :, :, :, (x + 2) % 4, :] == 0)


def test_squared_coarse_correction_is_least_squares():
    """With the squared coarse operator the exact coarse correction
    P (P^+ D^+ D P)^-1 P^+ D^+ r minimises |r - D x| over x in range(P)
    (numpy's lstsq on the dense D P)."""
    op = _op((4, 4, 4, 4), 2, 0.1, 0.4, 6)
    T = M.Transfer(_vectors(op, 4), op.dims, (2, 2, 2, 2))
    C = M.squared_coarse_operator(op, T)
    Ac = M.dense_matrix(C.apply, T.cshape)
    r = I.gaussian_source(op.dims, op.S, 7).reshape(op.shape)
    c = np.linalg.solve(Ac, T.restrict(op.apply_dag(r)).ravel()).reshape(T.cshape)
    Nc = int(np.prod(T.cshape))
    e = np.zeros(Nc, complex)
    DP = []
    for j in range(Nc):
        e[j] = 1.0
        DP.append(op.apply(T.prolong(e.reshape(T.cshape))).ravel())
        e[j] = 0.0
    cl, *_ = np.linalg.lstsq(np.stack(DP, axis=1), r.ravel(), rcond=None)
    assert np.abs(c.ravel() - cl).max() < 1e-10 * np.abs(cl).max()


def test_squared_vcycle_and_solve():
    """nu = 0 and an exact coarse solve: P^+ D^+ (b - D x) = 0 after the
    squared coarse correction; the adaptive MG with the squared coarsening
    reaches the dense-LU solution with true residual <= 1e-10."""
    op = _op((4, 4, 4, 4), 4, 0.1, 0.3, 1)
    p = M.MGParams(nvec=(8,), block=((2, 2, 2, 2),), nu_pre=0, nu_post=0, coarsest_tol=1e-14,
                   coarsest_maxiter=2000, coarse_restart=200, coarsen="squared")
    mg = M.MG(op, p)
    mg.build_from_vectors(0, _vectors(op, 4))
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    x = mg.vcycle(0, b)
    T = mg.levels[0].transfer
    g = T.restrict(op.apply_dag(b - op.apply(x)))
    assert np.abs(g).max() < 1e-11 * np.abs(T.restrict(op.apply_dag(b))).max()
    op = _op((2, 2, 2, 4), 4, 0.1, 0.3, 1)
    b = I.gaussian_source(op.dims, op.S, 2).reshape(op.shape)
    mg = M.adaptive_setup(op, M.MGParams(nvec=(8,), block=((2, 2, 2, 2),), coarsen="squared"), [_vectors(op, 4)])
    x, info = M.mg_solve(mg, b, tol=1e-10)
    xs = _dense_solution(op, b)
    assert info.converged and M.norm(b - op.apply(x)) / M.norm(b) <= 1e-10
    assert M.norm(x - xs) / M.norm(xs) < 1e-8
    with pytest.raises(ValueError):
        M.MG(op, M.MGParams(nvec=(8,), block=((1, 2, 2, 2),), coarsen="squared")).build_from_vectors(
            0, _vectors(op, 4))
