"""Pins of the oracle's fine operator D (and D^+) against what the physics fixes.

The paper names the operator (Shamir domain-wall fermions with fifth
dimension Ls, Sec. 2) and its stencil (Sec. 4) but does not write it out;
these tests pin the oracle's D by properties that do not restate its code:
the free-field momentum-space form, the known smallest singular value at
zero momentum, the Ls = 1 Wilson limit, gamma5-R5 hermiticity, gauge
covariance, the stencil size and the placement of the quark mass.
"""
import os

import numpy as np
import pytest

import oracle
import paper_1205_2933_gb300.inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gamma_algebra():
    g = [oracle.gamma(m) for m in range(4)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * np.eye(4) * (a == b))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def _plane_wave_matrix(dims, Ls, M5, mf, p, ap):
    """Apply the oracle's D (unit links) to e^{ip.x} chi for every (s, spin) basis
    vector chi and read the result at the origin: the 4Ls x 4Ls symbol D(p)."""
    U = I.unit_links(dims)
    dwf = oracle.DWF(U, dims, Ls, M5, mf, antiperiodic_t=ap)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    M = np.zeros((Ls * 4, Ls * 4), dtype=complex)
    for s in range(Ls):
        for a in range(4):
            f = np.zeros(dwf.shape, dtype=complex)
            f[s, ..., a, 0] = phase
            out = dwf.D(f)
            # D psi must again be a plane wave with the same momentum
            assert np.allclose(out[..., 0] / phase[None, ..., None], out[:, 0, 0, 0, 0, :, 0][:, None, None, None, None, :])
            assert np.abs(out[..., 1:]).max() == 0
            M[:, s * 4 + a] = out[:, 0, 0, 0, 0, :, 0].reshape(-1)
    return M


def _symbol(Ls, M5, mf, p):
    """Momentum-space form: [(5-M5) - sum cos p + i sum gamma_mu sin p] x 1_s plus the
    fifth-dimension hops -P_- (s->s+1), -P_+ (s->s-1) with +mf wrap-around."""
    g = [oracle.gamma(m) for m in range(4)]
    d4 = (5 - M5 - sum(np.cos(p))) * np.eye(4) + 1j * sum(g[m] * np.sin(p[m]) for m in range(4))
    Pp, Pm = np.diag([1, 1, 0, 0]), np.diag([0, 0, 1, 1])
    M = np.kron(np.eye(Ls), d4)
    for s in range(Ls):
        up = (s + 1) % Ls
        dn = (s - 1) % Ls
        cu = mf if s == Ls - 1 else -1.0
        cd = mf if s == 0 else -1.0
        M[s * 4:(s + 1) * 4, up * 4:(up + 1) * 4] += cu * Pm
        M[s * 4:(s + 1) * 4, dn * 4:(dn + 1) * 4] += cd * Pp
    return M


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 3), (2, 2, 0, 0)])
def test_free_field_plane_waves(n):
    dims = (4, 3, 4, 6)
    Ls, M5, mf = 4, 1.8, 0.05
    p = [2 * np.pi * n[m] / dims[m] for m in range(3)] + [2 * np.pi * (n[3] + 0.5) / dims[3]]
    M = _plane_wave_matrix(dims, Ls, M5, mf, p, True)
    assert np.abs(M - _symbol(Ls, M5, mf, p)).max() < 1e-13


def test_free_field_spectrum_union_over_momenta():
    """Full spectrum on a tiny free lattice = union over momenta of eig D(p), x3 colours."""
    dims, Ls, M5, mf = (2, 2, 2, 2), 2, 1.8, 0.1
    dwf = oracle.DWF(I.unit_links(dims), dims, Ls, M5, mf, antiperiodic_t=True)
    from oracle.mg import dense_matrix
    D = dense_matrix(dwf.D, dwf.shape)
    ev = np.linalg.eigvals(D)
    ref = []
    for nx in range(2):
        for ny in range(2):
            for nz in range(2):
                for nt in range(2):
                    p = [np.pi * nx, np.pi * ny, np.pi * nz, np.pi * (nt + 0.5)]
                    ref += list(np.linalg.eigvals(_symbol(Ls, M5, mf, p))) * 3
    ref = np.array(ref)
    # match every eigenvalue to its nearest reference (multisets agree)
    used = np.zeros(ref.size, bool)
    for e in ev:
        d = np.abs(ref - e) + used * 1e9
        k = np.argmin(d)
        assert d[k] < 1e-10
        used[k] = True


@pytest.mark.parametrize("mf", [0.001, 0.01])
def test_zero_momentum_smallest_singular_value(mf):
    """At p = 0 (periodic t) the light domain-wall mode has singular value
    ~ (1 - w0^2)(mf + |w0|^Ls), w0 = 1 - M5 (large-Ls asymptotics of the
    Shamir operator); at Ls = 16, M5 = 1.8 the two agree to about 0.5%."""
    Ls, M5 = 16, 1.8
    M = _plane_wave_matrix((2, 2, 2, 2), Ls, M5, mf, [0, 0, 0, 0], False)
    smin = np.linalg.svd(M, compute_uv=False).min()
    w0 = 1 - M5
    pred = (1 - w0 ** 2) * (mf + abs(w0) ** Ls)
    assert abs(smin / pred - 1) < 0.015, (smin, pred)


def test_ls1_is_wilson():
    """Ls = 1: D is the Wilson operator with mass m = 1 - M5 + mf, whose free
    eigenvalues are m + sum(1 - cos p) +- i |sin p| (textbook)."""
    M5, mf = 1.3, 0.2
    m = 1 - M5 + mf
    for n in [(0, 0, 0, 0), (1, 2, 0, 1), (3, 1, 2, 2)]:
        dims = (4, 4, 4, 4)
        p = np.array([2 * np.pi * n[k] / 4 for k in range(3)] + [2 * np.pi * (n[3] + 0.5) / 4])
        ev = np.linalg.eigvals(_plane_wave_matrix(dims, 1, M5, mf, p, True))
        ev = ev[np.argsort(ev.imag)]
        re = m + np.sum(1 - np.cos(p))
        im = np.sqrt(np.sum(np.sin(p) ** 2))
        ref = np.array([re - 1j * im, re - 1j * im, re + 1j * im, re + 1j * im])
        assert np.abs(ev - ref).max() < 1e-12


def _rand_op(dims=(4, 4, 2, 4), Ls=6, mf=0.07, seed=3):
    U = I.epsilon_links(dims, 0.6, seed)
    return oracle.DWF(U, dims, Ls, 1.8, mf)


def test_gamma5_r5_hermiticity_and_adjoint():
    """<chi, D psi> = <D^+ chi, psi> with D^+ = gamma5 R5 D gamma5 R5."""
    dwf = _rand_op()
    psi = I.gauss_complex(dwf.shape, 1, 50)
    chi = I.gauss_complex(dwf.shape, 2, 50)
    lhs = np.vdot(chi, dwf.D(psi))
    rhs = np.vdot(dwf.Ddag(chi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_dense_adjoint_tiny():
    dwf = _rand_op((2, 2, 2, 2), 2, 0.3, 9)
    from oracle.mg import dense_matrix
    D = dense_matrix(dwf.D, dwf.shape)
    Dd = dense_matrix(dwf.Ddag, dwf.shape)
    assert np.abs(Dd - D.conj().T).max() < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    dwf = _rand_op(dims)
    g = I.random_gauge_transform(dims, 4)                     # (T,Z,Y,X,3,3)
    U = dwf.U
    Ug = np.empty_like(U)
    for mu in range(4):
        gp = np.roll(g, -1, axis=3 - mu)                      # g(x + mu)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    dwfg = oracle.DWF(Ug, dims, dwf.Ls, dwf.M5, dwf.mf)
    psi = I.gauss_complex(dwf.shape, 3, 50)
    gpsi = np.einsum("tzyxab,stzyxsb->stzyxsa".replace("sb", "qb").replace("sa", "qa"), g, psi)
    lhs = dwfg.D(gpsi)
    rhs = np.einsum("tzyxab,stzyxqb->stzyxqa", g, dwf.D(psi))
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


def test_mass_term_affine_and_on_walls():
    """D(m1) - D(m0) = (m1 - m0) [P_- psi(s=0) at s = Ls-1, P_+ psi(s=Ls-1) at s = 0]."""
    dims = (2, 2, 2, 4)
    a = _rand_op(dims, 5, 0.0)
    b = oracle.DWF(a.U, dims, 5, 1.8, 0.25)
    psi = I.gauss_complex(a.shape, 4, 50)
    d = b.D(psi) - a.D(psi)
    assert np.abs(d[1:4]).max() < 1e-14
    assert np.abs(d[0, ..., :2, :] - 0.25 * psi[4, ..., :2, :]).max() < 1e-14
    assert np.abs(d[0, ..., 2:, :]).max() < 1e-14
    assert np.abs(d[4, ..., 2:, :] - 0.25 * psi[0, ..., 2:, :]).max() < 1e-14
    assert np.abs(d[4, ..., :2, :]).max() < 1e-14


def test_stencil_size():
    """Sec. 4: a fine site couples to itself and its 10 unit-distance neighbours in 5D."""
    expected = {}
    for line in open(os.path.join(GOLDEN, "stencil_sizes.txt")):
        if not line.startswith("#"):
            k, v = line.split()
            expected[k] = int(v)
    dwf = _rand_op((4, 4, 4, 4), 6, 0.1)
    # column of D: sites whose output depends on the input site (s=2, x=(1,2,1,2))
    f = np.zeros(dwf.shape, complex)
    f[2, 2, 1, 2, 1, 0, 0] = 1.0
    f[2, 2, 1, 2, 1, 2, 1] = 1.0
    out = np.abs(dwf.D(f)).sum(axis=(-1, -2))
    assert np.count_nonzero(out > 1e-15) == expected["fine_sites"]


def test_sites_and_hops_consistent():
    dwf = _rand_op()
    psi = I.gauss_complex(dwf.shape, 5, 50)
    full = dwf.D(psi)
    V = int(np.prod(dwf.dims))
    idx = np.array([0, 7, V + 3, 5 * V + V - 1])
    got = dwf.D_sites(psi, idx)
    flat = full.reshape(dwf.Ls * V, 4, 3)
    assert np.abs(got - flat[idx]).max() < 1e-15
    # D minus its 8 hopping terms couples no two different 4D sites
    rest = full - sum(dwf.hop(psi, mu, d) for mu in range(4) for d in (1, -1))
    psi2 = psi.copy()
    psi2[:, 1, 1, 2, 3] += 1.0  # change the field at one 4D site
    full2 = dwf.D(psi2)
    rest2 = full2 - sum(dwf.hop(psi2, mu, d) for mu in range(4) for d in (1, -1))
    diff = np.abs(rest2 - rest).sum(axis=(0, -1, -2))
    assert np.count_nonzero(diff > 1e-13) == 1 and diff[1, 1, 2, 3] > 0
