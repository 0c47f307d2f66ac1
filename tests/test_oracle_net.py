"""Pins of the network oracle (oracle/net.py) against facts that do not come
from the oracle itself: inner-product adjointness of the transports, gauge
covariance, central finite differences, and the loss's closed forms."""
import numpy as np
import pytest

from oracle import net as N
import paper_1205_2933_gb300.inputs as I

DIMS = (4, 4, 2, 2)      # X, Y, Z, T
BLOCK = (2, 2, 2, 2)
SHAPE = N.NetShape(c_in=2, hidden=3, layers=2, nout=2, Ls=4)


def _params(shape, seed):
    parts = []
    for k, sh in enumerate(N.param_shapes(shape)):
        fan_in = int(np.prod(sh[2:])) if k < shape.layers else int(np.prod(sh[3:]))
        parts.append(I.gauss_complex(sh, seed + k, I.STREAM_NETWORK) / np.sqrt(fan_in))
    return parts


def _input(shape, dims, seed):
    X, Y, Z, T = dims
    return I.gauss_complex((shape.c_in, 4, T, Z, Y, X, 3), seed, I.STREAM_NETWORK)


def _targets(nt, dims, Ls, seed):
    X, Y, Z, T = dims
    return I.gauss_complex((nt, Ls, T, Z, Y, X, 12), seed, I.STREAM_NETWORK)


def _vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def test_transport_adjoints():
    """<y, T_d h> = <T_d^+ y, h> for all nine directions (T_{+mu}^+ = T_{-mu})."""
    U = I.epsilon_links(DIMS, 0.4, 3)
    X, Y, Z, T = DIMS
    h = I.gauss_complex((2, 4, T, Z, Y, X, 3), 1, I.STREAM_NETWORK)
    y = I.gauss_complex((2, 4, T, Z, Y, X, 3), 2, I.STREAM_NETWORK)
    Ts = N.transports(U, h)
    for d in range(9):
        lhs = _vdot(y, Ts[d])
        rhs = _vdot(N.transport_adjoint(U, y, d), h)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_transport_unit_links_is_a_shift():
    """With U = 1 the transports are plain periodic shifts."""
    U = I.unit_links(DIMS)
    X, Y, Z, T = DIMS
    h = I.gauss_complex((1, 4, T, Z, Y, X, 3), 5, I.STREAM_NETWORK)
    # +x: value at x comes from x + 1
    t = N.transport(U, h, 0, +1)
    assert np.array_equal(t[..., 0, :], h[..., 1, :])
    t = N.transport(U, h, 3, -1)                 # -t: value at t comes from t - 1
    assert np.array_equal(t[:, :, 1], h[:, :, 0])


def test_gauge_covariance():
    """Links U^g, input g h0  ->  outputs g v; the loss with targets g q equals
    the loss with q (g is unitary and site-local, blocks are unions of sites)."""
    U = I.epsilon_links(DIMS, 0.5, 7)
    g = I.random_gauge_transform(DIMS, 8)
    Ug = N.gauge_transform_links(g, U)
    p = _params(SHAPE, 10)
    h0 = _input(SHAPE, DIMS, 20)
    v, _ = N.forward(SHAPE, p, U, h0, DIMS)
    vg, _ = N.forward(SHAPE, p, Ug, N.gauge_transform_field(g, h0), DIMS)
    X, Y, Z, T = DIMS
    v6 = v.reshape(v.shape[:6] + (4, 3))
    expect = np.einsum("tzyxab,jstzyxcb->jstzyxca", g, v6).reshape(v.shape)
    assert np.abs(vg - expect).max() < 1e-12 * np.abs(v).max()
    q = _targets(3, DIMS, SHAPE.Ls, 30)
    q6 = q.reshape(q.shape[:6] + (4, 3))
    qg = np.einsum("tzyxab,jstzyxcb->jstzyxca", g, q6).reshape(q.shape)
    L0 = N.projection_loss(v, q, DIMS, BLOCK)
    L1 = N.projection_loss(vg, qg, DIMS, BLOCK)
    assert abs(L0 - L1) < 1e-12


def test_loss_closed_forms():
    X, Y, Z, T = DIMS
    v = _targets(2, DIMS, 4, 40)
    # the targets are the network's own Gamma-split pieces: zero distance
    assert N.projection_loss(v, N.gamma_split(v), DIMS, BLOCK) < 1e-24
    # outputs on the upper spins (the Gamma split keeps them there), targets on
    # the lower spins: orthogonal, the loss is the targets' whole norm
    vu = v.copy()
    vu[..., 6:] = 0
    q = _targets(3, DIMS, 4, 41)
    q[..., :6] = 0
    nb = (X // 2) * (Y // 2) * (Z // 2) * (T // 2)
    expect = float(np.sum(np.abs(q) ** 2)) / (nb * 3)
    assert abs(N.projection_loss(vu, q, DIMS, BLOCK) - expect) < 1e-12 * expect
    # mixing the outputs with an invertible matrix, or scaling them by a
    # positive constant per block, leaves the block spans and the loss alone
    M = np.array([[1.0 + 0.5j, -0.3], [0.2j, 0.7]])
    vm = np.einsum("jk,k...->j...", M, v)
    L = N.projection_loss(v, q, DIMS, BLOCK)
    assert abs(N.projection_loss(vm, q, DIMS, BLOCK) - L) < 1e-12
    scale = np.ones((T, Z, Y, X))
    scale[:, :, :, 2:] = 3.0                     # the second block column in x
    vs = v * scale[None, None, :, :, :, :, None]
    assert abs(N.projection_loss(vs, q, DIMS, BLOCK) - L) < 1e-12


def test_gate():
    a = I.gauss_complex((2, 4, 1, 1, 1, 2, 3), 50, I.STREAM_NETWORK)
    big = 1e4 * a
    assert np.abs(N.gate(big) - big).max() < 1e-6 * np.abs(big).max()
    small = 1e-4 * a
    t = np.sum(np.abs(small) ** 2, axis=-1, keepdims=True)
    assert np.abs(N.gate(small) - t * small).max() < 1e-14


@pytest.mark.parametrize("group", [0, 1, 2])
def test_finite_differences(group):
    """dL = 2 Re <G, dtheta>: central differences along a random complex
    direction of one parameter group (layer 0, layer 1, the head)."""
    U = I.epsilon_links(DIMS, 0.4, 60)
    p = _params(SHAPE, 61)
    h0 = _input(SHAPE, DIMS, 62)
    q = _targets(3, DIMS, SHAPE.Ls, 63)
    L, grads = N.loss_and_grad(SHAPE, p, U, h0, q, DIMS, BLOCK)
    dirn = I.gauss_complex(p[group].shape, 64 + group, I.STREAM_NETWORK)
    eps = 1e-5

    def loss_at(e):
        pp = [x.copy() for x in p]
        pp[group] = p[group] + e * dirn
        v, _ = N.forward(SHAPE, pp, U, h0, DIMS)
        return N.projection_loss(v, q, DIMS, BLOCK)

    fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
    an = 2.0 * np.real(_vdot(grads[group], dirn))
    assert abs(fd - an) < 1e-6 * max(abs(an), 1e-3), (fd, an)


def test_finite_differences_input_gate_path():
    """The gate's derivative alone: L = sum |sigma(a)|^2 against its gradient."""
    a = I.gauss_complex((1, 4, 1, 1, 1, 2, 3), 70, I.STREAM_NETWORK)
    d = I.gauss_complex(a.shape, 71, I.STREAM_NETWORK)
    f = lambda x: float(np.sum(np.abs(N.gate(x)) ** 2))
    g = N.gate_backward(a, N.gate(a))        # dL/d conj(sigma) = sigma for L = |sigma|^2
    eps = 1e-6
    fd = (f(a + eps * d) - f(a - eps * d)) / (2 * eps)
    assert abs(fd - 2 * np.real(_vdot(g, d))) < 1e-6 * abs(fd)


RSHAPE = N.NetShape(c_in=4, hidden=3, layers=2, nout=1, Ls=4)


def test_refine_identity_and_covariance():
    """Zero head weights give back the input fields exactly; the refined fields
    transform like fermions under a gauge transform of links and inputs."""
    U = I.epsilon_links(DIMS, 0.4, 80)
    X, Y, Z, T = DIMS
    v = _targets(2, DIMS, RSHAPE.Ls, 81)
    p = _params(RSHAPE, 82)
    p0 = [x.copy() for x in p]
    p0[-1][:] = 0
    out, _ = N.forward_refine(RSHAPE, p0, U, v, DIMS)
    assert np.array_equal(out, v)
    g = I.random_gauge_transform(DIMS, 83)
    def gf(f):
        f6 = f.reshape(f.shape[:6] + (4, 3))
        return np.einsum("tzyxab,jstzyxcb->jstzyxca", g, f6).reshape(f.shape)
    out, _ = N.forward_refine(RSHAPE, p, U, v, DIMS)
    outg, _ = N.forward_refine(RSHAPE, p, N.gauge_transform_links(g, U), gf(v), DIMS)
    assert np.abs(outg - gf(out)).max() < 1e-12 * np.abs(out).max()


@pytest.mark.parametrize("group", [0, 2])
def test_refine_finite_differences(group):
    U = I.epsilon_links(DIMS, 0.4, 90)
    p = _params(RSHAPE, 91)
    v = _targets(2, DIMS, RSHAPE.Ls, 92)
    q = _targets(3, DIMS, RSHAPE.Ls, 93)
    L, grads = N.loss_and_grad_refine(RSHAPE, p, U, v, q, DIMS, BLOCK)
    dirn = I.gauss_complex(p[group].shape, 94 + group, I.STREAM_NETWORK)
    eps = 1e-5

    def loss_at(e):
        pp = [x.copy() for x in p]
        pp[group] = p[group] + e * dirn
        out, _ = N.forward_refine(RSHAPE, pp, U, v, DIMS)
        return N.projection_loss(out, q, DIMS, BLOCK)

    fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
    an = 2.0 * np.real(_vdot(grads[group], dirn))
    assert abs(fd - an) < 1e-6 * max(abs(an), 1e-3), (fd, an)
