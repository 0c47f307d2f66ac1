"""GPU parity of the learned near-null proposal (include/dwfnet.h) against the
FP64 network oracle (oracle/net.py) on identical seeded inputs: forward
outputs, the block-projection loss and every parameter gradient; plus gauge
covariance on the GPU and a few Adam steps lowering the loss."""
import numpy as np
import pytest

from oracle import net as N
import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = (4, 4, 4, 4)
LS = 8
BLOCK = (2, 2, 2, 2)
SHAPE = N.NetShape(c_in=2, hidden=4, layers=2, nout=3, Ls=LS)


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


def _params(shape, seed):
    parts = []
    for k, sh in enumerate(N.param_shapes(shape)):
        fan_in = int(np.prod(sh[2:])) if k < shape.layers else int(np.prod(sh[3:]))
        parts.append(I.gauss_complex(sh, seed + k, I.STREAM_NETWORK) / np.sqrt(fan_in))
    return parts


def _input(shape, dims, seed):
    X, Y, Z, T = dims
    return I.gauss_complex((shape.c_in, 4, T, Z, Y, X, 3), seed, I.STREAM_NETWORK)


class NetCase:
    def __init__(self, G, U, shape=SHAPE, pseed=10):
        from gpu_util import ctx_for
        self.G, self.U, self.shape = G, U, shape
        self.ctx = ctx_for(U, DIMS, shape.Ls, 1.8, 0.1)
        self.net = G.net_create(self.ctx.h, shape.c_in, shape.hidden, shape.layers, shape.nout, shape.Ls)
        self.p = _params(shape, pseed)
        flat = N.flatten(self.p)
        assert G.net_num_params(self.net) == flat.size
        G.net_set_params(self.net, np.ascontiguousarray(flat))

    def forward(self, h0=None, seed=0):
        out = torch.empty(self.shape.nout * self.ctx.field_elems, dtype=torch.complex128, device="cuda")
        inp = None if h0 is None else np.ascontiguousarray(h0)
        self.G.net_forward(self.net, self.ctx.h, out, input=inp, seed=seed)
        torch.cuda.synchronize()
        X, Y, Z, T = DIMS
        return out.cpu().numpy().reshape(self.shape.nout, self.shape.Ls, T, Z, Y, X, 12)

    def close(self):
        self.G.net_destroy(self.net)
        self.ctx.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forward_matches_oracle(G):
    U = I.epsilon_links(DIMS, 0.4, 3)
    c = NetCase(G, U)
    h0 = _input(SHAPE, DIMS, 20)
    got = c.forward(h0)
    ref, _ = N.forward(SHAPE, c.p, U, h0, DIMS)
    assert _rel(got, ref) < 1e-5
    # the device Philox input equals the host generator's field
    got2 = c.forward(None, seed=20)
    assert _rel(got2, got) < 1e-6
    # parameters round-trip through the device copy (FP32 storage)
    back = np.empty(G.net_num_params(c.net), dtype=np.complex128)
    G.net_get_params(c.net, back)
    flat = N.flatten(c.p)
    assert np.abs(back - flat).max() < 1e-6 * np.abs(flat).max()
    c.close()


def test_forward_gauge_covariance(G):
    U = I.epsilon_links(DIMS, 0.5, 4)
    g = I.random_gauge_transform(DIMS, 5)
    h0 = _input(SHAPE, DIMS, 21)
    c1 = NetCase(G, U)
    v = c1.forward(h0)
    c1.close()
    c2 = NetCase(G, N.gauge_transform_links(g, U))
    vg = c2.forward(N.gauge_transform_field(g, h0))
    c2.close()
    v6 = v.reshape(v.shape[:6] + (4, 3))
    expect = np.einsum("tzyxab,jstzyxcb->jstzyxca", g, v6).reshape(v.shape)
    assert _rel(vg, expect) < 1e-5


def test_loss_and_gradient_match_oracle(G):
    from gpu_util import to_internal
    U = I.epsilon_links(DIMS, 0.4, 6)
    c = NetCase(G, U, pseed=30)
    h0 = _input(SHAPE, DIMS, 31)
    X, Y, Z, T = DIMS
    nt = 4
    q = I.gauss_complex((nt, LS, T, Z, Y, X, 12), 32, I.STREAM_NETWORK)
    qt = to_internal(c.ctx, q, nrhs=nt)
    grad = np.empty(G.net_num_params(c.net), dtype=np.complex128)
    L = G.net_loss_grad(c.net, c.ctx.h, qt, nt, BLOCK, input=np.ascontiguousarray(h0), grad=grad)
    Lo, go = N.loss_and_grad(SHAPE, c.p, U, h0, q, DIMS, BLOCK)
    assert abs(L - Lo) < 1e-5 * Lo
    parts = N.unflatten(SHAPE, grad)
    for k, (a, b) in enumerate(zip(parts, go)):
        assert _rel(a, b) < 1e-4, (k, _rel(a, b))
    c.close()


def test_adam_lowers_the_loss_and_breakdown(G):
    from gpu_util import to_internal
    U = I.epsilon_links(DIMS, 0.4, 7)
    c = NetCase(G, U, pseed=40)
    X, Y, Z, T = DIMS
    nt = 6
    q = I.gauss_complex((nt, LS, T, Z, Y, X, 12), 41, I.STREAM_NETWORK)
    qt = to_internal(c.ctx, q, nrhs=nt)
    losses = []
    for _ in range(30):
        losses.append(G.net_loss_grad(c.net, c.ctx.h, qt, nt, BLOCK, seed=42))
        G.net_adam(c.net, 3e-3)
    # random targets: the loss (about the targets' whole norm) falls slowly but steadily
    assert all(b < a for a, b in zip(losses[:10], losses[1:11])), losses
    assert losses[-1] < 0.99 * losses[0], losses
    # a network with zero parameters proposes zero vectors: Gram-Schmidt breaks down
    G.net_set_params(c.net, np.zeros(G.net_num_params(c.net), dtype=np.complex128))
    with pytest.raises(G.DWFError) as e:
        G.net_loss_grad(c.net, c.ctx.h, qt, nt, BLOCK, seed=42)
    assert e.value.status == G.DWF_EBREAKDOWN
    with pytest.raises(G.DWFError):
        G.net_adam(c.net, 1e-3)   # no gradient since the parameters were set
    c.close()


def test_learned_setup_and_fallback(G):
    """mg_setup_learned: the network's proposal starts the setup and the solve
    converges; a probe limit that no solve meets triggers the plain setup."""
    from gpu_util import ctx_for, to_internal
    dims, Ls = (4, 4, 4, 4), 8
    U = I.epsilon_links(dims, 0.3, 8)
    ctx = ctx_for(U, dims, Ls, 1.8, 0.1)
    shape = N.NetShape(c_in=2, hidden=4, layers=2, nout=4, Ls=Ls)
    net = G.net_create(ctx.h, shape.c_in, shape.hidden, shape.layers, shape.nout, shape.Ls)
    G.net_set_params(net, np.ascontiguousarray(N.flatten(_params(shape, 50))))
    p = G.mg_default_params()
    p.setup_iters0 = 10
    b = to_internal(ctx, I.gaussian_source(dims, Ls, 51))
    assert not G.mg_setup_learned(ctx.h, net, 3, 2, [8], [(2, 2, 2, 2)], p)
    x = torch.zeros_like(b)
    st = G.mg_solve(ctx.h, b, x, 1e-10)
    assert st.true_res <= 1e-10
    assert G.mg_setup_learned(ctx.h, net, 3, 2, [8], [(2, 2, 2, 2)], p, fallback_iters0=50, probe_tol=1e-8,
                              probe_max_iters=1)
    x.zero_()
    assert G.mg_solve(ctx.h, b, x, 1e-10).true_res <= 1e-10
    with pytest.raises(G.DWFError):   # nout must be Nvec/2
        G.mg_setup_learned(ctx.h, net, 3, 2, [6], [(2, 2, 2, 2)], p)
    G.net_destroy(net)
    ctx.close()


def test_trained_weights_beat_untrained(G):
    """The committed network (trained on heatbath lattices 1000-1031 at 8^4,
    Ls = 16) against its own initialisation on a held-out lattice (seed 1035):
    the trained proposal is closer to the adaptive setup's subspace."""
    import pathlib
    from paper_1205_2933_gb300 import learned as Lm
    path = pathlib.Path(Lm.__file__).parent / "weights" / "near_null_8x8x8x8_Ls16.npz"
    shape, params, meta = Lm.load(path)
    assert shape == Lm.SHAPE
    ctx = Lm.lattice((8, 8, 8, 8), shape["Ls"], 1035)
    nvec, block = 2 * shape["nout"], (4, 4, 4, 4)
    q = Lm.adaptive_targets(ctx, nvec, block, Lm.solve_params())
    trained = Lm.make_net(ctx, shape, params)
    untrained = Lm.make_net(ctx, shape, Lm.init_params(shape, 77))
    lt = np.mean([G.net_loss_grad(trained, ctx.h, q, nvec, block, seed=s) for s in (1, 2)])
    lu = np.mean([G.net_loss_grad(untrained, ctx.h, q, nvec, block, seed=s) for s in (1, 2)])
    assert lt < lu - 0.02, (lt, lu)
    G.net_destroy(trained)
    G.net_destroy(untrained)
    ctx.close()


RSHAPE = N.NetShape(c_in=LS, hidden=4, layers=2, nout=1, Ls=LS)


def test_refine_matches_oracle(G):
    """Refinement mode: the refined fields, the projection loss and every
    gradient against the oracle's forward_refine / loss_and_grad_refine."""
    from gpu_util import to_internal, ctx_for
    U = I.epsilon_links(DIMS, 0.4, 12)
    ctx = ctx_for(U, DIMS, LS, 1.8, 0.1)
    net = G.net_create(ctx.h, RSHAPE.c_in, RSHAPE.hidden, RSHAPE.layers, RSHAPE.nout, RSHAPE.Ls)
    p = _params(RSHAPE, 60)
    G.net_set_params(net, np.ascontiguousarray(N.flatten(p)))
    X, Y, Z, T = DIMS
    B, nt = 3, 4
    v = I.gauss_complex((B, LS, T, Z, Y, X, 12), 61, I.STREAM_NETWORK)
    vt = to_internal(ctx, v, nrhs=B)
    out = torch.empty(B * ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.net_refine(net, ctx.h, vt, B, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(v.shape)
    ref, _ = N.forward_refine(RSHAPE, p, U, v, DIMS)
    assert _rel(got, ref) < 1e-5
    q = I.gauss_complex((nt, LS, T, Z, Y, X, 12), 62, I.STREAM_NETWORK)
    qt = to_internal(ctx, q, nrhs=nt)
    grad = np.empty(G.net_num_params(net), dtype=np.complex128)
    L = G.net_refine_loss_grad(net, ctx.h, vt, B, qt, nt, BLOCK, grad=grad)
    Lo, go = N.loss_and_grad_refine(RSHAPE, p, U, v, q, DIMS, BLOCK)
    assert abs(L - Lo) < 1e-5 * Lo
    for k, (a, b) in enumerate(zip(N.unflatten(RSHAPE, grad), go)):
        assert _rel(a, b) < 1e-4, (k, _rel(a, b))
    G.net_destroy(net)
    ctx.close()


def test_adaptive_vectors_and_refined_setup(G):
    """mg_get_adaptive_vectors returns the setup's globally orthonormal
    vectors; the learned setup with a refinement network (short relaxation,
    refinement, short relaxation) gives a converging solve."""
    from gpu_util import ctx_for, to_internal
    U = I.epsilon_links(DIMS, 0.3, 13)
    ctx = ctx_for(U, DIMS, LS, 1.8, 0.1)
    p = G.mg_default_params()
    p.setup_iters0 = 20
    G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p)
    a = torch.empty(4 * ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.mg_get_adaptive_vectors(ctx.h, 0, a)
    A = a.reshape(4, -1)
    gram = (A.conj() @ A.T).cpu().numpy()
    assert np.abs(gram - np.eye(4)).max() < 1e-10
    net = G.net_create(ctx.h, RSHAPE.c_in, RSHAPE.hidden, RSHAPE.layers, RSHAPE.nout, RSHAPE.Ls)
    pr = _params(RSHAPE, 70)
    pr[-1] *= 0.05
    G.net_set_params(net, np.ascontiguousarray(N.flatten(pr)))
    p.setup_iters0 = 10
    assert not G.mg_setup_learned(ctx.h, net, 3, 2, [8], [(2, 2, 2, 2)], p, pre_iters0=10)
    b = to_internal(ctx, I.gaussian_source(DIMS, LS, 71))
    x = torch.zeros_like(b)
    assert G.mg_solve(ctx.h, b, x, 1e-10).true_res <= 1e-10
    G.net_destroy(net)
    ctx.close()


def _bf16(x):
    """Round to BF16 (nearest even) through FP32, as a BF16 weight store holds them."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_weights(G):
    """BF16 inference weights: the forward pass equals the oracle's with the
    weights rounded to BF16 (FP32 arithmetic); training keeps FP32 masters."""
    U = I.epsilon_links(DIMS, 0.4, 14)
    c = NetCase(G, U, pseed=80)
    h0 = _input(SHAPE, DIMS, 81)
    f32 = c.forward(h0)
    G.net_set_weight_precision(c.net, G.DWF_BF16)
    b16 = c.forward(h0)
    pr = [_bf16(p.real) + 1j * _bf16(p.imag) for p in c.p]
    ref, _ = N.forward(SHAPE, pr, U, h0, DIMS)
    assert _rel(b16, ref) < 1e-5
    assert 1e-5 < _rel(b16, f32) < 5e-2
    back = np.empty(G.net_num_params(c.net), dtype=np.complex128)
    G.net_get_params(c.net, back)                      # masters unchanged
    assert np.abs(back - N.flatten(c.p)).max() < 1e-6 * np.abs(N.flatten(c.p)).max()
    with pytest.raises(G.DWFError):
        G.net_set_weight_precision(c.net, G.DWF_F16)
    c.close()
