"""GPU parity of the fine operator D / D^+ (FP64 and FP32) and of the layout
conversions, against the FP64 oracle on identical seeded inputs."""
import numpy as np
import pytest

import oracle
import paper_1205_2933_gb300.inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    from paper_1205_2933_gb300 import dwfmg
    return dwfmg


CASES = [
    # dims (X,Y,Z,T), Ls, mf, links, antiperiodic
    ((4, 4, 4, 4), 8, 0.1, "eps", True),       # the plain-method workload (4^4, Ls = 8)
    ((2, 4, 6, 4), 5, 0.03, "eps", True),      # ragged extents, odd Ls
    ((4, 4, 2, 6), 16, 0.001, "hb", False),    # heatbath links, periodic t, Ls = 16
    ((6, 2, 2, 2), 1, 0.2, "eps", True),       # Ls = 1 (Wilson limit)
    ((3, 3, 3, 3), 3, 0.5, "eps", True),       # odd extents everywhere, block tail of the CTA
]


def _links(dims, kind, seed=1):
    if kind == "hb":
        return I.heatbath_links(dims, 6.0, 10, seed)
    return I.epsilon_links(dims, 0.6, seed)


@pytest.mark.parametrize("dims,Ls,mf,kind,ap", CASES)
def test_pack_roundtrip(G, dims, Ls, mf, kind, ap):
    from gpu_util import ctx_for, to_internal, to_canonical
    U = _links(dims, kind)
    ctx = ctx_for(U, dims, Ls, 1.8, mf, ap)
    f = I.gaussian_source(dims, Ls, 3)
    t = to_internal(ctx, f)
    assert np.array_equal(to_canonical(ctx, t, f.shape), f)
    t32 = to_internal(ctx, f, G.DWF_F32)
    back = to_canonical(ctx, t32, f.shape, G.DWF_F32)
    assert np.array_equal(back, f.astype(np.complex64).astype(np.complex128))
    # internal order: (site*12 + comp)*Ls + s
    V = int(np.prod(dims))
    arr = t.cpu().numpy().reshape(V, 12, Ls)
    assert arr[5 % V, 7, Ls - 1] == f.reshape(Ls, V, 12)[Ls - 1, 5 % V, 7]
    ctx.close()


@pytest.mark.parametrize("dims,Ls,mf,kind,ap", CASES)
@pytest.mark.parametrize("dag", [False, True])
def test_dslash_f64_parity(G, dims, Ls, mf, kind, ap, dag):
    from gpu_util import ctx_for, to_internal, to_canonical, rel_max
    U = _links(dims, kind)
    ctx = ctx_for(U, dims, Ls, 1.8, mf, ap)
    f = I.gaussian_source(dims, Ls, 4)
    t = to_internal(ctx, f)
    out = torch.empty_like(t)
    G.dwf_apply(ctx.h, out, t, G.DWF_F64, dag)
    got = to_canonical(ctx, out, f.shape)
    o = oracle.DWF(U, dims, Ls, 1.8, mf, antiperiodic_t=ap)
    ref = o.Ddag(f) if dag else o.D(f)
    assert rel_max(got, ref) < 1e-13
    ctx.close()


@pytest.mark.parametrize("dims,Ls,mf,kind,ap", CASES)
@pytest.mark.parametrize("dag", [False, True])
def test_dslash_f32_parity(G, dims, Ls, mf, kind, ap, dag):
    from gpu_util import ctx_for, to_internal, to_canonical, rel_norm, rel_max
    U = _links(dims, kind)
    ctx = ctx_for(U, dims, Ls, 1.8, mf, ap)
    f = I.gaussian_source(dims, Ls, 5)
    t = to_internal(ctx, f, G.DWF_F32)
    out = torch.empty_like(t)
    G.dwf_apply(ctx.h, out, t, G.DWF_F32, dag)
    got = to_canonical(ctx, out, f.shape, G.DWF_F32)
    o = oracle.DWF(U, dims, Ls, 1.8, mf, antiperiodic_t=ap)
    ref = o.Ddag(f) if dag else o.D(f)
    assert rel_norm(got, ref) < 1e-6
    assert rel_max(got, ref) < 2e-6
    ctx.close()


def test_multi_rhs_equals_single(G):
    from gpu_util import ctx_for, to_internal
    dims, Ls = (4, 4, 4, 4), 8
    U = _links(dims, "eps")
    ctx = ctx_for(U, dims, Ls, 1.8, 0.1)
    fs = np.stack([I.gaussian_source(dims, Ls, 10 + i) for i in range(3)])
    t = to_internal(ctx, fs, G.DWF_F64, nrhs=3)
    out = torch.empty_like(t)
    G.dwf_apply(ctx.h, out, t, G.DWF_F64, False, 3)
    n = ctx.field_elems
    for i in range(3):
        one = torch.empty(n, dtype=torch.complex128, device="cuda")
        G.dwf_apply(ctx.h, one, t[i * n:(i + 1) * n].contiguous(), G.DWF_F64)
        assert torch.equal(one, out[i * n:(i + 1) * n])
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dslash_full_size_sampled(G, prec):
    """16^3 x 32, Ls = 16 (the mixed-precision workload's lattice), in the
    launch configuration the benchmark times; 384 output sites checked one by
    one against the oracle."""
    from gpu_util import ctx_for, to_internal
    dims, Ls, mf = (16, 16, 16, 32), 16, 0.001
    U = I.epsilon_links(dims, 0.5, 7)
    ctx = ctx_for(U, dims, Ls, 1.8, mf)
    f = I.gaussian_source(dims, Ls, 8)
    p = G.DWF_F64 if prec == "f64" else G.DWF_F32
    t = to_internal(ctx, f, p)
    out = torch.empty_like(t)
    G.dwf_apply(ctx.h, out, t, p)
    torch.cuda.synchronize()
    V = int(np.prod(dims))
    rng = np.random.default_rng(0)
    idx5 = np.concatenate([rng.integers(0, V * Ls, 380), [0, V * Ls - 1, V - 1, (Ls - 1) * V]])
    ref = oracle.DWF(U, dims, Ls, 1.8, mf).D_sites(f, idx5).reshape(len(idx5), 12)
    o = out.cpu().numpy().astype(np.complex128).reshape(V, 12, Ls)
    got = np.stack([o[i % V, :, i // V] for i in idx5])
    tol = 1e-13 if prec == "f64" else 2e-6
    assert np.abs(got - ref).max() / np.abs(ref).max() < tol
    ctx.close()


def test_invalid_arguments(G):
    from gpu_util import ctx_for, to_internal
    dims, Ls = (2, 2, 2, 2), 4
    ctx = ctx_for(I.epsilon_links(dims, 0.3, 1), dims, Ls, 1.8, 0.1)
    t = to_internal(ctx, I.gaussian_source(dims, Ls, 1))
    assert G.lib().dwf_apply(ctx.h, G._ptr(t), G._ptr(t), 0, 0, 1) == G.DWF_EINVAL      # in place
    assert G.lib().dwf_apply(ctx.h, G._ptr(t), G._ptr(t), G.DWF_BF16, 0, 1) == G.DWF_EINVAL
    assert G.lib().dwf_apply(ctx.h, G._ptr(t), G._ptr(t), 0, 0, 0) == G.DWF_EINVAL
    # component calls before mg_setup
    assert G.lib().mg_vcycle(ctx.h, G._ptr(t), G._ptr(torch.empty_like(t))) == G.DWF_ESTATE
    ctx.close()
