"""FP64 oracle of the learned near-null proposal (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no network: it finds the near-null vectors of the adaptive
setup (Sec. 2) by relaxing on D x = 0 from random vectors.  This module is
the plain reference of the project's gauge-covariant convolutional network
that proposes those vectors, and of the loss that trains it against the
vectors the adaptive setup generates.  Every function is written from its
definition, loop-free only where numpy's einsum states the contraction
directly.

Network (all fields complex)
  input   h_0(x): c_in channels x 4 spins x 3 colours per 4D site, seeded
          Gaussian (a gauge-covariant field in distribution)
  layer   a_{l+1}(x) = sum_{d=0..8} W_l[d] (T_d h_l)(x),
          T_0 h(x) = h(x),  T_{+mu} h(x) = U_mu(x) h(x+mu),
          T_{-mu} h(x) = U_mu(x-mu)^+ h(x-mu)
          (parallel transport with the links); W_l[d] acts on
          (channel, spin) and never on colour, so a_{l+1} is covariant.
  gate    h_{l+1} = sigma(a_{l+1}),  sigma(a) = a * t / (1 + t) with
          t = |a|^2 summed over colour for each (channel, spin, site):
          a gauge-invariant norm gate.
  head    v_j(x, s, spin, colour) = sum_{c, spin'} Hd[j, s, spin, c, spin']
          h_L(x, c, spin', colour): nout fine 5D fields (the fifth
          dimension enters only here).

Loss (block projection onto the adaptive subspace)
  H = the Gamma split of the outputs, [(1 + Gamma)/2 v_j, (1 - Gamma)/2 v_j]
  with Gamma = gamma_5 R_5 (the split the setup applies), cut into the
  blocks of the transfer.  For targets q_c (the setup's basis) and every
  block b:  L_b = min_Y || Q_b - H_b Y ||_F^2, the squared distance of the
  target pieces from the span of the network's pieces.
  L = sum_b L_b / (number of blocks * number of targets).

Gradients
  For a real loss of complex parameters theta the gradient returned is
  G = dL/d(conj theta), so that dL = 2 Re <G, d theta>.

Shapes
  U      (T, Z, Y, X, 4, 3, 3)          links, mu = x, y, z, t
  h      (C, 4, T, Z, Y, X, 3)          activations
  W_l    (C_out, 4, 9, C_in, 4)         direction d: 0 self, 1 + 2 mu: +mu,
                                        2 + 2 mu: -mu
  Hd     (nout, Ls, 4, C, 4)
  v      (nout, Ls, T, Z, Y, X, 12)     fine fields in the oracle layout

Refinement mode (forward_refine): the network maps each given fine field
v_b (its fifth dimension folded into c_in = Ls channels, scaled by
alpha = sqrt(Ls V 12) so that a unit-norm field has entries of order one)
to v_b + head(h_L) / alpha (nout = 1, a skip connection), for improving
vectors that a short relaxation produced.

Parity pins (tests/test_oracle_net.py): adjointness of the transports
(T_{+mu}^+ = T_{-mu}), gauge covariance of the forward pass and gauge
invariance of the loss, central finite differences of every parameter
group, the loss's closed forms (zero when the outputs span the targets,
the full norm when they are orthogonal to them, invariance under mixing
within a block).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from .mg import to_blocks


@dataclasses.dataclass
class NetShape:
    c_in: int = 4       # input channels
    hidden: int = 16    # hidden channels
    layers: int = 2     # convolution layers (the first maps c_in -> hidden)
    nout: int = 12      # output fine fields (Nvec / 2 with the Gamma split)
    Ls: int = 16


def param_shapes(s: NetShape):
    shapes = []
    cin = s.c_in
    for _ in range(s.layers):
        shapes.append((s.hidden, 4, 9, cin, 4))
        cin = s.hidden
    shapes.append((s.nout, s.Ls, 4, s.hidden, 4))
    return shapes


def unflatten(s: NetShape, flat):
    out, o = [], 0
    for sh in param_shapes(s):
        n = int(np.prod(sh))
        out.append(np.asarray(flat[o:o + n]).reshape(sh))
        o += n
    assert o == len(flat)
    return out


def flatten(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p).ravel() for p in parts])


# ---------------------------------------------------------------------------
# parallel transport
# ---------------------------------------------------------------------------

def _axis(mu):
    return 5 - mu  # h axes: (C, 4, T, Z, Y, X, 3): X is 5, T is 2


def transport(U, h, mu, d):
    """T_{+mu} h (d = +1) or T_{-mu} h (d = -1)."""
    Um = U[..., mu, :, :]
    if d > 0:
        hn = np.roll(h, -1, axis=_axis(mu))                # h(x + mu)
        return np.einsum("tzyxab,cstzyxb->cstzyxa", Um, hn)
    # U_mu(y)^+ h(y) at y = x - mu
    w = np.einsum("tzyxba,cstzyxb->cstzyxa", np.conj(Um), h)
    return np.roll(w, +1, axis=_axis(mu))


def transports(U, h):
    """[T_0 h, T_{+x} h, T_{-x} h, ..., T_{-t} h]."""
    out = [h]
    for mu in range(4):
        out.append(transport(U, h, mu, +1))
        out.append(transport(U, h, mu, -1))
    return out


def transport_adjoint(U, y, d):
    """T_d^+ y: T_0^+ = 1, T_{+mu}^+ = T_{-mu}, T_{-mu}^+ = T_{+mu}."""
    if d == 0:
        return y
    mu = (d - 1) // 2
    sgn = +1 if (d - 1) % 2 == 0 else -1
    return transport(U, y, mu, -sgn)


# ---------------------------------------------------------------------------
# layers
# ---------------------------------------------------------------------------

def conv(U, W, h):
    """a = sum_d W[d] (T_d h); W shape (Co, 4, 9, Ci, 4)."""
    T = transports(U, h)
    a = 0
    for d in range(9):
        a = a + np.einsum("oaib,ibtzyxc->oatzyxc", W[:, :, d], T[d])
    return a, T


def gate(a):
    """sigma(a) = a t/(1+t), t = sum over colour of |a|^2."""
    t = np.sum(np.abs(a) ** 2, axis=-1, keepdims=True)
    return a * (t / (1.0 + t))


def gate_backward(a, g):
    """dL/d(conj a) from dL/d(conj sigma) = g:
    g t/(1+t) + 2 (1+t)^-2 Re(sum_colour conj(a) g) a."""
    t = np.sum(np.abs(a) ** 2, axis=-1, keepdims=True)
    re = np.sum(np.conj(a) * g, axis=-1, keepdims=True).real
    return g * (t / (1.0 + t)) + 2.0 * re / (1.0 + t) ** 2 * a


def head(Hd, h, dims):
    """v_j (Ls, T, Z, Y, X, 12) from h (C, 4, T, Z, Y, X, 3)."""
    v = np.einsum("jsaib,ibtzyxc->jstzyxac", Hd, h)
    X, Y, Z, T = dims
    return v.reshape(v.shape[0], v.shape[1], T, Z, Y, X, 12)


def forward(s: NetShape, params, U, h0, dims):
    """Outputs v (nout, Ls, T, Z, Y, X, 12) and the cache for backward."""
    Ws, Hd = params[:-1], params[-1]
    h = h0
    cache = []
    for W in Ws:
        a, T = conv(U, W, h)
        cache.append((a, T))
        h = gate(a)
    return head(Hd, h, dims), (cache, h)


def backward(s: NetShape, params, U, cache, gv, dims):
    """Parameter gradients from gv = dL/d(conj v)."""
    Ws, Hd = params[:-1], params[-1]
    layers, hL = cache
    X, Y, Z, T = dims
    g6 = gv.reshape(gv.shape[0], gv.shape[1], T, Z, Y, X, 4, 3)
    gHd = np.einsum("jstzyxac,ibtzyxc->jsaib", g6, np.conj(hL))
    gh = np.einsum("jsaib,jstzyxac->ibtzyxc", np.conj(Hd), g6)
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        a, Tl = layers[l]
        ga = gate_backward(a, gh)
        W = Ws[l]
        gW = np.zeros_like(W)
        ghp = 0
        for d in range(9):
            gW[:, :, d] = np.einsum("oatzyxc,ibtzyxc->oaib", ga, np.conj(Tl[d]))
            y = np.einsum("oaib,oatzyxc->ibtzyxc", np.conj(W[:, :, d]), ga)
            ghp = ghp + transport_adjoint(U, y, d)
        grads[l] = gW
        gh = ghp
    return grads + [gHd]


# ---------------------------------------------------------------------------
# loss
# ---------------------------------------------------------------------------

def gamma_split(v):
    """[(1+G)/2 v_0, (1-G)/2 v_0, (1+G)/2 v_1, ...], G = gamma_5 R_5:
    (G v)(s) = diag(1,1,-1,-1) v(Ls-1-s)."""
    out = []
    for vj in v:
        g = vj[::-1].copy()
        g[..., 6:] *= -1
        out.append(0.5 * (vj + g))
        out.append(0.5 * (vj - g))
    return np.array(out)


def gamma_split_adjoint(g):
    """Adjoint of gamma_split: (1+G)/2 g_2j + (1-G)/2 g_2j+1 (G is Hermitian)."""
    out = []
    for j in range(g.shape[0] // 2):
        a, b = g[2 * j], g[2 * j + 1]
        ga, gb = a[::-1].copy(), b[::-1].copy()
        ga[..., 6:] *= -1
        gb[..., 6:] *= -1
        out.append(0.5 * (a + ga) + 0.5 * (b - gb))
    return np.array(out)


def projection_loss(v, targets, dims, block, grad=False):
    """L and (optionally) dL/d(conj v), see the module docstring.

    Per block: Y = argmin ||Q - H Y|| by least squares (numpy lstsq), the
    residual R = Q - H Y, L_b = ||R||^2 and dL_b/d(conj H) = -R Y^+."""
    Hs = gamma_split(v)
    Hb = np.stack([to_blocks(h, dims, block) for h in Hs])          # (Nh, Vc, bs)
    Qb = np.stack([to_blocks(q, dims, block) for q in targets])     # (Nt, Vc, bs)
    Vc = Hb.shape[1]
    nt = Qb.shape[0]
    scale = 1.0 / (Vc * nt)
    L = 0.0
    gHb = np.zeros_like(Hb)
    for b in range(Vc):
        Hm = Hb[:, b, :].T        # bs x Nh
        Qm = Qb[:, b, :].T        # bs x Nt
        Yb = np.linalg.lstsq(Hm, Qm, rcond=None)[0]
        R = Qm - Hm @ Yb
        L += float(np.sum(np.abs(R) ** 2))
        if grad:
            gHb[:, b, :] = (-(R @ np.conj(Yb.T))).T
    L *= scale
    if not grad:
        return L
    gH = np.stack([_from_blocks_like(gHb[k], Hs[k], dims, block) for k in range(Hb.shape[0])]) * scale
    return L, gamma_split_adjoint(gH)


def _from_blocks_like(g, like, dims, block):
    from .mg import from_blocks
    return from_blocks(g, like.shape[0], like.shape[-1], dims, block)


def loss_and_grad(s: NetShape, params, U, h0, targets, dims, block):
    """L and the gradient of every parameter group."""
    v, cache = forward(s, params, U, h0, dims)
    L, gv = projection_loss(v, targets, dims, block, grad=True)
    return L, backward(s, params, U, cache, gv, dims)


# ---------------------------------------------------------------------------
# refinement mode: the network improves given vectors instead of drawing them
# ---------------------------------------------------------------------------

def fields_to_input(v, dims):
    """Fine fields (B, Ls, T, Z, Y, X, 12) -> B network inputs with the fifth
    dimension as channels: (B, Ls, 4, T, Z, Y, X, 3)."""
    X, Y, Z, T = dims
    B, Ls = v.shape[0], v.shape[1]
    v8 = v.reshape(B, Ls, T, Z, Y, X, 4, 3)
    return np.ascontiguousarray(np.transpose(v8, (0, 1, 6, 2, 3, 4, 5, 7)))


def refine_scale(s: NetShape, dims):
    """alpha = sqrt(Ls * V * 12): a unit-norm field times alpha has entries of
    order one, the range in which the gate t/(1+t) is neither dead nor linear."""
    return float(np.sqrt(s.Ls * int(np.prod(dims)) * 12))


def forward_refine(s: NetShape, params, U, v, dims):
    """out_b = v_b + net(alpha v_b) / alpha: c_in = Ls channels (one per s),
    nout = 1, and a skip connection, so that zero head weights give out = v
    exactly."""
    assert s.c_in == s.Ls and s.nout == 1
    alpha = refine_scale(s, dims)
    h0s = fields_to_input(v, dims) * alpha
    outs, caches = [], []
    for b in range(v.shape[0]):
        o, cache = forward(s, params, U, h0s[b], dims)
        outs.append(v[b] + o[0] / alpha)
        caches.append(cache)
    return np.array(outs), caches


def loss_and_grad_refine(s: NetShape, params, U, v, targets, dims, block):
    """Projection loss of the refined fields and the parameter gradients
    (summed over the batch; the skip connection holds no parameters)."""
    out, caches = forward_refine(s, params, U, v, dims)
    L, gout = projection_loss(out, targets, dims, block, grad=True)
    alpha = refine_scale(s, dims)
    grads = None
    for b, cache in enumerate(caches):
        gb = backward(s, params, U, cache, gout[b:b + 1] / alpha, dims)
        grads = gb if grads is None else [x + y for x, y in zip(grads, gb)]
    return L, grads


def gauge_transform_field(g, h):
    """(g h)(x) for h (..., T, Z, Y, X, 3) and g (T, Z, Y, X, 3, 3)."""
    return np.einsum("tzyxab,...tzyxb->...tzyxa", g, h)


def gauge_transform_links(g, U):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^+."""
    out = np.empty_like(U)
    for mu in range(4):
        gn = np.roll(g, -1, axis=3 - mu)   # g(x + mu): axes (T, Z, Y, X)
        out[..., mu, :, :] = np.einsum("tzyxab,tzyxbc,tzyxdc->tzyxad", g, U[..., mu, :, :], np.conj(gn))
    return out
