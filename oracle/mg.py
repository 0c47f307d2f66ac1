"""FP64 oracle of the adaptive multigrid algorithm (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Cohen, Brower, Clark, Osborn, "Multigrid Algorithms for Domain-Wall
Fermions":
  * Sec. 1   restrictor R and prolongator P with R P = 1_c
  * Sec. 2   the five-step V-cycle (x1, b2, x2, b3, x), recursion through
             S2, the block subspace spanned by near-null vectors cut into
             blocks, the adaptive setup on A x = 0, blocks spanning the whole
             fifth dimension
  * Sec. 3   flexible GCR as the outer solver, CG on the squared operator as
             the comparison, cost counted in fine-operator applications
  * Sec. 4   the fine operator's one-hop stencil (here the coarse operator
             R D P of the unsquared operator is the 9-point stencil that one
             hop on the fine lattice produces on the coarse lattice), and the
             paper's own choice, the coarsened squared operator P^+ D^+ D P,
             whose coarse stencil reaches two hops (33 coarse offsets with
             blocks of extent >= 2 in every direction)

Parity pins (tests/test_oracle_*.py):
  D, D^+                  free-field momentum-space closed form, Ls=1 Wilson
                          limit, gamma5-R5 hermiticity, adjointness, gauge
                          covariance, m_f affinity
  block_orthonormalise    P^+ P = 1, span preserved, agrees with a QR
  Transfer.restrict/prolong  adjoint pair, R P = 1
  coarse_operator         equals the dense P^+ D P by brute force
  squared_coarse_operator equals the dense (D P)^+ (D P) by brute force; no
                          coupling beyond the 33 offsets; Hermitian positive;
                          its coarse correction is the least-squares fit of
                          the residual over range(P) (numpy lstsq)
  CoarseOp.apply          equals the dense coarse matrix
  gcr / cgnr              dense-LU solutions, residual monotonicity
  vcycle                  Galerkin orthogonality of the coarse correction
  (with oracle/dwf2d.py)  the same code runs the 2D U(1) toy of Sec. 3; its
                          whole solves are pinned by dense LU
  adaptive_setup          near-null Rayleigh quotients fall with sweeps
  mg_solve                dense-LU solution on tiny lattices, true residual
Nothing here is "parity unpinned".

Field convention: every level stores fields as arrays of shape
(S, T, Z, Y, X, n) where S = Ls and n = 12 (spin*3+colour) on the fine level,
S = 1 and n = Nvec on coarse levels.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np

from . import DWF


def vdot(a, b):
    """<a, b> = sum conj(a) b over all entries."""
    return np.vdot(a.ravel(), b.ravel())


def norm(a):
    return float(np.sqrt(np.vdot(a.ravel(), a.ravel()).real))


# ---------------------------------------------------------------------------
# Level operators
# ---------------------------------------------------------------------------

class FineOp:
    """The fine level: the Shamir DWF operator, fields (Ls, T, Z, Y, X, 12)."""

    def __init__(self, dwf: DWF):
        self.dwf = dwf
        self.dims = dwf.dims
        self.S = dwf.Ls
        self.n = 12
        X, Y, Z, T = self.dims
        self.shape = (self.S, T, Z, Y, X, 12)
        self.count = 0  # number of applications of the fine operator

    def apply(self, f):
        self.count += 1
        return self.dwf.D(f.reshape(self.dwf.shape)).reshape(self.shape)

    def apply_dag(self, f):
        self.count += 1
        return self.dwf.Ddag(f.reshape(self.dwf.shape)).reshape(self.shape)

    def hop(self, f, mu, d):
        return self.dwf.hop(f.reshape(self.dwf.shape), mu, d).reshape(self.shape)


def _shift(c, mu, d):
    """c(x + d*mu) on a periodic lattice, c shape (1, T, Z, Y, X, n)."""
    axis = 4 - mu  # X is axis 4, T is axis 1
    return np.roll(c, -d, axis=axis)


class CoarseOp:
    """A coarse level: 9-point stencil of dense n x n complex blocks.

    Y has shape (Tc, Zc, Yc, Xc, 9, n, n); direction 0 is the site itself,
    1 + 2*mu the +mu neighbour and 2 + 2*mu the -mu neighbour:
      (A c)(x) = Y0(x) c(x) + sum_{mu, d} Y_{mu,d}(x) c(x + d mu)
    with periodic neighbours (boundary signs of the fine lattice already sit
    inside the Y blocks).
    """

    def __init__(self, Y, dims):
        self.Y = Y
        self.dims = tuple(int(d) for d in dims)
        self.S = 1
        self.n = Y.shape[-1]
        X, Yd, Z, T = self.dims
        self.shape = (1, T, Z, Yd, X, self.n)
        self.count = 0

    @staticmethod
    def dir_index(mu, d):
        return 1 + 2 * mu + (0 if d > 0 else 1)

    def hop(self, c, mu, d):
        k = self.dir_index(mu, d)
        return np.einsum("tzyxab,stzyxb->stzyxa", self.Y[..., k, :, :], _shift(c, mu, d))

    def apply_self(self, c):
        return np.einsum("tzyxab,stzyxb->stzyxa", self.Y[..., 0, :, :], c)

    def apply(self, c):
        self.count += 1
        out = self.apply_self(c)
        for mu in range(4):
            for d in (+1, -1):
                out = out + self.hop(c, mu, d)
        return out

    def apply_dag(self, c):
        """A^+: (A^+ c)(x) = Y0(x)^+ c(x) + sum_{mu,d} Y_{mu,d}(x - d mu)^+ c(x - d mu)."""
        self.count += 1
        Yh = np.conj(np.swapaxes(self.Y, -1, -2))
        out = np.einsum("tzyxab,stzyxb->stzyxa", Yh[..., 0, :, :], c)
        for mu in range(4):
            for d in (+1, -1):
                k = self.dir_index(mu, d)
                out = out + _shift(np.einsum("tzyxab,stzyxb->stzyxa", Yh[..., k, :, :], c), mu, -d)
        return out


# ---------------------------------------------------------------------------
# Blocking, block Gram-Schmidt, restrictor / prolongator
# ---------------------------------------------------------------------------

def coarse_dims(dims, block):
    for L, b in zip(dims, block):
        if L % b:
            raise ValueError(f"block {block} does not divide lattice {dims}")
    return tuple(L // b for L, b in zip(dims, block))


def to_blocks(f, dims, block):
    """(S, T, Z, Y, X, n) -> (Vc, S*bt*bz*by*bx*n): one row per coarse site.

    A block holds B^4 sites of the 4D lattice and the whole fifth dimension
    (Sec. 2: the coarse blocks cover the entire fifth dimension)."""
    S = f.shape[0]
    n = f.shape[-1]
    X, Y, Z, T = dims
    bx, by, bz, bt = block
    Xc, Yc, Zc, Tc = coarse_dims(dims, block)
    g = f.reshape(S, Tc, bt, Zc, bz, Yc, by, Xc, bx, n)
    g = g.transpose(1, 3, 5, 7, 0, 2, 4, 6, 8, 9)
    return g.reshape(Tc * Zc * Yc * Xc, -1)


def from_blocks(g, S, n, dims, block):
    X, Y, Z, T = dims
    bx, by, bz, bt = block
    Xc, Yc, Zc, Tc = coarse_dims(dims, block)
    h = g.reshape(Tc, Zc, Yc, Xc, S, bt, bz, by, bx, n)
    h = h.transpose(4, 0, 5, 1, 6, 2, 7, 3, 8, 9)
    return h.reshape(S, T, Z, Y, X, n)


def block_orthonormalise(Vb):
    """Block Gram-Schmidt: Vb shape (Nv, Vc, bs), vector k restricted to block b.

    Within every block the Nv pieces are orthonormalised in order k = 0..Nv-1
    by modified Gram-Schmidt, run twice (re-orthogonalisation), each vector
    normalised to unit length with a real positive coefficient.  The result
    is Q = V R^-1 with R upper triangular with positive diagonal, so that
    P^+ P = 1 on the coarse space (R P = 1_c, Sec. 1).  Raises on a block
    whose pieces are linearly dependent.
    """
    Q = np.array(Vb, dtype=np.complex128, copy=True)
    Nv = Q.shape[0]
    for k in range(Nv):
        w = Q[k]
        for _pass in range(2):
            for j in range(k):
                c = np.einsum("bi,bi->b", np.conj(Q[j]), w)
                w = w - c[:, None] * Q[j]
        nrm = np.sqrt(np.einsum("bi,bi->b", np.conj(w), w).real)
        if np.any(nrm == 0.0) or not np.all(np.isfinite(nrm)):
            raise FloatingPointError("block Gram-Schmidt breakdown")
        Q[k] = w / nrm[:, None]
    return Q


class Transfer:
    """Prolongator P and restrictor R = P^+ built from near-null vectors.

    vectors: array (Nv, S, T, Z, Y, X, n) of fields on the fine level of this
    pair.  P maps a coarse field c (1, Tc, Zc, Yc, Xc, Nv) to
      (P c)(x, s, a) = sum_k q_k(x, s, a) c(block(x), k)
    where q_k are the block-orthonormalised vectors; R = P^+ sums
    conj(q_k) psi over each block (all s, all components)."""

    def __init__(self, vectors, dims, block):
        self.dims = tuple(dims)
        self.block = tuple(block)
        self.cdims = coarse_dims(dims, block)
        self.Nv = vectors.shape[0]
        self.S = vectors.shape[1]
        self.n = vectors.shape[-1]
        Vb = np.stack([to_blocks(v, self.dims, self.block) for v in vectors])
        self.Qb = block_orthonormalise(Vb)
        X, Y, Z, T = self.cdims
        self.cshape = (1, T, Z, Y, X, self.Nv)

    def restrict(self, f):
        fb = to_blocks(f, self.dims, self.block)
        c = np.einsum("kbi,bi->bk", np.conj(self.Qb), fb)
        return c.reshape(self.cshape)

    def prolong(self, c):
        cb = c.reshape(-1, self.Nv)
        fb = np.einsum("kbi,bk->bi", self.Qb, cb)
        return from_blocks(fb, self.S, self.n, self.dims, self.block)

    def vector(self, k):
        """The block-orthonormalised near-null vector q_k as a full field."""
        return from_blocks(self.Qb[k], self.S, self.n, self.dims, self.block)


def crossing_mask(dims, block, S, mu, d):
    """1 where the hop x -> x + d*mu leaves the block of x (before wrap-around)."""
    X, Y, Z, T = dims
    L = dims[mu]
    b = block[mu]
    x = np.arange(L)
    cross = ((x + d) // b != x // b).astype(np.float64)
    shape = [1, 1, 1, 1, 1, 1]
    shape[4 - mu] = L
    m = cross.reshape(shape)
    return np.broadcast_to(m, (S, T, Z, Y, X, 1))


def coarse_operator(op, T: Transfer) -> CoarseOp:
    """Galerkin coarse operator R A P as a 9-point stencil (Sec. 2 step 3).

    For every coarse direction l: take q_l, apply the level operator and each
    of its 8 hopping terms to it.  A hop from x to x + d*mu that leaves the
    block of x contributes (after restriction onto block(x)) to the link
    Y_{mu,d}(block(x)); everything else (diagonal, fifth-dimension hops,
    hops inside the block) contributes to Y0.
    """
    Nv = T.Nv
    Xc, Yc, Zc, Tc = T.cdims
    Y = np.zeros((Tc, Zc, Yc, Xc, 9, Nv, Nv), dtype=np.complex128)
    for l in range(Nv):
        q = T.vector(l)
        rest = op.apply(q)
        op.count -= 1  # construction applies are not solver cost
        for mu in range(4):
            for d in (+1, -1):
                h = op.hop(q, mu, d) * crossing_mask(op.dims, T.block, op.S, mu, d)
                rest = rest - h
                Y[..., CoarseOp.dir_index(mu, d), :, l] = T.restrict(h)[0]
        Y[..., 0, :, l] = T.restrict(rest)[0]
    return CoarseOp(Y, T.cdims)


# The squared operator's coarse stencil (Sec. 4): offset 0, the 8 one-hop
# offsets (1 + 2 mu: +mu, 2 + 2 mu: -mu) and the 24 two-hop diagonals
# +-mu +-nu (mu < nu), index 9 + 4 p + 2 a + b with p the pair's rank in
# (0,1), (0,2), (0,3), (1,2), (1,3), (2,3), a = 1 for -mu and b = 1 for -nu.
MU_NU_PAIRS = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def _offsets33():
    out = [(0, 0, 0, 0)]
    for mu in range(4):
        for d in (+1, -1):
            v = [0, 0, 0, 0]
            v[mu] = d
            out.append(tuple(v))
    for mu, nu in MU_NU_PAIRS:
        for a in (+1, -1):
            for b in (+1, -1):
                v = [0, 0, 0, 0]
                v[mu], v[nu] = a, b
                out.append(tuple(v))
    return out


OFFSETS33 = _offsets33()


def _shift_vec(c, off):
    """c(x + off) for a 4-vector offset (x, y, z, t), c shape (1, T, Z, Y, X, ...)."""
    for mu in range(4):
        if off[mu]:
            c = np.roll(c, -off[mu], axis=4 - mu)
    return c


class SquaredCoarseOp:
    """The coarsened squared operator P^+ D^+ D P (Sec. 4) as a 33-point
    stencil of dense n x n complex blocks, Y shape (Tc, Zc, Yc, Xc, 33, n, n):
      (A c)(x) = sum_j Y_j(x) c(x + OFFSETS33[j])   (periodic)."""

    def __init__(self, Y, dims):
        self.Y = Y
        self.dims = tuple(int(d) for d in dims)
        self.S = 1
        self.n = Y.shape[-1]
        X, Yd, Z, T = self.dims
        self.shape = (1, T, Z, Yd, X, self.n)
        self.count = 0

    def apply(self, c):
        self.count += 1
        out = np.zeros_like(c)
        for j, off in enumerate(OFFSETS33):
            out = out + np.einsum("tzyxab,stzyxb->stzyxa", self.Y[..., j, :, :], _shift_vec(c, off))
        return out

    def apply_dag(self, c):
        """(A^+ c)(x) = sum_j Y_j(x - o_j)^+ c(x - o_j)."""
        self.count += 1
        Yh = np.conj(np.swapaxes(self.Y, -1, -2))
        out = np.zeros_like(c)
        for j, off in enumerate(OFFSETS33):
            t = np.einsum("tzyxab,stzyxb->stzyxa", Yh[..., j, :, :], c)
            out = out + _shift_vec(t, tuple(-o for o in off))
        return out


def squared_coarse_operator(op, T: Transfer) -> SquaredCoarseOp:
    """P^+ D^+ D P as a 33-point stencil (Sec. 4 coarsens the squared operator).

    D q_l splits by where its terms read q_l: h_0 collects the terms that read
    inside the block of x (diagonal, fifth-dimension hops, hops within the
    block), h_{mu,d} the hop from x to x + d mu where it leaves the block.  So
    on block b'' the field D (q_l on block b' only) equals h_sigma with
    b' = b'' + sigma, and
      (P^+ D^+ D P)[b, k; b', l] = sum_{b''} <D q_k|_b, D q_l|_b'>_{b''}
                                 = sum over sigma1, sigma2 with b = b'' + sigma1,
                                   b' = b'' + sigma2 of <h_{sigma1,k}, h_{sigma2,l}>_{b''},
    the coarse offset b' - b = sigma2 - sigma1 kept as a vector (so that two
    offsets that reach the same site of a small periodic coarse lattice stay
    apart).  With every block extent >= 2, h_{+mu} (last layer of the block
    in mu) and h_{-mu} (first layer) never share a site, so the offsets +-2 mu
    vanish and 33 offsets remain.  A direction of lattice extent 1 (a lower-
    dimensional lattice embedded in four dimensions) has hops that return to
    the same site: they read inside the block and belong to h_0."""
    dirs = getattr(op, "hop_dirs", range(4))
    local = [mu for mu in range(4) if op.dims[mu] == 1]
    if min([T.block[mu] for mu in dirs if mu not in local] or [2]) < 2:
        raise ValueError("the squared coarse stencil needs block extents >= 2")
    Nv = T.Nv
    Xc, Yc, Zc, Tc = T.cdims
    src = [(0, 0, 0, 0)] + OFFSETS33[1:9]
    pieces = np.empty((9, Nv, int(np.prod(T.cdims)), T.S * int(np.prod(T.block)) * T.n), dtype=np.complex128)
    for l in range(Nv):
        q = T.vector(l)
        rest = op.apply(q)
        op.count -= 1  # construction applies are not solver cost
        for mu in range(4):
            for d in (+1, -1):
                if mu in local:
                    pieces[CoarseOp.dir_index(mu, d), l] = 0.0
                    continue
                h = op.hop(q, mu, d) * crossing_mask(op.dims, T.block, op.S, mu, d)
                rest = rest - h
                pieces[CoarseOp.dir_index(mu, d), l] = to_blocks(h, T.dims, T.block)
        pieces[0, l] = to_blocks(rest, T.dims, T.block)
    Y = np.zeros((Tc, Zc, Yc, Xc, 33, Nv, Nv), dtype=np.complex128)
    index = {o: j for j, o in enumerate(OFFSETS33)}
    for i1, s1 in enumerate(src):
        for i2, s2 in enumerate(src):
            delta = tuple(b - a for a, b in zip(s1, s2))
            if delta not in index:
                continue  # +-2 mu: disjoint supports (checked against brute force)
            G = np.einsum("kbi,lbi->bkl", np.conj(pieces[i1]), pieces[i2])
            G = G.reshape(1, Tc, Zc, Yc, Xc, Nv, Nv)
            # row b = b'' + sigma1: the value at b is G(b - sigma1)
            Y[..., index[delta], :, :] += _shift_vec(G, tuple(-o for o in s1))[0]
    return SquaredCoarseOp(Y, T.cdims)


def squared_coarse_bruteforce(op, T: Transfer) -> np.ndarray:
    """Dense (D P)^+ (D P) from the dense prolongator (tiny cases only)."""
    Nc = int(np.prod(T.cshape))
    e = np.zeros(Nc, dtype=np.complex128)
    cols = []
    for j in range(Nc):
        e[j] = 1.0
        cols.append(op.apply(T.prolong(e.reshape(T.cshape))).ravel())
        e[j] = 0.0
    DP = np.stack(cols, axis=1)
    return DP.conj().T @ DP


def dense_matrix(apply: Callable, shape) -> np.ndarray:
    """Dense matrix of a linear map by applying it to every unit vector (tiny cases)."""
    N = int(np.prod(shape))
    M = np.empty((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        e[j] = 1.0
        M[:, j] = apply(e.reshape(shape)).ravel()
        e[j] = 0.0
    return M


def coarse_operator_bruteforce(op, T: Transfer) -> np.ndarray:
    """Dense P^+ A P from the dense prolongator and dense A (tiny cases only)."""
    Nc = int(np.prod(T.cshape))
    cols = []
    e = np.zeros(Nc, dtype=np.complex128)
    for j in range(Nc):
        e[j] = 1.0
        cols.append(T.prolong(e.reshape(T.cshape)).ravel())
        e[j] = 0.0
    P = np.stack(cols, axis=1)
    AP = np.stack([op.apply(P[:, j].reshape(op.shape)).ravel() for j in range(Nc)], axis=1)
    return P.conj().T @ AP


# ---------------------------------------------------------------------------
# Krylov solvers
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class SolveInfo:
    iters: int = 0
    converged: bool = False
    rel_res: float = float("nan")
    history: List[float] = dataclasses.field(default_factory=list)


def gcr(A: Callable, b, x0=None, tol=1e-10, maxiter=1000, restart=10,
        M: Optional[Callable] = None, info: Optional[SolveInfo] = None, min_iter: int = 0):
    """Flexible GCR with right preconditioner M (Sec. 3: the outer solver must
    tolerate a preconditioner that changes between applications).

    Per iteration: z = M(r), w = A z, w orthogonalised against the stored
    directions by modified Gram-Schmidt (z updated alike), both scaled so
    |w| = 1, then x += <w, r> z and r -= <w, r> w.  After `restart`
    directions the history is dropped and r recomputed from b - A x.
    Stops when |r| / |b| <= tol (the iterated residual) or after maxiter.
    """
    info = info if info is not None else SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = norm(b)
    if bnorm == 0.0:
        if x0 is None:
            info.converged = True
            info.rel_res = 0.0
            return np.zeros_like(b), info
        bnorm = 1.0  # A x = 0 from a nonzero start (adaptive setup): absolute residual
    r = b - A(x) if x0 is not None else b.copy()
    rn = norm(r)
    info.history.append(rn / bnorm)
    Z: list = []
    W: list = []
    it = 0
    while it < maxiter and (rn / bnorm > tol or it < min_iter):
        z = M(r) if M is not None else r.copy()
        w = A(z)
        for zi, wi in zip(Z, W):
            beta = vdot(wi, w)
            w = w - beta * wi
            z = z - beta * zi
        wn = norm(w)
        if wn == 0.0 or not np.isfinite(wn):
            break
        w = w / wn
        z = z / wn
        alpha = vdot(w, r)
        x = x + alpha * z
        r = r - alpha * w
        it += 1
        rn = norm(r)
        info.history.append(rn / bnorm)
        Z.append(z)
        W.append(w)
        if len(Z) == restart:
            Z, W = [], []
            r = b - A(x)
            rn = norm(r)
    info.iters = it
    info.rel_res = rn / bnorm
    info.converged = rn / bnorm <= tol
    return x, info


def cgnr(A: Callable, Adag: Callable, b, tol=1e-10, maxiter=100000, x0=None, info=None, check_every=1):
    """CG on the normal equations A^+ A x = A^+ b (the paper's comparison solver,
    Sec. 3: CG on the squared operator).  Stops on |b - A x| / |b| <= tol,
    using the recursively updated residual of the unsquared system, tested
    every `check_every` iterations.  For A x = 0 from a nonzero start the
    test is relative to the initial residual |A x0|."""
    info = info if info is not None else SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    bnorm = norm(b) or norm(r) or 1.0
    z = Adag(r)
    p = z.copy()
    zz = vdot(z, z).real
    it = 0
    rn = norm(r)
    info.history.append(rn / bnorm)
    while it < maxiter and (rn / bnorm > tol or it % check_every):
        w = A(p)
        a = zz / vdot(w, w).real
        x = x + a * p
        r = r - a * w
        z = Adag(r)
        zz_new = vdot(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
        it += 1
        rn = norm(r)
        info.history.append(rn / bnorm)
    info.iters = it
    info.rel_res = rn / bnorm
    info.converged = rn / bnorm <= tol
    return x, info


# ---------------------------------------------------------------------------
# Multigrid
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class MGParams:
    """Multigrid parameters.  The paper leaves the smoothers S1, S3, the coarse
    solver S2 and the nu's open; these defaults are this library's choices.

    Smoother: nu steps of CG on the normal equations (CGNR).  Minimal-residual
    relaxation on D itself does not smooth the Shamir operator, whose
    eigenvalues lie on both sides of the imaginary axis around the origin."""
    nvec: tuple = (8,)                 # coarse components per site (Nvec) per transfer
    block: tuple = ((2, 2, 2, 2),)     # 4D block per transfer (fifth dim collapsed)
    nu_pre: int = 0                    # nu_1
    nu_post: int = 8                   # nu_3
    coarse_tol: float = 0.1            # S2 tolerance on intermediate levels
    coarse_maxiter: int = 24
    coarsest_tol: float = 0.1          # S2 on the coarsest level
    coarsest_maxiter: int = 64
    coarse_restart: int = 16
    setup_iters0: int = 1000           # CGNR iterations on A x = 0 for the initial vectors, at most
    setup_tol0: float = 1e-6           # ... or until |A x| <= setup_tol0 |A x0| (tested every 8)
    setup_sweeps: int = 0              # inverse-iteration sweeps with the current MG
    setup_sweep_iters: int = 8         # MG-GCR iterations per vector per sweep, at most
    setup_sweep_tol: float = 0.1       # MG-GCR relative tolerance of a sweep's solve
    split: bool = True                 # split each vector into its Gamma = +1 / -1 halves:
                                       # Nvec/2 adaptive vectors give Nvec coarse components
    cycle: str = "K"                   # S2 on intermediate levels: "K" = GCR preconditioned by
                                       # the next V-cycle; "W" = two V-cycles (Sec. 2's W-cycle)
    coarsen: str = "unsquared"         # "unsquared": R D P (9 points); "squared": the paper's
                                       # P^+ D^+ D P (Sec. 4), two levels only


def gamma_halves(op, v):
    """(1 + Gamma)/2 v and (1 - Gamma)/2 v.  On the fine level Gamma = gamma_5 R_5
    (spin sign +,+,-,- and s -> Ls-1-s); on a coarse level built from split
    vectors Gamma is +1 on even and -1 on odd coarse components."""
    if hasattr(op, "gamma5r5"):
        g = op.gamma5r5(v)
    elif isinstance(op, FineOp):
        g = v[::-1].copy()
        g[..., 6:] *= -1
    else:
        g = v.copy()
        g[..., 1::2] *= -1
    return 0.5 * (v + g), 0.5 * (v - g)


class Level:
    def __init__(self, op):
        self.op = op
        self.transfer: Optional[Transfer] = None


class MG:
    """Levels 0..L-1: level 0 is the fine DWF operator, level l+1 = R_l A_l P_l."""

    def __init__(self, fine_op, params: MGParams):
        self.p = params
        self.levels: List[Level] = [Level(fine_op)]
        self.vectors: List = []  # the (unsplit, normalised) adaptive vectors per level

    @property
    def nlevels(self):
        return len(self.levels)

    def build_from_vectors(self, l: int, vectors):
        """Build the transfer at level l from the given near-null vectors and
        the Galerkin coarse operator of level l+1 (drops deeper levels)."""
        lev = self.levels[l]
        del self.vectors[l:]
        self.vectors.append(vectors)
        if self.p.split:
            vectors = np.stack([h for v in vectors for h in gamma_halves(lev.op, v)])
        T = Transfer(vectors, lev.op.dims, self.p.block[l])
        lev.transfer = T
        if self.p.coarsen == "squared":
            if len(self.p.nvec) != 1:
                raise ValueError("the squared coarsening is built for two levels")
            coarse = squared_coarse_operator(lev.op, T)
        else:
            coarse = coarse_operator(lev.op, T)
        del self.levels[l + 1:]
        self.levels.append(Level(coarse))

    # -- the V-cycle (Sec. 2) ------------------------------------------------
    def smooth(self, l, b, nu):
        """S1 / S3: nu CGNR iterations on A_l x = b from x = 0."""
        if nu == 0:
            return np.zeros_like(b)
        op = self.levels[l].op
        x, _ = cgnr(op.apply, op.apply_dag, b, tol=0.0, maxiter=nu)
        return x

    def coarse_solve(self, l, b):
        """S2 on level l >= 1: GCR on R A P, preconditioned by the V-cycle of the
        next level when there is one (the recursion of Sec. 2); with cycle "W"
        S2 is two V-cycles of level l instead (Sec. 2: replacing S2 by two
        V-cycles gives the W-cycle): x = V(b), then x += V(b - A x)."""
        A = self.levels[l].op.apply
        if l == self.nlevels - 1:
            x, _ = gcr(A, b, tol=self.p.coarsest_tol, maxiter=self.p.coarsest_maxiter,
                       restart=self.p.coarse_restart)
        elif self.p.cycle == "W":
            x = self.vcycle(l, b)
            x = x + self.vcycle(l, b - A(x))
        else:
            x, _ = gcr(A, b, tol=self.p.coarse_tol, maxiter=self.p.coarse_maxiter,
                       restart=self.p.coarse_restart, M=lambda r: self.vcycle(l, r))
        return x

    def vcycle(self, l, b):
        """One V-cycle for A_l x = b, the five steps of Sec. 2:
          x1 = S1^nu1(A, b)
          b2 = R (b - A x1)
          x2 = S2^nu2(R A P, b2)
          b3 = b - A (P x2 + x1)
          x  = x1 + P x2 + S3^nu3(A, b3)
        With the squared coarsening the coarse problem is that of the normal
        equations, D^+ D x = D^+ r, so b2 = R D^+ (b - A x1) (Sec. 4)."""
        A = self.levels[l].op.apply
        T = self.levels[l].transfer
        x1 = self.smooth(l, b, self.p.nu_pre)
        r1 = b - A(x1) if self.p.nu_pre else b
        if self.p.coarsen == "squared" and l == 0:
            r1 = self.levels[0].op.apply_dag(r1)
        b2 = T.restrict(r1)
        x2 = self.coarse_solve(l + 1, b2)
        Px2 = T.prolong(x2)
        b3 = b - A(Px2 + x1)
        return x1 + Px2 + self.smooth(l, b3, self.p.nu_post)

    def precondition(self, r):
        return self.vcycle(0, r)


def initial_vectors(op, nvec, random_vectors, p: MGParams):
    """Adaptive start (Sec. 2): a Krylov solver (CGNR) on A x = 0 from each
    random vector; what it fails to remove is near-null.  Each result is
    normalised."""
    out = []
    for k in range(nvec):
        x0 = random_vectors[k].reshape(op.shape)
        x, _ = cgnr(op.apply, op.apply_dag, np.zeros_like(x0), x0=x0, tol=p.setup_tol0,
                    maxiter=p.setup_iters0, check_every=8)
        out.append(x / norm(x))
    return np.stack(out)


def nvectors(p: MGParams, l: int) -> int:
    """Adaptive vectors needed at level l: Nvec, or Nvec/2 when they are split."""
    if p.split:
        if p.nvec[l] % 2:
            raise ValueError("split coarse spaces need an even Nvec")
        return p.nvec[l] // 2
    return p.nvec[l]


def orthonormalise_global(vecs):
    """Two passes of modified Gram-Schmidt over the whole set of vectors."""
    out = [np.array(v, copy=True) for v in vecs]
    for _pass in range(2):
        for j in range(len(out)):
            for i in range(j):
                out[j] = out[j] - vdot(out[i], out[j]) * out[i]
            out[j] = out[j] / norm(out[j])
    return np.stack(out)


def adaptive_setup(fine_op, p: MGParams, random_vectors_per_level) -> MG:
    """The adaptive setup of Sec. 2, level by level:
      1. start vectors: Krylov iterations (CGNR) on A x = 0 from random
         vectors, normalised, then orthonormalised as a set;
      2. build the transfer (block Gram-Schmidt) and R A P;
      3. sweeps: each vector is replaced by an approximate solution of
         A x = v with the current multigrid (GCR preconditioned by the
         V-cycle, loose tolerance) -- inverse iteration, which amplifies
         exactly the modes the solver finds hard -- the set is
         re-orthonormalised, and the multigrid rebuilt ("repeated for as long
         as necessary").
    random_vectors_per_level[l] holds nvectors(p, l) random fields of level l."""
    mg = MG(fine_op, p)
    nl = len(p.nvec)
    for l in range(nl):
        op = mg.levels[l].op
        nv = nvectors(p, l)
        vecs = orthonormalise_global(initial_vectors(op, nv, random_vectors_per_level[l], p))
        mg.build_from_vectors(l, vecs)
        for _ in range(p.setup_sweeps):
            new = []
            for k in range(nv):
                x, _ = gcr(op.apply, vecs[k], tol=p.setup_sweep_tol, maxiter=p.setup_sweep_iters,
                           restart=p.setup_sweep_iters + 1, M=lambda r, l=l: mg.vcycle(l, r))
                new.append(x / norm(x))
            vecs = orthonormalise_global(np.stack(new))
            mg.build_from_vectors(l, vecs)
    return mg


def mg_solve(mg: MG, b, tol=1e-10, maxiter=500, restart=20, x0=None):
    """Outer flexible GCR on the fine operator, preconditioned by one V-cycle
    per iteration (Sec. 3)."""
    A = mg.levels[0].op.apply
    return gcr(A, b, x0=x0, tol=tol, maxiter=maxiter, restart=restart, M=mg.precondition)
