"""FP64 oracle of the two-dimensional U(1) domain-wall operator, the paper's
toy model (Sec. 3: a 20^2 x 8 quenched U(1) lattice, 16 near-null vectors,
4^2 x 8 blocks, masses 0.01 to 0.10).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper writes no formula for the operator; this is the two-dimensional
analogue of the Shamir operator of the four-dimensional oracle, with
2-component spinors: gamma_x = sigma_1, gamma_y = sigma_2, chirality sigma_3
(P_+ keeps spin 0, P_- spin 1), diagonal d + 1 - M5 with d = 2, hops
-1/2 (1 -+ gamma_mu) U, fifth-dimension hops -P_-+ and wall terms +m_f,
periodic in x and (flag) antiperiodic in y, D^+ = Gamma D Gamma with
Gamma = sigma_3 R_5.

Fields have the multigrid oracle's layout (S, T, Z, Y, X, n) with T = Z = 1,
S = Ls and n = 2, so that oracle/mg.py (blocking, transfers, coarse
operators, solvers, V-cycle, setup) runs on it unchanged; lattice dims are
(X, Y, 1, 1).

Parity pins (tests/test_oracle_u1.py): free-field spectrum against the
momentum-space block matrix, the Ls = 1 Wilson limit against its closed
form, Gamma-hermiticity (adjointness), U(1) gauge covariance, m_f confined
to the walls.  Nothing here is "parity unpinned".
"""
from __future__ import annotations

import numpy as np

SIGMA = (np.array([[0, 1], [1, 0]], dtype=np.complex128),
         np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
         np.array([[1, 0], [0, -1]], dtype=np.complex128))
P_PLUS = np.diag([1.0, 0.0]).astype(np.complex128)
P_MINUS = np.diag([0.0, 1.0]).astype(np.complex128)


class DWF2D:
    """The 2D U(1) Shamir operator on link angles theta (2, Y, X)."""

    def __init__(self, theta, dims2, Ls, M5, mf, antiperiodic_y=True):
        self.X, self.Y = int(dims2[0]), int(dims2[1])
        self.dims = (self.X, self.Y, 1, 1)
        self.S = int(Ls)
        self.n = 2
        self.M5, self.mf = float(M5), float(mf)
        self.ap = bool(antiperiodic_y)
        self.U = np.exp(1j * np.asarray(theta, dtype=np.float64))  # (2, Y, X)
        self.shape = (self.S, 1, 1, self.Y, self.X, 2)
        self.hop_dirs = (0, 1)
        self.count = 0

    # -- pieces --------------------------------------------------------------
    def _shift(self, f, mu, d):
        """f(x + d mu) (fields (S, 1, 1, Y, X, 2)), with the antiperiodic sign
        when a y-hop wraps around."""
        axis = 4 if mu == 0 else 3
        g = np.roll(f, -d, axis=axis)
        if mu == 1 and self.ap:
            g = g.copy()
            if d > 0:
                g[:, :, :, self.Y - 1] *= -1
            else:
                g[:, :, :, 0] *= -1
        return g

    def _link(self, mu, d):
        """U_mu(x) for d = +1, conj(U_mu(x - mu)) for d = -1, shaped to broadcast over fields."""
        u = self.U[mu]
        if d < 0:
            u = np.conj(np.roll(u, 1, axis=(1 if mu == 0 else 0)))
        return u[None, None, None, :, :, None]

    def hop(self, f, mu, d):
        """-1/2 (1 - d sigma_mu) U^(d) f(x + d mu); zero for mu = 2, 3 (no such directions)."""
        f = f.reshape(self.shape)
        if mu >= 2:
            return np.zeros_like(f)
        proj = np.eye(2) - d * SIGMA[mu]
        t = self._link(mu, d) * self._shift(f, mu, d)
        return -0.5 * np.einsum("ab,...b->...a", proj, t)

    def gamma5r5(self, f):
        """Gamma f: (Gamma f)(s) = sigma_3 f(Ls - 1 - s)."""
        g = f.reshape(self.shape)[::-1].copy()
        g[..., 1] *= -1
        return g

    # -- the operator --------------------------------------------------------
    def apply(self, f):
        self.count += 1
        f = f.reshape(self.shape)
        out = (3.0 - self.M5) * f
        for mu in range(2):
            for d in (+1, -1):
                out = out + self.hop(f, mu, d)
        # fifth dimension: -P_- f(s + 1) - P_+ f(s - 1), walls +m_f
        up = np.roll(f, -1, axis=0)    # f(s + 1), s = Ls-1 reads f(0)
        dn = np.roll(f, 1, axis=0)     # f(s - 1), s = 0 reads f(Ls-1)
        cu = np.full(self.S, -1.0)
        cu[self.S - 1] = self.mf
        cd = np.full(self.S, -1.0)
        cd[0] = self.mf
        out = out + cu[:, None, None, None, None, None] * np.einsum("ab,...b->...a", P_MINUS, up)
        out = out + cd[:, None, None, None, None, None] * np.einsum("ab,...b->...a", P_PLUS, dn)
        return out

    def apply_dag(self, f):
        """D^+ = Gamma D Gamma (counted as one application by the inner apply)."""
        return self.gamma5r5(self.apply(self.gamma5r5(f)))


def momentum_matrix(p, Ls, M5, mf):
    """D(p) on plane waves e^{i p.x} (free field): a (2 Ls) x (2 Ls) matrix,
    index s * 2 + spin, written out from the operator's definition in momentum
    space: W(p) = 3 - M5 - sum cos p_mu + i sum sigma_mu sin p_mu on the
    diagonal, -P_- / -P_+ to s + 1 / s - 1, +m_f at the walls."""
    W = (3.0 - M5 - np.cos(p[0]) - np.cos(p[1])) * np.eye(2) + 1j * (np.sin(p[0]) * SIGMA[0] + np.sin(p[1]) * SIGMA[1])
    M = np.zeros((2 * Ls, 2 * Ls), dtype=np.complex128)
    for s in range(Ls):
        M[2 * s:2 * s + 2, 2 * s:2 * s + 2] += W
        su, sd = (s + 1) % Ls, (s - 1) % Ls
        M[2 * s:2 * s + 2, 2 * su:2 * su + 2] += (mf if s == Ls - 1 else -1.0) * P_MINUS
        M[2 * s:2 * s + 2, 2 * sd:2 * sd + 2] += (mf if s == 0 else -1.0) * P_PLUS
    return M
