"""Pins of the low-mode diagnostic oracle (oracle/eig.py)."""
import numpy as np
import pytest

import oracle
from oracle import eig as E
from oracle import mg as OM
import paper_1205_2933_gb300.inputs as I
from test_oracle_dwf import _symbol


def test_free_field_lowest_modes_are_squared_singular_values():
    """Unit links: the spectrum of D^+ D is the union over momenta of the
    squared singular values of the symbol D(p), each three times (colour)."""
    dims, Ls, M5, mf = (2, 2, 2, 2), 2, 1.8, 0.1
    op = OM.FineOp(oracle.DWF(I.unit_links(dims), dims, Ls, M5, mf, antiperiodic_t=True))
    k = 24
    w, V = E.lowest_modes(op, k)
    ref = []
    for nx in range(2):
        for ny in range(2):
            for nz in range(2):
                for nt in range(2):
                    p = [np.pi * nx, np.pi * ny, np.pi * nz, np.pi * (nt + 0.5)]
                    ref += list(np.linalg.svd(_symbol(Ls, M5, mf, p), compute_uv=False) ** 2) * 3
    ref = np.sort(np.array(ref))[:k]
    assert np.abs(w - ref).max() < 1e-12 * ref.max()


def test_eigenpairs_residual_and_orthonormality():
    dims, Ls = (2, 2, 2, 4), 4
    op = OM.FineOp(oracle.DWF(I.epsilon_links(dims, 0.4, 5), dims, Ls, 1.8, 0.01))
    w, V = E.lowest_modes(op, 6)
    assert np.all(np.diff(w) >= 0) and w[0] > 0
    for j in range(6):
        r = op.apply_dag(op.apply(V[j])) - w[j] * V[j]
        assert OM.norm(r) < 1e-10 * max(w[j], 1e-3)
    G = np.array([[OM.vdot(V[i], V[j]) for j in range(6)] for i in range(6)])
    assert np.abs(G - np.eye(6)).max() < 1e-12


def test_coarse_overlap_closed_forms():
    dims, Ls, block = (4, 4, 2, 2), 4, (2, 2, 2, 2)
    op = OM.FineOp(oracle.DWF(I.epsilon_links(dims, 0.4, 6), dims, Ls, 1.8, 0.05))
    vecs = I.random_vectors(3, dims, Ls, 7).reshape((3,) + op.shape)
    T = OM.Transfer(vecs, dims, block)
    v = vecs[1]
    assert abs(E.coarse_overlap(T, v) - 1.0) < 1e-12           # the vectors themselves
    f = I.gaussian_source(dims, Ls, 9).reshape(op.shape)
    perp = f - T.prolong(T.restrict(f))
    assert E.coarse_overlap(T, perp) < 1e-24                     # the orthogonal complement
    a = E.coarse_overlap(T, f)
    assert 0.0 < a < 1.0
