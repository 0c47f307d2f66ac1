"""FP64 oracle of the low-mode diagnostic (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Sec. 2, Fig. 1) judges a coarse space by how much of each low
eigenmode of the Dirac operator it contains.  Here: the smallest eigenpairs
of the Hermitian positive operator D^+ D, and the fraction |P P^+ v|^2 / |v|^2
of a field v that lies in the coarse space of a transfer (P block-orthonormal,
so P P^+ is the orthogonal projector onto that space).

Parity pins (tests/test_oracle_eig.py): on a free lattice the eigenvalues of
D^+ D are the squared singular values of the momentum-space symbol over all
momenta (three colours each); eigen-residuals and orthonormality; the
projector fraction is 1 on the coarse space and 0 on its orthogonal
complement.
"""
from __future__ import annotations

import numpy as np

from .mg import Transfer, dense_matrix, norm


def lowest_modes(op, k):
    """The k smallest eigenvalues (ascending) and eigenvectors of D^+ D by a
    dense Hermitian eigensolver (numpy eigh of the explicit matrix; tiny
    lattices only).  Vectors come back in the level's field shape."""
    M = dense_matrix(lambda f: op.apply_dag(op.apply(f)), op.shape)
    M = 0.5 * (M + M.conj().T)
    w, V = np.linalg.eigh(M)
    return w[:k], np.ascontiguousarray(V[:, :k].T).reshape((k,) + tuple(op.shape))


def coarse_overlap(T: Transfer, v):
    """|P P^+ v|^2 / |v|^2: the share of v inside the coarse space."""
    pv = T.prolong(T.restrict(v))
    return norm(pv) ** 2 / norm(v) ** 2
