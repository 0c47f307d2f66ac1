"""The forms of CGNR the FP32 batched smoother takes, checked on the CPU
against the oracle's CGNR (CG on the normal equations, the comparison
solver of Sec. 3 and the smoother of the V-cycle) on a small dense system.

The oracle updates r <- r - a w, forms z = A^+ r and keeps a direction p
with x <- x + a p.  The batched smoother instead keeps the normal-equations
residuals z_k, carries w = A p by w_{k+1} = A z_{k+1} + b_k w_k, and forms x
from the kept z: all at once (the post-smoother) or chunk by chunk (the
setup's relaxation, which also carries the first direction of each chunk).
In exact arithmetic all are the same iterates; in FP64 they agree to
rounding.  The formulas are written out here from that algebra, not taken
from the library."""
import numpy as np
import pytest

from oracle import mg as OM


def _system(n=48, seed=3):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 3.0 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def _oracle_x(A, b, nu):
    x, info = OM.cgnr(lambda v: A @ v, lambda v: A.conj().T @ v, b, tol=0.0, maxiter=nu)
    assert info.iters == nu
    return x


def _nrm2(v):
    return float(np.vdot(v, v).real)


def _kept_residuals(A, b, nu):
    """The post-smoother's form: z_0 .. z_{nu-1} kept, w by recursion, x once."""
    Ah = A.conj().T
    z = [Ah @ b]
    w = A @ z[0]
    zz, ww = [_nrm2(z[0])], [_nrm2(w)]
    for k in range(nu - 1):
        a = zz[k] / ww[k]
        z.append(z[k] - a * (Ah @ w))
        zz.append(_nrm2(z[k + 1]))
        beta = zz[k + 1] / zz[k]
        w = A @ z[k + 1] + beta * w
        ww.append(_nrm2(w))
    g = 0.0
    x = np.zeros_like(b)
    for j in range(nu - 1, -1, -1):
        a = zz[j] / ww[j]
        beta = zz[j + 1] / zz[j] if j + 1 < nu else 0.0
        g = a + beta * g
        x = x + g * z[j]
    return x


def _chunks(A, b, nu, m):
    """The setup relaxation's form: chunks of m iterations; each chunk's end adds
    sum a_k p_k to x and forms the next chunk's first direction from the
    chunk's first direction and its kept residuals."""
    Ah = A.conj().T
    z = {0: Ah @ b}
    p = z[0].copy()
    w = A @ p
    zz, ww = {0: _nrm2(z[0])}, {0: _nrm2(w)}
    x = np.zeros_like(b)
    k0 = 0
    while k0 < nu:
        k1 = min(k0 + m, nu)
        last = k1 == nu
        for k in range(k0, k1 - 1 if last else k1):
            a = zz[k] / ww[k]
            z[k + 1] = z[k] - a * (Ah @ w)
            zz[k + 1] = _nrm2(z[k + 1])
            w = A @ z[k + 1] + (zz[k + 1] / zz[k]) * w
            ww[k + 1] = _nrm2(w)
        mm = k1 - k0
        G = [0.0] * mm
        P = [0.0] * (mm + 1)
        g, q = 0.0, 1.0
        P[mm] = 1.0
        for t in range(mm - 1, -1, -1):
            a = zz[k0 + t] / ww[k0 + t]
            beta = zz[k0 + t + 1] / zz[k0 + t] if (t + 1 < mm or not last) else 0.0
            g = a + (beta * g if t + 1 < mm else 0.0)
            G[t] = g
            q *= beta
            P[t] = q
        x = x + G[0] * p + sum(G[t] * z[k0 + t] for t in range(1, mm))
        if not last:
            p = P[0] * p + sum(P[t] * z[k0 + t] for t in range(1, mm + 1))
        k0 = k1
    return x


@pytest.mark.parametrize("nu", [1, 2, 5, 16])
def test_kept_residual_form_equals_cgnr(nu):
    A, b = _system()
    ref = _oracle_x(A, b, nu)
    got = _kept_residuals(A, b, nu)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("nu,m", [(16, 8), (17, 8), (8, 8), (7, 3), (1, 8)])
def test_chunked_form_equals_cgnr(nu, m):
    A, b = _system(seed=5)
    ref = _oracle_x(A, b, nu)
    got = _chunks(A, b, nu, m)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


def test_forms_differ_from_a_wrong_recursion():
    """A sign slip in the w recursion (w = A z - b w) must not pass."""
    A, b = _system(seed=7)
    nu = 6
    Ah = A.conj().T
    z = [Ah @ b]
    w = A @ z[0]
    zz, ww = [_nrm2(z[0])], [_nrm2(w)]
    for k in range(nu - 1):
        z.append(z[k] - zz[k] / ww[k] * (Ah @ w))
        zz.append(_nrm2(z[k + 1]))
        w = A @ z[k + 1] - (zz[k + 1] / zz[k]) * w
        ww.append(_nrm2(w))
    g, x = 0.0, np.zeros_like(b)
    for j in range(nu - 1, -1, -1):
        g = zz[j] / ww[j] + (zz[j + 1] / zz[j] if j + 1 < nu else 0.0) * g
        x = x + g * z[j]
    ref = _oracle_x(A, b, nu)
    assert np.linalg.norm(x - ref) > 1e-3 * np.linalg.norm(ref)
