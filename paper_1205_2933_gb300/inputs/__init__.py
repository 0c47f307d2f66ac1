"""Seeded synthetic inputs shared by the GPU path and the FP64 oracle.

Nothing here computes any part of the multigrid solve.  The module makes
gauge fields (epsilon-random SU(3) links, or a quenched Wilson-gauge
heatbath) and random 5D fields (Gaussian sources, point and Z2 wall
sources, random starting vectors for the adaptive setup).

Array conventions (numpy, complex128):
  links   : shape (T, Z, Y, X, 4, 3, 3); mu = 0..3 is x, y, z, t
  fermion : shape (Ls, T, Z, Y, X, 4, 3)  -- s slowest, then the 4D site
            (x fastest), then spin, then colour.  This is the canonical
            ("user") layout of the library's pack/unpack calls.
Dimensions are always given as dims = (X, Y, Z, T).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SO = _HERE / "libdwfinputs.so"
_lib = None

# Stream identifiers of the counter-based generator (second key word).
STREAM_LINKS_EPS = 1
STREAM_HOTSTART = 2
STREAM_SOURCE = 3
STREAM_NULLVEC = 4
STREAM_Z2 = 5
STREAM_GAUGE_TRANSFORM = 6
STREAM_NETWORK = 7
STREAM_U1 = 8


def build(force: bool = False) -> pathlib.Path:
    """Compile the input generator's C code into an in-tree shared library."""
    src = _HERE / "dwfinputs.c"
    if force or not _SO.exists() or _SO.stat().st_mtime < src.stat().st_mtime:
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", str(src), "-o",
               str(_SO) + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(str(_SO) + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_SO))
        dp = ctypes.POINTER(ctypes.c_double)
        u32 = ctypes.c_uint32
        i64 = ctypes.c_int64
        L.dwfin_philox4x32_10.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
        L.dwfin_uniform.argtypes = [dp, i64, u32, u32, u32, u32]
        L.dwfin_gauss_complex.argtypes = [dp, i64, ctypes.c_double, u32, u32]
        L.dwfin_project_su3_field.argtypes = [dp, i64]
        L.dwfin_plaquette.argtypes = [dp, ctypes.POINTER(ctypes.c_int)]
        L.dwfin_plaquette.restype = ctypes.c_double
        L.dwfin_kp_samples.argtypes = [dp, i64, ctypes.c_double, u32]
        L.dwfin_random_su3.argtypes = [dp, i64, u32, u32]
        L.dwfin_heatbath.argtypes = [dp, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, u32]
        L.dwfin_heatbath.restype = ctypes.c_int
        L.dwfin_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def philox(counter, key):
    """One Philox-4x32-10 block: four 32-bit words for a 4-word counter and 2-word key."""
    c = (ctypes.c_uint32 * 4)(*counter)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().dwfin_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(n: int, seed: int, stream: int, c1: int = 0, c2: int = 0) -> np.ndarray:
    out = np.empty(int(n), dtype=np.float64)
    lib().dwfin_uniform(_dp(out), int(n), seed, stream, c1, c2)
    return out


def gauss_complex(shape, seed: int, stream: int, sigma: float = 1.0) -> np.ndarray:
    """Complex array whose real and imaginary parts are i.i.d. N(0, sigma^2)."""
    out = np.empty(tuple(shape), dtype=np.complex128)
    lib().dwfin_gauss_complex(_dp(out.view(np.float64)), out.size, float(sigma), seed, stream)
    return out


def lattice_shape(dims):
    X, Y, Z, T = [int(d) for d in dims]
    return (T, Z, Y, X)


def project_su3(U: np.ndarray) -> np.ndarray:
    """Project every 3x3 matrix onto SU(3) (row Gram-Schmidt, row 2 = conj(row0 x row1))."""
    U = np.ascontiguousarray(U, dtype=np.complex128)
    lib().dwfin_project_su3_field(_dp(U.view(np.float64)), U.size // 9)
    return U


def epsilon_links(dims, eps: float, seed: int) -> np.ndarray:
    """U = exp(i eps H) with H random traceless Hermitian built from Gaussian entries.

    A has real and imaginary parts ~ N(0, 1/2); H = (A + A^+)/2 - tr(.)/3.
    The exponential is taken through the eigendecomposition of H, then each
    matrix is projected onto SU(3) so that it is unitary with det 1 to
    rounding.
    """
    shape = lattice_shape(dims) + (4, 3, 3)
    A = gauss_complex(shape, seed, STREAM_LINKS_EPS, sigma=np.sqrt(0.5))
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    w, Q = np.linalg.eigh(H)
    U = np.einsum("...ab,...b,...cb->...ac", Q, np.exp(1j * eps * w), np.conj(Q))
    return project_su3(U)


def unit_links(dims) -> np.ndarray:
    shape = lattice_shape(dims) + (4, 3, 3)
    U = np.zeros(shape, dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def random_su3(n: int, seed: int, stream: int = STREAM_HOTSTART) -> np.ndarray:
    U = np.empty((int(n), 3, 3), dtype=np.complex128)
    lib().dwfin_random_su3(_dp(U.view(np.float64)), int(n), seed, stream)
    return U


def plaquette(U: np.ndarray, dims) -> float:
    U = np.ascontiguousarray(U)
    return float(lib().dwfin_plaquette(_dp(U.view(np.float64)), _dims(dims)))


def kp_samples(n: int, bp: float, seed: int) -> np.ndarray:
    out = np.empty(int(n), dtype=np.float64)
    lib().dwfin_kp_samples(_dp(out), int(n), float(bp), seed)
    return out


def _cache_dir():
    d = os.environ.get("DWFMG_CACHE", "/tmp/dwfmg_cache")
    pathlib.Path(d).mkdir(parents=True, exist_ok=True)
    return pathlib.Path(d)


def heatbath_links(dims, beta: float, sweeps: int, seed: int, cache: bool = True) -> np.ndarray:
    """Quenched Wilson-gauge links: hot start then `sweeps` Cabibbo-Marinari sweeps.

    Results are cached on local disk keyed by (dims, beta, sweeps, seed) since
    a 16^3x32 field at 200 sweeps costs seconds to minutes of host time.
    """
    dims = [int(d) for d in dims]
    key = hashlib.sha1(repr(("hb1", dims, float(beta), int(sweeps), int(seed))).encode()).hexdigest()[:16]
    path = _cache_dir() / f"hb_{key}.npy"
    if cache and path.exists():
        U = np.load(path)
        if U.shape == lattice_shape(dims) + (4, 3, 3):
            return U
    V = int(np.prod(dims))
    U = random_su3(4 * V, seed, STREAM_HOTSTART).reshape(lattice_shape(dims) + (4, 3, 3))
    U = np.ascontiguousarray(U)
    rc = lib().dwfin_heatbath(_dp(U.view(np.float64)), _dims(dims), float(beta), int(sweeps), 0, seed)
    if rc != 0:
        raise ValueError("heatbath needs even lattice extents")
    if cache:
        tmp = path.with_suffix(".tmp.npy")
        np.save(tmp, U)
        os.replace(tmp, path)
    return U


def fermion_shape(dims, Ls: int):
    return (int(Ls),) + lattice_shape(dims) + (4, 3)


def gaussian_source(dims, Ls: int, seed: int, stream: int = STREAM_SOURCE) -> np.ndarray:
    """5D source with real and imaginary parts i.i.d. N(0,1)."""
    return gauss_complex(fermion_shape(dims, Ls), seed, stream, 1.0)


def random_vectors(n: int, dims, Ls: int, seed: int) -> np.ndarray:
    """n Gaussian 5D fields, the starting vectors of the adaptive setup."""
    return gauss_complex((int(n),) + fermion_shape(dims, Ls), seed, STREAM_NULLVEC, 1.0)


def wall_source(eta4: np.ndarray, Ls: int) -> np.ndarray:
    """Place a 4D spinor eta (shape (T,Z,Y,X,4,3)) on the domain walls:
    b(s=0) = P_- eta, b(s=Ls-1) = P_+ eta, zero elsewhere, with
    P_+ keeping spins 0,1 and P_- keeping spins 2,3 (gamma_5 = diag(1,1,-1,-1))."""
    b = np.zeros((int(Ls),) + eta4.shape, dtype=np.complex128)
    b[0, ..., 2:, :] = eta4[..., 2:, :]
    b[Ls - 1, ..., :2, :] = eta4[..., :2, :]
    return b


def point_sources(dims, Ls: int) -> np.ndarray:
    """12 wall sources from a point at the origin, one per (spin, colour)."""
    out = []
    for sp in range(4):
        for c in range(3):
            eta = np.zeros(lattice_shape(dims) + (4, 3), dtype=np.complex128)
            eta[0, 0, 0, 0, sp, c] = 1.0
            out.append(wall_source(eta, Ls))
    return np.stack(out)


def z2_source(dims, Ls: int, seed: int) -> np.ndarray:
    """Wall source from a real Z2 4D noise field (+1 or -1 per spin-colour entry)."""
    u = uniform(int(np.prod(dims)) * 12, seed, STREAM_Z2)
    eta = np.where(u < 0.5, -1.0, 1.0).astype(np.complex128).reshape(lattice_shape(dims) + (4, 3))
    return wall_source(eta, Ls)


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix g(x) per 4D site, shape (T,Z,Y,X,3,3)."""
    V = int(np.prod(dims))
    return random_su3(V, seed, STREAM_GAUGE_TRANSFORM).reshape(lattice_shape(dims) + (3, 3))


# ---------------------------------------------------------------------------
# Two-dimensional compact U(1) gauge fields (the paper's 20^2 x 8 toy, Sec. 3)
# ---------------------------------------------------------------------------

def u1_plaquette_angles(theta: np.ndarray) -> np.ndarray:
    """theta_P(x) = theta_x(x) + theta_y(x + x^) - theta_x(x + y^) - theta_y(x);
    theta shape (2, Y, X), mu = 0 is x (axis 1 of each slice), 1 is y."""
    tx, ty = theta[0], theta[1]
    return tx + np.roll(ty, -1, axis=1) - np.roll(tx, -1, axis=0) - ty


def u1_plaquette(theta: np.ndarray) -> float:
    """Average of cos theta_P over the lattice."""
    return float(np.mean(np.cos(u1_plaquette_angles(theta))))


def u1_links_2d(dims2, beta: float, sweeps: int, seed: int, hits: int = 2, delta: float = 1.5,
                trace: list | None = None) -> np.ndarray:
    """Quenched 2D U(1) link angles, Wilson action beta * sum_P (1 - cos theta_P),
    by Metropolis from a hot start: per sweep, for each direction and
    checkerboard parity, `hits` proposals theta' = theta + delta (2u - 1)
    accepted with probability min(1, exp(-dS)).  Links of one direction and
    parity share no plaquette, so they are updated together.  Uniforms come
    from the counter-based generator (stream STREAM_U1, one block of draws per
    sweep).  Returns theta, shape (2, Y, X); `trace`, when given, receives the
    average plaquette after every sweep."""
    X, Y = int(dims2[0]), int(dims2[1])
    V = X * Y
    theta = (2.0 * uniform(2 * V, seed, STREAM_U1, 0xFFFF, 0) - 1.0).reshape(2, Y, X) * np.pi
    yy, xx = np.meshgrid(np.arange(Y), np.arange(X), indexing="ij")
    parity = (xx + yy) % 2
    nk = 2 * 2 * int(hits) * 2
    for sw in range(int(sweeps)):
        u = uniform(nk * V, seed, STREAM_U1, sw, 0).reshape(nk, Y, X)
        for mu in range(2):
            for par in range(2):
                mask = parity == par
                for h in range(int(hits)):
                    k = ((mu * 2 + par) * int(hits) + h) * 2
                    new = theta.copy()
                    new[mu] = np.where(mask, theta[mu] + delta * (2.0 * u[k] - 1.0), theta[mu])
                    d = np.cos(u1_plaquette_angles(theta)) - np.cos(u1_plaquette_angles(new))
                    # the two plaquettes holding link (mu, x): P(x) and P(x - nu^), nu the other direction
                    dS = beta * (d + np.roll(d, 1, axis=(0 if mu == 0 else 1)))
                    take = mask & (u[k + 1] < np.exp(-np.minimum(dS, 50.0)))
                    theta[mu] = np.where(take, new[mu], theta[mu])
        if trace is not None:
            trace.append(u1_plaquette(theta))
    return np.angle(np.exp(1j * theta))


def u1_gauss_field(dims2, Ls: int, n: int, seed: int, stream: int = STREAM_SOURCE) -> np.ndarray:
    """n Gaussian 2D-toy fermion fields, shape (n, Ls, 1, 1, Y, X, 2)."""
    X, Y = int(dims2[0]), int(dims2[1])
    return gauss_complex((int(n), int(Ls), 1, 1, Y, X, 2), seed, stream, 1.0)


def embed_u1_2d(theta: np.ndarray, charges=(1, 1, -2)):
    """The 2D U(1) field theta (2, Y, X) as SU(3) links of a 4D lattice
    X x 1 x 1 x Y: the 2D x-links on mu = 0, the 2D y-links on mu = 3 (so that
    the antiperiodic direction is the 4D t), identity on mu = 1, 2; colour c
    carries charge charges[c] (diag(e^{i q_c theta}), det 1 for charges summing
    to 0).  Returns (links (Y, 1, 1, X, 4, 3, 3), dims (X, 1, 1, Y))."""
    Y, X = theta.shape[1], theta.shape[2]
    U = np.zeros((Y, 1, 1, X, 4, 3, 3), dtype=np.complex128)
    for mu in (1, 2):
        U[..., mu, :, :] = np.eye(3)
    for c, q in enumerate(charges):
        U[:, 0, 0, :, 0, c, c] = np.exp(1j * q * theta[0])
        U[:, 0, 0, :, 3, c, c] = np.exp(1j * q * theta[1])
    return U, (X, 1, 1, Y)
