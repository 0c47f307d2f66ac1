"""Python binding of the dwfmg C ABI (include/dwfmg.h, include/dwfnet.h).

Argument marshalling only: every computation runs in the CUDA library
libdwfmg.so.  The functions keep the C names; arrays are torch tensors
(device or host) or numpy arrays (host), passed by pointer.  If the library
is missing the import of this module fails loudly: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import pathlib

_PKG = pathlib.Path(__file__).resolve().parent
LIB_PATH = _PKG / "libdwfmg.so"

DWF_OK, DWF_EINVAL, DWF_ECUDA, DWF_ENOMEM, DWF_ENOCONV, DWF_EBREAKDOWN, DWF_ENAN, DWF_ETIMEOUT, DWF_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
DWF_F64, DWF_F32, DWF_BF16, DWF_F16 = 0, 1, 2, 3


class mg_params(ctypes.Structure):
    _fields_ = [
        ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("coarse_tol", ctypes.c_double),
        ("coarse_maxiter", ctypes.c_int),
        ("coarsest_tol", ctypes.c_double),
        ("coarsest_maxiter", ctypes.c_int),
        ("coarse_restart", ctypes.c_int),
        ("outer_restart", ctypes.c_int),
        ("outer_maxiter", ctypes.c_int),
        ("setup_iters0", ctypes.c_int),
        ("setup_tol0", ctypes.c_double),
        ("setup_sweeps", ctypes.c_int),
        ("setup_sweep_iters", ctypes.c_int),
        ("setup_sweep_tol", ctypes.c_double),
        ("split", ctypes.c_int),
        ("smoother_prec", ctypes.c_int),
        ("coarse_prec", ctypes.c_int * 4),
        ("basis_prec", ctypes.c_int),
        ("seed", ctypes.c_uint32),
        ("cycle", ctypes.c_int),
        ("coarsen", ctypes.c_int),
        ("graph", ctypes.c_int),
    ]


class mg_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("fine_applies_f64", ctypes.c_longlong),
        ("fine_applies_f32", ctypes.c_longlong),
        ("coarse_applies", ctypes.c_longlong * 4),
        ("true_res", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {"iters": self.iters, "restarts": self.restarts, "fine_applies_f64": self.fine_applies_f64,
                "fine_applies_f32": self.fine_applies_f32, "coarse_applies": list(self.coarse_applies),
                "true_res": self.true_res, "seconds": self.seconds}


class dwf_net_shape(ctypes.Structure):
    _fields_ = [("c_in", ctypes.c_int), ("hidden", ctypes.c_int), ("layers", ctypes.c_int),
                ("nout", ctypes.c_int), ("Ls", ctypes.c_int)]


class DWFError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.dwf_strerror(status).decode()
        detail = _lib.dwf_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f": {detail}" if detail else ""))


def _load():
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is not built; run paper_1205_2933_gb300.build.build() "
                          "(the library has no CPU fallback)")
    L = ctypes.CDLL(str(LIB_PATH))
    vp, ip, st, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int
    L.mg_default_params.argtypes = [ctypes.POINTER(mg_params)]
    L.mg_default_params.restype = None
    L.dwf_strerror.argtypes = [st]
    L.dwf_strerror.restype = ctypes.c_char_p
    L.dwf_last_error.argtypes = []
    L.dwf_last_error.restype = ctypes.c_char_p
    L.dwf_create.argtypes = [ctypes.POINTER(vp), i, vp, i, ctypes.c_double, ctypes.c_double, vp, i, vp]
    L.dwf_lattice.argtypes = [vp, i, ctypes.POINTER(vp)]
    L.dwf_lattice.restype = st
    L.dwf_destroy.argtypes = [vp]
    L.dwf_destroy.restype = None
    L.dwf_apply.argtypes = [vp, vp, vp, st, i, i]
    L.dwf_pack.argtypes = [vp, vp, vp, st, i]
    L.dwf_unpack.argtypes = [vp, vp, vp, st, i]
    L.mg_setup.argtypes = [vp, i, ip, ip, ctypes.POINTER(mg_params), vp]
    L.mg_solve.argtypes = [vp, vp, vp, ctypes.c_double, i, ctypes.POINTER(mg_stats)]
    L.mg_level_info.argtypes = [vp, i, ip, ip]
    L.mg_get_vectors.argtypes = [vp, i, vp]
    L.mg_get_coarse_links.argtypes = [vp, i, vp]
    L.mg_restrict.argtypes = [vp, i, vp, vp]
    L.mg_prolong.argtypes = [vp, i, vp, vp]
    L.mg_coarse_apply.argtypes = [vp, i, vp, vp, i, st]
    L.mg_vcycle.argtypes = [vp, vp, vp]
    L.mg_vcycle_batch.argtypes = [vp, vp, vp, i]
    L.mg_coarse_solve.argtypes = [vp, i, vp, vp]
    L.mg_coarse_solve.restype = st
    L.mg_coarse_solve_static.argtypes = [vp, i, vp, vp]
    L.mg_coarse_solve_static.restype = st
    L.dwf_cg_solve.argtypes = [vp, vp, vp, ctypes.c_double, i, i, st, ctypes.POINTER(mg_stats)]
    L.dwf_cg_solve.restype = st
    L.dwf_profile.argtypes = [vp, i]
    L.dwf_profile_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
    L.dwf_profile_units.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong)]
    L.dwf_profile_units.restype = st
    L.dwf_launch_count.argtypes = []
    L.dwf_launch_count.restype = ctypes.c_ulonglong
    L.net_create.argtypes = [vp, ctypes.POINTER(dwf_net_shape), ctypes.POINTER(vp)]
    L.net_num_params.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.net_set_params.argtypes = [vp, vp]
    L.net_get_params.argtypes = [vp, vp]
    L.net_forward.argtypes = [vp, vp, vp, ctypes.c_uint, vp]
    L.net_loss_grad.argtypes = [vp, vp, vp, ctypes.c_uint, vp, i, ip, ctypes.POINTER(ctypes.c_double), vp]
    L.net_adam.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.net_destroy.argtypes = [vp]
    L.net_destroy.restype = None
    L.net_set_weight_precision.argtypes = [vp, st]
    L.net_set_weight_precision.restype = st
    L.mg_setup_learned.argtypes = [vp, vp, ctypes.c_uint, i, ip, ip, ctypes.POINTER(mg_params), i, i, ctypes.c_double,
                                   i, ip]
    L.mg_setup_learned.restype = st
    L.net_refine.argtypes = [vp, vp, vp, i, vp]
    L.net_refine.restype = st
    L.net_refine_loss_grad.argtypes = [vp, vp, vp, i, vp, i, ip, ctypes.POINTER(ctypes.c_double), vp]
    L.net_refine_loss_grad.restype = st
    L.mg_get_adaptive_vectors.argtypes = [vp, i, vp]
    L.mg_get_adaptive_vectors.restype = st
    dp = ctypes.POINTER(ctypes.c_double)
    L.dwf_lowest_modes.argtypes = [vp, i, i, ctypes.c_double, ctypes.c_uint, dp, vp, dp, ip]
    L.dwf_lowest_modes.restype = st
    L.mg_coarse_overlap.argtypes = [vp, i, vp, i, dp]
    L.mg_coarse_overlap.restype = st
    for name in ("net_create", "net_num_params", "net_set_params", "net_get_params", "net_forward",
                 "net_loss_grad", "net_adam"):
        getattr(L, name).restype = st
    for name in ("dwf_profile", "dwf_profile_read", "dwf_create", "dwf_apply", "dwf_pack", "dwf_unpack", "mg_setup", "mg_solve", "mg_level_info",
                 "mg_get_vectors", "mg_get_coarse_links", "mg_restrict", "mg_prolong", "mg_coarse_apply",
                 "mg_vcycle", "mg_vcycle_batch"):
        getattr(L, name).restype = st
    return L


_lib = _load()


def lib():
    return _lib


def _ptr(a):
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "ctypes"):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError(f"cannot take the address of {type(a)}")


def _check(status, where):
    if status != DWF_OK:
        raise DWFError(status, where)
    return status


def mg_default_params() -> mg_params:
    p = mg_params()
    _lib.mg_default_params(ctypes.byref(p))
    return p


def dwf_create(dims, Ls, M5, mf, links, antiperiodic_t=True, stream=None):
    """Context handle (ctypes.c_void_p) for one lattice; links complex128 [V][4][3][3]."""
    return dwf_create_batch([dims], Ls, M5, mf, [links], antiperiodic_t, stream)


def dwf_create_batch(dims_list, Ls, M5, mf, links_list, antiperiodic_t=True, stream=None):
    """Context handle for len(dims_list) independent lattices (one handle, fields of the
    lattices one after another); links_list[i] complex128 [V_i][4][3][3]."""
    n = len(dims_list)
    if n != len(links_list):
        raise ValueError("one links array per lattice")
    h = ctypes.c_void_p()
    d = (ctypes.c_int * (4 * n))(*[int(x) for dims in dims_list for x in dims])
    lk = (ctypes.c_void_p * n)(*[_ptr(u) for u in links_list])
    s = ctypes.c_void_p(int(stream)) if stream is not None else None
    _check(_lib.dwf_create(ctypes.byref(h), n, ctypes.cast(d, ctypes.c_void_p), int(Ls), float(M5), float(mf),
                           ctypes.cast(lk, ctypes.c_void_p), 1 if antiperiodic_t else 0, s), "dwf_create")
    return h


def dwf_lattice(ctx, i):
    """Borrowed handle of lattice i of a batch context."""
    h = ctypes.c_void_p()
    _check(_lib.dwf_lattice(ctx, int(i), ctypes.byref(h)), "dwf_lattice")
    return h


def dwf_destroy(ctx):
    _lib.dwf_destroy(ctx)


def dwf_apply(ctx, out, inp, prec=DWF_F64, dagger=False, nrhs=1):
    return _check(_lib.dwf_apply(ctx, _ptr(out), _ptr(inp), prec, 1 if dagger else 0, int(nrhs)), "dwf_apply")


def dwf_pack(ctx, internal, canonical, prec=DWF_F64, nrhs=1):
    return _check(_lib.dwf_pack(ctx, _ptr(internal), _ptr(canonical), prec, int(nrhs)), "dwf_pack")


def dwf_unpack(ctx, canonical, internal, prec=DWF_F64, nrhs=1):
    return _check(_lib.dwf_unpack(ctx, _ptr(canonical), _ptr(internal), prec, int(nrhs)), "dwf_unpack")


def mg_setup(ctx, levels, nvec, block, params=None, start=None):
    nv = (ctypes.c_int * (levels - 1))(*[int(v) for v in nvec])
    bl = (ctypes.c_int * (4 * (levels - 1)))(*[int(b) for blk in block for b in blk])
    p = ctypes.byref(params) if params is not None else None
    return _check(_lib.mg_setup(ctx, int(levels), nv, bl, p, _ptr(start)), "mg_setup")


def mg_solve(ctx, b, x, tol, nrhs=1, check=True) -> mg_stats:
    st = mg_stats()
    status = _lib.mg_solve(ctx, _ptr(b), _ptr(x), float(tol), int(nrhs), ctypes.byref(st))
    if check:
        _check(status, "mg_solve")
    st.status = status
    return st


def dwf_cg_solve(ctx, b, x, tol, maxiter, nrhs=1, prec=DWF_F32, check=True) -> mg_stats:
    st = mg_stats()
    status = _lib.dwf_cg_solve(ctx, _ptr(b), _ptr(x), float(tol), int(maxiter), int(nrhs), prec, ctypes.byref(st))
    if check:
        _check(status, "dwf_cg_solve")
    st.status = status
    return st


def mg_level_info(ctx, level):
    d = (ctypes.c_int * 4)()
    n = ctypes.c_int()
    _check(_lib.mg_level_info(ctx, int(level), d, ctypes.byref(n)), "mg_level_info")
    return tuple(d), n.value


def mg_get_vectors(ctx, level, out):
    return _check(_lib.mg_get_vectors(ctx, int(level), _ptr(out)), "mg_get_vectors")


def mg_get_coarse_links(ctx, level, out):
    return _check(_lib.mg_get_coarse_links(ctx, int(level), _ptr(out)), "mg_get_coarse_links")


def mg_restrict(ctx, level, coarse_out, fine_in):
    return _check(_lib.mg_restrict(ctx, int(level), _ptr(coarse_out), _ptr(fine_in)), "mg_restrict")


def mg_prolong(ctx, level, fine_out, coarse_in):
    return _check(_lib.mg_prolong(ctx, int(level), _ptr(fine_out), _ptr(coarse_in)), "mg_prolong")


def mg_coarse_apply(ctx, level, out, inp, dagger=False, prec=DWF_F64):
    return _check(_lib.mg_coarse_apply(ctx, int(level), _ptr(out), _ptr(inp), 1 if dagger else 0, prec),
                  "mg_coarse_apply")


def mg_coarse_solve(ctx, level, x, b):
    return _check(_lib.mg_coarse_solve(ctx, int(level), _ptr(x), _ptr(b)), "mg_coarse_solve")


def mg_coarse_solve_static(ctx, level, x, b):
    """mg_coarse_solve without any device allocation (static scratch; see dwfmg.h)."""
    return _check(_lib.mg_coarse_solve_static(ctx, int(level), _ptr(x), _ptr(b)), "mg_coarse_solve_static")


def mg_vcycle(ctx, x, b):
    return _check(_lib.mg_vcycle(ctx, _ptr(x), _ptr(b)), "mg_vcycle")


def mg_vcycle_batch(ctx, x, b, nrhs):
    return _check(_lib.mg_vcycle_batch(ctx, _ptr(x), _ptr(b), int(nrhs)), "mg_vcycle_batch")


K_DSLASH_F64, K_DSLASH_F32, K_RESTRICT, K_PROLONG, K_COARSE, K_DSLASH_F32_Z = 0, 1, 2, 3, 4, 5


def dwf_profile(ctx, enable):
    return _check(_lib.dwf_profile(ctx, 1 if enable else 0), "dwf_profile")


def dwf_profile_read(ctx, kernel_class):
    """(launches, total device milliseconds) of one kernel class since dwf_profile(ctx, True)."""
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(_lib.dwf_profile_read(ctx, int(kernel_class), ctypes.byref(n), ctypes.byref(ms)), "dwf_profile_read")
    return n.value, ms.value


def dwf_profile_units(ctx, kernel_class):
    """Fields processed by the recorded launches of one class (a batched launch counts its nrhs)."""
    n = ctypes.c_longlong()
    _check(_lib.dwf_profile_units(ctx, int(kernel_class), ctypes.byref(n)), "dwf_profile_units")
    return n.value


def dwf_launch_count():
    return int(_lib.dwf_launch_count())


class Context:
    """Owns one dwf_ctx; fields are torch tensors in the library's internal layout."""

    def __init__(self, dims, Ls, M5, mf, links, antiperiodic_t=True, stream=None):
        import torch
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.h = dwf_create(dims, Ls, M5, mf, links, antiperiodic_t, stream)

    @property
    def field_elems(self):
        return self.V * 12 * self.Ls

    def close(self):
        if self.h is not None:
            dwf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchContext:
    """Owns one dwf_ctx holding several independent lattices (same Ls, M5, mf);
    fields hold the lattices one after another (nrhs fields of each in turn)."""

    def __init__(self, dims_list, Ls, M5, mf, links_list, antiperiodic_t=True, stream=None):
        import torch
        self.dims = [tuple(int(d) for d in dims) for dims in dims_list]
        self.Ls = int(Ls)
        self.V = [d[0] * d[1] * d[2] * d[3] for d in self.dims]
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.h = dwf_create_batch(self.dims, Ls, M5, mf, links_list, antiperiodic_t, stream)

    def field_elems(self, i=None):
        """Complex elements of one field of lattice i (all lattices when i is None)."""
        if i is None:
            return sum(v * 12 * self.Ls for v in self.V)
        return self.V[i] * 12 * self.Ls

    def offset(self, i, nrhs=1):
        """Element offset of lattice i's first field in a batch array of nrhs fields per lattice."""
        return sum(self.V[j] * 12 * self.Ls for j in range(i)) * nrhs

    def lattice(self, i):
        return dwf_lattice(self.h, i)

    def close(self):
        if self.h is not None:
            dwf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned near-null proposal (include/dwfnet.h) ----

def net_create(ctx, c_in, hidden, layers, nout, Ls):
    h = ctypes.c_void_p()
    sh = dwf_net_shape(int(c_in), int(hidden), int(layers), int(nout), int(Ls))
    _check(_lib.net_create(ctx, ctypes.byref(sh), ctypes.byref(h)), "net_create")
    return h


def net_num_params(net):
    n = ctypes.c_longlong()
    _check(_lib.net_num_params(net, ctypes.byref(n)), "net_num_params")
    return n.value


def net_set_params(net, params):
    return _check(_lib.net_set_params(net, _ptr(params)), "net_set_params")


def net_get_params(net, params):
    return _check(_lib.net_get_params(net, _ptr(params)), "net_get_params")


def net_forward(net, ctx, out, input=None, seed=0):
    return _check(_lib.net_forward(net, ctx, _ptr(input), int(seed), _ptr(out)), "net_forward")


def net_loss_grad(net, ctx, targets, nt, block, input=None, seed=0, grad=None):
    b = (ctypes.c_int * 4)(*[int(x) for x in block])
    loss = ctypes.c_double()
    _check(_lib.net_loss_grad(net, ctx, _ptr(input), int(seed), _ptr(targets), int(nt), b, ctypes.byref(loss),
                              _ptr(grad)), "net_loss_grad")
    return loss.value


def net_set_weight_precision(net, prec):
    return _check(_lib.net_set_weight_precision(net, int(prec)), "net_set_weight_precision")


def net_adam(net, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    return _check(_lib.net_adam(net, float(lr), float(beta1), float(beta2), float(eps)), "net_adam")


def net_destroy(net):
    _lib.net_destroy(net)


def mg_setup_learned(ctx, net, seed, levels, nvec, block, params=None, pre_iters0=0, fallback_iters0=1000,
                     probe_tol=1e-4, probe_max_iters=0):
    """mg_setup from the network's vectors; returns True when the plain setup was used as fallback."""
    nv = (ctypes.c_int * (levels - 1))(*[int(v) for v in nvec])
    bl = (ctypes.c_int * (4 * (levels - 1)))(*[int(b) for blk in block for b in blk])
    p = ctypes.byref(params) if params is not None else None
    used = ctypes.c_int(0)
    _check(_lib.mg_setup_learned(ctx, net, int(seed), int(levels), nv, bl, p, int(pre_iters0), int(fallback_iters0),
                                 float(probe_tol), int(probe_max_iters), ctypes.byref(used)), "mg_setup_learned")
    return bool(used.value)


def net_refine(net, ctx, fields, nfields, out):
    return _check(_lib.net_refine(net, ctx, _ptr(fields), int(nfields), _ptr(out)), "net_refine")


def net_refine_loss_grad(net, ctx, fields, nfields, targets, nt, block, grad=None):
    b = (ctypes.c_int * 4)(*[int(x) for x in block])
    loss = ctypes.c_double()
    _check(_lib.net_refine_loss_grad(net, ctx, _ptr(fields), int(nfields), _ptr(targets), int(nt), b,
                                     ctypes.byref(loss), _ptr(grad)), "net_refine_loss_grad")
    return loss.value


def mg_get_adaptive_vectors(ctx, level, out):
    return _check(_lib.mg_get_adaptive_vectors(ctx, int(level), _ptr(out)), "mg_get_adaptive_vectors")


def dwf_lowest_modes(ctx, k, evecs, max_iters=50, tol=1e-8, seed=1):
    """(eigenvalues, residuals, iterations) of the k smallest eigenpairs of D^+ D; vectors into evecs."""
    ev = (ctypes.c_double * k)()
    rs = (ctypes.c_double * k)()
    it = ctypes.c_int()
    _check(_lib.dwf_lowest_modes(ctx, int(k), int(max_iters), float(tol), int(seed), ev, _ptr(evecs), rs,
                                 ctypes.byref(it)), "dwf_lowest_modes")
    return list(ev), list(rs), it.value


def mg_coarse_overlap(ctx, level, fields, nfields):
    out = (ctypes.c_double * nfields)()
    _check(_lib.mg_coarse_overlap(ctx, int(level), _ptr(fields), int(nfields), out), "mg_coarse_overlap")
    return list(out)

