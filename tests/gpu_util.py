"""Helpers for GPU tests: move seeded inputs between the oracle's canonical
numpy arrays and the library's internal layout through the C ABI."""
import numpy as np
import torch

from paper_1205_2933_gb300 import dwfmg as G


def ctx_for(U, dims, Ls, M5, mf, ap=True):
    return G.Context(dims, Ls, M5, mf, torch.from_numpy(np.ascontiguousarray(U)).cuda(), antiperiodic_t=ap)


def to_internal(ctx, f, prec=G.DWF_F64, nrhs=1):
    c = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    dt = torch.complex128 if prec == G.DWF_F64 else torch.complex64
    out = torch.empty(ctx.field_elems * nrhs, dtype=dt, device="cuda")
    G.dwf_pack(ctx.h, out, c, prec, nrhs)
    return out


def to_canonical(ctx, t, shape, prec=G.DWF_F64, nrhs=1):
    out = torch.empty(int(np.prod(shape)), dtype=torch.complex128, device="cuda")
    G.dwf_unpack(ctx.h, out, t, prec, nrhs)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(shape)


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_norm(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
