#!/usr/bin/env python
"""Benchmark of the domain-wall multigrid solve on GB300.

Metric: wall time per solve of D x = b to |b - D x| / |b| <= 1e-10 (FP64 true
residual), with the multigrid setup amortised over the right-hand sides of
one step; plus the fine Dslash's achieved HBM bandwidth (roofline).

Workload (one GPU): 16^3 x 32 lattice, Ls = 16, M5 = 1.8, m_f = 0.001, links
from 200 sweeps of a seeded quenched Wilson-gauge heatbath at beta = 6.0,
2-level multigrid with 4^4 blocks and Nvec = 24, mixed precision (FP32 fine
V-cycle, BF16 coarse stencil with FP32 accumulation, FP64 outer GCR with
reliable updates), 12 Gaussian right-hand sides.  A step = mg_setup + the 12
solves (every part of the solve path runs in each step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own independent problem
(replicas; the path has no exchange step) and rank 0 prints the job line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import paper_1205_2933_gb300.inputs as I  # noqa: E402

DIMS = (16, 16, 16, 32)
LS = 16
M5 = 1.8
MF = 0.001
BETA = 6.0
HB_SWEEPS = 200
HB_SEED = 100
NVEC = 24
BLOCK = (4, 4, 4, 4)
NRHS = 12
TOL = 1e-10
METRIC = "DWF MG solve time to |r|/|b|\u226410^-10 (chosen vs FP64 plain); Dslash HBM GB/s"
FINE_BYTES_F32 = 204   # algorithmic bytes per 5D site of the FP32 Dslash
# dram__bytes_read.sum + dram__bytes_write.sum of the FP32 Dslash with fused
# output norms (the instantiation of nearly all timed launches) per 2,097,152
# 5D sites (one 16^3x32x16 field), from an ncu capture of a two-field launch on
# 16^3x16x16; None until the kernel as it stands has been captured
DSLASH_TRAFFIC_PER_FIELD = 425732864  # 251.68 MB read + 174.05 MB written
DSLASH_Z_TRAFFIC_PER_FIELD = 630616832  # 453.86 MB read + 176.76 MB written
FINE_BYTES_F64 = 408
FINE_BYTES_F32_Z = FINE_BYTES_F32 + 96  # the fused residual kernels also read b (or z) at every 5D site
# fine-operator applications per solve of this workload on the GPU path (FP32 and
# FP64, the setup's amortised over 12 right-hand sides), from the timed bench steps;
# the reference arm scales its timed oracle applications by it
APPLIES_PER_SOLVE = 3866  # fine applications per solve of the GPU path on this workload (setup amortised)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nrhs", type=int, default=NRHS)
    ap.add_argument("--coarsen", choices=["unsquared", "squared"], default="unsquared",
                    help="coarse operator: R D P (9-point, default) or the squared operator's P^+ D^+ D P "
                         "(33-point, Sec. 4; right-hand sides solved one after another)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--plain-nrhs", type=int, default=2,
                    help="right-hand sides solved by the plain FP64 method (their solutions are the FP64 "
                         "reference of the per-solve errors)")
    ap.add_argument("--e2e-steps", type=int, default=2, help="timed end-to-end steps (after one warm-up)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-setup comparison")
    ap.add_argument("--workload", choices=["headline", "point-sources-24x48", "uneven-batch"], default="headline",
                    help="point-sources-24x48: 24^3x48 Ls=16 batched point (+Z2) sources; uneven-batch: the uneven batch "
                         "8^4 + 12^3x24 + 16^3x32 in one context and a 3-level solve (one JSON line each; "
                         "the default is the headline workload)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="profiling mode: setup, then one solve inside cudaProfilerStart/Stop (for ncu)")
    ap.add_argument("--dslash-only", action="store_true",
                    help="profiling mode: a few FP32 Dslash applications of the workload (for ncu)")
    ap.add_argument("--profile-coarse", action="store_true",
                    help="profiling mode: four batched V-cycles of 12 right-hand sides on 16^3x32 with Ls=2 "
                         "(the workload's coarse problem, 512 sites x 24, with small fine fields; for ncu)")
    ap.add_argument("--profile-vcycle", action="store_true",
                    help="profiling mode: two batched V-cycles of 2 right-hand sides on 16^3x16, Ls=16, Nvec=8 "
                         "(the FP32 Dslash with fused output norms at 2 x 101 MB per launch; for ncu)")
    return ap.parse_args()


def workload_config(nrhs, coarsen="unsquared"):
    coarse = ("BF16 coarse stencil" if coarsen == "unsquared" else
              "BF16 33-point coarse stencil of the squared operator P^+D^+DP (RHS one after another)")
    return {"workload": f"DWF MG solve, 16^3x32 Ls=16 M5=1.8 mf=0.001, heatbath beta=6.0 ({HB_SWEEPS} sweeps, "
                        f"seed {HB_SEED}), 2-level Nvec=24 blocks 4^4, FP32 V-cycle + {coarse} + "
                        f"FP64 outer GCR, 16 CGNR post-smoothing steps, coarsest GCR to 0.03, 600 setup iterations, "
                        f"setup amortised over "
                        f"{nrhs} Gaussian RHS",
            "lattice": "16x16x16x32", "Ls": LS, "mf": MF, "nvec": NVEC, "block": list(BLOCK), "nrhs": nrhs,
            "tol": TOL, "l2": "inputs larger than L2 (FP32 fine field 201 MB, FP64 403 MB; working set ~10 GB)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dslash_roofline(prof, units, V5, peak, peak_kind):
    """Roofline object of the dominant FP32 Dslash class by summed device time:
    the plain kernels (204 B per 5D site) or those with a fused second field
    (300 B per 5D site); the other class goes in `other_dslash`.  prof maps a
    class name to (launches, ms), units to the fields its launches covered
    (a batched launch over nrhs fields counts nrhs); achieved = algorithmic
    bytes of all those fields over their summed device time."""
    def one(name, bytes_site, traffic, note):
        n, ms = prof[name]
        if not n or not ms:
            return None
        u = units[name]
        achieved = bytes_site * V5 * u / (ms * 1e-3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "avg_launch_us": ms / n * 1e3, "launches": n, "fields": u, "ms": ms,
                "bytes_per_launch": bytes_site * V5 * u / n, "bytes_per_site": bytes_site, "traffic_note": note}

    roofs = [r for r in (
        one("dslash_f32", FINE_BYTES_F32, DSLASH_TRAFFIC_PER_FIELD,
            "ncu dram bytes per field application of the norm-epilogue kernel (two-field launch of "
            "2 x 16^3x16x16 = one 16^3x32x16 field of sites)"),
        one("dslash_f32_z", FINE_BYTES_F32_Z, DSLASH_Z_TRAFFIC_PER_FIELD,
            "ncu dram bytes per field application of the residual-update kernel z - a D^+ w (same launch "
            "shape); the class also holds the w updates D z + b w and the V-cycle's b - D x (same bytes)"))
             if r]
    roofs.sort(key=lambda r: -r["ms"])
    roof = roofs[0] if roofs else None
    if roof and len(roofs) > 1:
        o = roofs[1]
        roof["other_dslash"] = {k: o[k] for k in ("kernel", "achieved", "frac", "ms", "fields", "bytes_per_site",
                                                  "traffic")}
    return roof


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def replica_reduce(ms_total, steps, nrhs, world, dist=None, dev="cpu"):
    """Replicas only (one independent set of right-hand sides per rank, no
    collective on the data path): the job's time is the slowest rank's, and
    the job solved nrhs x world systems per step.  Returns (ms per step,
    seconds per solve)."""
    import torch
    if dist is not None:
        t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / steps
    return ms_step, ms_step / 1000.0 / (nrhs * world)


def gen_inputs(nrhs, rank=0):
    U = I.heatbath_links(DIMS, BETA, HB_SWEEPS, HB_SEED)
    bs = np.stack([I.gaussian_source(DIMS, LS, 101 + 1000 * rank + i) for i in range(nrhs)])
    return U, bs


def mixed_params(G, coarsen="unsquared"):
    """Mixed precision: FP32 fine V-cycle, BF16 coarse stencil, FP64 outer GCR;
    16 CGNR post-smoothing steps, coarsest GCR to 0.03 (at most 128
    iterations) and 600 setup relaxation iterations: the fastest of measured
    sweeps on this workload (s/solve with the setup amortised: 2.02 at the
    library defaults 8 / 0.1 / 1000, 1.50 at 16 / 0.03 / 1000, 1.23 at
    16 / 0.03 / 600; with another setup seed 600 gave 1.52)."""
    p = G.mg_default_params()
    p.smoother_prec = G.DWF_F32
    p.coarse_prec[0] = G.DWF_BF16
    p.nu_post = 16
    p.coarsest_tol = 0.03
    p.coarsest_maxiter = 128
    p.setup_iters0 = 600
    p.coarsen = 1 if coarsen == "squared" else 0
    return p


def cpu_baseline_sample(U, b, seconds_target=15.0):
    """The FP64 oracle as it stands, on the host cores: time applications of
    its fine operator at the full lattice (the paper's cost unit, Sec. 3)."""
    import oracle
    dwf = oracle.DWF(U, DIMS, LS, M5, MF)
    t0 = time.perf_counter()
    dwf.D(b)
    t1 = time.perf_counter()
    per = t1 - t0
    n = max(1, min(20, int(seconds_target / max(per, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(n):
        dwf.D(b)
    per = (time.perf_counter() - t0) / n
    return per, n, host_threads()


def host_threads():
    threads = os.environ.get("OMP_NUM_THREADS")
    return int(threads) if threads else os.cpu_count()


# The plain method's small case: 4^4 lattice, Ls = 8, M5 = 1.8, m_f = 0.1,
# eps-random links (eps = 0.3, seed 1), Gaussian source (seed 2), 2-level
# FP64 multigrid with 2^4 blocks, Nvec = 8, 3 inverse-iteration setup sweeps.
SMALL_DIMS, SMALL_LS, SMALL_MF = (4, 4, 4, 4), 8, 0.1


def small_case_oracle():
    """Full setup + solve of the small plain-FP64 case by the oracle on the host
    cores (measured, not extrapolated); returns (seconds, iterations, solution)."""
    import oracle
    from oracle import mg as OM
    U = I.epsilon_links(SMALL_DIMS, 0.3, 1)
    b = I.gaussian_source(SMALL_DIMS, SMALL_LS, 2)
    rv = I.random_vectors(4, SMALL_DIMS, SMALL_LS, 3)
    t0 = time.perf_counter()
    op = OM.FineOp(oracle.DWF(U, SMALL_DIMS, SMALL_LS, M5, SMALL_MF))
    prm = OM.MGParams(nvec=(8,), block=((2, 2, 2, 2),), setup_sweeps=3)
    mg = OM.adaptive_setup(op, prm, [rv.reshape((4,) + op.shape)])
    x, info = OM.mg_solve(mg, b.reshape(op.shape), tol=TOL, restart=20)
    return time.perf_counter() - t0, info.iters, x.reshape(b.shape)


def small_case_gpu(G, torch):
    """The same small case through the library (CUDA events around setup + solve)."""
    U = I.epsilon_links(SMALL_DIMS, 0.3, 1)
    b = I.gaussian_source(SMALL_DIMS, SMALL_LS, 2)
    rv = torch.from_numpy(I.random_vectors(4, SMALL_DIMS, SMALL_LS, 3)).cuda()
    ctx = G.Context(SMALL_DIMS, SMALL_LS, M5, SMALL_MF, torch.from_numpy(U).cuda())
    bt = torch.empty(ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.dwf_pack(ctx.h, bt, torch.from_numpy(b).cuda(), G.DWF_F64, 1)
    p = G.mg_default_params()
    p.setup_sweeps = 3
    times = []
    for _ in range(4):  # one warm-up, three timed
        x = torch.zeros_like(bt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.mg_setup(ctx.h, 2, [8], [(2, 2, 2, 2)], p, rv)
        st = G.mg_solve(ctx.h, bt, x, TOL)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    xc = torch.empty_like(bt)
    G.dwf_unpack(ctx.h, xc, x, G.DWF_F64, 1)
    torch.cuda.synchronize()
    out = xc.cpu().numpy().reshape(b.shape)
    ctx.close()
    return statistics.median(times[1:]), st.iters, st.true_res, out


def run_reference(args):
    """--impl reference: the FP64 oracle timed on the host cores on bounded
    samples of this workload, scaled to seconds per solve."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    U, bs = gen_inputs(1)
    b = bs[0]
    # cost of one solve in fine-operator applications, as measured on the GPU
    # path for this workload (FP64 + FP32 applications per solve, the setup's
    # amortised over the 12 right-hand sides)
    applies = float(os.environ.get("DWF_APPLIES_PER_SOLVE", str(APPLIES_PER_SOLVE)))
    times = []
    for _ in range(args.warmup):
        cpu_baseline_sample(U, b, 1.0)
    n = cores = 0
    for _ in range(args.steps):
        per, n, cores = cpu_baseline_sample(U, b, 5.0)
        times.append(per * applies)
    v = statistics.median(times)
    t_small, it_small, _ = small_case_oracle()
    line = {"impl": "reference", "metric": METRIC,
            "value": v, "unit": "s/solve", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.nrhs, args.coarsen),
            "cpu_baseline": {"value": v, "unit": "s/solve", "cores": cores, "kind": "oracle",
                             "method": "extrapolated",
                             "sample": f"per step {n} applications of the oracle's FP64 fine operator at "
                                       f"16^3x32x16, scaled by {applies:.0f} fine applications per solve "
                                       f"(the GPU path's count for this workload, setup amortised)"},
            "small_case": {"workload": "4^4x8 plain FP64 MG (Nvec 8, 2^4 blocks, 3 setup sweeps), m_f=0.1",
                           "oracle_s": t_small, "oracle_iters": it_small, "kind": "measured"},
            "e2e": {"value": v, "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_modes(args):
    """Small commands for ncu captures of the workload's kernels."""
    import torch
    from paper_1205_2933_gb300 import dwfmg as G
    U, bs = gen_inputs(1)
    ctx = G.Context(DIMS, LS, M5, MF, torch.from_numpy(U).cuda())
    canon = torch.from_numpy(bs).cuda()
    if args.dslash_only:
        f = torch.empty(ctx.field_elems, dtype=torch.complex64, device="cuda")
        G.dwf_pack(ctx.h, f, canon, G.DWF_F32, 1)
        out = torch.empty_like(f)
        for _ in range(4):
            G.dwf_apply(ctx.h, out, f, G.DWF_F32)
        torch.cuda.synchronize()
        print("dslash-only ok")
    else:
        # one solve of args.nrhs right-hand sides (batched when nrhs > 1)
        U, bs = gen_inputs(args.nrhs)
        canon = torch.from_numpy(bs).cuda()
        b = torch.empty(ctx.field_elems * args.nrhs, dtype=torch.complex128, device="cuda")
        G.dwf_pack(ctx.h, b, canon, G.DWF_F64, args.nrhs)
        G.mg_setup(ctx.h, 2, [NVEC], [BLOCK], mixed_params(G, args.coarsen))
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        st = G.mg_solve(ctx.h, b, x, TOL, args.nrhs)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("profile-solve ok", st.iters, st.true_res)
    ctx.close()


def _timed(torch, f):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = f()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, r


def run_workload(args):
    """The other measured configurations (one JSON line each):
    point-sources-24x48: 24^3 x 48, Ls = 16, m_f = 0.001, heatbath beta = 6.0 (seed 200),
      12 spin-colour point sources at the origin (plus args.nrhs - 12 Z2 noise
      sources, seeds 201...), all solved as one batch with the chosen mixed
      precision; per-RHS time, Dslash GB/s and the coarse solver's share.
    uneven-batch: 8^4, 12^3 x 24 and 16^3 x 32 at Ls = 16, m_f = 0.002, heatbath
      beta = 5.9 (seeds 300-302) in one batch context (one setup call, one
      solve call over all three lattices) against the three lattices one after
      another in contexts of their own; then a 3-level solve of the 16^3 x 32
      lattice (4^4 then 2^4 blocks, Nvec 24 then 32)."""
    import torch
    from paper_1205_2933_gb300 import dwfmg as G
    p = mixed_params(G)
    line = {"metric": f"{args.workload}: solve time per right-hand side (setup amortised)", "unit": "s/rhs",
            "higher_is_better": False, "dtype": "f32+bf16 (fp64 outer)", "data": "synthetic"}
    if args.workload == "point-sources-24x48":
        dims, mf = (24, 24, 24, 48), 0.001
        nr = max(12, args.nrhs)
        U = I.heatbath_links(dims, BETA, HB_SWEEPS, 200)
        ctx = G.Context(dims, LS, M5, mf, torch.from_numpy(U).cuda())
        N = ctx.field_elems
        b = torch.empty(N * nr, dtype=torch.complex128, device="cuda")
        for i in range(nr):  # one canonical source (2 GB) at a time on the host
            if i < 12:  # spin-colour point source at the origin on the walls
                eta = np.zeros(I.lattice_shape(dims) + (4, 3), dtype=np.complex128)
                eta[0, 0, 0, 0, i // 3, i % 3] = 1.0
                src = I.wall_source(eta, LS)
            else:
                src = I.z2_source(dims, LS, 201 + i - 12)
            G.dwf_pack(ctx.h, b[i * N:(i + 1) * N], torch.from_numpy(src).cuda(), G.DWF_F64, 1)
            del src
        torch.cuda.synchronize()
        x = torch.zeros_like(b)
        G.dwf_profile(ctx.h, True)
        ts, _ = _timed(torch, lambda: G.mg_setup(ctx.h, 2, [NVEC], [BLOCK], p))
        tv, st = _timed(torch, lambda: G.mg_solve(ctx.h, b, x, TOL, nr, check=False))
        n32, ms32 = G.dwf_profile_read(ctx.h, G.K_DSLASH_F32)
        u32 = G.dwf_profile_units(ctx.h, G.K_DSLASH_F32)
        nz, msz = G.dwf_profile_read(ctx.h, G.K_DSLASH_F32_Z)
        uz = G.dwf_profile_units(ctx.h, G.K_DSLASH_F32_Z)
        nco, msco = G.dwf_profile_read(ctx.h, G.K_COARSE)
        G.dwf_profile(ctx.h, False)
        V5 = ctx.V * LS
        line.update({"value": (ts + tv) / nr, "config": {"workload": f"24^3x48 Ls=16 mf=0.001 heatbath beta=6.0 "
                     f"(200 sweeps, seed 200), 12 point + {nr - 12} Z2 sources in one batch, Nvec 24, 4^4 blocks",
                     "nrhs": nr},
                     "setup_s": ts, "solve_s": tv, "status": st.status, "iters": st.iters, "true_res": st.true_res,
                     "dslash_f32_gbs": FINE_BYTES_F32 * V5 * u32 / (ms32 * 1e-3) / 1e9 if n32 else None,
                     "dslash_f32_z_gbs": FINE_BYTES_F32_Z * V5 * uz / (msz * 1e-3) / 1e9 if nz else None,
                     "coarse_ms": msco, "coarse_launches": nco, "wall_s": ts + tv})
        ctx.close()
    else:
        dims_l = [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32)]
        mf = 0.002
        Us = [I.heatbath_links(d, 5.9, HB_SWEEPS, 300 + i) for i, d in enumerate(dims_l)]
        bs = [I.gaussian_source(d, LS, 310 + i) for i, d in enumerate(dims_l)]
        # one context holding all three lattices: one setup call, one solve call
        bc = G.BatchContext(dims_l, LS, M5, mf, [torch.from_numpy(u).cuda() for u in Us])
        canon = torch.from_numpy(np.concatenate([s.reshape(-1) for s in bs])).cuda()
        bb = torch.empty(bc.field_elems(), dtype=torch.complex128, device="cuda")
        G.dwf_pack(bc.h, bb, canon, G.DWF_F64, 1)
        xb = torch.zeros_like(bb)
        G.mg_setup(bc.h, 2, [NVEC], [BLOCK], p)  # warm-up of both paths' kernels and workspaces
        G.mg_solve(bc.h, bb, xb, TOL, 1)
        xb.zero_()
        ts_b, _ = _timed(torch, lambda: G.mg_setup(bc.h, 2, [NVEC], [BLOCK], p))
        tv_b, st_b = _timed(torch, lambda: G.mg_solve(bc.h, bb, xb, TOL, 1, check=False))
        bc.close()
        seq = []
        for i, d in enumerate(dims_l):
            ctx = G.Context(d, LS, M5, mf, torch.from_numpy(Us[i]).cuda())
            b1 = torch.empty(ctx.field_elems, dtype=torch.complex128, device="cuda")
            G.dwf_pack(ctx.h, b1, torch.from_numpy(bs[i]).cuda(), G.DWF_F64, 1)
            x1 = torch.zeros_like(b1)
            ts, _ = _timed(torch, lambda: G.mg_setup(ctx.h, 2, [NVEC], [BLOCK], p))
            tv, st = _timed(torch, lambda: G.mg_solve(ctx.h, b1, x1, TOL, 1, check=False))
            seq.append({"dims": d, "setup_s": ts, "solve_s": tv, "iters": st.iters, "true_res": st.true_res,
                        "status": st.status})
            if i == 2:
                # 3 levels: 4^4 blocks then 2^4 (coarse 4^3x8 -> 2^3x4), Nvec 24 then 32
                p3 = mixed_params(G)
                p3.coarse_prec[1] = G.DWF_BF16
                x1.zero_()
                ts3, _ = _timed(torch, lambda: G.mg_setup(ctx.h, 3, [NVEC, 32], [BLOCK, (2, 2, 2, 2)], p3))
                tv3, st3 = _timed(torch, lambda: G.mg_solve(ctx.h, b1, x1, TOL, 1, check=False))
                three = {"dims": d, "levels": 3, "nvec": [NVEC, 32], "blocks": [list(BLOCK), [2, 2, 2, 2]],
                         "setup_s": ts3, "solve_s": tv3, "iters": st3.iters, "true_res": st3.true_res,
                         "status": st3.status, "coarse_applies": list(st3.coarse_applies)}
            ctx.close()
        tseq = sum(r["setup_s"] + r["solve_s"] for r in seq)
        line.update({"value": (ts_b + tv_b) / 3,
                     "config": {"workload": "uneven batch 8^4 + 12^3x24 + 16^3x32, Ls=16, mf=0.002, heatbath "
                                            "beta=5.9 (200 sweeps, seeds 300-302), one Gaussian source per lattice, "
                                            "Nvec 24, 4^4 blocks, one batch context", "nrhs": 3},
                     "batch": {"setup_s": ts_b, "solve_s": tv_b, "iters": st_b.iters, "true_res": st_b.true_res,
                               "status": st_b.status},
                     "one_after_another": seq, "one_after_another_s": tseq, "batch_s": ts_b + tv_b,
                     "three_level_16x16x16x32": three,
                     "note": "32^3x64 with three levels is not run: at Nvec 24 its FP32 basis, the FP64 "
                             "adaptive vectors and the coarse construction's D q_k take 231 GB of the 288 GB"})
    print(json.dumps(line), flush=True)


def profile_small(args):
    """Small device-memory cases of the timed kernels for ncu captures: the
    batched coarsest solve at the workload's coarse size (--profile-coarse) and
    the FP32 Dslash with fused norms inside the batched smoother (--profile-vcycle)."""
    import torch
    from paper_1205_2933_gb300 import dwfmg as G
    if args.profile_coarse:
        dims, Ls, nvec, nr = DIMS, 2, NVEC, 12
    else:
        dims, Ls, nvec, nr = (16, 16, 16, 16), LS, 8, 2
    U = I.heatbath_links(dims, BETA, 20, HB_SEED)
    ctx = G.Context(dims, Ls, M5, MF, torch.from_numpy(U).cuda())
    p = mixed_params(G)
    p.setup_iters0 = 50
    G.mg_setup(ctx.h, 2, [nvec], [BLOCK], p)
    bs = np.stack([I.gaussian_source(dims, Ls, 101 + i) for i in range(nr)])
    canon = torch.from_numpy(bs).cuda()
    b = torch.empty(ctx.field_elems * nr, dtype=torch.complex128, device="cuda")
    G.dwf_pack(ctx.h, b, canon, G.DWF_F64, nr)
    x = torch.empty_like(b)
    G.mg_vcycle_batch(ctx.h, x, b, nr)  # workspaces allocated outside the profiled range
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(4 if args.profile_coarse else 2):
        G.mg_vcycle_batch(ctx.h, x, b, nr)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print("profile ok", float(x.abs().max()))
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_solve or args.dslash_only:
        profile_modes(args)
        return
    if args.profile_coarse or args.profile_vcycle:
        profile_small(args)
        return
    if args.workload != "headline":
        run_workload(args)
        return
    import torch
    from paper_1205_2933_gb300 import dwfmg as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nrhs = args.nrhs

    U, bs = gen_inputs(nrhs, rank)
    stream = torch.cuda.current_stream()
    ctx = G.Context(DIMS, LS, M5, MF, torch.from_numpy(U).to(dev))
    N = ctx.field_elems
    canon = torch.from_numpy(bs).to(dev)
    b = torch.empty(N * nrhs, dtype=torch.complex128, device=dev)
    G.dwf_pack(ctx.h, b, canon, G.DWF_F64, nrhs)
    x = torch.zeros_like(b)
    del canon
    p = mixed_params(G, args.coarsen)

    def step(stats_out=None):
        G.mg_setup(ctx.h, 2, [NVEC], [BLOCK], p)
        x.zero_()
        st = G.mg_solve(ctx.h, b, x, TOL, nrhs)
        if stats_out is not None:
            stats_out.append(st.as_dict())
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    G.dwf_profile(ctx.h, True)
    launches0 = G.dwf_launch_count()
    stats = []
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(stats)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = G.dwf_launch_count() - launches0
    ms_total = t0.elapsed_time(t1)
    clk = clocks.stop()
    classes = (("dslash_f32", G.K_DSLASH_F32), ("dslash_f32_z", G.K_DSLASH_F32_Z), ("dslash_f64", G.K_DSLASH_F64),
               ("restrict", G.K_RESTRICT), ("prolong", G.K_PROLONG), ("coarse", G.K_COARSE))
    prof = {name: G.dwf_profile_read(ctx.h, k) for name, k in classes}
    units = {name: G.dwf_profile_units(ctx.h, k) for name, k in classes}
    G.dwf_profile(ctx.h, False)
    ms_step, value = replica_reduce(ms_total, args.steps, nrhs, world, dist, dev)

    V5 = ctx.V * LS
    peak, peak_kind = measured_peaks()

    roof = dslash_roofline(prof, units, V5, peak, peak_kind)

    # fine-operator applications per solve in the timed region, setup included
    # (the paper's cost unit, Sec. 3): all fields the FP32 and FP64 Dslash processed
    applies_per_solve = (units["dslash_f32"] + units["dslash_f32_z"] + units["dslash_f64"]) / (nrhs * args.steps) \
        or None

    line = {"metric": METRIC,
            "value": value, "unit": "s/solve", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+bf16 (fp64 outer)", "data": "synthetic (seeded heatbath links, Gaussian sources)",
            "config": workload_config(nrhs, args.coarsen), "gpu_launches": int(launches), "clocks": clk,
            "roofline": roof, "solve_stats": stats[-1] if stats else None,
            "applies_per_solve": applies_per_solve,
            "kernel_time_ms": {k: {"launches": v[0], "fields": units[k], "ms": v[1]} for k, v in prof.items()}}
    # the chosen solutions of the last timed step stay on the device for the error check
    ctx.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_plain:
        line["plain_fp64"] = run_plain(G, torch, U, b, x, min(args.plain_nrhs, nrhs), value)
    if rank == 0 and not args.no_learned:
        line["learned_setup"] = run_learned(G, torch, U, b, p)
    del b, x
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_e2e:
        line["e2e"] = run_e2e(G, torch, U, bs, p, nrhs, args.e2e_steps)
    if rank == 0 and not args.no_cpu_baseline:
        per, n, cores = cpu_baseline_sample(U, bs[0])
        if applies_per_solve:
            line["cpu_baseline"] = {"value": per * applies_per_solve, "unit": "s/solve", "cores": cores,
                                    "kind": "oracle", "method": "extrapolated",
                                    "sample": f"{n} applications of the oracle's FP64 fine operator at 16^3x32x16, "
                                              f"scaled by the {applies_per_solve:.0f} fine applications per solve "
                                              f"(setup amortised) of the timed GPU steps (the paper's cost unit)"}
        t_or, it_or, x_or = small_case_oracle()
        t_gpu, it_gpu, res_gpu, x_gpu = small_case_gpu(G, torch)
        line["small_case"] = {"workload": "4^4x8 plain FP64 MG (Nvec 8, 2^4 blocks, 3 setup sweeps), m_f=0.1, "
                                          "full setup + solve",
                              "oracle_s": t_or, "oracle_iters": it_or, "oracle_cores": host_threads(),
                              "gpu_s": t_gpu, "gpu_iters": it_gpu, "gpu_true_res": res_gpu,
                              "rel_diff_vs_oracle": float(np.linalg.norm(x_gpu - x_or) / np.linalg.norm(x_or)),
                              "kind": "measured"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_e2e(G, torch, U, bs, p, nrhs, steps):
    """Same metric through the public API with host buffers: every step creates
    the context from pinned host links, copies the canonical host sources to
    the device, converts them to the internal layout, runs the setup and the
    solves, converts the solutions back and copies them to pinned host memory.
    One warm-up step, then the median of `steps` timed steps."""
    Uh = torch.from_numpy(U).pin_memory()
    bh = torch.from_numpy(bs).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    times = []
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = G.Context(DIMS, LS, M5, MF, Uh)
        bd = bh.to("cuda", non_blocking=True)
        bi = torch.empty(ctx.field_elems * nrhs, dtype=torch.complex128, device="cuda")
        G.dwf_pack(ctx.h, bi, bd, G.DWF_F64, nrhs)
        xi = torch.zeros_like(bi)
        G.mg_setup(ctx.h, 2, [NVEC], [BLOCK], p)
        G.mg_solve(ctx.h, bi, xi, TOL, nrhs)
        G.dwf_unpack(ctx.h, bd, xi, G.DWF_F64, nrhs)
        xh.copy_(bd, non_blocking=True)
        torch.cuda.synchronize()
        if i > 0:
            times.append(time.perf_counter() - t0)
        ctx.close()
        del bd, bi, xi
        torch.cuda.empty_cache()
    return {"value": statistics.median(times) / nrhs, "unit": "s/solve", "steps": steps,
            "h2d_bytes_per_step": int(Uh.numel() * 16 + bh.numel() * 16),
            "d2h_bytes_per_step": int(xh.numel() * 16)}


def run_learned(G, torch, U, b, p):
    """The learned setup on this workload against the method without it: the
    committed refinement network (trained at 8^4 x 16) refines the adaptive
    vectors after 50 relaxation iterations and the setup relaxes 550 more,
    against the chosen setup's 600 relaxation iterations from random vectors;
    setup time and outer iterations of the first source's solve."""
    import pathlib
    from paper_1205_2933_gb300 import learned as Lm
    shape, params, meta = Lm.load(pathlib.Path(Lm.__file__).parent / "weights" / "near_null_refine_8x8x8x8_Ls16.npz")
    ctx = G.Context(DIMS, LS, M5, MF, torch.from_numpy(U).cuda())
    N = ctx.field_elems
    b0 = b[:N].contiguous()
    net = Lm.make_net(ctx, shape, params)
    out = {}
    for name in ("plain", "learned"):
        q = G.mg_params.from_buffer_copy(p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name == "learned":
            q.setup_iters0 = p.setup_iters0 - meta["pre_iters"]
            G.mg_setup_learned(ctx.h, net, 11, 2, [NVEC], [BLOCK], q, pre_iters0=meta["pre_iters"])
        else:
            G.mg_setup(ctx.h, 2, [NVEC], [BLOCK], q)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        x0 = torch.zeros_like(b0)
        st = G.mg_solve(ctx.h, b0, x0, TOL, 1, check=False)
        torch.cuda.synchronize()
        out[name] = {"setup_s": ts, "iters": st.iters, "solve_s": st.seconds, "true_res": st.true_res,
                     "status": st.status}
    G.net_destroy(net)
    ctx.close()
    out["note"] = ("refinement network (8^4 x 16 training) after 50 relaxation iterations, then 550 more, "
                   "against 600 relaxation iterations from random vectors; first source, one-RHS solve")
    return out


def run_plain(G, torch, U, b, x_chosen, nplain, chosen_value):
    """The plain method, FP64 throughout (smoother, V-cycle, coarse stencil and
    coarsest solve), with the chosen configuration's solver parameters, on the
    same lattice: one setup and nplain solves.  Its solutions are the FP64
    reference for the chosen solutions' errors."""
    ctx = G.Context(DIMS, LS, M5, MF, torch.from_numpy(U).cuda())
    N = ctx.field_elems
    p = mixed_params(G)
    p.smoother_prec = G.DWF_F64
    p.coarse_prec[0] = G.DWF_F64
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G.mg_setup(ctx.h, 2, [NVEC], [BLOCK], p)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    solves, errors, iters, res = [], [], [], []
    for i in range(nplain):
        bi = b[i * N:(i + 1) * N].contiguous()
        xp = torch.zeros_like(bi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = G.mg_solve(ctx.h, bi, xp, TOL, 1, check=False)
        torch.cuda.synchronize()
        solves.append(time.perf_counter() - t0)
        iters.append(st.iters)
        res.append(st.true_res)
        xc = x_chosen[i * N:(i + 1) * N]
        errors.append(float(torch.linalg.vector_norm(xc - xp) / torch.linalg.vector_norm(xp)))
    ctx.close()
    per = t_setup / NRHS + statistics.mean(solves)
    return {"setup_s": t_setup, "solve_s": solves, "iters": iters, "true_res": res,
            "per_solve_amortised_12": per, "chosen_over_plain": chosen_value / per,
            "speedup_vs_plain": per / chosen_value,
            "chosen_rel_error_vs_fp64": errors,
            "note": f"plain FP64 MG (same parameters, FP64 everywhere) on the first {nplain} sources; "
                    f"the errors compare the chosen solutions of the last timed step with these FP64 solutions"}


if __name__ == "__main__":
    main()
