"""Training and evaluation of the learned near-null proposal (include/dwfnet.h).

Host-side control only: the network's forward and backward passes, the
projection loss, the optimiser steps, the adaptive setups that produce the
training targets and the solves that judge the result all run in
libdwfmg.so on the GPU.  The paper has no network (its setup relaxes on
D x = 0 from random vectors, Sec. 2); this module trains one on the vectors
that relaxation produces and measures what it saves.

Command line (one GPU):
  python -m paper_1205_2933_gb300.learned --out weights.npz [--train 32 --heldout 8]
trains on seeded heatbath lattices, evaluates on held-out ones and writes
the weights and a JSON report.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import dwfmg as G
from . import inputs as I

SHAPE = dict(c_in=4, hidden=16, layers=3, nout=12, Ls=16)            # proposal from noise
REFINE_SHAPE = dict(c_in=16, hidden=16, layers=3, nout=1, Ls=16)     # refinement of relaxed vectors


def param_shapes(c_in, hidden, layers, nout, Ls):
    """Shapes of the parameter groups in the order of the flat vector (dwfnet.h)."""
    out, cin = [], c_in
    for _ in range(layers):
        out.append((hidden, 4, 9, cin, 4))
        cin = hidden
    out.append((nout, Ls, 4, hidden, 4))
    return out


def init_params(shape: dict, seed: int, head_scale: float = 1.0) -> np.ndarray:
    """Gaussian weights scaled by 1/sqrt(fan-in) (complex), seeded; the head
    additionally by head_scale (small for a refinement network, which then
    starts near the identity through its skip connection)."""
    parts = []
    for k, sh in enumerate(param_shapes(**shape)):
        fan_in = int(np.prod(sh[2:])) if k < shape["layers"] else int(np.prod(sh[3:]))
        w = I.gauss_complex(sh, seed + k, I.STREAM_NETWORK).ravel() / np.sqrt(2.0 * fan_in)
        parts.append(w * (head_scale if k == shape["layers"] else 1.0))
    return np.concatenate(parts)


def save(path, shape: dict, params: np.ndarray, meta: dict | None = None):
    np.savez(path, params=params.astype(np.complex64), shape=json.dumps(shape), meta=json.dumps(meta or {}))


def load(path):
    z = np.load(path)
    return json.loads(str(z["shape"])), z["params"].astype(np.complex128), json.loads(str(z["meta"]))


def make_net(ctx, shape: dict, params: np.ndarray):
    net = G.net_create(ctx.h, shape["c_in"], shape["hidden"], shape["layers"], shape["nout"], shape["Ls"])
    G.net_set_params(net, np.ascontiguousarray(params))
    return net


def solve_params(setup_iters0=1000):
    """The mixed-precision solver of the benchmark (FP32 V-cycle, BF16 coarse stencil)."""
    p = G.mg_default_params()
    p.smoother_prec = G.DWF_F32
    p.coarse_prec[0] = G.DWF_BF16
    p.setup_iters0 = int(setup_iters0)
    return p


def adaptive_targets(ctx, nvec, block, params):
    """Run the plain adaptive setup and return its basis (nvec internal FP64
    fields on the device) as the training target."""
    import torch
    G.mg_setup(ctx.h, 2, [nvec], [block], params)
    q = torch.empty(nvec * ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.mg_get_vectors(ctx.h, 0, q)
    return q


def lattice(dims, Ls, seed, beta=6.0, sweeps=200, M5=1.8, mf=0.001):
    import torch
    U = I.heatbath_links(dims, beta, sweeps, seed)
    return G.Context(dims, Ls, M5, mf, torch.from_numpy(U).cuda())


def relaxed_vectors(ctx, nvec, block, pre_iters, seed):
    """The adaptive vectors after a short relaxation (pre_iters CGNR iterations
    from seeded random vectors): the refinement network's input."""
    import torch
    p = solve_params(pre_iters)
    p.seed = seed
    G.mg_setup(ctx.h, 2, [nvec], [block], p)
    v = torch.empty(nvec // 2 * ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.mg_get_adaptive_vectors(ctx.h, 0, v)
    return v


def train_refine(net, data, nvec, block, epochs, lr, seed=0, log=None):
    """Adam on the projection loss of refined vectors: data holds (context,
    relaxed vectors, targets)."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        tot = 0.0
        for i in rng.permutation(len(data)):
            ctx, v, q = data[i]
            tot += G.net_refine_loss_grad(net, ctx.h, v, nvec // 2, q, nvec, block)
            G.net_adam(net, lr)
        hist.append(tot / len(data))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.5f}")
    return hist


def train(net, data, nvec, block, epochs, lr, seed=0, log=None):
    """Adam on the projection loss over (context, targets) pairs; a fresh
    seeded network input every step.  Returns the mean loss of each epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    step = 0
    for ep in range(epochs):
        tot = 0.0
        for i in rng.permutation(len(data)):
            ctx, q = data[i]
            tot += G.net_loss_grad(net, ctx.h, q, nvec, block, seed=1_000_000 + seed * 100_000 + step)
            G.net_adam(net, lr)
            step += 1
        hist.append(tot / len(data))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.5f}")
    return hist


def solve_iterations(ctx, src_seed, tol=1e-10):
    import torch
    b = torch.from_numpy(I.gaussian_source(ctx.dims, ctx.Ls, src_seed)).cuda()
    bi = torch.empty(ctx.field_elems, dtype=torch.complex128, device="cuda")
    G.dwf_pack(ctx.h, bi, b, G.DWF_F64, 1)
    x = torch.zeros_like(bi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = G.mg_solve(ctx.h, bi, x, tol, 1, check=False)
    torch.cuda.synchronize()
    return {"iters": st.iters, "true_res": st.true_res, "status": st.status, "seconds": time.perf_counter() - t0}


def compare_setups(ctx, net, nvec, block, refine_iters, seed, src_seed, full_iters=1000, pre_iters=0,
                   names=("adaptive", "random", "learned")):
    """Setup time and solve iterations of (a) the plain adaptive setup, (b)
    random vectors + pre_iters + refine_iters relaxation iterations, (c) the
    network's vectors (a refinement network: after pre_iters relaxation
    iterations) + refine_iters relaxation iterations."""
    import torch
    out = {}
    for name in names:
        p = solve_params(full_iters if name == "adaptive" else
                         (refine_iters + pre_iters if name == "random" else refine_iters))
        p.seed = seed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name == "learned":
            G.mg_setup_learned(ctx.h, net, seed, 2, [nvec], [block], p, pre_iters0=pre_iters)
        else:
            G.mg_setup(ctx.h, 2, [nvec], [block], p)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        r = solve_iterations(ctx, src_seed)
        r["setup_s"] = ts
        out[name] = r
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--report", default=None)
    ap.add_argument("--dims", type=int, nargs=4, default=[8, 8, 8, 8])
    ap.add_argument("--train", type=int, default=32)
    ap.add_argument("--heldout", type=int, default=8)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--refine", type=int, nargs="+", default=[0, 25, 100])
    ap.add_argument("--eval-dims", type=int, nargs=4, default=None)
    ap.add_argument("--eval-seeds", type=int, nargs="*", default=[])
    ap.add_argument("--mode", choices=["proposal", "refine"], default="proposal")
    ap.add_argument("--pre", type=int, default=50, help="relaxation iterations before a refinement")
    args = ap.parse_args(argv)
    if args.mode == "refine":
        return main_refine(args)
    import torch
    nvec, block, Ls = 2 * SHAPE["nout"], (4, 4, 4, 4), SHAPE["Ls"]
    log = lambda m: print(f"[learned] {m}", flush=True)
    t0 = time.time()
    train_data, held = [], []
    for k in range(args.train + args.heldout):
        ctx = lattice(tuple(args.dims), Ls, args.seed0 + k)
        q = adaptive_targets(ctx, nvec, block, solve_params())
        (train_data if k < args.train else held).append((ctx, q))
    log(f"targets for {len(train_data)} + {len(held)} lattices in {time.time() - t0:.1f}s")
    params = init_params(SHAPE, 77)
    net = make_net(train_data[0][0], SHAPE, params)
    init_loss = [G.net_loss_grad(net, c.h, q, nvec, block, seed=5) for c, q in held]
    t1 = time.time()
    hist = train(net, train_data, nvec, block, args.epochs, args.lr, log=log)
    train_s = time.time() - t1
    held_loss = [G.net_loss_grad(net, c.h, q, nvec, block, seed=5) for c, q in held]
    log(f"held-out loss {np.mean(init_loss):.4f} (initial) -> {np.mean(held_loss):.4f} (trained), {train_s:.1f}s")
    trained = np.empty(G.net_num_params(net), dtype=np.complex128)
    G.net_get_params(net, trained)
    report = {"shape": SHAPE, "dims": args.dims, "train": args.train, "heldout": args.heldout,
              "epochs": args.epochs, "lr": args.lr, "train_seconds": train_s, "loss_history": hist,
              "heldout_loss_initial": init_loss, "heldout_loss_trained": held_loss, "compare": []}
    # judge on held-out lattices: iterations after each refinement length
    for k, (ctx, _) in enumerate(held):
        for it in args.refine:
            r = compare_setups(ctx, net, nvec, block, it, seed=11 + k, src_seed=500 + k)
            report["compare"].append({"lattice": args.seed0 + args.train + k, "refine": it, **r})
            log(f"held-out {k} refine {it}: " + ", ".join(f"{n} {v['iters']} it" for n, v in r.items() if v))
    if args.eval_dims:
        for s in args.eval_seeds:
            ctx = lattice(tuple(args.eval_dims), Ls, s)
            for it in args.refine:
                r = compare_setups(ctx, net, nvec, block, it, seed=31, src_seed=101)
                report["compare"].append({"lattice": s, "dims": args.eval_dims, "refine": it, **r})
                log(f"eval {args.eval_dims} seed {s} refine {it}: " +
                    ", ".join(f"{n} {v['iters']} it {v['setup_s']:.2f}s" for n, v in r.items() if v))
            ctx.close()
    save(args.out, SHAPE, trained, {"dims": args.dims, "train_seeds": [args.seed0, args.seed0 + args.train - 1],
                                    "epochs": args.epochs, "lr": args.lr})
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)
    G.net_destroy(net)
    for c, _ in train_data + held:
        c.close()


def main_refine(args):
    """Train and judge a refinement network: inputs are the adaptive vectors
    after args.pre relaxation iterations, targets the full setup's basis."""
    import torch
    shape = REFINE_SHAPE
    nvec, block, Ls = 24, (4, 4, 4, 4), shape["Ls"]
    log = lambda m: print(f"[learned] {m}", flush=True)
    t0 = time.time()
    train_data, held = [], []
    for k in range(args.train + args.heldout):
        ctx = lattice(tuple(args.dims), Ls, args.seed0 + k)
        q = adaptive_targets(ctx, nvec, block, solve_params())
        v = relaxed_vectors(ctx, nvec, block, args.pre, seed=3 + k)
        (train_data if k < args.train else held).append((ctx, v, q))
    log(f"targets and relaxed inputs for {len(train_data)} + {len(held)} lattices in {time.time() - t0:.1f}s")
    params = init_params(shape, 78, head_scale=0.01)
    net = make_net(train_data[0][0], shape, params)
    ident = make_net(train_data[0][0], shape, init_params(shape, 78, head_scale=0.0))
    base_loss = [G.net_refine_loss_grad(ident, c.h, v, nvec // 2, q, nvec, block) for c, v, q in held]
    init_loss = [G.net_refine_loss_grad(net, c.h, v, nvec // 2, q, nvec, block) for c, v, q in held]
    t1 = time.time()
    hist = train_refine(net, train_data, nvec, block, args.epochs, args.lr, log=log)
    train_s = time.time() - t1
    held_loss = [G.net_refine_loss_grad(net, c.h, v, nvec // 2, q, nvec, block) for c, v, q in held]
    log(f"held-out loss: relaxed vectors {np.mean(base_loss):.4f}, initial net {np.mean(init_loss):.4f}, "
        f"trained net {np.mean(held_loss):.4f} ({train_s:.1f}s)")
    trained = np.empty(G.net_num_params(net), dtype=np.complex128)
    G.net_get_params(net, trained)
    report = {"mode": "refine", "shape": shape, "dims": args.dims, "pre_iters": args.pre, "train": args.train,
              "heldout": args.heldout, "epochs": args.epochs, "lr": args.lr, "train_seconds": train_s,
              "loss_history": hist, "heldout_loss_relaxed": base_loss, "heldout_loss_initial": init_loss,
              "heldout_loss_trained": held_loss, "compare": []}
    for k, (ctx, _, _) in enumerate(held):
        for it in args.refine:
            r = compare_setups(ctx, net, nvec, block, it, seed=11 + k, src_seed=500 + k, pre_iters=args.pre)
            report["compare"].append({"lattice": args.seed0 + args.train + k, "refine": it, **r})
            log(f"held-out {k} pre {args.pre} refine {it}: " + ", ".join(f"{n} {v['iters']} it" for n, v in r.items()))
    if args.eval_dims:
        for s_ in args.eval_seeds:
            ctx = lattice(tuple(args.eval_dims), Ls, s_)
            for it in args.refine:
                r = compare_setups(ctx, net, nvec, block, it, seed=31, src_seed=101, pre_iters=args.pre)
                report["compare"].append({"lattice": s_, "dims": args.eval_dims, "refine": it, **r})
                log(f"eval {args.eval_dims} seed {s_} pre {args.pre} refine {it}: " +
                    ", ".join(f"{n} {v['iters']} it {v['setup_s']:.2f}s" for n, v in r.items()))
            ctx.close()
    save(args.out, shape, trained, {"mode": "refine", "dims": args.dims, "pre_iters": args.pre,
                                    "train_seeds": [args.seed0, args.seed0 + args.train - 1], "epochs": args.epochs})
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)
    G.net_destroy(net)
    G.net_destroy(ident)
    for c, _, _ in train_data + held:
        c.close()


if __name__ == "__main__":
    main()
