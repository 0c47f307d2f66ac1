"""The learned near-null setup judged by the method without it (the adaptive
setup of Sec. 2 relaxing random vectors).

The committed refinement network (trained on the GPU by the library's own
forward, backward and Adam kernels on heatbath lattices 1000-1031 at 8^4,
Ls = 16, beta = 6.0, m_f = 0.001) refines the adaptive vectors after 50
relaxation iterations, and the setup then relaxes them 50 more.  The method
without the network relaxes random vectors for the same 100 iterations.  On
the 8 held-out lattices (seeds 1032-1039) the learned setup must need no
more outer iterations than the plain one on at least 6 and fewer in total;
it costs more setup time (one network inference), which the test records
but does not judge."""
import pathlib

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_refinement_network_against_plain_relaxation():
    from paper_1205_2933_gb300 import dwfmg as G
    from paper_1205_2933_gb300 import learned as Lm
    path = pathlib.Path(Lm.__file__).parent / "weights" / "near_null_refine_8x8x8x8_Ls16.npz"
    shape, params, meta = Lm.load(path)
    assert shape == Lm.REFINE_SHAPE and meta["pre_iters"] == 50
    nvec, block, pre, refine = 24, (4, 4, 4, 4), 50, 50
    rows = []
    for k, seed in enumerate(range(1032, 1040)):
        ctx = Lm.lattice((8, 8, 8, 8), shape["Ls"], seed)
        net = Lm.make_net(ctx, shape, params)
        r = Lm.compare_setups(ctx, net, nvec, block, refine, seed=11 + k, src_seed=500 + k, pre_iters=pre,
                              names=("random", "learned"))
        rows.append((seed, r["random"]["iters"], r["learned"]["iters"], r["random"]["setup_s"], r["learned"]["setup_s"]))
        G.net_destroy(net)
        ctx.close()
    print("seed, iterations plain / learned, setup s plain / learned:", rows)
    plain = np.array([x[1] for x in rows])
    learned = np.array([x[2] for x in rows])
    assert (learned <= plain).sum() >= 6, rows
    assert learned.sum() < plain.sum(), rows
