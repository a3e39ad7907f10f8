"""The graph-capturable pipeline (include/kitc_pipeline.h) against the eager
entry points.

The pipeline plans every stage on the device (tree levels, work items of the
weights pass, the paired-record plan, list lengths) in buffers sized once from
example inputs.  On inputs that fit, each stage must take exactly the eager
path's decisions in the same order, so the output is compared bit for bit
with kitc_build_tree / kitc_build_forest + kitc_modified_weights +
kitc_evaluate(_forest) on the same inputs (which the parity tests compare
with the oracle):
* one system, six kernel / precision / MAC / weights-mode combinations,
  separate and self targets, on coordinates and weights other than the
  example's;
* a forest of 12 systems through the handle's CUDA graph (hi/lo and
  leaf-offset near fields), replayed on new values written into the same
  buffers, with exact interaction counts and no allocation across replays;
* a forest whose systems have target sets of their own (rotlet, per-target
  MAC, batches of 48), through run() and the graph;
* the degenerate trees of the eager tree tests (one particle, a root leaf,
  coincident points, chains to the depth limit, a slab);
* an input that needs more levels and entries than reserved: the run stays in
  bounds, reports KITC_ERR_TOO_LARGE, and the next run that fits is exact again.
"""
import gc

import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

from devpool import USED_MEM_HIGH, Pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_02250_gb300 import build, kitc
    build.build()
    torch.cuda.set_device(0)
    return kitc


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def jitter(x, seed, scale=1e-3):
    return x + scale * wl.rng(seed).uniform(-1.0, 1.0, size=x.shape)


def eager(K, x, f, p, y=None, sc=None, tc=None):
    """The eager entry points: (output, stats)."""
    if sc is None:
        return K.treecode(x, f, p, tgt_xyz=y)
    t = K.kitc_build_forest(x, sc, p)
    try:
        K.kitc_modified_weights(t, f)
        out = K.kitc_evaluate_forest(t, x if y is None else y, sc if tc is None else tc)
        return out, t.stats()
    finally:
        t.free()


def same_counts(a, b):
    for k in ("n_clusters", "depth", "n_leaves", "n_batches", "far_entries", "near_entries",
              "near_pairs", "far_points", "near_exec", "far_exec"):
        assert a[k] == b[k], (k, a[k], b[k])


CASES = [  # kernel, precision, MAC, weights mode, batch, separate targets
    ("stokeslet mixed all-targets", 0, 1, 2, 0, 64, True),
    ("rotlet mixed per-target", 1, 1, 0, 0, 64, False),
    ("stokeslet+rotlet mixed batch", 2, 1, 1, 0, 32, True),
    ("stokeslet fp64 batch algorithm1", 0, 0, 1, 1, 64, False),
    ("stokeslet leaf-offsets all-targets", 0, 2, 2, 0, 64, True),
    ("rotlet leaf-offsets per-target", 1, 2, 0, 0, 64, False),
]


@pytest.mark.parametrize("name,kernel,prec,mac,wmode,batch,separate", CASES,
                         ids=[c[0] for c in CASES])
def test_pipeline_matches_eager_bit_for_bit(K, name, kernel, prec, mac, wmode, batch, separate):
    import torch
    win = 6 if kernel == 2 else 3
    x0, f0 = wl.uniform_cube(60_000, 81, win=win)
    y0 = wl.uniform_cube(23_456, 82)[0] if separate else None
    p = K.Params(theta=0.7, degree=6, leaf_size=700, eps=0.003, kernel=kernel, precision=prec,
                 mac=mac, target_batch=batch, weights=wmode)
    pipe = K.Pipeline(dev(x0), p, tgt_xyz=None if y0 is None else dev(y0))
    try:
        for step in range(2):  # the example itself, then other coordinates and weights
            x = x0 if step == 0 else jitter(x0, 90 + step)
            f = f0 if step == 0 else wl.uniform_cube(len(x0), 95 + step, win=win)[1]
            y = None if y0 is None else (y0 if step == 0 else jitter(y0, 97 + step))
            xd, fd = dev(x), dev(f)
            yd = None if y is None else dev(y)
            out = pipe.run(xd, fd, yd)
            st = pipe.check()
            ref, rst = eager(K, xd, fd, p, y=yd)
            assert torch.equal(out, ref), (name, step, float((out - ref).abs().max()))
            same_counts(st, rst)
    finally:
        pipe.free()


@pytest.mark.parametrize("prec", ["MIXED", "MIXED_LEAF"])
def test_pipeline_forest_graph_replay_bit_for_bit(K, prec):
    """A forest through the handle's CUDA graph: replayed on new coordinates
    and weights written into the captured buffers, bit-identical to the eager
    forest each time, and no device memory allocated across replays."""
    import torch
    systems = wl.batched_systems(12, 83, nmin=2000, nmax=40_000)
    sc = np.array([len(s[0]) for s in systems], np.int64)
    x0 = np.concatenate([s[0] for s in systems])
    f0 = np.concatenate([s[1] for s in systems])
    p = K.Params(theta=0.7, degree=7, leaf_size=1000, eps=1e-3, precision=getattr(K, prec),
                 mac=K.MAC_ALL, target_batch=64)
    pipe = K.Pipeline(dev(x0), p, src_counts=sc)
    try:
        xb, fb = dev(x0), dev(f0)
        out = torch.empty((len(x0), 3), dtype=torch.float64, device="cuda")
        pool = Pool(torch.cuda.current_device())
        for step in range(4):
            x = x0 if step == 0 else jitter(x0, 100 + step, scale=2e-3)
            f = f0 if step == 0 else wl.uniform_cube(len(x0), 110 + step)[1]
            xb.copy_(dev(x))
            fb.copy_(dev(f))
            if step == 2:  # no collection inside the window: it frees test temporaries
                gc.collect()
                gc.disable()
                torch.cuda.synchronize()
                before = pool.snapshot()
                pool.reset_high()
            pipe.replay(xb, fb, out=out)
            if step == 2:
                torch.cuda.synchronize()
                after = pool.snapshot()
                gc.enable()
                assert after == before, (before, after)
                assert pool.get(USED_MEM_HIGH) == before[1]
            st = pipe.check()
            ref, rst = eager(K, dev(x), dev(f), p, sc=sc)
            assert torch.equal(out, ref), (step, float((out - ref).abs().max()))
            same_counts(st, rst)
        assert pipe.graph_launches() > 20
    finally:
        pipe.free()


def test_pipeline_forest_with_own_targets(K):
    """A forest whose systems have target sets of their own, of other sizes than
    their sources (rotlet, per-target MAC, batches of 48), through run() and
    replay(): bit-identical to the eager forest, exact counts."""
    import torch
    systems = wl.batched_systems(7, 87, nmin=1500, nmax=25_000)
    sc = np.array([len(s[0]) for s in systems], np.int64)
    g = wl.rng(88)
    tgts = []
    for xs, _ in systems:
        lo, hi = xs.min(0), xs.max(0)
        tgts.append(lo + (hi - lo) * g.uniform(0.0, 1.0, size=(int(g.integers(100, 9000)), 3)))
    tc = np.array([len(t) for t in tgts], np.int64)
    x = np.concatenate([s[0] for s in systems])
    f = np.concatenate([s[1] for s in systems])
    y = np.concatenate(tgts)
    p = K.Params(theta=0.65, degree=6, leaf_size=800, eps=2e-3, kernel=K.ROTLET, precision=K.MIXED,
                 mac=K.MAC_PARTICLE, target_batch=48)
    xd, fd, yd = dev(x), dev(f), dev(y)
    pipe = K.Pipeline(xd, p, src_counts=sc, tgt_xyz=yd, tgt_counts=tc)
    try:
        ref, rst = eager(K, xd, fd, p, y=yd, sc=sc, tc=tc)
        out = pipe.run(xd, fd, yd)
        same_counts(pipe.check(), rst)
        assert torch.equal(out, ref), float((out - ref).abs().max())
        out2 = torch.empty_like(ref)
        for _ in range(2):  # capture, then a launch of the graph
            pipe.replay(xd, fd, yd, out=out2)
            same_counts(pipe.check(), rst)
            assert torch.equal(out2, ref)
    finally:
        pipe.free()


DEGENERATE = {
    # one particle; a root that is already a leaf; 300 coincident points among
    # 700 others; ten groups of 200 coincident points with N0 = 100, whose
    # chains run to the depth limit (41 levels queued, 40 upward levels); a slab
    "one": lambda: (np.array([[0.25, -0.5, 1.0]]), 4),
    "root_leaf": lambda: (wl.uniform_cube(500, 34)[0], 500),
    "duplicates": lambda: (np.vstack([np.full((300, 3), 0.125), wl.uniform_cube(700, 35)[0]]), 50),
    "chains": lambda: (np.repeat(wl.uniform_cube(10, 36)[0], 200, axis=0), 100),
    "slab": lambda: (np.column_stack([wl.rng(1).uniform(0, 16, 30000), wl.rng(2).uniform(0, 16, 30000),
                                      wl.rng(3).uniform(0, 9, 30000)]), 400),
}


@pytest.mark.parametrize("case", sorted(DEGENERATE))
def test_pipeline_degenerate_trees(K, case):
    """The trees of the eager tree tests, through the whole pipeline (mixed
    Stokeslet, all-targets MAC): bit-identical to the eager calls."""
    import torch
    x, N0 = DEGENERATE[case]()
    f = wl.rng(89).uniform(-1.0, 1.0, size=(len(x), 3))
    p = K.Params(theta=0.7, degree=4, leaf_size=N0, eps=0.01, precision=K.MIXED, mac=K.MAC_ALL,
                 target_batch=64)
    xd, fd = dev(x), dev(f)
    pipe = K.Pipeline(xd, p)
    try:
        out = pipe.run(xd, fd)
        st = pipe.check()
        ref, rst = eager(K, xd, fd, p)
        assert torch.equal(out, ref), (case, float((out - ref).abs().max()))
        same_counts(st, rst)
    finally:
        pipe.free()


def test_pipeline_overflow_is_reported_and_recoverable(K):
    """Created on a uniform cube with no slack, run on a centrally concentrated
    input of the same size, whose tree is deeper than the handle's levels:
    the status is KITC_ERR_TOO_LARGE; then a run on the uniform input is
    exact again."""
    import torch
    n = 40_000
    xu, f = wl.uniform_cube(n, 84)
    xp, _ = wl.plummer_with_background(n, 85)
    p = K.Params(theta=0.7, degree=5, leaf_size=200, eps=1e-3, precision=K.MIXED,
                 mac=K.MAC_ALL, target_batch=64)
    fd = dev(f)
    _, su = eager(K, dev(xu), fd, p)
    _, sp = eager(K, dev(xp), fd, p)
    assert sp["depth"] > su["depth"] + 2  # the handle holds depth + 2 levels
    pipe = K.Pipeline(dev(xu), p, slack=1.0)
    try:
        pipe.run(dev(xp), fd)
        code, _ = pipe.status()
        assert code == 6
        out = pipe.run(dev(xu), fd)
        st = pipe.check()
        ref, rst = eager(K, dev(xu), fd, p)
        assert torch.equal(out, ref)
        same_counts(st, rst)
    finally:
        pipe.free()


def test_pipeline_argument_checks(K):
    x, f = wl.uniform_cube(5000, 86)
    xd, fd = dev(x), dev(f)
    with pytest.raises(K.KitcError) as e:
        K.Pipeline(xd, K.Params(), slack=0.5)
    assert e.value.status == 1
    pipe = K.Pipeline(xd, K.Params(leaf_size=300))
    try:
        code, st = pipe.status()  # before any run: no error, no counts
        assert code == 0 and st["far_points"] == 0 and st["near_pairs"] == 0 and st["n_clusters"] == 0
        with pytest.raises(K.KitcError) as e:  # created with the sources as targets
            pipe.run(xd, fd, tgt_xyz=xd)
        assert e.value.status == 1
        with pytest.raises(ValueError):
            pipe.run(dev(x[:4000]), fd)
    finally:
        pipe.free()
