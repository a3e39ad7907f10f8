"""Per-cluster interpolation degrees (kitc_set_degrees) against the FP64 CPU
oracle: modified weights of Eq. modified_weights at each cluster's own degree,
Algorithm 2 and its batch-MAC variant with (n_c+1)^3 grid points per accepted
cluster, the interaction counts, and the error paths.

Tolerances as in the fixed-degree parity tests: FP64 to 1e-12 relative L2,
the mixed form to MIXED_TOL, counts exact.
"""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

from mixed_parity import check_mixed

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6
ST, RO, SR = 0, 1, 2


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


def random_degrees(m, seed, lo=1, hi=12):
    return np.random.default_rng(seed).integers(lo, hi + 1, m).astype(np.int32)


@pytest.mark.parametrize("hi", [16, 12, 9])
def test_weights_per_cluster_degree(K, orc, hi):
    """hi = 16: Algorithm 1 on every cluster (the upward form's shared memory
    does not fit); hi <= 12: leaves at the largest degree on their root path,
    parents from children, then each cluster down to its own degree."""
    x, f = wl.plummer_with_background(12000, 61)
    p = K.Params(theta=0.7, degree=6, leaf_size=150, eps=0.01)
    t = K.kitc_build_tree(dev(x), p)
    m = t.stats()["n_clusters"]
    deg = random_degrees(m, 62 + hi, 0, hi)
    deg[0] = 0
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    got = t.weights()
    o = orc.Tree(x, 150)
    ref, foff = o.modified_weights_var(f, deg)
    assert got.shape == ref[:len(got)].shape and len(got) == int(
        ((deg.astype(np.int64) + 1) ** 3 * (deg > 0)).sum() * 3)
    for c in range(m):
        if deg[c] == 0:
            continue
        k = (int(deg[c]) + 1) ** 3 * 3
        a, b = got[foff[c]:foff[c] + k], ref[foff[c]:foff[c] + k]
        assert np.linalg.norm(a - b) <= FP64_TOL * max(np.linalg.norm(b), 1e-300), c
    t.free()


def test_weights_per_cluster_degree_six_components(K, orc):
    """Stokeslet + rotlet weights (w_in = 6) in the upward form (degrees <= 9)."""
    x, f = wl.uniform_cube(9000, 60, win=6)
    p = K.Params(theta=0.7, degree=5, leaf_size=150, eps=0.01, kernel=SR)
    t = K.kitc_build_tree(dev(x), p)
    m = t.stats()["n_clusters"]
    deg = random_degrees(m, 59, 0, 9)
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    got = t.weights()
    ref, foff = orc.Tree(x, 150).modified_weights_var(f, deg)
    assert len(got) == len(ref)
    for c in np.nonzero(deg)[0]:
        k = (int(deg[c]) + 1) ** 3 * 6
        a, b = got[foff[c]:foff[c] + k], ref[foff[c]:foff[c] + k]
        assert np.linalg.norm(a - b) <= FP64_TOL * max(np.linalg.norm(b), 1e-300), c
    t.free()


@pytest.mark.parametrize("kernel", [ST, RO, SR])
def test_fp64_particle_mac_per_cluster_degree(K, orc, kernel):
    win = 6 if kernel == SR else 3
    x, f = wl.uniform_cube(9001, 63, win=win)
    tg = wl.uniform_cube(3001, 64)[0]
    p = K.Params(theta=0.7, degree=5, leaf_size=120, eps=0.02, kernel=kernel, mac=K.MAC_PARTICLE)
    t = K.kitc_build_tree(dev(x), p)
    deg = random_degrees(t.stats()["n_clusters"], 65)
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    got = K.kitc_evaluate(t, dev(tg)).cpu().numpy()
    st = t.stats()
    o = orc.Tree(x, 120)
    fh, foff = o.modified_weights_var(f, deg)
    ref, cnt, bad = o.treecode_var(f, fh, deg, foff, kernel, 0.02, 0.7, tg)
    assert bad == 0
    assert st["far_points"] == cnt[1] and st["near_pairs"] == cnt[0] and cnt[1] > 0
    assert orc.rel_l2(ref, got) <= FP64_TOL
    t.free()


def test_fp64_batch_mac_per_cluster_degree_zero_where_unused(K, orc):
    """Clusters that no batch accepts get degree 0 (no weights at all)."""
    x, f = wl.plummer_with_background(10007, 66)
    B = 64
    o = orc.Tree(x, 100)
    lists = o.treecode_batch(f, o.modified_weights(f, 1), 1, ST, 0.01, 0.7, x, B, B, lists=True,
                             evaluate=False)
    used = np.zeros(o.nclusters, bool)
    used[lists["far_list"]] = True
    deg = np.where(used, random_degrees(o.nclusters, 67, 2, 12), 0).astype(np.int32)
    assert (deg == 0).sum() > 0 and used.sum() > 0
    p = K.Params(theta=0.7, degree=4, leaf_size=100, eps=0.01, mac=K.MAC_BATCH, target_batch=B)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    got = K.kitc_evaluate(t, dev(x)).cpu().numpy()
    st = t.stats()
    fh, foff = o.modified_weights_var(f, deg)
    sel = wl.sample_indices(len(x), 2500, 68)
    ref, cnt = o.treecode_batch_var(f, fh, deg, foff, ST, 0.01, 0.7, x, B, B, select=sel)
    assert st["far_points"] == cnt[1] and st["near_pairs"] == cnt[0]
    assert orc.rel_l2(ref[sel], got[sel]) <= FP64_TOL
    t.free()


@pytest.mark.parametrize("kernel", [ST, RO])
@pytest.mark.parametrize("mac", [0, 1])
@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_per_cluster_degree(K, orc, kernel, mac, prec):
    """FP32x2 paired grid records of every degree, with the near field's
    hi/lo (KITC_MIXED) or leaf-offset (KITC_MIXED_LEAF) source records."""
    x, f = wl.uniform_cube(20000, 69)
    p = K.Params(theta=0.6, degree=6, leaf_size=300, eps=0.005, kernel=kernel, mac=mac,
                 precision=prec)
    t = K.kitc_build_tree(dev(x), p)
    deg = random_degrees(t.stats()["n_clusters"], 70, 2, 16)
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    got = K.kitc_evaluate(t, dev(x)).cpu().numpy()
    o = orc.Tree(x, 300)
    fh, foff = o.modified_weights_var(f, deg)
    sel = wl.sample_indices(len(x), 3000, 71)
    if mac == 0:
        ref, _, bad = o.treecode_var(f, fh, deg, foff, kernel, 0.005, 0.6, x[sel])
        assert bad == 0
    else:
        ref = o.treecode_batch_var(f, fh, deg, foff, kernel, 0.005, 0.6, x, 64, 64,
                                   select=sel)[0][sel]
    check_mixed(ref, got[sel], "per-cluster degree kernel=%d mac=%d precision=%d" % (kernel, mac, prec))
    t.free()


def test_uniform_map_equals_fixed_degree(K):
    """A map with n_c = n everywhere reproduces the fixed-degree path with the
    upward pass (leaves by Algorithm 1, parents from children: the same sums in
    the same order)."""
    x, f = wl.uniform_cube(30000, 72)
    for prec in (K.FP64, K.MIXED):
        p = K.Params(theta=0.7, degree=7, leaf_size=400, eps=0.001, precision=prec,
                     weights=K.WEIGHTS_UPWARD, mac=K.MAC_BATCH)
        t = K.kitc_build_tree(dev(x), p)
        K.kitc_modified_weights(t, dev(f))
        a = K.kitc_evaluate(t, dev(x)).cpu().numpy()
        fa = t.weights().ravel()
        K.kitc_set_degrees(t, np.full(t.stats()["n_clusters"], 7, np.int32))
        K.kitc_modified_weights(t, dev(f))
        b = K.kitc_evaluate(t, dev(x)).cpu().numpy()
        assert np.array_equal(fa, t.weights())
        assert np.array_equal(a, b)
        K.kitc_set_degrees(t, None)   # back to the uniform path
        K.kitc_modified_weights(t, dev(f))
        assert np.array_equal(a, K.kitc_evaluate(t, dev(x)).cpu().numpy())
        t.free()


def test_degree_errors(K):
    import torch
    x, f = wl.uniform_cube(5000, 73)
    p = K.Params(theta=0.7, degree=4, leaf_size=100, eps=0.01, mac=K.MAC_BATCH)
    t = K.kitc_build_tree(dev(x), p)
    m = t.stats()["n_clusters"]
    with pytest.raises(RuntimeError):
        K.kitc_set_degrees(t, np.full(m, 17, np.int32))
    with pytest.raises(RuntimeError):
        K.kitc_set_degrees(t, np.full(m, -1, np.int32))
    # every cluster at degree 0: any accepted cluster is an error, not a wrong sum
    K.kitc_set_degrees(t, np.zeros(m, np.int32))
    K.kitc_modified_weights(t, dev(f))
    with pytest.raises(K.KitcError) as e:
        K.kitc_evaluate(t, dev(x))
    assert e.value.status == 1
    # a device-resident map and kitc_apply (graph replay) with it
    d = torch.from_numpy(random_degrees(m, 74, 3, 9)).cuda()
    K.kitc_set_degrees(t, d)
    K.kitc_modified_weights(t, dev(f))
    out = K.kitc_evaluate(t, dev(x))
    ref = out.clone()
    f2 = dev(f)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):              # eager run + capture + replay, then replay
            out.zero_()
            K.kitc_apply(t, f2, out)
            assert torch.equal(out, ref)
    t.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_evaluate_planned_equals_evaluate(K, prec):
    """Lists built before the degree map (kitc_plan_targets) serve the
    evaluation after it: same bits and counts as a full kitc_evaluate."""
    x, f = wl.plummer_with_background(25000, 75)
    p = K.Params(theta=0.7, degree=6, leaf_size=300, eps=0.001, precision=prec, mac=K.MAC_BATCH)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_plan_targets(t, dev(x))
    st0 = t.stats()
    assert st0["n_targets"] == len(x) and st0["far_entries"] > 0
    deg = random_degrees(st0["n_clusters"], 76, 2, 12)
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    a = K.kitc_evaluate_planned(t).cpu().numpy()
    sa = t.stats()
    b = K.kitc_evaluate(t, dev(x)).cpu().numpy()
    sb = t.stats()
    assert np.array_equal(a, b)
    for k in ("far_points", "near_pairs", "far_exec", "near_exec", "far_entries"):
        assert sa[k] == sb[k], k
    # a map with degree 0 on an accepted cluster is refused at evaluation
    deg0 = deg.copy()
    lists = t.lists()
    deg0[lists["far"][0]] = 0
    K.kitc_set_degrees(t, deg0)
    K.kitc_modified_weights(t, dev(f))
    with pytest.raises(K.KitcError) as e:
        K.kitc_evaluate_planned(t)
    assert e.value.status == 1
    t.free()


def test_evaluate_planned_needs_a_plan(K):
    x, f = wl.uniform_cube(3000, 77)
    p = K.Params(theta=0.7, degree=4, leaf_size=100, eps=0.01)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_modified_weights(t, dev(f))
    import torch
    out = torch.empty((len(x), 3), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KitcError) as e:
        K.kitc_evaluate_planned(t, out)
    assert e.value.status == 5
    t.free()


def test_plan_on_side_stream_beside_weights(K):
    """The target tree and lists built on a second stream while the modified
    weights run on the first (they need only the source tree) give the same
    bits as the serial kitc_evaluate."""
    import torch
    x, f = wl.uniform_cube(200000, 78)
    p = K.Params(theta=0.7, degree=9, leaf_size=2000, eps=0.001, precision=K.MIXED, mac=K.MAC_BATCH)
    xd, fd = dev(x), dev(f)
    t = K.kitc_build_tree(xd, p)
    K.kitc_modified_weights(t, fd)
    ref = K.kitc_evaluate(t, xd).cpu().numpy()
    t.free()
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    for _ in range(3):
        t = K.kitc_build_tree(xd, p)
        built = torch.cuda.Event()
        built.record(main)
        K.kitc_modified_weights(t, fd)
        side.wait_event(built)
        K.kitc_plan_targets(t, xd, stream=side)
        main.wait_stream(side)
        out = K.kitc_evaluate_planned(t)
        assert np.array_equal(out.cpu().numpy(), ref)
        t.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_forest_with_degree_map(K, orc, prec):
    """Per-cluster degrees on a forest of independent systems: a uniform map
    reproduces the fixed-degree forest bit for bit, and a random map matches
    the oracle system by system."""
    systems = wl.batched_systems(5, 79, nmin=400, nmax=5000)
    counts = [len(s[0]) for s in systems]
    x = np.vstack([s[0] for s in systems])
    f = np.vstack([s[1] for s in systems])
    p = K.Params(theta=0.7, degree=5, leaf_size=250, eps=0.01, precision=prec, mac=K.MAC_BATCH)
    t = K.kitc_build_forest(dev(x), counts, p)
    K.kitc_modified_weights(t, dev(f))
    a = K.kitc_evaluate_forest(t, dev(x), counts).cpu().numpy()
    m = t.stats()["n_clusters"]
    K.kitc_set_degrees(t, np.full(m, 5, np.int32))
    K.kitc_modified_weights(t, dev(f))
    assert np.array_equal(a, K.kitc_evaluate_forest(t, dev(x), counts).cpu().numpy())
    if prec == 1:
        t.free()
        return
    # a random map: compare each system with the oracle on that system alone
    tr = t.download()
    deg = np.random.default_rng(80).integers(2, 10, m).astype(np.int32)
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    got = K.kitc_evaluate_forest(t, dev(x), counts).cpu().numpy()
    t.free()
    off = np.concatenate([[0], np.cumsum(counts)])
    # clusters of system k: its root and descendants; roots are the clusters without parent
    roots = np.nonzero(tr["parent"] < 0)[0]
    assert len(roots) == len(counts)
    sys_of = np.empty(m, np.int64)
    for c in range(m):
        sys_of[c] = np.searchsorted(roots, c, side="right") - 1 if tr["parent"][c] < 0 else sys_of[tr["parent"][c]]
    for k in range(len(counts)):
        xs, fs = x[off[k]:off[k + 1]], f[off[k]:off[k + 1]]
        o = orc.Tree(xs, 250)
        dk = deg[sys_of == k]
        assert len(dk) == o.nclusters
        fh, foff = o.modified_weights_var(fs, dk)
        ref = o.treecode_batch_var(fs, fh, dk, foff, 0, 0.01, 0.7, xs, 64, 64)[0]
        assert orc.rel_l2(ref, got[off[k]:off[k + 1]]) <= FP64_TOL, k


def test_forest_plan_on_side_stream(K):
    """Forest: target trees and lists planned on a second stream beside the
    weights, then kitc_evaluate_planned, equal kitc_evaluate_forest bit for bit."""
    import torch
    systems = wl.batched_systems(6, 81, nmin=500, nmax=8000)
    counts = [len(s[0]) for s in systems]
    x = np.vstack([s[0] for s in systems])
    f = np.vstack([s[1] for s in systems])
    xd, fd = dev(x), dev(f)
    p = K.Params(theta=0.7, degree=6, leaf_size=400, eps=0.001, precision=K.MIXED)
    t = K.kitc_build_forest(xd, counts, p)
    K.kitc_modified_weights(t, fd)
    ref = K.kitc_evaluate_forest(t, xd, counts).cpu().numpy()
    st_ref = t.stats()
    t.free()
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    t = K.kitc_build_forest(xd, counts, p)
    built = torch.cuda.Event()
    built.record(main)
    K.kitc_modified_weights(t, fd)
    side.wait_event(built)
    K.kitc_plan_targets_forest(t, xd, counts, stream=side)
    main.wait_stream(side)
    out = K.kitc_evaluate_planned(t)
    st = t.stats()
    assert np.array_equal(out.cpu().numpy(), ref)
    assert st["far_points"] == st_ref["far_points"] and st["near_pairs"] == st_ref["near_pairs"]
    t.free()
