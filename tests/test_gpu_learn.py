"""The degree selector's CUDA kernels against the CPU oracle: cluster features,
measured per-cluster far-field errors, and the network's forward pass,
gradient (checked against the chain rule of oracle/mlp.py) and Adam step.

Tolerances: features are FP32 roundings of FP64 values (relative 1e-5);
sample counts are exact (both sides draw SplitMix64 of the same keys);
squared errors are squares of FP64 differences of nearly equal sums taken
in another order (their roots to 1e-7 relative plus 1e-11 absolute); the network
runs in FP32 (relative 2e-5 on logits and loss, 1e-4 on the gradient norm),
and its argmax is compared only where the oracle's top two logits differ by
more than the FP32 tolerance.
"""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ST, RO = 0, 1


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_02250_gb300 import build, kitc
    build.build()
    torch.cuda.set_device(0)
    return kitc


@pytest.fixture(scope="module")
def L(orc):
    from oracle import learn
    return learn


@pytest.fixture(scope="module")
def M(orc):
    from oracle import mlp
    return mlp


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda()


def _setup(K, orc, x, f, leaf, kernel=ST, B=64, theta=0.7, eps=0.01, degree=4):
    p = K.Params(theta=theta, degree=degree, leaf_size=leaf, eps=eps, kernel=kernel,
                 mac=K.MAC_BATCH, target_batch=B)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_plan_targets(t, dev(x))
    o = orc.Tree(x, leaf)
    lists = o.treecode_batch(f, o.modified_weights(f, 1), 1, kernel, eps, theta, x, B, B,
                             lists=True, evaluate=False)
    return t, o, lists


def test_features_match_oracle(K, orc, L):
    x, f = wl.plummer_with_background(9000, 85)
    t, o, lists = _setup(K, orc, x, f, 100)
    got = K.kitc_cluster_features(t, dev(f)).cpu().numpy()
    ref = L.features(o, f, x, lists, 64, 0.01).astype(np.float32)
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-6), np.abs(got - ref).max(axis=0)
    assert (ref[:, 4] > 0).sum() > 10          # clusters accepted by some targets
    t.free()


@pytest.mark.parametrize("kernel", [ST, RO])
@pytest.mark.parametrize("var", [False, True])
def test_far_errors_match_oracle(K, orc, L, kernel, var):
    x, f = wl.uniform_cube(8000, 86)
    n = 5
    t, o, lists = _setup(K, orc, x, f, 120, kernel=kernel, degree=n)
    m = o.nclusters
    if var:
        deg = np.random.default_rng(87).integers(2, 13, m).astype(np.int32)
        K.kitc_set_degrees(t, deg)
        fh, foff = o.modified_weights_var(f, deg)
        fhat_of = lambda c: fh[foff[c]:foff[c] + (deg[c] + 1) ** 3 * 3].reshape(-1, 3)  # noqa: E731
        degree_of = lambda c: int(deg[c])  # noqa: E731
    else:
        fh = o.modified_weights(f, n)
        fhat_of = lambda c: fh[c].reshape(-1, 3)  # noqa: E731
        degree_of = lambda c: n  # noqa: E731
    K.kitc_modified_weights(t, dev(f))
    e2, ns = K.kitc_cluster_far_errors(t, dev(f), max_samples=6, seed=123)
    e2, ns = e2.cpu().numpy(), ns.cpu().numpy()
    r2, rns = L.far_errors(o, f, fhat_of, degree_of, kernel, 0.01, x, lists, 64, 6, 123)
    assert np.array_equal(ns, rns) and rns.sum() > 50
    # err2 is the square of a difference of two nearly equal FP64 sums taken in
    # different orders: compare its root, to 1e-7 relative plus 1e-11 absolute
    # (about 1e-15 of the velocities of these sums)
    assert np.allclose(np.sqrt(e2), np.sqrt(r2), rtol=1e-7, atol=1e-11)
    t.free()


def test_far_errors_need_lists_and_weights(K):
    x, f = wl.uniform_cube(3000, 88)
    p = K.Params(theta=0.7, degree=4, leaf_size=100, eps=0.01, mac=K.MAC_BATCH)
    t = K.kitc_build_tree(dev(x), p)
    with pytest.raises(K.KitcError) as e:
        K.kitc_cluster_features(t, dev(f))
    assert e.value.status == 5
    K.kitc_plan_targets(t, dev(x))
    with pytest.raises(K.KitcError) as e:
        K.kitc_cluster_far_errors(t, dev(f))
    assert e.value.status == 5
    K.kitc_modified_weights(t, dev(f))
    e2, ns = K.kitc_cluster_far_errors(t, dev(f), max_samples=4, seed=1)
    assert int(ns.sum()) > 0 and float(e2.sum()) > 0
    t.free()


# ------------------------------------------------------------------- network
def _net(M, seed, m):
    g = np.random.default_rng(seed)
    X = g.normal(size=(m, 12)) * 2.0 + 1.0
    y = g.integers(0, 6, m).astype(np.int32)
    p = M.init(seed, X.mean(axis=0), X.std(axis=0) + 0.1)
    # nonzero biases so that every term of the chain rule is exercised
    d = M.unpack(p.copy())
    for k in ("b1", "b2", "b3"):
        d[k][:] = g.normal(size=d[k].shape) * 0.1
    return M.pack(d), X, y


@pytest.mark.parametrize("m", [1, 63, 64, 1000, 4097])
def test_forward_matches_oracle(K, M, m):
    import torch
    p, X, _ = _net(M, 90 + m, m)
    lg, deg = K.kitc_mlp_forward(dev(p, torch.float32), dev(X, torch.float32),
                                 class_degree=[2, 4, 6, 8, 10, 12])
    lg, deg = lg.cpu().numpy(), deg.cpu().numpy()
    ref, _ = M.forward(p.astype(np.float32).astype(np.float64),
                       X.astype(np.float32).astype(np.float64))
    scale = np.abs(ref).max() + 1e-30
    assert np.abs(lg - ref).max() <= 2e-5 * scale
    top = np.sort(ref, axis=1)
    clear = top[:, -1] - top[:, -2] > 1e-4 * scale
    want = np.array([2, 4, 6, 8, 10, 12])[np.argmax(ref, axis=1)]
    assert np.array_equal(deg[clear], want[clear]) and clear.sum() >= 0.9 * m


@pytest.mark.parametrize("m", [1, 64, 65, 3000])
def test_gradient_matches_oracle(K, M, m):
    import torch
    p, X, y = _net(M, 100 + m, m)
    p32 = p.astype(np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    tr = K.MLPTrainer(dev(p, torch.float32), m)
    loss, grad = tr.loss_grad(dev(X, torch.float32), dev(y))
    loss, grad = loss.cpu().numpy(), grad.cpu().numpy()
    rl, rg = M.loss_and_grad(p32, X32, y)
    assert abs(loss[0] - rl) <= 2e-5 * abs(rl) and loss[1] == 0
    assert np.linalg.norm(grad - rg) <= 1e-4 * np.linalg.norm(rg)
    assert np.all(grad[:24] == 0)
    # every parameter block, separately
    for name, sl in (("W1", slice(24, 792)), ("W2", slice(856, 4952)), ("W3", slice(5016, 5400)),
                     ("b3", slice(5400, 5406))):
        assert np.linalg.norm(grad[sl] - rg[sl]) <= 2e-4 * np.linalg.norm(rg[sl]) + 1e-12, name
    # the same call twice: the same bits
    _, grad2 = tr.loss_grad(dev(X, torch.float32), dev(y))
    assert np.array_equal(grad, grad2.cpu().numpy())


def test_gradient_against_finite_differences(K, M):
    """The oracle's chain rule, pinned independently by central differences
    in FP64, agrees with the device gradient."""
    import torch
    p, X, y = _net(M, 110, 200)
    p = p.astype(np.float32).astype(np.float64)
    X = X.astype(np.float32).astype(np.float64)
    tr = K.MLPTrainer(dev(p, torch.float32), 200)
    _, g = tr.loss_grad(dev(X, torch.float32), dev(y))
    g = g.cpu().numpy()
    rng = np.random.default_rng(111)
    for k in rng.choice(np.arange(24, M.NPARAM), 40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss_and_grad(pp, X, y)[0] - M.loss_and_grad(pm, X, y)[0]) / (2 * h)
        assert abs(g[k] - fd) <= 1e-3 * max(abs(fd), 1e-3), k


def test_rejected_labels_are_counted(K, M):
    import torch
    p, X, y = _net(M, 120, 130)
    y[[3, 77]] = [6, -1]
    tr = K.MLPTrainer(dev(p, torch.float32), 130)
    loss, _ = tr.loss_grad(dev(X, torch.float32), dev(y))
    assert loss.cpu().numpy()[1] == 2


def test_adam_matches_oracle_and_training_lowers_the_loss(K, M):
    import torch
    p, X, y = _net(M, 130, 2000)
    # labels a function of the inputs, so that the loss can fall
    y = (np.digitize(X[:, 0] + 0.5 * X[:, 1], [-2, -0.5, 1, 2.5, 4])).astype(np.int32)
    pd = dev(p, torch.float32)
    tr = K.MLPTrainer(pd, 2000)
    Xd, yd = dev(X, torch.float32), dev(y)
    p64 = p.astype(np.float32).astype(np.float64)
    m1 = np.zeros_like(p64)
    m2 = np.zeros_like(p64)
    for step in range(1, 4):
        _, g = tr.loss_grad(Xd, yd)
        g64 = g.cpu().numpy().astype(np.float64)
        tr.adam(1e-3)
        p64, m1, m2 = M.adam_step(p64, g64, m1, m2, step, 1e-3)
        assert np.abs(pd.cpu().numpy() - p64).max() <= 1e-6
    l0 = float(tr.loss_grad(Xd, yd)[0][0])
    for _ in range(300):
        tr.step(Xd, yd, 3e-3)
    l1 = float(tr.loss_grad(Xd, yd)[0][0])
    assert l1 < 0.5 * l0
    assert np.all(pd.cpu().numpy()[:24] == p.astype(np.float32)[:24])
