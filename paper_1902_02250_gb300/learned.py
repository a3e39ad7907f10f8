"""Interpolation degree per cluster, chosen by a small trained network.

The paper interpolates every cluster at one degree n (Sec. 3), so the degree
that a few hard clusters need is paid by all of them.  Here the degree of
cluster c is picked from classes (6, 7, 8, 9, 10, 11) by a 12-64-64-6
perceptron (FP32) that reads the cluster features of kitc_cluster_features.
Consecutive degrees around the ones the Plummer workloads need most let a
cluster stop one degree short of the next even one.

Training data come from the treecode itself: on a training system, the
library measures each cluster's far-field error at sampled accepting targets
against the direct sum over the cluster's own sources
(kitc_cluster_far_errors), at every class degree.  The label of cluster c is
the smallest class degree whose RMS error over the samples is within

    tau = budget * u_rms / sqrt(m_far),

u_rms being the RMS velocity (direct sum at sampled targets) and m_far the mean
number of accepted clusters per target: if the errors of different clusters
add like independent terms, the far-field part of the relative L2 error of the
whole sum then stays near `budget`.  Clusters that no target accepts carry no
label and get degree 0 (no modified weights) at inference.  The network is
trained on the GPU by the library's own forward/gradient/Adam kernels.

The fixed-degree treecode is the fallback: a caller measures the learned
run's error against the direct sum and keeps the fixed degree if the budget is
missed (bench.py does).
"""
import math

import numpy as np

from . import kitc as K

CLASSES = (6, 7, 8, 9, 10, 11)


def init_params(seed, mu, sd):
    """He-style initial weights (seeded), zero biases, fixed normalisation."""
    g = np.random.Generator(np.random.PCG64(seed))
    nf, nh, nc = K.NFEAT, K.MLP_HIDDEN, K.MLP_CLASSES
    parts = [np.asarray(mu, np.float64), np.asarray(sd, np.float64),
             g.standard_normal((nh, nf)) * math.sqrt(2.0 / nf), np.zeros(nh),
             g.standard_normal((nh, nh)) * math.sqrt(2.0 / nh), np.zeros(nh),
             g.standard_normal((nc, nh)) * math.sqrt(1.0 / nh), np.zeros(nc)]
    p = np.concatenate([a.ravel() for a in parts]).astype(np.float32)
    assert p.size == K.MLP_NPARAM
    return p


def _u_rms(xd, fd, p, n_sample, seed):
    import torch
    n = xd.shape[0]
    idx = np.random.Generator(np.random.PCG64(seed)).choice(n, min(n, n_sample), replace=False)
    q = K.Params(theta=p.theta, degree=p.degree, leaf_size=p.leaf_size, eps=p.eps, kernel=p.kernel,
                 precision=K.FP64)
    u = K.kitc_direct(xd[torch.from_numpy(idx).to(xd.device)].contiguous(), xd, fd, q)
    return float(torch.sqrt((u ** 2).sum(dim=1).mean()))


def measure(xd, fd, p, samples=32, seed=7, u_samples=4000, log=None):
    """Features and measured far-field errors of every cluster of one system at
    every class degree.  p: the treecode parameters (theta, N0, batch, MAC)."""
    import torch
    t = K.kitc_build_tree(xd, p)
    try:
        K.kitc_plan_targets(t, xd)
        st = t.stats()
        m = st["n_clusters"]
        m_far = st["far_points"] / float((p.degree + 1) ** 3) / float(xd.shape[0])
        feats = K.kitc_cluster_features(t, fd)
        err2 = torch.empty((len(CLASSES), m), dtype=torch.float64, device=xd.device)
        ns = torch.empty((len(CLASSES), m), dtype=torch.int32, device=xd.device)
        for k, n in enumerate(CLASSES):
            K.kitc_set_degrees(t, np.full(m, n, np.int32))
            K.kitc_modified_weights(t, fd)
            e, c = K.kitc_cluster_far_errors(t, fd, max_samples=samples, seed=seed)
            err2[k].copy_(e)
            ns[k].copy_(c)
            if log:
                log(dict(degree=n, rms_far=math.sqrt(float(e.sum()) / max(1, int(c.sum())))))
    finally:
        t.free()
    return dict(features=feats, err2=err2, n_samples=ns, m_far=m_far,
                u_rms=_u_rms(xd, fd, p, u_samples, seed + 1))


def labels(meas, budget):
    """(labels, valid rows, tau): the smallest class meeting tau per cluster."""
    err2 = meas["err2"].cpu().numpy()
    ns = meas["n_samples"].cpu().numpy()
    tau = budget * meas["u_rms"] / math.sqrt(max(meas["m_far"], 1.0))
    valid = ns[0] > 0
    rms = np.sqrt(err2 / np.maximum(ns, 1))
    ok = rms <= tau
    lab = np.where(ok.any(axis=0), ok.argmax(axis=0), len(CLASSES) - 1).astype(np.int32)
    return lab, valid, tau


def train(features, lab, steps=3000, lr=3e-3, seed=11, log=None):
    """Network parameters (CUDA float32) fitted to (features, labels) with
    full-batch Adam on the GPU."""
    import torch
    X = features.contiguous()
    Xh = X.cpu().numpy().astype(np.float64)
    params = torch.from_numpy(init_params(seed, Xh.mean(axis=0), Xh.std(axis=0) + 1e-3)).to(X.device)
    y = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).to(X.device)
    tr = K.MLPTrainer(params, X.shape[0])
    hist = []
    for s in range(steps):
        tr.step(X, y, lr)
        if log and (s % 500 == 0 or s == steps - 1):
            loss = float(tr.loss[0])
            hist.append((s, loss))
            log(dict(step=s, loss=loss))
    _, pred = K.kitc_mlp_forward(params, X, class_degree=list(range(len(CLASSES))), logits=False)
    acc = float((pred.cpu().numpy() == lab).mean())
    return params, dict(loss=hist, accuracy=acc)


def calibrate(xd, fd, p, meas, budgets=(0.25e-6, 0.35e-6, 0.5e-6, 0.7e-6, 1.0e-6, 1.4e-6, 2.0e-6),
              target=0.8e-6,
              n_sample=4000, seed=21, steps=3000, log=None):
    """Trains one selector per label budget (ascending) and keeps the last whose
    learned run on the training system itself stays within `target` relative
    L2 error against the FP64 direct sum on sampled targets.  Returns
    (params, budget, record) or None when even the first budget misses."""
    import torch
    n = xd.shape[0]
    idx = np.random.Generator(np.random.PCG64(seed)).choice(n, min(n, n_sample), replace=False)
    idx_d = torch.from_numpy(idx).to(xd.device)
    q = K.Params(eps=p.eps, kernel=p.kernel, precision=K.FP64)
    ref = K.kitc_direct(xd[idx_d].contiguous(), xd, fd, q)
    out = torch.empty((n, K.kernel_wout(p.kernel)), dtype=torch.float64, device=xd.device)
    rows = None
    best = None
    for b in budgets:
        lab, valid, tau = labels(meas, b)
        if rows is None:
            rows = torch.from_numpy(np.nonzero(valid)[0]).to(xd.device)
        params, rep = train(meas["features"][rows].contiguous(), lab[valid], steps=steps)
        st = learned_step(xd, fd, p, params, out)
        d = out[idx_d] - ref
        E = float(torch.sqrt((d ** 2).sum() / (ref ** 2).sum()))
        rec = dict(budget=b, tau=tau, E_train=E, accuracy=rep["accuracy"],
                   far_points=st["far_points"],
                   label_hist=np.bincount(lab[valid], minlength=len(CLASSES)).tolist())
        if log:
            log(rec)
        if E > target:
            break
        best = (params, b, rec)
    return best


def select_degrees(tree, fd, params):
    """Degree per cluster (CUDA int32) from the network; the tree's lists must
    exist (kitc_plan_targets or kitc_evaluate)."""
    feats = K.kitc_cluster_features(tree, fd)
    _, deg = K.kitc_mlp_forward(params, feats, class_degree=CLASSES, logits=False, zero_unused=True)
    return deg


def learned_step(xd, fd, p, params, out):
    """One treecode pass with learned degrees: tree, lists, features, network,
    degree map, modified weights, evaluation.  Returns the tree's stats."""
    t = K.kitc_build_tree(xd, p)
    try:
        K.kitc_plan_targets(t, xd)
        K.kitc_set_degrees(t, select_degrees(t, fd, params))
        K.kitc_modified_weights(t, fd)
        K.kitc_evaluate_planned(t, out)
        return t.stats()
    finally:
        t.free()
