"""Plain numpy reference of the per-cluster degree selector (FP64).

Test infrastructure, like the rest of ``oracle/``.  The network is
    z0 = (x - mu) / sd                       (12 features, fixed normalisation)
    h1 = relu(W1 z0 + b1)                    (64)
    h2 = relu(W2 h1 + b2)                    (64)
    logits = W3 h2 + b3                      (6 classes)
trained with the mean softmax cross-entropy and Adam.  Gradients are the chain
rule written out layer by layer.  Parameter vector layout (floats):
    mu[12] sd[12] W1[64][12] b1[64] W2[64][64] b2[64] W3[6][64] b3[6]
mu and sd are not trained (their gradient is zero).
"""
import numpy as np

NF, NH, NC = 12, 64, 6
SHAPES = [("mu", (NF,)), ("sd", (NF,)), ("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)),
          ("b2", (NH,)), ("W3", (NC, NH)), ("b3", (NC,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def init(seed, mu, sd):
    """He-style initial weights (seeded), zero biases."""
    g = np.random.Generator(np.random.PCG64(seed))
    d = {"mu": np.asarray(mu, np.float64), "sd": np.asarray(sd, np.float64),
         "W1": g.standard_normal((NH, NF)) * np.sqrt(2.0 / NF), "b1": np.zeros(NH),
         "W2": g.standard_normal((NH, NH)) * np.sqrt(2.0 / NH), "b2": np.zeros(NH),
         "W3": g.standard_normal((NC, NH)) * np.sqrt(1.0 / NH), "b3": np.zeros(NC)}
    return pack(d)


def forward(p, X):
    d = unpack(np.asarray(p, np.float64))
    X = np.asarray(X, np.float64)
    z0 = (X - d["mu"]) / d["sd"]
    a1 = z0 @ d["W1"].T + d["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ d["W2"].T + d["b2"]
    h2 = np.maximum(a2, 0.0)
    logits = h2 @ d["W3"].T + d["b3"]
    return logits, (z0, a1, h1, a2, h2)


def softmax(logits):
    z = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss_and_grad(p, X, labels):
    """Mean cross-entropy and its gradient with respect to p."""
    d = unpack(np.asarray(p, np.float64))
    logits, (z0, a1, h1, a2, h2) = forward(p, X)
    n = len(labels)
    P = softmax(logits)
    loss = -np.mean(np.log(P[np.arange(n), labels]))
    g3 = P.copy()
    g3[np.arange(n), labels] -= 1.0
    g3 /= n                                   # dL/dlogits
    gW3 = g3.T @ h2
    gb3 = g3.sum(axis=0)
    gh2 = g3 @ d["W3"]
    ga2 = gh2 * (a2 > 0)
    gW2 = ga2.T @ h1
    gb2 = ga2.sum(axis=0)
    gh1 = ga2 @ d["W2"]
    ga1 = gh1 * (a1 > 0)
    gW1 = ga1.T @ z0
    gb1 = ga1.sum(axis=0)
    grad = pack({"mu": np.zeros(NF), "sd": np.zeros(NF), "W1": gW1, "b1": gb1, "W2": gW2,
                 "b2": gb2, "W3": gW3, "b3": gb3})
    return loss, grad


def adam_step(p, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); mu and sd stay fixed."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    step = lr * mh / (np.sqrt(vh) + eps)
    step[:2 * NF] = 0.0
    return p - step, m, v
