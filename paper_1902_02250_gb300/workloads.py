"""Seeded synthetic particle sets shaped like the paper's workloads.

This module only draws random numbers (numpy ``Generator(PCG64(seed))``); it
holds none of the treecode's arithmetic.  Both the CUDA path and the CPU
oracle take their inputs from here.  Every array is float64, row-major.
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(n, seed, lo=-1.0, hi=1.0, win=3):
    """n points uniform in [lo, hi]^3 with weights uniform in [-1, 1]^win
    (the Stokeslet workloads with N = 10^4 and N = 10^6)."""
    g = rng(seed)
    x = g.uniform(lo, hi, size=(n, 3))
    f = g.uniform(-1.0, 1.0, size=(n, win))
    return x, f


def sphere_surface(n, seed, win=3):
    """n points uniform on the unit sphere (x = g/|g|, g ~ N(0, I3)), with
    N(0, 1) weights: a boundary-element-like quadrature set."""
    g = rng(seed)
    v = g.standard_normal(size=(n, 3))
    x = v / np.linalg.norm(v, axis=1, keepdims=True)
    f = g.standard_normal(size=(n, win))
    return x, f


def plummer_with_background(n, seed, a=0.1, rmax=2.0, frac_uniform=0.1, box=2.0, win=3):
    """(1 - frac_uniform) n points from a Plummer sphere of scale a, truncated
    at radius rmax (r = a (u^(-2/3) - 1)^(-1/2), isotropic direction,
    rejection of r > rmax), plus frac_uniform n points uniform in
    [-box, box]^3; weights uniform in [-1, 1]^win."""
    g = rng(seed)
    nb = int(round(frac_uniform * n))
    npl = n - nb
    pts = []
    have = 0
    while have < npl:
        m = int(1.3 * (npl - have)) + 16
        u = g.uniform(0.0, 1.0, size=m)
        u = np.clip(u, 1e-300, None)
        r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        r = r[np.isfinite(r) & (r <= rmax)]
        d = g.standard_normal(size=(len(r), 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts.append(d * r[:, None])
        have += len(r)
    xp = np.concatenate(pts)[:npl]
    xb = g.uniform(-box, box, size=(nb, 3))
    x = np.concatenate([xp, xb])
    x = x[g.permutation(n)]
    f = g.uniform(-1.0, 1.0, size=(n, win))
    return np.ascontiguousarray(x), f


def batched_systems(num, seed, nmin=1000, nmax=200000, side=(0.5, 2.0), origin=10.0, win=3):
    """num independent systems; N_s = round(exp(U[ln nmin, ln nmax])), each
    uniform in its own box of side U[side] with origin U[-origin, origin]^3;
    weights uniform in [-1, 1]^win.  Returns a list of (x, f)."""
    g = rng(seed)
    sizes = np.rint(np.exp(g.uniform(np.log(nmin), np.log(nmax), size=num))).astype(np.int64)
    out = []
    for ns in sizes:
        s = g.uniform(side[0], side[1])
        o = g.uniform(-origin, origin, size=3)
        x = o + s * g.uniform(0.0, 1.0, size=(int(ns), 3))
        f = g.uniform(-1.0, 1.0, size=(int(ns), win))
        out.append((x, f))
    return out


def organisms(n_pairs, seed, length=10.0, ell=0.02, orientation="random"):
    """Example 1 shape: n_pairs organisms with uniform centres in [0, length]^3;
    each is two particles ell apart carrying unit forces of opposite sign along
    the organism axis.  The paper does not state the orientations:
    "random" draws each axis uniformly on the sphere, "aligned" gives every
    organism the axis z (the draws of the centres are the same)."""
    g = rng(seed)
    c = g.uniform(0.0, length, size=(n_pairs, 3))
    d = g.standard_normal(size=(n_pairs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    if orientation == "aligned":
        d = np.zeros((n_pairs, 3))
        d[:, 2] = 1.0
    elif orientation != "random":
        raise ValueError("orientation must be 'random' or 'aligned'")
    x = np.empty((2 * n_pairs, 3))
    f = np.empty((2 * n_pairs, 3))
    x[0::2] = c + 0.5 * ell * d
    x[1::2] = c - 0.5 * ell * d
    f[0::2] = d
    f[1::2] = -d
    return x, f


def helical_rods(n_side, seed, segments=150, spacing=16.0 / 14.0, height=9.0):
    """Example 2 shape: n_side^2 helical rods (x0 + 0.3 cos 2z, y0 + 0.3 sin 2z, z),
    0 <= z <= height, segments+1 points each, base points on a square grid of
    the given spacing; force and torque components uniform in [-1, 1]."""
    g = rng(seed)
    z = np.linspace(0.0, height, segments + 1)
    grid = (np.arange(n_side) - 0.5 * (n_side - 1)) * spacing
    x0, y0 = np.meshgrid(grid, grid, indexing="ij")
    x0 = x0.ravel()[:, None]
    y0 = y0.ravel()[:, None]
    X = np.stack([x0 + 0.3 * np.cos(2 * z)[None, :], y0 + 0.3 * np.sin(2 * z)[None, :],
                  np.broadcast_to(z[None, :], (len(x0), len(z)))], axis=-1).reshape(-1, 3)
    f = g.uniform(-1.0, 1.0, size=(len(X), 6))
    return np.ascontiguousarray(X), f


def sample_indices(n, k, seed):
    """k distinct indices of range(n), drawn without replacement."""
    g = rng(seed)
    k = min(k, n)
    return np.sort(g.choice(n, size=k, replace=False))
