"""Comparison of a mixed-precision result (FP32 kernel values, FP64 sums) with
the FP64 oracle, shared by the GPU parity tests.

Two bounds, both needed:

* MIXED_TOL on the relative L2 error over all targets, ||u - u_ref|| / ||u_ref||
  (the error measure of the paper's Sec. 8, here of GPU against oracle);
* MIXED_TARGET_TOL on every single target,
      |u_i - u_ref,i| / max(|u_ref,i|, rms_i |u_ref,i|),
  with |.| the Euclidean norm of the target's w_out components.  The floor
  rms|u| keeps a target whose velocity nearly cancels from dominating.  A
  global norm alone lets a wrong sum at a few targets through (1% of targets
  off by 1e-5 moves the global error by only 1e-6); the per-target bound
  catches any single target that is off.

Both tolerances come from FP32 rounding of the kernel values (a few units of
2^-24 ~ 6e-8 relative per value) and of the FP32 partial sums (runs of <= 8
terms, three levels deep, before the FP64 sum: about 4 units more), which puts
the relative L2 error near 4e-7 at worst and a single target's error at a few
times that when its terms have random signs; the measured per-target maxima
are printed.
"""
import numpy as np

FP64_TOL = 1e-12
MIXED_TOL = 1e-6
MIXED_TARGET_TOL = 5e-6


def target_errors(ref, got):
    """Per-target relative error |u_i - u_ref,i| / max(|u_ref,i|, rms |u_ref|)."""
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    got = np.asarray(got, np.float64).reshape(len(got), -1)
    nr = np.sqrt((ref ** 2).sum(axis=1))
    rms = float(np.sqrt((nr ** 2).mean()))
    return np.sqrt(((got - ref) ** 2).sum(axis=1)) / np.maximum(nr, rms)


def rel_l2(ref, got):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    return float(np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum()))


def check_mixed(ref, got, what=""):
    """Asserts both mixed-precision bounds; returns (relative L2, worst target)."""
    e = rel_l2(ref, got)
    t = target_errors(ref, got)
    worst = float(t.max()) if len(t) else 0.0
    print("%s mixed rel_l2=%.3e worst_target=%.3e (target %d)"
          % (what, e, worst, int(t.argmax()) if len(t) else -1))
    assert np.all(np.isfinite(got)), what
    assert e <= MIXED_TOL, (what, e)
    assert worst <= MIXED_TARGET_TOL, (what, worst)
    return e, worst
