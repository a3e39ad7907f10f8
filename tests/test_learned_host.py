"""Host-side logic of the learned degree selector (no GPU): the labelling rule
and the initial parameters."""
import math

import numpy as np
import torch

from paper_1902_02250_gb300 import learned as LD


def test_label_rule():
    # 4 clusters x 6 classes of measured squared errors and sample counts
    rms = np.array([[1e-2, 1e-4, 1e-7, 1e-9],    # class 0 (degree 6)
                    [1e-3, 1e-5, 1e-8, 1e-9],    # 1 (7)
                    [1e-4, 1e-6, 1e-9, 1e-9],    # 2 (8)
                    [1e-5, 5e-8, 1e-9, 1e-9],    # 3 (9)
                    [1e-6, 1e-8, 1e-9, 1e-9],    # 4 (10)
                    [1e-6, 1e-9, 1e-9, 1e-9]])   # 5 (11)
    ns = np.array([[4, 9, 1, 0]] * 6, np.int32)
    meas = {"err2": torch.from_numpy(rms ** 2 * ns), "n_samples": torch.from_numpy(ns),
            "m_far": 100.0, "u_rms": 2.0}
    lab, valid, tau = LD.labels(meas, 5e-7)
    assert math.isclose(tau, 5e-7 * 2.0 / 10.0)            # budget * u_rms / sqrt(m_far)
    assert valid.tolist() == [True, True, True, False]      # no sample: no label
    # cluster 0 never reaches tau = 1e-7: the largest class; cluster 1 reaches it at
    # class 3; cluster 2 already at the smallest class
    assert lab[:3].tolist() == [5, 3, 0]


def test_initial_parameters():
    mu, sd = np.arange(12.0), np.full(12, 2.0)
    p = LD.init_params(3, mu, sd)
    assert p.dtype == np.float32 and p.size == 2 * 12 + 64 * 12 + 64 + 64 * 64 + 64 + 6 * 64 + 6
    assert np.array_equal(p[:12], mu.astype(np.float32)) and np.array_equal(p[12:24], sd)
    assert np.array_equal(p, LD.init_params(3, mu, sd))
    assert LD.CLASSES == (6, 7, 8, 9, 10, 11)
