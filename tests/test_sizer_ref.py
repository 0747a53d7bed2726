"""Pins of the sizer's CPU reference (no GPU)."""
import numpy as np

from oracle import sizer_ref as R
from paper_2210_16998_gb300 import cfggen as G

from .test_oracle import fig1_cfg


def test_gradient_matches_central_differences():
    cfgs = [G.config1_cfg(), G.diamond_chain(2), G.random_cfg(G.TRAIN_SEED0 + 1)]
    X, A = R.batch_inputs(cfgs)
    rng = np.random.default_rng(7)
    p = rng.normal(0.0, 0.2, R.NPARAM)
    T = rng.normal(1.0, 1.0, (X.shape[0], 3))
    loss, g = R.loss_grad(p, X, A, T)
    idx = np.concatenate([rng.choice(R.NPARAM, 48, replace=False),
                          [R.OFF_B0 + 3, R.OFF_WO + 5, R.OFF_BO + 1, R.OFF_WL + R.H * R.K + 2]])
    eps = 1e-6
    for i in idx:
        pp = p.copy()
        pp[i] += eps
        pm = p.copy()
        pm[i] -= eps
        fd = (R.loss_grad(pp, X, A, T)[0] - R.loss_grad(pm, X, A, T)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-4 * max(abs(fd), 1e-3), (i, fd, g[i])


def test_features_of_the_worked_example():
    cfg, _ = fig1_cfg()
    x = R.features(cfg)
    n = 11
    # vertex 2: in {1, 8}, out {3, 9}; SCC {2,3,4,5,6,8}; 0->1->2; 2->9->10
    np.testing.assert_allclose(x[2], [np.log1p(2), np.log1p(2), 0, 0, np.log1p(6), 2 / n, 2 / n, np.log(n) / 5])
    # the entry: no predecessors, one successor, its own SCC, 0->1->2->9->10
    np.testing.assert_allclose(x[0], [0, np.log1p(1), 1, 0, np.log1p(1), 0, 4 / n, np.log(n) / 5])
    # the exit: cannot be left
    assert x[10][3] == 1 and x[10][6] == 0 and x[10][1] == 0


def test_bf16_rounding_is_round_to_nearest_even():
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 3.0e-39], np.float32)
    got = R.bf16(vals)
    np.testing.assert_array_equal(got[:4], [1.0, 1.0, 1 + 2 ** -6, -2.5])
    assert abs(got[4] - 3.0e-39) < 1e-40


def test_bf16_reference_stays_close_to_fp64():
    cfgs = [G.random_cfg(G.TRAIN_SEED0 + i) for i in range(4)]
    X, A = R.batch_inputs(cfgs)
    rng = np.random.default_rng(3)
    p = rng.normal(0.0, 0.1, R.NPARAM)
    T = rng.normal(2.0, 1.0, (X.shape[0], 3))
    l64, g64 = R.loss_grad(p, X, A, T)
    l16, g16 = R.loss_grad(p, X, A, T, bf=True)
    assert abs(l16 - l64) / l64 < 0.02
    assert np.linalg.norm(g16 - g64) / np.linalg.norm(g64) < 0.05
