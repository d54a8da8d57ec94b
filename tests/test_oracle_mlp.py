"""Pins of the FP64 reference network used to check the training kernels,
and of the dimensionless form of the coupling the network learns.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import mlp as M


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = M.init(1) + 0.05 * rng.standard_normal(M.NPARAM)
    X = rng.uniform(-2, 2, (17, 2))
    t = rng.standard_normal(17)
    loss, g = M.loss_and_grad(theta, X, t)
    idx = rng.choice(M.NPARAM, 300, replace=False)
    idx = np.r_[idx, [0, 1, 127, 128, 191, 192, M.NPARAM - 65, M.NPARAM - 1]]
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (M.loss_and_grad(tp, X, t)[0] - M.loss_and_grad(tm, X, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_zero_weights_give_the_output_bias_and_layout_is_complete():
    assert M.NPARAM == 8577
    theta = np.zeros(M.NPARAM)
    theta[-1] = 0.37
    out, _ = M.forward(theta, np.random.default_rng(1).uniform(-1, 1, (5, 2)))
    np.testing.assert_allclose(out, 0.37)
    # a single path: x1 -> unit 0 of every layer -> output
    p = M.unpack(np.zeros(M.NPARAM))
    p["W1"][0, 0] = 0.5
    p["W2"][0, 0] = 2.0
    p["W3"][0, 0] = -1.5
    p["w4"][0] = 3.0
    x = np.array([[0.8, 0.3]])
    out, _ = M.forward(M.pack(p), x)
    assert out[0] == pytest.approx(3.0 * np.tanh(-1.5 * np.tanh(2.0 * np.tanh(0.4))))


def test_first_adam_step_is_lr_times_sign():
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = M.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    # bias correction makes the first step exactly -lr g / (|g| + eps)
    np.testing.assert_allclose(new - theta, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_dimensionless_root_is_the_coupling_solution():
    """y = T^{n+1}/T^n from (alpha, eps) equals the oracle's converged Newton
    coupling (Sect. 2.8 iterated) for random cells."""
    import workloads as W
    p = W.uniform_state("cartesian", (4, 1, 1), 1)
    p.implicit_mode = "newton"
    p.chat, p.c = 1.0, 3.0
    o = oracle.Oracle(p)
    rng = np.random.default_rng(3)
    n = 200
    rho = 10 ** rng.uniform(-1, 1, n)
    Tn = 10 ** rng.uniform(-0.5, 0.5, n)
    kp = 10 ** rng.uniform(-2, 2, n)
    Es = Tn ** 4 * 10 ** rng.uniform(-2, 2, n)
    dt = 0.01
    E, T, _, _ = o.couple_cells(dt, rho, Tn, kp, Es)
    Cv = o.heat_capacity(rho)
    g = dt * p.c * kp * rho
    gr = dt * p.chat * kp * rho
    alpha = g * Tn ** 3 / ((1 + gr) * Cv)
    eps = Es / Tn ** 4
    y = M.coupling_root(alpha, eps)
    np.testing.assert_allclose(y * Tn, T, rtol=1e-12)
