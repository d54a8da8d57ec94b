"""FP64 reference of the small MLP that supplies the starting temperature of
the coupling iteration (test infrastructure only; never imported by the CUDA
library).

Network: x (2 features) -> 64 tanh -> 64 tanh -> 64 tanh -> 1 (linear).
Parameters are one flat vector in the order
    W1 (64 x 2, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (64 x 64),
    b3 (64), w4 (64), b4 (1)                                 -> 8577 values,
the same layout the library's rad_mlp_set / rad_mlp_get use.  Loss: mean
squared error of the output against the target.  Adam with the usual bias
correction (Kingma & Ba 2015, Algorithm 1).
"""
from __future__ import annotations

import numpy as np

H = 64
NIN = 2
SHAPES = [("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
          ("b3", (H,)), ("w4", (H,)), ("b4", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init(seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = shape[1] if len(shape) == 2 else shape[0]
            fan_out = shape[0] if len(shape) == 2 else 1
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            p[name] = rng.uniform(-lim, lim, shape)
    return pack(p)


def forward(theta: np.ndarray, X: np.ndarray):
    """X: (n, 2).  Returns the outputs (n,) and the activations."""
    p = unpack(theta)
    h1 = np.tanh(X @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    h3 = np.tanh(h2 @ p["W3"].T + p["b3"])
    out = h3 @ p["w4"] + p["b4"][0]
    return out, (X, h1, h2, h3)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray):
    """Mean squared error and its gradient by backpropagation."""
    p = unpack(theta)
    out, (X, h1, h2, h3) = forward(theta, X)
    n = X.shape[0]
    r = out - t
    loss = float(np.mean(r * r))
    dout = 2.0 * r / n
    g = {"w4": h3.T @ dout, "b4": np.array([dout.sum()])}
    d3 = np.outer(dout, p["w4"]) * (1.0 - h3 * h3)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ p["W3"]) * (1.0 - h2 * h2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def coupling_root(alpha: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """y = T^{n+1}/T^n of the converged coupling: the positive root of
    (y - 1) + alpha (y^4 - eps) = 0, the dimensionless form of
    C_v (T - T^n) + g/(1 + g_r) (a T^4 - E*) = 0 with
    alpha = g a T^n^3 / ((1 + g_r) C_v) and eps = E* / (a T^n^4).  Bisection
    in log y (brute force, independent of Newton's method)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    lo = np.minimum(1.0, eps ** 0.25) * 0.5
    hi = np.maximum(1.0, eps ** 0.25) * 2.0 + 1.0
    f = lambda y: (y - 1.0) + alpha * (y ** 4 - eps)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        neg = f(mid) < 0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    return 0.5 * (lo + hi)
