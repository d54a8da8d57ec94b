"""The benchmark's headline form checked against the oracle directly: FP32
transport, the coupling of Sect. 2.8 iterated by Newton with rtol 1e-7 from
the learned guess (trained by the benchmark's own routine on logged solves
of the 2D non-equilibrium box, gate 1e-2, evaluated on the tensor cores in
the queue pass), the TMA-staged non-overlapping step kernel (launch variants
9, 7 and 6: 16 x 16 and 32 x 8 tiles, marches of 19, 16 and 8 cells), on a
hot-sphere box that spans several full tiles and a ragged tail in x and y
and several march chunks in z."""
import argparse

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import rounded

pytestmark = pytest.mark.gpu

NSTEPS = 100


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26268_b300 import build
    build.build()
    import paper_2606_26268_b300 as R
    import bench
    args = argparse.Namespace(train_n=512, train_steps=4, train_epochs=4, precision="split")
    theta, info = bench.train_guess(R, torch, torch.device("cuda", 0), args)
    assert info["records"] > 0
    p = W.hot_sphere_3d(ns=(72, 40, 36), nsteps=NSTEPS)
    q = rounded(p, np.float32)
    q.implicit_mode = "newton"
    q.newton_rtol = 1e-7
    dt = oracle.Oracle(q).dt()
    # the FP64 oracle, iterated to convergence, and its spread under 1e-7
    # perturbations of the inputs (the box amplifies them)
    ref = q.copy()
    ref.newton_rtol = 1e-12
    o = oracle.Oracle(ref)
    o1 = oracle.Oracle(ref)
    o1.step(1, dt)
    o.step(NSTEPS, dt)
    q2 = ref.copy()
    rng = np.random.default_rng(0)
    for k in ("E", "rho", "T"):
        a = getattr(q2, k)
        setattr(q2, k, a * (1 + 1e-7 * rng.standard_normal(a.shape)))
    o2 = oracle.Oracle(q2)
    o2.step(NSTEPS, dt)
    return dict(R=R, theta=theta, q=q, dt=dt, o=o, o1=o1, o2=o2)


def _run(s, launch, nsteps, guess=True):
    R = s["R"]
    extra = dict(use_mlp=1, mlp_gate=1e-2) if guess else {}
    r = R.from_problem(s["q"], "split", implicit_mode="newton", **extra)
    if guess:
        r.mlp_set(s["theta"])
    r.set_launch(*launch)
    r.step(nsteps, s["dt"])
    st = r.sync()
    out = {k: np.asarray(r.read(k), dtype=np.float64) for k in ("E", "F", "e")}
    out["stats"] = r.stats()
    r.close()
    assert st == R.RAD_OK
    return out


@pytest.mark.parametrize("launch", [(9, 19), (9, 16), (7, 16), (6, 8)])
def test_headline_form_one_step_matches_the_oracle_cell_by_cell(setup, launch):
    """One step: every cell within FP32 rounding of the converged FP64
    coupling (per-cell relative error of E and e below 1e-5; F against E),
    with and without the learned guess, and the two runs within a few units
    in the last place of each other (both iterate to the same root)."""
    s = setup
    o1 = s["o1"]
    g = _run(s, launch, 1)
    h = _run(s, launch, 1, guess=False)
    assert g["stats"]["iters"] > 0
    for out in (g, h):
        assert np.max(np.abs(out["E"] - o1.E) / o1.E) <= 1e-5
        assert np.max(np.abs(out["e"] - o1.e) / o1.e) <= 1e-5
        assert np.max(np.abs(out["F"] - o1.F) / o1.E) <= 1e-5
    assert np.max(np.abs(g["E"] - h["E"]) / h["E"]) <= 1e-6
    assert np.max(np.abs(g["e"] - h["e"]) / h["e"]) <= 1e-6


@pytest.mark.parametrize("launch", [(9, 19), (9, 16), (7, 16), (6, 8)])
def test_headline_form_100_steps_within_the_problems_own_sensitivity(setup, launch):
    """100 steps: normwise and per-cell errors against the FP64 oracle within
    20x the oracle's own response to 1e-7 input perturbations of E, rho and
    T, with and without the learned guess."""
    s = setup
    o, o2 = s["o"], s["o2"]
    sens = np.linalg.norm(o2.E - o.E) / np.linalg.norm(o.E)
    sens_cell = np.max(np.abs(o2.E - o.E) / o.E)
    for guess in (True, False):
        g = _run(s, launch, NSTEPS, guess=guess)
        norm_E = np.linalg.norm(g["E"] - o.E) / np.linalg.norm(o.E)
        norm_e = np.linalg.norm(g["e"] - o.e) / np.linalg.norm(o.e)
        cell_E = np.max(np.abs(g["E"] - o.E) / o.E)
        assert norm_E <= max(20 * sens, 1e-5), (guess, norm_E, sens)
        assert norm_e <= max(20 * sens, 1e-5), (guess, norm_e, sens)
        assert cell_E <= max(20 * sens_cell, 1e-5), (guess, cell_E, sens_cell)
