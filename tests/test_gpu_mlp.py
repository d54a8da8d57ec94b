"""The learned starting guess: training kernels against the FP64 reference
network, logged training records against the exact coupling root, and the
gain of the trained guess over starting the iteration from T^n."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26268_b300 import build
    build.build()
    return torch


def _ctx(precision="fp64", **kw):
    import paper_2606_26268_b300 as R
    p = W.turbulent_2d((64, 48), nonequilibrium=True)
    p.implicit_mode = "newton"
    return R.from_problem(p, precision, **kw), p


def _records(torch, n, seed):
    rng = np.random.default_rng(seed)
    rec = np.zeros((n, 4), dtype=np.float32)
    rec[:, :2] = rng.uniform(-2, 2, (n, 2))
    rec[:, 2] = rng.standard_normal(n)
    return rec, torch.tensor(rec, device="cuda")


def test_gradient_kernel_matches_fp64_backprop(torch_mod):
    r, _ = _ctx()
    theta = M.init(5).astype(np.float32)
    r.mlp_set(theta)
    rec, drec = _records(torch_mod, 3000, 1)
    loss, g = r.mlp_grad(drec)
    ref_loss, ref = M.loss_and_grad(theta.astype(np.float64), rec[:, :2].astype(np.float64),
                                    rec[:, 2].astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(g - ref)) <= 1e-4 * scale
    r.close()


def test_forward_and_adam_match_the_reference(torch_mod):
    r, _ = _ctx()
    theta = M.init(6).astype(np.float32)
    r.mlp_set(theta)
    rec, drec = _records(torch_mod, 2048, 2)
    out = r.mlp_predict(drec).cpu().numpy()
    ref, _ = M.forward(theta.astype(np.float64), rec[:, :2].astype(np.float64))
    assert np.max(np.abs(out - ref)) <= 5e-3 * max(1.0, np.max(np.abs(ref)))  # tanh.approx
    # the tensor-core path of the queue pass (bf16 hidden layers): 2048 records
    # is 16 full products; bf16 keeps about three significant digits
    tc = r.mlp_predict(drec, tensor_cores=True).cpu().numpy()
    assert r.sync() == 0
    assert np.max(np.abs(tc - ref)) <= 2e-2 * max(1.0, np.max(np.abs(ref)))
    assert np.corrcoef(tc, ref)[0, 1] > 0.999
    # one Adam step over one full batch
    r.mlp_train(drec, epochs=1, batch=2048, lr=1e-3, seed=3)
    new = r.mlp_get()
    _, g = M.loss_and_grad(theta.astype(np.float64), rec[:, :2].astype(np.float64),
                           rec[:, 2].astype(np.float64))
    want, _, _ = M.adam_step(theta.astype(np.float64), g, np.zeros(M.NPARAM),
                             np.zeros(M.NPARAM), 1, 1e-3)
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))  # sign(g) is unstable where g ~ 0
    np.testing.assert_allclose(new[big], want[big], atol=2e-6)
    r.close()


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_logged_records_are_exact_coupling_roots(torch_mod, precision):
    r, p = _ctx(precision)
    buf = torch_mod.zeros((20000, 4), dtype=torch_mod.float32, device="cuda")
    r.log_bind(buf, stride=1)
    r.step(3)
    n = r.log_count()
    assert n > 1000
    rec = buf[:n].cpu().numpy().astype(np.float64)
    alpha = 10 ** (4 * rec[:, 0])
    eps = 10 ** (4 * rec[:, 1])
    inside = (np.abs(rec[:, 0]) < 1.99) & (np.abs(rec[:, 1]) < 1.99)
    y = M.coupling_root(alpha[inside], eps[inside])
    err = np.abs(np.log(y) - rec[inside, 2])
    # features are float32 logs: the root is recovered to their precision
    assert np.median(err) < 2e-5 and np.max(err) < 5e-3, (np.median(err), np.max(err))
    r.close()


def test_trained_guess_saves_iterations_and_keeps_the_answer(torch_mod):
    """Train on solves logged from the 2D non-equilibrium turbulent box, then
    advance a fresh copy with and without the learned guess: same answer to
    the convergence tolerance, fewer Newton iterations on the queued cells."""
    import paper_2606_26268_b300 as R
    torch = torch_mod
    p = W.turbulent_2d((256, 256), nonequilibrium=True)
    p.implicit_mode = "newton"
    rt = R.from_problem(p, "fp64")
    buf = torch.zeros((400000, 4), dtype=torch.float32, device="cuda")
    rt.log_bind(buf, stride=1)
    rt.step(6)
    n = rt.log_count()
    loss = rt.mlp_train(buf[:n].contiguous(), epochs=8, batch=1024, lr=2e-3, seed=1)
    theta = rt.mlp_get()
    rt.close()
    assert loss < 1e-3, loss
    runs = {}
    for use in (0, 1):
        r = R.from_problem(p, "fp64", use_mlp=use, mlp_gate=1e-3)
        if use:
            r.mlp_set(theta)
        r.step(5)
        assert r.sync() == R.RAD_OK
        runs[use] = (r.read("E").copy(), r.read("T").copy(), r.stats())
        r.close()
    (E0, T0, s0), (E1, T1, s1) = runs[0], runs[1]
    np.testing.assert_allclose(E1, E0, rtol=1e-9)
    np.testing.assert_allclose(T1, T0, rtol=1e-9)
    assert s1["noconv"] == 0
    print("iterations without / with the learned guess:", s0["iters"], s1["iters"])
    assert s1["iters"] < s0["iters"]
