"""rad_mlp_grad_noalloc: the training-loss gradient for callers that cannot
allocate device memory (frameworks that own every byte of device memory
through a pre-sized pool, or code that must not let an allocation synchronise
the device).  It must agree with rad_mlp_grad, which keeps its accumulators in
a context's workspace, and the FP64 backpropagation of the oracle, on two
calls in a row, and refuse sets larger than its fixed scratch.  This file is
collected last on purpose."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as M

pytestmark = pytest.mark.gpu


def test_noalloc_gradient_matches_the_workspace_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26268_b300 import build
    build.build()
    import paper_2606_26268_b300 as R

    p = W.turbulent_2d((32, 24), nonequilibrium=True)
    p.implicit_mode = "newton"
    ctx = R.from_problem(p, "fp64")
    theta = (M.init(11) + 0.02 * np.random.default_rng(4).standard_normal(M.NPARAM)).astype(np.float32)
    ctx.mlp_set(theta)
    d_params = torch.tensor(theta, device="cuda")
    grad = torch.empty(M.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(5)
    # two calls in a row; the second uses fewer records than the first, so
    # partial gradients left in the shared scratch by the first must not leak
    for n in (R.NOALLOC_MAX_RECORDS - 37, 1000):
        rec = np.zeros((n, 4), dtype=np.float32)
        rec[:, :2] = rng.uniform(-2, 2, (n, 2))
        rec[:, 2] = rng.standard_normal(n)
        d_rec = torch.tensor(rec, device="cuda")
        ref_loss, ref_grad = ctx.mlp_grad(d_rec)
        assert R.mlp_grad_noalloc(d_params, d_rec, grad, loss) == R.RAD_OK
        torch.cuda.synchronize()
        g = grad.cpu().numpy()
        scale = np.max(np.abs(ref_grad))
        assert np.max(np.abs(g - ref_grad)) <= 1e-4 * scale
        assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)
        # and the FP64 backpropagation of the oracle on the same records
        o_loss, o_grad = M.loss_and_grad(theta.astype(np.float64), rec[:, :2].astype(np.float64),
                                         rec[:, 2].astype(np.float64))
        assert np.max(np.abs(g - o_grad)) <= 1e-4 * np.max(np.abs(o_grad))
        assert float(loss.item()) == pytest.approx(o_loss, rel=1e-4)
    # beyond the scratch: a clear error, nothing launched
    big = torch.zeros((R.NOALLOC_MAX_RECORDS + 1, 4), dtype=torch.float32, device="cuda")
    assert R.mlp_grad_noalloc(d_params, big, grad, loss) == R.RAD_EINVAL
    ctx.close()
