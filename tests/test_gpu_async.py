"""The asynchronous host transfers (rad_set_gas_host_async,
rad_set_rad_host_async, rad_read_host_async): three steps, each uploading a
different state from host arrays and reading the result back, enqueued
without waiting and synchronised once, give bit for bit what the
synchronous calls give step by step, in both precisions and with the gas
evolved."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26268_b300 import build
    build.build()


def _inputs(p, k, dtype, pinned):
    import torch
    nc = p.ncomp

    def host(a):
        a = np.ascontiguousarray(np.asarray(a, dtype=dtype).reshape(-1))
        if not pinned:
            return a
        t = torch.empty(a.size, dtype=torch.float64 if dtype == np.float64 else torch.float32,
                        pin_memory=True)
        t.numpy()[:] = a
        return t.numpy()

    return (host(p.rho), host(np.asarray(p.v)[:nc]), host(p.T * (1 + 0.01 * k)),
            host(p.E * (1 + 0.02 * k)), host(np.asarray(p.F)[:nc] * (1 - 0.01 * k)))


FIELDS = ("E", "F", "e", "m", "T", "rho")


@pytest.mark.parametrize("precision,hydro,pinned", [("split", False, True), ("fp64", False, False),
                                                    ("split", True, True)])
def test_async_host_transfers_equal_the_synchronous_calls(precision, hydro, pinned):
    import paper_2606_26268_b300 as R
    p = W.random_smooth("cartesian", (40, 24, 20), 3, seed=1900, bc="periodic", ncomp=3,
                        fmax=0.8)
    if hydro:
        p.hydro = True
        p.integrator = "rk2"
    dtype = np.float64 if precision == "fp64" else np.float32
    rs = R.from_problem(p, precision)
    dt = rs.dt()
    ref = []
    for k in range(3):
        rho, v, T, E, F = _inputs(p, k, dtype, False)
        rs.set_gas(rho, v, T)
        rs.set_rad(E, F)
        rs.step(1, dt)
        ref.append({f: np.asarray(rs.read(f)).reshape(-1).copy() for f in FIELDS})
    assert rs.sync() == 0
    rs.close()

    ra = R.from_problem(p, precision)
    keep, outs = [], []
    for k in range(3):
        ins = _inputs(p, k, dtype, pinned)
        keep.append(ins)
        ra.set_gas_async(*ins[:3])
        ra.set_rad_async(*ins[3:])
        ra.step(1, dt)
        o = {f: np.empty(p.N * (p.ncomp if f in ("F", "m") else 1), dtype=dtype) for f in FIELDS}
        for f in FIELDS:
            ra.read_async(f, o[f])
        outs.append(o)
    assert ra.sync() == 0
    ra.close()
    for k in range(3):
        for f in FIELDS:
            np.testing.assert_array_equal(outs[k][f], ref[k][f], err_msg="step %d %s" % (k, f))
    assert not np.array_equal(outs[0]["E"], outs[2]["E"])

