"""Failure paths on the GPU, made without a fault: a coupling iteration that
cannot converge in its iteration budget (RAD_ENOCONV, with the oracle's
counters), non-physical values handed to the setters (RAD_ENONPHYS), and a
bounded wait of the TMA-staged step kernel made to run out (RAD_ETIMEOUT),
after which the context keeps working."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import rounded, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26268_b300 import build
    build.build()
    import paper_2606_26268_b300 as R
    return R


def test_newton_iteration_budget_exhausted_reports_enoconv_with_the_oracles_counters(R):
    """One Newton iteration with rtol 1e-15 converges in no out-of-equilibrium
    cell (Sect. 2.8 iterated, reading 12): each cell restarts once from T^n
    and then gives up, so the fallback and non-convergence counts equal the
    number of cells whose first solve moves T, on both sides."""
    p = W.turbulent_2d((40, 32), nonequilibrium=True)
    p.implicit_mode = "newton"
    p.newton_maxit = 1
    p.newton_rtol = 1e-15
    r = R.from_problem(p, "fp64")
    dt = r.dt()
    r.step(1, dt)
    st = r.sync()
    stats = r.stats()
    r.close()
    assert st == R.RAD_ENOCONV
    o = oracle.Oracle(p)
    o.step(1, dt)
    names = oracle.STAT_NAMES
    want = {k: int(o.stats[names.index(k)]) for k in ("fallback", "noconv", "iters", "itmax")}
    assert want["noconv"] > 0.9 * p.N
    for k, v in want.items():
        assert stats[k] == v, (k, stats[k], v)


@pytest.mark.parametrize("field", ["E_nan", "E_neg", "F_inf", "rho_zero", "T_nan", "v_nan"])
@pytest.mark.parametrize("where", ["host", "device"])
def test_nonphysical_uploads_return_enonphys(R, field, where):
    import torch
    p = W.turbulent_2d((24, 20), nonequilibrium=True)
    r = R.from_problem(p, "fp64")
    rho, v, T, E, F = (np.array(p.rho), np.array(p.v[:2]), np.array(p.T), np.array(p.E),
                       np.array(p.F[:2]))
    k = 37
    if field == "E_nan":
        E[k] = np.nan
    elif field == "E_neg":
        E[k] = -1.0
    elif field == "F_inf":
        F[1, k] = np.inf
    elif field == "rho_zero":
        rho[k] = 0.0
    elif field == "T_nan":
        T[k] = np.nan
    else:
        v[0, k] = np.nan
    dev = (lambda a: torch.tensor(np.ascontiguousarray(a).ravel(), device="cuda")) \
        if where == "device" else (lambda a: a)
    with pytest.raises(R.RadError) as err:
        if field.split("_")[0] in ("E", "F"):
            r.set_rad(dev(E), dev(F))
        else:
            r.set_gas(dev(rho), dev(v), dev(T))
    assert err.value.status == R.RAD_ENONPHYS
    # the word is consumed: good values are accepted again and a step runs
    r.set_gas(p.rho, p.v[:2], p.T)
    r.set_rad(p.E, p.F[:2])
    r.step(1)
    assert r.sync() == R.RAD_OK
    r.close()


def test_nonphysical_asynchronous_upload_surfaces_at_sync(R):
    p = W.turbulent_2d((24, 20), nonequilibrium=True)
    r = R.from_problem(p, "fp64")
    E = np.array(p.E)
    E[5] = np.nan
    r.set_rad_async(E, np.array(p.F[:2]))
    assert r.sync() == R.RAD_ENONPHYS
    r.set_rad(p.E, p.F[:2])
    r.step(1)
    assert r.sync() == R.RAD_OK
    r.close()


@pytest.mark.parametrize("variant", [4, 7, 9])
def test_staged_plane_wait_that_runs_out_reports_etimeout_and_the_context_recovers(R, variant):
    """The TMA-staged kernels (launch variants 4-9 on split 3D Cartesian
    grids) stop a CTA whose wait for a plane runs out, after letting the
    copies in flight land.  With one non-blocking test per wait, the first
    wait (issued a moment before) cannot have completed, so every CTA stops:
    rad_sync returns RAD_ETIMEOUT.  With the default bound restored and the
    state set again, the same context steps to the same result as a fresh
    one."""
    p = rounded(W.hot_sphere_3d(ns=(72, 40, 36)), np.float32)
    r = R.from_problem(p, "split")
    dt = r.dt()
    r.set_launch(variant, 16)
    r.set_wait_limit(1)
    r.step(1, dt)
    assert r.sync() == R.RAD_ETIMEOUT
    r.set_wait_limit(0)
    r.set_gas(p.rho, p.v, p.T)
    r.set_rad(p.E, p.F)
    r.reset_stats()
    r.step(2, dt)
    assert r.sync() == R.RAD_OK
    got = {k: np.asarray(r.read(k), dtype=np.float64) for k in ("E", "F", "e")}
    r.close()
    f = R.from_problem(p, "split")
    f.set_launch(variant, 16)
    f.step(2, dt)
    assert f.sync() == R.RAD_OK
    for k in ("E", "F", "e"):
        np.testing.assert_array_equal(got[k], np.asarray(f.read(k), dtype=np.float64))
    f.close()
