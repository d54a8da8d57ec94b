"""Seeded random combinations of geometry, dimension, sizes, boundary kinds,
face options, coupling mode, integrator, opacity model, irradiation and
evolved gas, each stepped on the GPU in FP64 and compared per cell with the
oracle (within 1e-11).  The clipping face treatment is left out: it makes
f = 1 face states, where the signal speeds depend on rounding (its own test
bounds it by the oracle's spread)."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import errors, run_gpu, run_oracle
from test_gpu_options import with_bcs
from test_gpu_parity import _opacity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26268_b300 import build
    build.build()


def random_case(seed):
    rng = np.random.default_rng(7000 + seed)
    geom = ["cartesian", "cylindrical", "spherical"][rng.integers(3)]
    ndim = int(rng.integers(1, 4))
    n = tuple(int(rng.integers(6, 30 if ndim == 3 else 60)) for _ in range(3))
    nc = int(rng.integers(ndim, 4)) if geom == "cartesian" else 3
    kind = [None, "powerlaw", "table"][rng.integers(3)]
    p = W.random_smooth(geom, n, ndim, seed=8000 + seed, bc="outflow", opacity=_opacity(kind),
                        log_r=bool(geom == "spherical" and rng.integers(2)), ncomp=nc, fmax=0.8)
    kinds = ["outflow", "reflective", "fixed", "lte", "periodic"]
    lo, hi = [], []
    for d in range(ndim):
        a = kinds[rng.integers(len(kinds))]
        b = "periodic" if a == "periodic" else kinds[rng.integers(4)]
        if geom != "cartesian" and d == 0:  # keep the radial sides simple
            a, b = "outflow", "outflow"
        lo.append(a)
        hi.append(b)
    p = with_bcs(p, lo, hi, seed=seed)
    p.recon = ["plm", "limo3"][rng.integers(2)]
    p.face_fix = ["fpreserve", "pluto"][rng.integers(2)]
    p.riemann = ["hll", "lf"][rng.integers(2)]
    p.implicit_mode = ["once", "newton", "absorb"][rng.integers(3)]
    p.integrator = ["euler", "rk2"][rng.integers(2)]
    if rng.integers(2):
        p.qirr = rng.uniform(-0.1, 0.3, p.N) * p.rho * p.T
    p.hydro = bool(geom == "cartesian" and rng.integers(2))
    return p


@pytest.mark.parametrize("seed", range(64))
def test_random_configuration_fp64_matches_oracle(seed):
    p = random_case(seed)
    dt = oracle.Oracle(p).dt()
    g = run_gpu(p, 3, "fp64", dt=dt)
    o = run_oracle(p, 3, dt=dt)
    assert g["status"] == 0, (seed, g["status"])
    err = errors(g, o, p.ncomp, p.chat, p.c / p.chat, 3)
    if p.hydro:
        err["rho"] = np.max(np.abs(g["rho"] - o["rho"]) / o["rho"])
        pgas = (p.gamma_gas - 1.0) * o["e"]
        scale = (np.sqrt(np.sum(o["m"] ** 2, axis=0)) + o["E"] / p.chat +
                 np.sqrt(p.gamma_gas * o["rho"] * pgas))
        err["m"] = max(np.max(np.abs(g["m"][q] - o["m"][q]) / scale) for q in range(p.ncomp))
    desc = (p.geometry, p.ndim, p.n, p.bc_lo[:p.ndim], p.bc_hi[:p.ndim], p.recon, p.face_fix,
            p.riemann, p.implicit_mode, p.integrator, p.qirr is not None, p.hydro)
    for k, v in err.items():
        assert v <= 1e-11, (desc, k, v)


@pytest.mark.parametrize("seed", range(32))
def test_random_configuration_split_within_its_sensitivity(seed):
    """The split form on the same random combinations (float-rounded inputs),
    on a random launch shape, normwise within max(1e-5, 20x the oracle's own
    change under input perturbations of FP32 size)."""
    import paper_2606_26268_b300 as R
    from helpers import rounded
    p = rounded(random_case(seed), np.float32)
    dt = oracle.Oracle(p).dt()
    r = R.from_problem(p, "split")
    nvar = r.get_launch()[2]
    r.set_launch(int(np.random.default_rng(seed).integers(nvar)), 0)
    r.step(3, dt)
    assert r.sync() == 0, seed
    g = {k: np.asarray(r.read(k), dtype=np.float64) for k in ("E", "e")}
    r.close()
    o = run_oracle(p, 3, dt=dt)
    q = p.copy()
    q.E = p.E * (1 + 1e-7 * np.random.default_rng(seed + 1).standard_normal(p.N))
    o2 = run_oracle(q, 3, dt=dt)
    for k in ("E", "e"):
        err = np.linalg.norm(g[k] - o[k]) / np.linalg.norm(o[k])
        sens = np.linalg.norm(o2[k] - o[k]) / np.linalg.norm(o[k])
        assert err <= max(1e-5, 20 * sens), (seed, k, err, sens)
