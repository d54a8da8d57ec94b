"""Shared helpers of the parity tests: run a problem on the GPU through the
C ABI and on the CPU oracle, and compare them with the per-cell error metric
(|dE|/|E|, |dF|/E, |de|/(|e| + 5e-5 n (c/chat) E), |dm|/(|m| + E/chat)).

The internal energy follows from the conservation of E_gas + (c/chat) E_r
(Sect. 2.7): each step changes it by the difference of (c/chat) E_r before
and after the coupling, which the definition (and so the oracle) forms by
subtracting two rounded radiation energies.  After n steps e therefore
carries up to about n units in the last place of (c/chat) E (2.2e-16 n
(c/chat) E) even when computed exactly as defined.  Where e is so small that
this floor exceeds the 1e-11 bound relative to e, the metric measures e
against 5e-5 n (c/chat) E instead: the FP64 bound then allows about two
units in the last place of (c/chat) E per step."""
import numpy as np

import oracle
import workloads as W


def rounded(p, dtype):
    """Copy of the problem with every field rounded to the storage dtype."""
    q = p.copy()
    for k in ("rho", "v", "T", "E", "F"):
        setattr(q, k, np.asarray(getattr(q, k)).astype(dtype).astype(np.float64))
    q.bc_value = {key: tuple(float(dtype(x)) for x in v)
                  for key, v in getattr(p, "bc_value", {}).items()}
    if getattr(p, "qirr", None) is not None:
        q.qirr = np.asarray(p.qirr).astype(dtype).astype(np.float64)
    return q


def run_gpu(p, nsteps, precision="fp64", dt=None, **overrides):
    import paper_2606_26268_b300 as R
    r = R.from_problem(p, precision=precision, **overrides)
    if dt is None:
        dt = r.dt()
        # the library's CFL step must be the oracle's (Sect. 2.4, item 10),
        # so that parity runs that hand the GPU's dt to the oracle do not
        # share a mistake in it; the split form takes the gas CFL reduction
        # in FP32
        want = oracle.Oracle(p).dt()
        tol = 1e-13 if precision == "fp64" else 1e-6
        assert abs(dt - want) <= tol * want, (dt, want)
    r.step(nsteps, dt)
    st = r.sync()
    out = {k: np.asarray(r.read(k), dtype=np.float64) for k in ("E", "F", "e", "m", "T", "rho")}
    out["stats"] = r.stats()
    out["status"] = st
    out["dt"] = dt
    r.close()
    return out


def run_oracle(p, nsteps, dt=None, nthreads=0):
    o = oracle.Oracle(p, nthreads=nthreads)
    if dt is None:
        dt = o.dt()
    o.step(nsteps, dt)
    return {"E": o.E, "F": o.F, "e": o.e, "m": o.m, "T": o.temperature(), "rho": o.rho,
            "stats": o.stats, "dt": dt}


def errors(g, o, ncomp, chat, ratio=1.0, nsteps=1):
    E = o["E"]
    escale = np.abs(o["e"]) + 5e-5 * nsteps * ratio * np.abs(E)
    out = {"E": np.max(np.abs(g["E"] - E) / np.abs(E)),
           "e": np.max(np.abs(g["e"] - o["e"]) / escale)}
    out["F"] = max(np.max(np.abs(g["F"][q] - o["F"][q]) / E) for q in range(ncomp))
    scale = np.sqrt(np.sum(o["m"] ** 2, axis=0)) + E / chat
    out["m"] = max(np.max(np.abs(g["m"][q] - o["m"][q]) / scale) for q in range(ncomp))
    return out


def _stencil_scale(ref, shape):
    """Largest |value| in each cell's 5-cell stencil, for one or more fields
    of the grid `shape` (n0, n1, n2), x fastest, stored one after the other."""
    from scipy.ndimage import maximum_filter
    grid = tuple(int(k) for k in shape)[::-1]
    a = np.abs(np.asarray(ref, dtype=np.float64)).reshape((-1,) + grid)
    return np.stack([maximum_filter(f, size=5, mode="nearest") for f in a]).ravel()


def _agreement(out, ref, shape):
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    norm = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    cell = np.max(np.abs(out - ref) / _stencil_scale(ref, shape))
    return norm, cell


def oracle_spread(p, nsteps, dt, seeds=(0, 1)):
    """The problem's own response to rounding: the largest change of the FP64
    oracle's E after `nsteps` steps when its E and F inputs are perturbed by
    6e-8 relative (half a unit in the last place of FP32), normwise and per
    cell against the stencil's largest E, over the given seeds."""
    o = oracle.Oracle(p)
    o.step(nsteps, dt)
    E0 = o.E.copy()
    norm = cell = 0.0
    for k in seeds:
        q = p.copy()
        rng = np.random.default_rng(k)
        q.E = p.E * (1.0 + 6e-8 * rng.standard_normal(p.N))
        q.F = p.F * (1.0 + 6e-8 * rng.standard_normal(np.shape(p.F)))
        o2 = oracle.Oracle(q)
        o2.step(nsteps, dt)
        n, c = _agreement(o2.E, E0, p.n)
        norm, cell = max(norm, n), max(cell, c)
    return norm, cell


def assert_shapes_agree(out, ref, variant, shape, spread=(0.0, 0.0)):
    """Two launch shapes of the split form after a few steps.  The kernels
    sum the flux divergence in different orders (the TMA-staged one on packed
    FP32 pairs), so they agree to FP32 rounding, amplified in a few cells by
    the discontinuous f-fix and limiter switches: normwise within 3e-7, and
    per cell within 1e-5 of the largest value in the cell's 5-cell stencil,
    or within the problem's own response to rounding (`spread`, normwise and
    per cell, from oracle_spread) where that is larger.  The FP32 rounding of
    a flux divergence scales with the largest flux it sums, hence with the
    stencil's largest E, not with the cell's own: where E varies by 10^3
    between neighbours the cell's relative rounding is 10^3 times FP32's.
    `out` and `ref` hold one or more fields of the grid `shape` (n0, n1, n2),
    x fastest, one after the other."""
    ncell = int(np.prod(shape))
    assert np.size(out) % ncell == 0
    norm, cell = _agreement(out, ref, shape)
    assert norm <= max(3e-7, spread[0]) and cell <= max(1e-5, spread[1]), \
        (variant, norm, cell, spread)
