"""The split form takes the opacities of Sect. 2.8 from (rho, e) rather than
from T = e / (rho C_v/rho): log2 T = log2 e - log2 rho - log2 (C_v/rho), so
the power law k0 rho^a T^b is k0 2^((a - b) log2 rho + b log2 e - b log2
(C_v/rho)) and the table's log10 T axis is read at (log2 e - log2 rho -
log2 (C_v/rho)) log10 2.  A float32 host emulation of that reading agrees
with the oracle's kappa(rho, T) over decades of rho and T to float rounding
of the exponent, and the same emulation with the log2 (C_v/rho) term
dropped (a planted mistake) does not.  CPU only."""
import math

import numpy as np

import oracle
import workloads as W

F = np.float32
LOG10_2 = F(0.30102999566398120)
LOG2_10 = F(3.32192809488736235)


def _samples(n=400, seed=17):
    rng = np.random.default_rng(seed)
    rho = (10.0 ** rng.uniform(-3.0, 2.0, n)).astype(F)
    T = 10.0 ** rng.uniform(-0.5, 1.2, n)
    return rho, T


def _emulate(op, rho, e, cvfac, drop_cv=False):
    """kappa_P from (rho, e) in float32, as the split form forms it."""
    lr = np.log2(rho.astype(F))
    le = np.log2(e.astype(F))
    lcv = F(0.0) if drop_cv else F(math.log2(cvfac))
    if op["kind"] == "powerlaw":
        amb = F(op["a_rho"] - op["b_T"])
        b = F(op["b_T"])
        blcv = F(0.0) if drop_cv else F(op["b_T"] * math.log2(cvfac))
        k = F(op["k0"]) * np.exp2(amb * lr + (b * le - blcv))
        return np.clip(k, F(op["kmin"]), F(op["kmax"]))
    nr, nt = op["nrho"], op["nT"]
    sr = F((nr - 1) / (op["lrho1"] - op["lrho0"]))
    sT = F((nt - 1) / (op["lT1"] - op["lT0"]))
    xr = (lr * LOG10_2 - F(op["lrho0"])) * sr
    xt = ((le - lr - lcv) * LOG10_2 - F(op["lT0"])) * sT
    xr = np.clip(xr, F(0), F(nr - 1))
    xt = np.clip(xt, F(0), F(nt - 1))
    ir = np.minimum(xr.astype(np.int64), nr - 2)
    it = np.minimum(xt.astype(np.int64), nt - 2)
    wr, wt = xr - ir.astype(F), xt - it.astype(F)
    t = np.asarray(op["table"], dtype=F).reshape(nt, nr)
    lk = ((F(1) - wr) * ((F(1) - wt) * t[it, ir] + wt * t[it + 1, ir])
          + wr * ((F(1) - wt) * t[it, ir + 1] + wt * t[it + 1, ir + 1]))
    return np.exp2(lk * LOG2_10)


def _oracle_kappa(op, rho, T):
    p = W.uniform_state("cartesian", (2, 1, 1), 1)
    p.opacity = op
    o = oracle.Oracle(p)
    cvfac = 1.0 / (p.mu * (p.gamma_gas - 1.0))
    return np.array([o.opacity(float(r), float(t))[0] for r, t in zip(rho, T)]), cvfac


def _check(op, tol):
    rho, T = _samples()
    p = W.uniform_state("cartesian", (2, 1, 1), 1)
    cvfac = 1.0 / (p.mu * (p.gamma_gas - 1.0))
    # e as the split form stores it (float, rho C_v/rho T), and the T the
    # oracle takes from it
    e = (rho.astype(np.float64) * cvfac * T).astype(F)
    Tq = e.astype(np.float64) / (rho.astype(np.float64) * cvfac)
    ref, _ = _oracle_kappa(op, rho, Tq)
    got = _emulate(op, rho, e, cvfac).astype(np.float64)
    rel = np.max(np.abs(got - ref) / ref)
    assert rel <= tol, rel
    bad = _emulate(op, rho, e, cvfac, drop_cv=True).astype(np.float64)
    assert np.max(np.abs(bad - ref) / ref) > 100 * tol


def test_power_laws_from_the_gas_energy():
    for op in ({"kind": "powerlaw", "k0": 2.0, "a_rho": 1.0, "b_T": -3.5, "kmin": 1e-3,
                "kmax": 1e3},
               {"kind": "powerlaw", "k0": 2.0, "a_rho": 0.5, "b_T": -2.0, "kmin": 1e-4,
                "kmax": 1e4}):
        # the exponent's terms reach |b log2 e| ~ 20; their float rounding
        # (about 1e-6 absolute each) moves kappa by a few 1e-6 relative
        # (4.5e-6 at most on these samples)
        _check(op, 2e-5)


def test_table_from_the_gas_energy():
    op = W.opacity_table(24, 20, seed=3)
    op.update(lrho0=-3.0, lrho1=2.0, lT0=-1.0, lT1=1.5)
    # float32 interpolation weights and the 2^(lk log2 10) of a log10 kappa
    # of order 10: a few 1e-6 (2.3e-6 at most on these samples)
    _check(op, 2e-5)
