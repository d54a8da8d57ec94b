"""Pins of the oracle's two-stage integration (RK2 / IMEX1, Sect. 2.4): the
transport + coupling split applied in each stage of the two-stage scheme,
U1 = S(U^n), U2 = S(U1), U^{n+1} = (U^n + U2) / 2 for the conserved
variables.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_step import volumes


def free_streaming_wave(n, integrator):
    """Periodic 1D wave E = 1 + 0.4 sin(2 pi x) with F = E (f = 1): every
    state moves at +chat without change of shape, so E(x, t) = E(x - chat t, 0)."""
    xf = W.uniform_faces(n, 0.0, 1.0)
    one = W.uniform_faces(1, 0.0, 1.0)
    p = W.Problem(name="wave", ndim=1, n=(n, 1, 1), geometry="cartesian",
                  bc_lo=("periodic",) * 3, bc_hi=("periodic",) * 3, xfaces=[xf, one, one],
                  chat=1.0, c=1.0, ncomp=1, integrator=integrator)
    x = W.cell_centres(xf)
    # cell averages of the exact profile
    p.E = 1.0 + 0.4 * (np.cos(2 * math.pi * xf[:-1]) - np.cos(2 * math.pi * xf[1:])) / (
        2 * math.pi * np.diff(xf))
    p.F = np.zeros((3, n))
    p.F[0] = p.E
    p.rho, p.T, p.v = np.ones(n), np.full(n, 1e-3), np.zeros((3, n))
    return p, xf


def wave_error(n, integrator, t_end=0.25):
    p, xf = free_streaming_wave(n, integrator)
    o = oracle.Oracle(p)
    dt = 0.4 / n  # CFL 0.4 at chat = 1
    steps = int(round(t_end / dt))
    o.step(steps, dt)
    t = steps * dt
    exact = 1.0 + 0.4 * (np.cos(2 * math.pi * (xf[:-1] - t)) - np.cos(2 * math.pi * (xf[1:] - t))) / (
        2 * math.pi * np.diff(xf))
    return np.mean(np.abs(o.E - exact))


def test_two_stage_scheme_is_second_order_in_time_on_a_smooth_wave():
    """At fixed CFL the Euler step is first order (its time error dominates),
    the two-stage step second order except where the limiter flattens the
    extrema."""
    ns = [32, 64, 128, 256]
    eu = [wave_error(n, "euler") for n in ns]
    rk = [wave_error(n, "rk2") for n in ns]
    s_eu = -np.polyfit(np.log(ns), np.log(eu), 1)[0]
    s_rk = -np.polyfit(np.log(ns), np.log(rk), 1)[0]
    assert s_eu < 1.3, (s_eu, eu)
    assert s_rk > 1.6, (s_rk, rk)
    assert rk[-1] < 0.2 * eu[-1]


def test_two_stage_conserves_total_energy_and_momentum_with_coupling():
    """Both stages conserve E_gas + (c/chat) E_r and m + F/chat (Sect. 2.7),
    and so does their average, the average being taken of E_gas, not of e."""
    p = W.random_smooth("cartesian", (12, 10, 1), 2, seed=21, bc="periodic", fmax=0.3,
                        chat=2.0, c=20.0,
                        opacity={"kind": "const", "kappa_p": 3.0, "kappa_r": 2.0, "sigma": 1.0})
    p.integrator = "rk2"
    o = oracle.Oracle(p)
    V = volumes(p)
    ratio = p.c / p.chat

    def totals():
        ke = np.sum(o.m * o.m, axis=0) / (2 * o.rho)
        return (np.sum(V * (o.e + ke)) + ratio * np.sum(V * o.E),
                (V * (o.m + o.F / p.chat)).sum(axis=1))

    t0, m0 = totals()
    o.step(4)
    t1, m1 = totals()
    assert o.stats[1] == 0 and o.stats[2] == 0
    assert abs(t1 - t0) / t0 < 1e-13
    np.testing.assert_allclose(m1, m0, atol=1e-13 * np.abs(m0).max() + 1e-15)


@pytest.mark.parametrize("geom,ndim,logr", [("cartesian", 3, False), ("cylindrical", 2, False),
                                            ("spherical", 3, True)])
def test_uniform_state_stays_uniform_with_two_stages(geom, ndim, logr):
    p = W.uniform_state(geom, (10, 8, 6), ndim, log_r=logr)
    p.integrator = "rk2"
    o = oracle.Oracle(p)
    e0 = o.e.copy()
    o.step(2)
    assert np.max(np.abs(o.E - 2.0)) / 2.0 < 1e-13
    assert np.max(np.abs(o.F)) / 2.0 < 1e-13
    assert np.max(np.abs(o.e - e0) / e0) < 1e-13


def test_uniform_relaxation_is_the_average_of_two_couplings():
    """Without transport a stage is the coupling of Sect. 2.8, so the step is
    (U^n + C(C(U^n))) / 2 with C the single-cell coupling."""
    p = W.uniform_state("cartesian", (5, 4, 1), 2, E=3.0, kappa=2.0)
    p.T = np.full(p.N, 0.7)
    p.integrator = "rk2"
    o = oracle.Oracle(p)
    dt = o.dt()
    rho, T0, E0 = o.rho[:1].copy(), o.temperature()[:1].copy(), o.E[:1].copy()
    cv = o.heat_capacity(rho)
    E1, T1, _, _ = o.couple_cells(dt, rho, T0, np.array([2.0]), E0)
    E2, T2, _, _ = o.couple_cells(dt, rho, T1, np.array([2.0]), E1)
    o.step(1)
    np.testing.assert_allclose(o.E, 0.5 * (E0[0] + E2[0]), rtol=1e-14)
    np.testing.assert_allclose(o.e, 0.5 * (cv[0] * T0[0] + cv[0] * T2[0]), rtol=1e-13)
