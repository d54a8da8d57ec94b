"""Pins of the oracle's gas step (the hydrodynamic step that precedes the
radiation transport in every substep, Sect. 2.4): Sod's shock tube against
the exact Riemann solution, exact uniform flow, second-order advection of a
smooth density wave, conservation with the radiation coupling on, and the
first step of a static uniform gas equal to the radiation-only step.  CPU
only."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
import workloads as W
from test_oracle_step import volumes


def exact_riemann(wl, wr, gamma, xi):
    """Exact solution of the Euler Riemann problem (left/right primitive
    states (rho, u, p)) at similarity coordinates xi = (x - x0) / t, by the
    two-wave pressure function: shock branch (p > p_K) from the
    Rankine-Hugoniot conditions, rarefaction branch from the isentropic
    Riemann invariants."""
    rl, ul, pl = wl
    rr, ur, pr = wr
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)

    def f(p, rk, pk, ck):
        if p > pk:
            a = 2.0 / ((gamma + 1) * rk)
            b = (gamma - 1) / (gamma + 1) * pk
            return (p - pk) * math.sqrt(a / (p + b))
        return 2 * ck / (gamma - 1) * ((p / pk) ** ((gamma - 1) / (2 * gamma)) - 1)

    ps = brentq(lambda p: f(p, rl, pl, cl) + f(p, rr, pr, cr) + ur - ul, 1e-12, 1e3)
    us = 0.5 * (ul + ur) + 0.5 * (f(ps, rr, pr, cr) - f(ps, rl, pl, cl))
    g1 = (gamma - 1) / (gamma + 1)
    out = np.zeros((3, xi.size))
    for k, s in enumerate(xi):
        if s < us:  # left of the contact
            if ps > pl:
                sh = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl +
                                         (gamma - 1) / (2 * gamma))
                w = (rl, ul, pl) if s < sh else (rl * (ps / pl + g1) / (g1 * ps / pl + 1), us, ps)
            else:
                cs = cl * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s < ul - cl:
                    w = (rl, ul, pl)
                elif s > us - cs:
                    w = (rl * (ps / pl) ** (1 / gamma), us, ps)
                else:
                    u = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * ul + s)
                    c = 2 / (gamma + 1) * (cl + (gamma - 1) / 2 * (ul - s))
                    w = (rl * (c / cl) ** (2 / (gamma - 1)), u, pl * (c / cl) ** (2 * gamma / (gamma - 1)))
        else:
            if ps > pr:
                sh = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr +
                                         (gamma - 1) / (2 * gamma))
                w = (rr, ur, pr) if s > sh else (rr * (ps / pr + g1) / (g1 * ps / pr + 1), us, ps)
            else:
                cs = cr * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s > ur + cr:
                    w = (rr, ur, pr)
                elif s < us + cs:
                    w = (rr * (ps / pr) ** (1 / gamma), us, ps)
                else:
                    u = 2 / (gamma + 1) * (-cr + (gamma - 1) / 2 * ur + s)
                    c = 2 / (gamma + 1) * (cr - (gamma - 1) / 2 * (ur - s))
                    w = (rr * (c / cr) ** (2 / (gamma - 1)), u, pr * (c / cr) ** (2 * gamma / (gamma - 1)))
        out[:, k] = w
    return out


def gas_1d(n, rho, u, pr, *, gamma=1.4, bc="outflow", extent=(0.0, 1.0), integrator="rk2"):
    """A 1D gas problem with the radiation inert (no opacity, tiny E, chat
    far below the gas speeds so that the gas sets the step)."""
    xf = W.uniform_faces(n, *extent)
    one = W.uniform_faces(1, 0.0, 1.0)
    p = W.Problem(name="gas1d", ndim=1, n=(n, 1, 1), geometry="cartesian",
                  bc_lo=(bc, "outflow", "outflow"), bc_hi=(bc, "outflow", "outflow"),
                  xfaces=[xf, one, one], chat=1e-6, c=1e-6, ncomp=1, gamma_gas=gamma,
                  integrator=integrator, hydro=True)
    x = W.cell_centres(xf)
    p.rho = np.asarray(rho(x), dtype=np.float64)
    p.v = np.zeros((3, n))
    p.v[0] = u(x)
    p.T = np.asarray(pr(x), dtype=np.float64) / p.rho  # p = rho T / mu, mu = 1
    p.E = np.full(n, 1e-10)
    p.F = np.zeros((3, n))
    return p, x


def evolve(p, t_end):
    o = oracle.Oracle(p)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.dt(), t_end - t)
        o.step(1, dt)
        t += dt
    return o


def test_gas_cfl_step_uses_the_sound_speed():
    p, _ = gas_1d(50, lambda x: np.ones_like(x), lambda x: np.full_like(x, 0.5),
                  lambda x: np.full_like(x, 1.4))
    o = oracle.Oracle(p)
    # c_s = sqrt(1.4 * 1.4 / 1) = 1.4, |v| + c_s = 1.9, dx = 1/50
    assert o.dt() == pytest.approx(0.4 / (1.9 * 50), rel=1e-14)


@pytest.mark.parametrize("n", [200, 400])
def test_sod_shock_tube_matches_the_exact_solution(n):
    p, x = gas_1d(n, lambda x: np.where(x < 0.5, 1.0, 0.125), lambda x: np.zeros_like(x),
                  lambda x: np.where(x < 0.5, 1.0, 0.1))
    o = evolve(p, 0.2)
    ex = exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, (x - 0.5) / 0.2)
    l1 = np.mean(np.abs(o.rho - ex[0]))
    assert l1 < (0.0022 if n == 400 else 0.004), l1
    # plateau between the contact and the shock: p* and u* to 1 %
    sel = (x > 0.72) & (x < 0.82)
    pr = (1.4 - 1) * o.e[sel]
    np.testing.assert_allclose(pr, ex[2][sel], rtol=1e-2)
    np.testing.assert_allclose(o.m[0][sel] / o.rho[sel], ex[1][sel], rtol=1e-2)


def test_uniform_moving_gas_stays_uniform():
    p = W.uniform_state("cartesian", (12, 10, 1), 2, kappa=0.3)
    p.hydro = True
    p.bc_lo = p.bc_hi = ("periodic", "periodic", "outflow")
    p.v = np.zeros((3, p.N))
    p.v[0], p.v[1], p.v[2] = 0.3, -0.2, 0.1
    o = oracle.Oracle(p)
    rho0, m0, e0 = o.rho.copy(), o.m.copy(), o.e.copy()
    o.step(3, 0.01)
    np.testing.assert_allclose(o.rho, rho0, rtol=1e-14)
    np.testing.assert_allclose(o.m, m0, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(o.e, e0, rtol=1e-13)


def test_smooth_density_wave_advects_at_second_order():
    errs = []
    ns = [32, 64, 128, 256]
    for n in ns:
        p, x = gas_1d(n, lambda x: 1 + 0.2 * np.sin(2 * np.pi * x), lambda x: np.ones_like(x),
                      lambda x: np.ones_like(x), bc="periodic")
        xf = p.xfaces[0]
        # cell averages of the initial density
        p.rho = 1 + 0.2 * (np.cos(2 * np.pi * xf[:-1]) - np.cos(2 * np.pi * xf[1:])) / (
            2 * np.pi * np.diff(xf))
        p.T = 1.0 / p.rho
        o = evolve(p, 1.0)
        errs.append(np.mean(np.abs(o.rho - p.rho)))
    order = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert order > 1.6, (order, errs)


def test_gas_and_radiation_conserve_mass_momentum_and_energy():
    """Periodic 2D box with opacities: the gas step is in flux form and the
    coupling conserves E_gas + (c/chat) E_r and m + F/chat (Sect. 2.7)."""
    p = W.random_smooth("cartesian", (16, 12, 1), 2, seed=31, bc="periodic", chat=2.0, c=20.0,
                        fmax=0.5)
    p.hydro = True
    p.integrator = "rk2"
    o = oracle.Oracle(p)
    V = volumes(p)
    r = p.c / p.chat

    def totals():
        ke = np.sum(o.m * o.m, axis=0) / (2 * o.rho)
        return (np.sum(V * o.rho), (V * (o.m + o.F / p.chat)).sum(axis=1),
                np.sum(V * (o.e + ke)) + r * np.sum(V * o.E))

    M0, P0, E0 = totals()
    o.step(4, 0.5 * o.dt())
    M1, P1, E1 = totals()
    assert o.stats[1] == 0 and o.stats[2] == 0
    assert abs(M1 - M0) / M0 < 1e-14
    np.testing.assert_allclose(P1, P0, atol=1e-13 * np.abs(P0).max())
    assert abs(E1 - E0) / E0 < 1e-13


def test_closed_reflective_box_conserves_mass_and_energy():
    p = W.random_smooth("cartesian", (12, 10, 1), 2, seed=33, chat=2.0, c=10.0, fmax=0.5)
    p.hydro = True
    p.bc_lo = ("reflective", "reflective", "outflow")
    p.bc_hi = ("reflective", "reflective", "outflow")
    o = oracle.Oracle(p)
    V = volumes(p)

    def totals():
        ke = np.sum(o.m * o.m, axis=0) / (2 * o.rho)
        return np.sum(V * o.rho), np.sum(V * (o.e + ke)) + (p.c / p.chat) * np.sum(V * o.E)

    M0, E0 = totals()
    o.step(3, 0.5 * o.dt())
    M1, E1 = totals()
    assert abs(M1 - M0) / M0 < 1e-14
    assert abs(E1 - E0) / E0 < 1e-13


def test_first_step_of_a_static_uniform_gas_is_the_radiation_step():
    p = W.random_smooth("cartesian", (14, 10, 1), 2, seed=35, bc="periodic")
    p.rho = np.full(p.N, 1.3)
    p.v = np.zeros((3, p.N))
    p.T = np.full(p.N, 0.9)
    ref = oracle.Oracle(p)
    dt = ref.dt()
    ref.step(1, dt)
    q = p.copy()
    q.hydro = True
    o = oracle.Oracle(q).step(1, dt)
    np.testing.assert_array_equal(o.E, ref.E)
    np.testing.assert_array_equal(o.e, ref.e)
    np.testing.assert_array_equal(o.rho, ref.rho)
