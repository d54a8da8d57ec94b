"""Pins of the oracle's irradiation term (Sect. 2.9): the energy deposited by
an external irradiation flux, q = -div F_irr per unit volume and time, enters
the gas row of the implicit system (S_1 + dt q) and the gas energy
bookkeeping (E_gas + (c/chat) E_r gains dt q per step).  CPU only."""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
import workloads as W
from test_oracle_step import volumes


def test_solve_satisfies_both_rows_of_the_linear_system():
    """The irradiated solve is the solution of the linear system written out:
    radiation row (1 + gr) E - 4 gr a Tk^3 T = E* - 3 gr a Tk^4, gas row
    -g E + (Cv + 4 g a Tk^3) T = Cv Tn + 3 g a Tk^4 + sq (residuals in long
    double)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        Es, Tn, Tk = rng.uniform(0.1, 5), rng.uniform(0.2, 3), rng.uniform(0.2, 3)
        Cv, g, a = rng.uniform(0.1, 5), 10 ** rng.uniform(-3, 2), rng.uniform(0.3, 2)
        gr = g * rng.uniform(0.01, 1)
        sq = rng.uniform(-0.5, 2) * Cv * Tn
        E, T = oracle.solve2x2(Es, Tn, Tk, Cv, g, gr, a, sq)
        L = np.longdouble
        aT3, aT4 = L(a) * L(Tk) ** 3, L(a) * L(Tk) ** 4
        r1 = (1 + L(gr)) * L(E) - 4 * L(gr) * aT3 * L(T) - (L(Es) - 3 * L(gr) * aT4)
        r2 = -L(g) * L(E) + (L(Cv) + 4 * L(g) * aT3) * L(T) - (L(Cv) * L(Tn) + 3 * L(g) * aT4 + L(sq))
        scale1 = abs(L(Es)) + abs(L(gr) * aT4) + abs(L(E)) * (1 + L(gr))
        scale2 = abs(L(Cv) * L(Tn)) + abs(L(g) * aT4) + abs(L(sq)) + abs(L(g) * L(E))
        assert abs(r1) <= 1e-13 * scale1 and abs(r2) <= 1e-13 * scale2
    # sq = 0 is the plain solve
    assert oracle.solve2x2(2.0, 1.0, 1.1, 1.5, 0.3, 0.2, 1.0, 0.0) == \
        oracle.solve2x2(2.0, 1.0, 1.1, 1.5, 0.3, 0.2, 1.0)


def uniform_box(q, kappa):
    p = W.uniform_state("cartesian", (6, 5, 4), 3, E=1.0, kappa=kappa)
    p.qirr = np.full(p.N, q)
    return p


def test_without_opacity_the_gas_gains_dt_q_per_step():
    p = uniform_box(0.7, 0.0)
    o = oracle.Oracle(p)
    e0, E0 = o.e.copy(), o.E.copy()
    dt = o.dt()
    o.step(5, dt)
    np.testing.assert_allclose(o.e, e0 + 5 * dt * 0.7, rtol=1e-14)
    np.testing.assert_allclose(o.E, E0, rtol=1e-15)


@pytest.mark.parametrize("integrator", ["euler", "rk2"])
def test_total_energy_gains_the_deposited_energy(integrator):
    """With coupling and transport on a periodic box, sum V (E_gas + (c/chat)
    E_r) grows by dt sum V q per step and m + F/chat is conserved."""
    p = W.random_smooth("cartesian", (12, 10, 1), 2, seed=31, bc="periodic", fmax=0.3,
                        chat=2.0, c=10.0,
                        opacity={"kind": "const", "kappa_p": 3.0, "kappa_r": 2.0, "sigma": 1.0})
    rng = np.random.default_rng(5)
    p.qirr = rng.uniform(0.0, 2.0, p.N)
    p.integrator = integrator
    o = oracle.Oracle(p)
    V = volumes(p)
    ratio = p.c / p.chat

    def total():
        ke = np.sum(o.m * o.m, axis=0) / (2 * o.rho)
        return np.sum(V * (o.e + ke)) + ratio * np.sum(V * o.E)

    t0 = total()
    dt = o.dt()
    o.step(3, dt)
    want = t0 + 3 * dt * np.sum(V * p.qirr)
    assert abs(total() - want) / want < 1e-13


def test_newton_with_irradiation_finds_the_root_of_the_heated_balance():
    """Newton mode converges to the root of
    Cv (T - Tn) - dt q + g / (1 + gr) (a T^4 - E*) = 0."""
    p = uniform_box(3.0, 2.0)
    p.implicit_mode = "newton"
    p.T = np.full(p.N, 0.8)
    o = oracle.Oracle(p)
    dt = o.dt()
    rho, Tn, E0 = o.rho[0], o.temperature()[0], o.E[0]
    Cv = o.heat_capacity(rho)
    g = dt * p.c * 2.0 * rho
    gr = dt * p.chat * 2.0 * rho
    f = lambda T: Cv * (T - Tn) - dt * 3.0 + g / (1 + gr) * (p.a_rad * T ** 4 - E0)
    root = brentq(f, 1e-3, 10.0, xtol=1e-15, rtol=1e-15)
    o.step(1, dt)
    assert o.temperature()[0] == pytest.approx(root, rel=1e-11)
