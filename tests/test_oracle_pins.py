"""Pins of the oracle's pointwise pieces against what the paper and the
mathematics fix (closed forms, printed limits, brute force, exact rational
solves).  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_closure():
    rows = []
    for line in open(os.path.join(GOLD, "closure_limits.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        name, f, c, v = line.split()
        rows.append((name, float(f), float(c), float(v)))
    return rows


# ---------------------------------------------------------------------------
# closure (Sect. 2.1) and signal speeds (Sect. 2.6)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("row", _golden_closure())
def test_closure_and_speed_limits_printed_by_the_paper(row):
    name, f, cth, value = row
    if name == "xi":
        assert oracle.xi(f) == pytest.approx(value, rel=1e-15, abs=1e-16)
        return
    # a state with reduced flux f at angle theta to direction x
    sth = math.sqrt(max(0.0, 1.0 - cth * cth))
    E = 2.0
    F = np.array([cth, sth, 0.0]) * f * E
    lm, lp = oracle.eigen(E, F, 0)
    got = lp if name == "lambda_plus" else lm
    assert got == pytest.approx(value, abs=1e-12)


def test_eddington_tensor_limits_and_trace():
    rng = np.random.default_rng(0)
    # f = 0: isotropic D = delta / 3
    D, f = oracle.closure(3.0, [0.0, 0.0, 0.0])
    assert f == 0.0
    np.testing.assert_allclose(D, np.eye(3) / 3.0, atol=1e-16)
    for _ in range(200):
        u = rng.standard_normal(3)
        n = u / np.linalg.norm(u)
        fval = rng.uniform(0, 1)
        E = 10 ** rng.uniform(-3, 3)
        D, f = oracle.closure(E, n * fval * E)
        assert f == pytest.approx(fval, rel=1e-14)
        # trace of the Eddington tensor is 1 for every f (closed form)
        assert np.trace(D) == pytest.approx(1.0, abs=1e-14)
        # D is symmetric, n is an eigenvector with eigenvalue xi, and the
        # transverse eigenvalue is (1 - xi) / 2
        np.testing.assert_allclose(D, D.T, atol=1e-15)
        xi = oracle.xi(fval)
        np.testing.assert_allclose(D @ n, xi * n, atol=1e-14)
        t = np.cross(n, rng.standard_normal(3))
        t /= np.linalg.norm(t)
        np.testing.assert_allclose(D @ t, 0.5 * (1 - xi) * t, atol=1e-14)
    # f = 1: D = n n
    n = np.array([0.6, 0.0, 0.8])
    D, f = oracle.closure(1.0, n)
    np.testing.assert_allclose(D, np.outer(n, n), atol=1e-15)


def test_xi_monotone_between_limits():
    fs = np.linspace(0, 1, 1001)
    x = np.array([oracle.xi(f) for f in fs])
    assert np.all(np.diff(x) > 0)
    assert x[0] == pytest.approx(1 / 3, abs=1e-16) and x[-1] == 1.0


def _flux_jacobian(E, F, d, h=1e-6):
    """Central-difference Jacobian of the physical flux of (E, F) along d."""
    u0 = np.array([E, *F])
    J = np.zeros((4, 4))
    for q in range(4):
        du = np.zeros(4)
        du[q] = h * max(abs(u0[q]), E)
        fp = oracle.phys_flux(1.0, u0[0] + du[0], u0[1:] + du[1:], d)
        fm = oracle.phys_flux(1.0, u0[0] - du[0], u0[1:] - du[1:], d)
        J[:, q] = (fp - fm) / (2 * du[q])
    return J


def test_signal_speeds_are_extreme_eigenvalues_of_the_flux_jacobian():
    """Brute force: the eigenvalues of the numerical Jacobian of the closure
    flux must contain lambda_1 and lambda_3 of Sect. 2.6 as their extremes,
    and lambda_2 = (3 xi - 1) cos(theta) / (2 f) among them."""
    rng = np.random.default_rng(1)
    for _ in range(60):
        f = rng.uniform(0.05, 0.95)
        u = rng.standard_normal(3)
        n = u / np.linalg.norm(u)
        E = 10 ** rng.uniform(-1, 1)
        F = n * f * E
        d = int(rng.integers(0, 3))
        ev = np.linalg.eigvals(_flux_jacobian(E, F, d)).real
        lm, lp = oracle.eigen(E, F, d)
        assert max(ev) == pytest.approx(lp, abs=2e-6)
        assert min(ev) == pytest.approx(lm, abs=2e-6)
        lam2 = (3 * oracle.xi(f) - 1) * n[d] / (2 * f)
        assert np.min(np.abs(ev - lam2)) < 2e-6


def test_signal_speeds_bounded_by_light_speed():
    for f in np.linspace(0, 1, 41):
        for cth in np.linspace(-1, 1, 41):
            sth = math.sqrt(max(0.0, 1 - cth * cth))
            lm, lp = oracle.eigen(1.0, [f * cth, f * sth, 0.0], 0)
            assert -1 - 1e-14 <= lm <= lp <= 1 + 1e-14


# ---------------------------------------------------------------------------
# reconstruction and the f-fix (Sect. 2.5)
# ---------------------------------------------------------------------------

def test_vanleer_limiter_properties():
    rng = np.random.default_rng(2)
    for _ in range(500):
        a, b = rng.standard_normal(2)
        s = oracle.vanleer(a, b)
        if a * b <= 0:
            assert s == 0.0
        else:
            assert abs(s) <= 2 * min(abs(a), abs(b)) + 1e-15
            assert np.sign(s) == np.sign(a)
            assert min(abs(a), abs(b)) - 1e-15 <= abs(s) <= max(abs(a), abs(b)) + 1e-15
        assert oracle.vanleer(a, a) == pytest.approx(a, rel=1e-15)


def test_plm_is_exact_for_linear_data_on_a_stretched_grid():
    import workloads as W
    p = W.random_smooth("cartesian", (24, 1, 1), 1, seed=3, log_r=False)
    xf = np.cumsum(np.r_[0.0, 0.02 * 1.07 ** np.arange(24)])
    p.xfaces[0] = xf
    xc = 0.5 * (xf[1:] + xf[:-1])
    p.E = 3.0 + 2.0 * xc
    p.F = np.zeros((3, 24))
    p.F[0] = 0.5 + 0.1 * xc
    o = oracle.Oracle(p)
    for i in range(2, 23):
        raw, _ = o.face_states(i, 0, 0, 0)
        xface = xf[i]
        assert raw[0] == pytest.approx(3.0 + 2.0 * xface, rel=1e-13)
        assert raw[4] == pytest.approx(3.0 + 2.0 * xface, rel=1e-13)
        assert raw[1] == pytest.approx(0.5 + 0.1 * xface, rel=1e-13)
        assert raw[5] == pytest.approx(0.5 + 0.1 * xface, rel=1e-13)


def test_f_fix_cases_of_eq_f_reconstruct():
    Ec, Fc = 2.0, np.array([0.8, 0.0, 0.0])  # f_c = 0.4
    # kept: f_face in (f_c, 1]
    Ff, fixed = oracle.fix_face(2.2, [1.1, 0.0, 0.0], Ec, Fc)
    assert not fixed and Ff[0] == 1.1
    # f_face > 1: recomputed from the centre with f = f_c
    Ff, fixed = oracle.fix_face(1.0, [1.5, 0.2, 0.0], Ec, Fc)
    assert fixed
    np.testing.assert_allclose(Ff, Fc * (1.0 / Ec), rtol=1e-15)
    # f_face < f_c: recomputed
    Ff, fixed = oracle.fix_face(2.0, [0.1, 0.1, 0.0], Ec, Fc)
    assert fixed
    np.testing.assert_allclose(np.linalg.norm(Ff) / 2.0, 0.4, rtol=1e-15)
    # tie f_face == f_c: recomputed (strict inequality of the equation)
    Ff, fixed = oracle.fix_face(4.0, [1.6, 0.0, 0.0], Ec, Fc)
    assert fixed
    # random: the result always satisfies f_c <= f_face <= 1 (up to rounding)
    rng = np.random.default_rng(4)
    for _ in range(1000):
        Ec = 10 ** rng.uniform(-2, 2)
        Fc = rng.standard_normal(3)
        Fc *= rng.uniform(0, 1) * Ec / np.linalg.norm(Fc)
        Ef = Ec * rng.uniform(0.3, 3)
        Ff = rng.standard_normal(3) * Ef * rng.uniform(0, 1.5)
        out, _ = oracle.fix_face(Ef, Ff, Ec, Fc)
        ff = np.linalg.norm(out) / Ef
        assert ff <= 1 + 1e-14
        assert ff >= np.linalg.norm(Fc) / Ec - 1e-14


# ---------------------------------------------------------------------------
# HLL
# ---------------------------------------------------------------------------

def test_hll_consistency_upwinding_and_rankine_hugoniot():
    rng = np.random.default_rng(5)
    for _ in range(300):
        E = 10 ** rng.uniform(-1, 1)
        F = rng.standard_normal(3)
        F *= rng.uniform(0, 0.99) * E / np.linalg.norm(F)
        d = int(rng.integers(0, 3))
        # consistency: equal states give the physical flux
        np.testing.assert_allclose(oracle.face_flux_states(2.0, d, E, F, E, F),
                                   oracle.phys_flux(2.0, E, F, d), rtol=1e-13, atol=1e-14)
        # two distinct states, explicit wave speeds
        uL = np.r_[E, F]
        E2 = E * rng.uniform(0.5, 2)
        F2 = rng.standard_normal(3)
        F2 *= rng.uniform(0, 0.99) * E2 / np.linalg.norm(F2)
        uR = np.r_[E2, F2]
        fL = oracle.phys_flux(1.0, E, F, d)
        fR = oracle.phys_flux(1.0, E2, F2, d)
        sl, sr = -rng.uniform(0.1, 1), rng.uniform(0.1, 1)
        fh = oracle.hll(sl, sr, uL, uR, fL, fR)
        # the HLL intermediate state from the integral form, and the
        # Rankine-Hugoniot condition across each outer wave
        ustar = (sr * uR - sl * uL - fR + fL) / (sr - sl)
        np.testing.assert_allclose(fh, fL + sl * (ustar - uL), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(fh, fR + sr * (ustar - uR), rtol=1e-12, atol=1e-13)
        # supersonic cases are upwind
        np.testing.assert_array_equal(oracle.hll(0.1, 0.5, uL, uR, fL, fR), fL)
        np.testing.assert_array_equal(oracle.hll(-0.5, -0.1, uL, uR, fL, fR), fR)


def test_thick_correction_limits_the_speeds():
    """With tau -> inf the HLL flux tends to the central average of the
    physical fluxes (the diffusion-limit fix of Sect. 2.6)."""
    E1, F1 = 1.0, np.array([0.1, 0.0, 0.0])
    E2, F2 = 0.5, np.array([0.0, 0.05, 0.0])
    f1 = oracle.phys_flux(1.0, E1, F1, 0)
    f2 = oracle.phys_flux(1.0, E2, F2, 0)
    out = oracle.face_flux_states(1.0, 0, E1, F1, E2, F2, tau=1e12)
    np.testing.assert_allclose(out, 0.5 * (f1 + f2), rtol=1e-9, atol=1e-11)
    # free streaming along +x is purely upwind (both speeds are +1)
    out = oracle.face_flux_states(1.0, 0, 1.0, [1.0, 0, 0], 0.3, [0.3, 0, 0])
    np.testing.assert_allclose(out, oracle.phys_flux(1.0, 1.0, [1.0, 0, 0], 0), rtol=1e-14)


# ---------------------------------------------------------------------------
# implicit coupling (Sect. 2.8)
# ---------------------------------------------------------------------------

def test_closed_form_matches_exact_rational_solve_of_the_printed_matrix():
    import sympy as sp
    rng = np.random.default_rng(6)
    for _ in range(40):
        Es, Tn, Tk = 10 ** rng.uniform(-2, 2), 10 ** rng.uniform(-1, 1), 10 ** rng.uniform(-1, 1)
        Cv, g, a = 10 ** rng.uniform(-2, 2), 10 ** rng.uniform(-4, 4), 10 ** rng.uniform(-1, 1)
        gr = g * 10 ** rng.uniform(-4, 0)
        R = [sp.Rational(float(x)) for x in (Es, Tn, Tk, Cv, g, gr, a)]
        es, tn, tk, cv, gg, ggr, aa = R
        M = sp.Matrix([[1 + ggr, -4 * ggr * aa * tk ** 3], [-gg, cv + 4 * gg * aa * tk ** 3]])
        rhs = sp.Matrix([es - 3 * ggr * aa * tk ** 4, cv * tn + 3 * gg * aa * tk ** 4])
        sol = M.LUsolve(rhs)
        E, T = oracle.solve2x2(Es, Tn, Tk, Cv, g, gr, a)
        assert E == pytest.approx(float(sol[0]), rel=1e-13)
        assert T == pytest.approx(float(sol[1]), rel=1e-13)


def _oracle_for_coupling(c_over_chat=1.0, mode="once", kappa=1.0):
    import workloads as W
    p = W.uniform_state("cartesian", (4, 1, 1), 1)
    p.chat = 1.0
    p.c = c_over_chat
    p.implicit_mode = mode
    p.opacity = {"kind": "const", "kappa_p": kappa, "kappa_r": kappa, "sigma": 0.0}
    return oracle.Oracle(p)


@pytest.mark.parametrize("ratio", [1.0, 1e4])
def test_coupling_fixed_point_and_energy_conservation(ratio):
    o = _oracle_for_coupling(ratio)
    rng = np.random.default_rng(7)
    n = 200
    rho = 10 ** rng.uniform(-1, 1, n)
    Tn = 10 ** rng.uniform(-0.5, 0.5, n)
    kp = 10 ** rng.uniform(-2, 2, n)
    Cv = o.heat_capacity(rho)
    dt = 0.01
    # equilibrium E = a T^4 is a fixed point
    E, T, _, _ = o.couple_cells(dt, rho, Tn, kp, Tn ** 4)
    np.testing.assert_allclose(E, Tn ** 4, rtol=1e-14)
    np.testing.assert_allclose(T, Tn, rtol=1e-14)
    # away from equilibrium: C_v dT + (c/chat) dE = 0 (Sect. 2.7)
    Es = Tn ** 4 * 10 ** rng.uniform(-1, 1, n)
    E, T, _, _ = o.couple_cells(dt, rho, Tn, kp, Es)
    resid = Cv * (T - Tn) + ratio * (E - Es)
    scale = Cv * Tn + ratio * Es
    assert np.max(np.abs(resid) / scale) < 1e-14


def test_newton_mode_converges_to_the_root_of_the_scalar_equation():
    from scipy.optimize import brentq
    o = _oracle_for_coupling(1.0, mode="newton")
    rng = np.random.default_rng(8)
    n = 300
    rho = 10 ** rng.uniform(-1, 1, n)
    Tn = 10 ** rng.uniform(-0.5, 0.5, n)
    kp = 10 ** rng.uniform(-2, 3, n)
    Es = Tn ** 4 * 10 ** rng.uniform(-3, 3, n)
    dt = 0.01
    E, T, it, st = o.couple_cells(dt, rho, Tn, kp, Es)
    assert np.all(st == 0)
    Cv = o.heat_capacity(rho)
    for q in range(n):
        g = dt * kp[q] * rho[q]
        fn = lambda x: Cv[q] * (x - Tn[q]) + g / (1 + g) * (x ** 4 - Es[q])
        root = brentq(fn, 1e-6, 1e3, xtol=1e-300, rtol=1e-15, maxiter=500)
        assert T[q] == pytest.approx(root, rel=2e-14)
        # E^{n+1} then follows from the first row at the root
        assert E[q] == pytest.approx((Es[q] + g * root ** 4) / (1 + g), rel=1e-12)
    # starting from any guess gives the same root
    E2, T2, _, _ = o.couple_cells(dt, rho, Tn, kp, Es, T0=Tn * 7.0)
    np.testing.assert_allclose(T2, T, rtol=1e-13)


def test_small_perturbations_decay_at_the_linear_rate():
    """E = a T^4 (1 + d): one coupling step multiplies E - a T^4 by
    1 / (1 + k dt), k = kappa rho (chat + 4 c a T^3 / C_v), up to O(d^2)."""
    o = _oracle_for_coupling(3.0)
    rho, Tn, kp, dt = np.array([2.0]), np.array([1.3]), np.array([0.7]), 0.05
    Cv = o.heat_capacity(rho)[0]
    k = kp[0] * rho[0] * (1.0 + 4 * 3.0 * Tn[0] ** 3 / Cv)
    errs = []
    for d in (1e-3, 1e-4):
        E, T, _, _ = o.couple_cells(dt, rho, Tn, kp, Tn ** 4 * (1 + d))
        ratio = (E[0] - T[0] ** 4) / (Tn[0] ** 4 * d)
        errs.append(abs(ratio - 1 / (1 + k * dt)))
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 5  # O(d) error in the ratio


def test_many_small_steps_converge_to_the_ode_solution_at_first_order():
    """Backward Euler on dE/dt = -chat k rho (E - a T^4), C_v dT/dt = c k rho
    (E - a T^4): error against a tight RK solution falls like dt."""
    from scipy.integrate import solve_ivp
    o = _oracle_for_coupling(2.0, mode="newton")
    rho, kp, T0, E0, tend = 1.5, 2.0, 1.0, 5.0, 0.3
    Cv = o.heat_capacity(np.array([rho]))[0]

    def rhs(t, y):
        E, T = y
        s = kp * rho * (E - T ** 4)
        return [-1.0 * s, 2.0 * s / Cv]

    ref = solve_ivp(rhs, (0, tend), [E0, T0], rtol=1e-12, atol=1e-14, method="DOP853").y[:, -1]
    errs = []
    for nst in (100, 200, 400):
        dt = tend / nst
        E, T = np.array([E0]), np.array([T0])
        for _ in range(nst):
            E, T, _, _ = o.couple_cells(dt, np.array([rho]), T, np.array([kp]), E)
        errs.append(abs(T[0] - ref[1]))
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
    assert errs[2] / errs[1] == pytest.approx(0.5, abs=0.08)


# ---------------------------------------------------------------------------
# opacities
# ---------------------------------------------------------------------------

def test_powerlaw_opacity_and_its_clip_bounds():
    import workloads as W
    p = W.uniform_state("cartesian", (2, 1, 1), 1)
    p.opacity = {"kind": "powerlaw", "k0": 1.0, "a_rho": 1.0, "b_T": -3.5, "kmin": 1e-4,
                 "kmax": 1e4, "sigma_ratio": 0.25}
    o = oracle.Oracle(p)
    kp, kr, sg = o.opacity(2.0, 3.0)
    assert kp == pytest.approx(2.0 * 3.0 ** -3.5, rel=1e-15) and kr == kp
    assert sg == pytest.approx(0.25 * kp, rel=1e-15)
    assert o.opacity(1e-3, 100.0)[0] == 1e-4       # below kmin
    assert o.opacity(1e3, 1e-3)[0] == 1e4          # above kmax


def test_table_opacity_nodes_linear_exactness_and_clamping():
    import workloads as W
    p = W.uniform_state("cartesian", (2, 1, 1), 1)
    nr, nt = 9, 7
    lr = np.linspace(-4, 0, nr)
    lt = np.linspace(0, 3, nt)
    LT, LR = np.meshgrid(lt, lr, indexing="ij")
    tab = (0.5 * LR - 1.25 * LT + 0.75).astype(np.float32).ravel()
    p.opacity = {"kind": "table", "nrho": nr, "nT": nt, "lrho0": -4.0, "lrho1": 0.0,
                 "lT0": 0.0, "lT1": 3.0, "table": tab, "sigma_ratio": 0.0}
    o = oracle.Oracle(p)
    t64 = tab.astype(np.float64).reshape(nt, nr)
    for it in range(nt):
        for ir in range(nr):
            k = o.opacity(10 ** lr[ir], 10 ** lt[it])[0]
            assert math.log10(k) == pytest.approx(t64[it, ir], abs=1e-12)
    rng = np.random.default_rng(9)
    for _ in range(200):
        a, b = rng.uniform(-4, 0), rng.uniform(0, 3)
        k = o.opacity(10 ** a, 10 ** b)[0]
        assert math.log10(k) == pytest.approx(0.5 * a - 1.25 * b + 0.75, abs=2e-6)  # float32 nodes
    # clamped outside the table
    assert o.opacity(1e-9, 1.0)[0] == pytest.approx(o.opacity(1e-4, 1.0)[0], rel=1e-14)
    assert o.opacity(1.0, 1e9)[0] == pytest.approx(o.opacity(1.0, 1e3)[0], rel=1e-14)
