"""Pins of the oracle's options: the LimO3 reconstruction, the flat ("PLUTO")
and clipping treatments of f_face > 1 and the Lax-Friedrichs-Rusanov flux
(Sect. 2.5), the absorption-only coupling of the shadow test (Sect. 3) and
the reflective, fixed (injection) and LTE boundary conditions of the tests
of Sect. 3.  Each is checked against exact values, invariants or an
equivalent problem.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_step import volumes


def one_d(n, E, F, *, bc=("outflow", "outflow"), chat=1.0, kappa=0.0, xf=None, **kw):
    xf = W.uniform_faces(n, 0.0, 1.0) if xf is None else xf
    one = W.uniform_faces(1, 0.0, 1.0)
    p = W.Problem(name="opt1d", ndim=1, n=(n, 1, 1), geometry="cartesian",
                  bc_lo=(bc[0], "outflow", "outflow"), bc_hi=(bc[1], "outflow", "outflow"),
                  xfaces=[xf, one, one], chat=chat, c=chat, ncomp=3,
                  opacity={"kind": "const", "kappa_p": kappa, "kappa_r": kappa, "sigma": 0.0},
                  **kw)
    p.E = np.asarray(E, dtype=np.float64).copy()
    p.F = np.asarray(F, dtype=np.float64).copy()
    p.rho = np.ones(n)
    p.v = np.zeros((3, n))
    p.T = np.ones(n)
    return p


# ---------------------------------------------------------------------------
# LimO3
# ---------------------------------------------------------------------------

def test_limo3_is_exact_for_linear_data_and_zero_at_flat_sides():
    for d in (0.3, -2.0, 1e-7):
        assert oracle.limo3(d, d) == pytest.approx(0.5 * d, rel=1e-15)
    assert oracle.limo3(1.0, 0.0) == 0.0
    assert oracle.limo3(0.0, 1.0) == 0.0  # theta = 0: phi = min(phi3, max(0, 0)) = 0


def test_limo3_face_values_of_a_parabola_are_exact():
    """Cell averages of u = x^2 on a uniform grid: where the limiter is not
    active the third-order face value is the point value (Sect. 2.5 offers
    LimO3 as the third-order option).  Checked through the whole face-state
    path of the step."""
    n = 8
    xf = W.uniform_faces(n, 1.0, 9.0)
    avg = (xf[1:] ** 3 - xf[:-1] ** 3) / 3.0
    p = one_d(n, avg, np.zeros((3, n)), recon="limo3")
    o = oracle.Oracle(p)
    for i in range(2, n - 1):
        raw, _ = o.face_states(i, 0, 0, 0)
        assert raw[0] == pytest.approx(xf[i] ** 2, rel=1e-14)  # upper state of cell i-1
        assert raw[4] == pytest.approx(xf[i] ** 2, rel=1e-14)  # lower state of cell i


def test_limo3_faces_stay_between_the_neighbouring_values():
    """No new extrema: each face value lies between the cell value and the
    neighbour on that side, for any data."""
    rng = np.random.default_rng(3)
    for _ in range(2000):
        um, uc, up = rng.standard_normal(3) * rng.choice([1e-3, 1.0, 1e3])
        hi = uc + oracle.limo3(uc - um, up - uc)
        lo = uc - oracle.limo3(up - uc, uc - um)
        assert min(uc, up) - 1e-12 * abs(uc) <= hi <= max(uc, up) + 1e-12 * abs(uc)
        assert min(uc, um) - 1e-12 * abs(uc) <= lo <= max(uc, um) + 1e-12 * abs(uc)


def test_limo3_face_error_is_third_order_on_smooth_monotone_data():
    errs = []
    ns = [16, 32, 64, 128]
    for n in ns:
        xf = np.linspace(0.2, 1.2, n + 1)
        avg = (np.cos(xf[:-1]) - np.cos(xf[1:])) / np.diff(xf)  # averages of sin
        e = 0.0
        for i in range(1, n - 1):
            hi = avg[i] + oracle.limo3(avg[i] - avg[i - 1], avg[i + 1] - avg[i])
            e = max(e, abs(hi - math.sin(xf[i + 1])))
        errs.append(e)
    slope = -np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert slope > 2.8, (slope, errs)


def test_limo3_wave_is_more_accurate_than_plm():
    """Smooth periodic free-streaming wave with the two-stage integrator: the
    third-order reconstruction leaves a smaller error than PLM."""
    from test_oracle_rk2 import free_streaming_wave

    def err(recon):
        p, xf = free_streaming_wave(128, "rk2")
        p.recon = recon
        o = oracle.Oracle(p)
        dt = 0.2 / 128
        steps = int(round(0.25 / dt))
        o.step(steps, dt)
        t = steps * dt
        exact = 1.0 + 0.4 * (np.cos(2 * math.pi * (xf[:-1] - t)) -
                             np.cos(2 * math.pi * (xf[1:] - t))) / (2 * math.pi * np.diff(xf))
        return np.mean(np.abs(o.E - exact))

    assert err("limo3") < 0.5 * err("plm")


# ---------------------------------------------------------------------------
# the free-streaming shock tube of Sect. 3.1 with the face treatments
# ---------------------------------------------------------------------------

def pressure_analog(o):
    """Pi = (1 - xi) E / 2, the pressure analog of Sect. 3.1."""
    f = np.minimum(np.linalg.norm(o.F, axis=0) / o.E, 1.0)
    xi = (3 + 4 * f * f) / (5 + 2 * np.sqrt(4 - 3 * f * f))
    return (1 - xi) * o.E / 2


def excess_variation(x, Pi, x_end=4.2):
    """Total variation of Pi on x < x_end beyond a monotone rise from its
    first value to its maximum (zero for a clean shock-plateau profile).  In
    tube 2 the contact-like discontinuity sits at x = 4.7 at t = 20."""
    w = Pi[x < x_end]
    return np.sum(np.abs(np.diff(w))) - (w.max() - w[0])


def test_tube2_flat_treatment_with_limo3_oscillates_left_of_the_contact():
    """Sect. 3.1, second tube (f = 1 on both sides), 2^8 cells, RK2: with
    LimO3 the flat face treatment leaves spurious oscillations of Pi on the
    left of the contact; the f-preserving faces do not.  Here their excess
    variation is 15x the f-preserving one and 4x that of the flat treatment
    with PLM."""
    from test_oracle_step import run_tube
    ex = {}
    for recon in ("plm", "limo3"):
        for fix in ("fpreserve", "pluto"):
            x, o = run_tube(2, 256, recon=recon, face_fix=fix, integrator="rk2")
            ex[recon, fix] = excess_variation(x, pressure_analog(o))
    assert ex["limo3", "pluto"] > 5 * ex["limo3", "fpreserve"], ex
    assert ex["limo3", "pluto"] > 2 * ex["plm", "pluto"], ex
    assert ex["limo3", "fpreserve"] < 0.005 and ex["plm", "fpreserve"] < 0.005, ex


@pytest.mark.parametrize("recon", ["plm", "limo3"])
def test_tube2_f_preserving_faces_leave_a_small_peak_of_pi_at_the_contact(recon):
    """Sect. 3.1, second tube: with the f-preserving faces Pi is flat behind
    the left shock and shows a small peak just left of the contact (here 4-5%
    above the plateau at 2^8 cells)."""
    from test_oracle_step import run_tube
    x, o = run_tube(2, 256, recon=recon, face_fix="fpreserve", integrator="rk2")
    Pi = pressure_analog(o)
    plateau = Pi[(x > 0) & (x < 3)]
    peak = Pi[(x > 3) & (x < 4.7)].max()
    assert np.ptp(plateau) < 0.01 * plateau.mean(), np.ptp(plateau)
    assert 1.02 < peak / plateau.mean() < 1.08, peak / plateau.mean()


# ---------------------------------------------------------------------------
# f <= 1 treatments of face states
# ---------------------------------------------------------------------------

def test_pluto_treatment_takes_the_flat_state_only_when_f_exceeds_one():
    Ec, Fc = 1.0, [0.5, 0.0, 0.0]
    E, F, ch = oracle.fix_face_mode("pluto", 1.2, [1.3, 0.0, 0.0], Ec, Fc)
    assert ch and E == 1.0 and list(F) == [0.5, 0.0, 0.0]
    # f_face = 0.25 < f_centre = 0.5: the f-preserving fix rescales, PLUTO keeps
    E, F, ch = oracle.fix_face_mode("pluto", 1.2, [0.3, 0.0, 0.0], Ec, Fc)
    assert not ch and E == 1.2 and list(F) == [0.3, 0.0, 0.0]
    E, F, ch = oracle.fix_face_mode("fpreserve", 1.2, [0.3, 0.0, 0.0], Ec, Fc)
    assert ch and E == 1.2 and F[0] == pytest.approx(0.6, rel=1e-15)


def test_clip_treatment_rescales_to_f_equal_one_along_the_same_direction():
    rng = np.random.default_rng(5)
    for _ in range(500):
        Ef = rng.uniform(0.1, 2.0)
        Ff = rng.standard_normal(3) * 2.0
        E, F, ch = oracle.fix_face_mode("clip", Ef, Ff, 1.0, [0.0, 0.0, 0.0])
        nf = np.linalg.norm(Ff)
        assert E == Ef
        if nf > Ef:
            assert ch
            assert np.linalg.norm(F) == pytest.approx(Ef, rel=1e-14)
            np.testing.assert_allclose(F / np.linalg.norm(F), Ff / nf, rtol=1e-13)
        else:
            assert not ch and np.array_equal(F, Ff)


@pytest.mark.parametrize("mode", ["fpreserve", "pluto", "clip"])
def test_every_treatment_leaves_faces_with_f_at_most_one(mode):
    p = W.random_smooth("cartesian", (24, 20, 1), 2, seed=41, fmax=0.999)
    p.face_fix = mode
    o = oracle.Oracle(p)
    for (i, j) in [(3, 4), (10, 7), (20, 15), (1, 1), (23, 19)]:
        for d in (0, 1):
            _, fx = o.face_states(i, j, 0, d)
            for s in (0, 4):
                assert np.linalg.norm(fx[s + 1:s + 4]) <= fx[s] * (1 + 1e-14)


# ---------------------------------------------------------------------------
# Lax-Friedrichs-Rusanov
# ---------------------------------------------------------------------------

def test_lf_equals_hll_when_the_signal_speeds_are_symmetric():
    """HLL with S_L = -S_R is the Rusanov flux: an identity that pins the
    halves and the sign of the dissipation."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        uL, uR, fL, fR = rng.standard_normal((4, 4))
        s = rng.uniform(0.1, 3.0)
        np.testing.assert_allclose(oracle.lf(-s, s, uL, uR, fL, fR),
                                   oracle.hll(-s, s, uL, uR, fL, fR), rtol=1e-13, atol=1e-14)


def test_lf_takes_the_largest_speed_and_is_more_dissipative_than_hll():
    uL = np.array([2.0, 0.5, 0.0, 0.0])
    uR = np.array([1.0, 0.1, 0.0, 0.0])
    fL = np.array([0.5, 0.9, 0.0, 0.0])
    fR = np.array([0.1, 0.4, 0.0, 0.0])
    out = oracle.lf(-0.2, 0.7, uL, uR, fL, fR)
    np.testing.assert_allclose(out, 0.5 * (fL + fR) - 0.35 * (uR - uL), rtol=1e-15)
    # with speeds (-0.2, 0.7) HLL weights F_R by 0.2/0.9 and dissipates less
    hll = oracle.hll(-0.2, 0.7, uL, uR, fL, fR)
    assert out[0] > hll[0]  # E jumps down to the right: more dissipation pushes right


def test_lf_and_hll_give_the_upwind_step_in_the_free_streaming_limit():
    """f = 1 along +x everywhere: both solvers reduce to upwinding (up to the
    rounding of lambda near f = 1, where it varies like sqrt(1 - f^2))."""
    n = 64
    x = W.cell_centres(W.uniform_faces(n, 0.0, 1.0))
    E = 1.0 + np.exp(-(x - 0.4) ** 2 / 0.01)
    F = np.zeros((3, n))
    F[0] = E
    res = []
    for r in ("hll", "lf"):
        p = one_d(n, E, F, riemann=r, bc=("periodic", "periodic"))
        o = oracle.Oracle(p)
        o.step(5)
        res.append(o.E.copy())
    np.testing.assert_allclose(res[1], res[0], rtol=1e-10)


def test_lf_step_conserves_energy_and_momentum():
    p = W.random_smooth("cartesian", (16, 12, 1), 2, seed=8, bc="periodic", chat=2.0, c=20.0)
    p.riemann = "lf"
    o = oracle.Oracle(p)
    V = volumes(p)
    r = p.c / p.chat

    def tot():
        ke = np.sum(o.m * o.m, axis=0) / (2 * o.rho)
        return np.sum(V * (o.e + ke)) + r * np.sum(V * o.E), (V * (o.m + o.F / p.chat)).sum(axis=1)

    t0, m0 = tot()
    o.step(3)
    t1, m1 = tot()
    assert o.stats[1] == 0 and o.stats[2] == 0
    assert abs(t1 - t0) / t0 < 1e-13
    np.testing.assert_allclose(m1, m0, atol=1e-13 * np.abs(m0).max())


# ---------------------------------------------------------------------------
# absorption-only coupling
# ---------------------------------------------------------------------------

def test_absorption_only_decays_E_geometrically_and_heats_the_gas():
    """No emission: E^{n+1} = E^n / (1 + chat dt kappa_P rho) per step; the
    lost energy goes into the gas (Sect. 2.7)."""
    p = W.uniform_state("cartesian", (6, 5, 1), 2, E=3.0, kappa=2.0)
    p.implicit_mode = "absorb"
    p.c = 10.0
    o = oracle.Oracle(p)
    dt = o.dt()
    g = p.chat * dt * 2.0 * 1.0
    e0 = o.e.copy()
    o.step(4, dt)
    np.testing.assert_allclose(o.E, 3.0 / (1 + g) ** 4, rtol=1e-14)
    np.testing.assert_allclose(o.e - e0, (p.c / p.chat) * (3.0 - o.E), rtol=1e-13)
    out = oracle.Oracle(p).step_cells([0], dt)
    assert out["T"][0] == pytest.approx(out["e"][0] / o.heat_capacity(1.0), rel=1e-15)


def test_absorption_only_with_transport_conserves_total_energy():
    p = W.random_smooth("cartesian", (14, 10, 1), 2, seed=13, bc="periodic", chat=2.0, c=50.0)
    p.implicit_mode = "absorb"
    o = oracle.Oracle(p)
    V = volumes(p)

    def tot():
        ke = np.sum(o.m * o.m, axis=0) / (2 * o.rho)
        return np.sum(V * (o.e + ke)) + (p.c / p.chat) * np.sum(V * o.E)

    t0 = tot()
    o.step(3)
    assert abs(tot() - t0) / t0 < 1e-13


# ---------------------------------------------------------------------------
# boundary conditions
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("side", ["lo", "hi"])
def test_reflective_wall_equals_the_mirror_symmetric_problem(side):
    """A reflective side is the symmetry plane of the doubled problem whose
    mirror half has E, F_y, F_z even and F_x odd (Sect. 3 uses the wall for
    the shadow test)."""
    n, ny = 12, 10
    rng = np.random.default_rng(17)
    w = rng.uniform(0.5, 1.5, n)
    xf = np.concatenate([[0.0], np.cumsum(w)]) / w.sum()   # stretched, [0, 1]
    full = W.random_smooth("cartesian", (2 * n, ny, 1), 2, seed=19, bc="periodic", chat=2.0,
                           c=5.0, fmax=0.8)
    xf2 = np.concatenate([-xf[::-1], xf[1:]])
    full.xfaces[0] = xf2
    full.bc_lo = ("outflow", "periodic", "outflow")
    full.bc_hi = ("outflow", "periodic", "outflow")
    shp = (ny, 2 * n)
    right = (slice(None), slice(n, 2 * n))
    left = (slice(None), slice(n - 1, None, -1))

    def mirror(a, odd=False):
        a = a.reshape(shp).copy()
        a[left] = -a[right] if odd else a[right]
        return a.ravel()

    full.E = mirror(full.E)
    full.F = np.stack([mirror(full.F[0], True), mirror(full.F[1]), mirror(full.F[2])])
    full.rho = mirror(full.rho)
    full.T = mirror(full.T)
    full.v = np.stack([mirror(full.v[0], True), mirror(full.v[1]), mirror(full.v[2])])

    half = full.copy()
    half.n = (n, ny, 1)
    half.xfaces = [xf.copy(), full.xfaces[1].copy(), full.xfaces[2].copy()]

    def take(a):
        return a.reshape(shp)[right].ravel().copy()

    for k in ("E", "rho", "T"):
        setattr(half, k, take(getattr(full, k)))
    half.F = np.stack([take(full.F[q]) for q in range(3)])
    half.v = np.stack([take(full.v[q]) for q in range(3)])
    half.bc_lo = ("reflective", "periodic", "outflow")
    half.bc_hi = ("outflow", "periodic", "outflow")
    if side == "hi":
        # the same problem seen from the other side: x -> 1 - x
        flipx = (slice(None), slice(None, None, -1))

        def fl(a, odd=False):
            b = a.reshape(ny, n)[flipx].ravel().copy()
            return -b if odd else b

        half.xfaces[0] = (1.0 - xf[::-1]).copy()
        for k in ("E", "rho", "T"):
            setattr(half, k, fl(getattr(half, k)))
        half.F = np.stack([fl(half.F[0], True), fl(half.F[1]), fl(half.F[2])])
        half.v = np.stack([fl(half.v[0], True), fl(half.v[1]), fl(half.v[2])])
        half.bc_lo = ("outflow", "periodic", "outflow")
        half.bc_hi = ("reflective", "periodic", "outflow")
    of = oracle.Oracle(full)
    oh = oracle.Oracle(half)
    dt = min(of.dt(), oh.dt())
    of.step(3, dt)
    oh.step(3, dt)
    E = take(of.E)
    F0 = take(of.F[0])
    e = take(of.e)
    if side == "hi":
        E, F0, e = (a.reshape(ny, n)[flipx].ravel() for a in (E, F0, e))
        F0 = -F0
    np.testing.assert_allclose(oh.E, E, rtol=1e-13)
    np.testing.assert_allclose(oh.F[0], F0, rtol=1e-12, atol=1e-13 * np.abs(F0).max())
    np.testing.assert_allclose(oh.e, e, rtol=1e-13)


def test_closed_reflective_box_conserves_total_energy():
    p = W.random_smooth("cartesian", (12, 10, 1), 2, seed=23, chat=2.0, c=10.0)
    p.bc_lo = ("reflective", "reflective", "outflow")
    p.bc_hi = ("reflective", "reflective", "outflow")
    o = oracle.Oracle(p)
    V = volumes(p)

    def tot():
        ke = np.sum(o.m * o.m, axis=0) / (2 * o.rho)
        return np.sum(V * (o.e + ke)) + (p.c / p.chat) * np.sum(V * o.E)

    t0 = tot()
    o.step(4)
    assert abs(tot() - t0) / t0 < 1e-13


def test_fixed_injection_feeds_the_upwind_flux_of_the_boundary_state():
    """A free-streaming (f = 1) interior fed by an injected f = 1 state: the
    first cell changes by chat dt / dx (E_b - E_0) exactly."""
    n = 16
    E0, Eb = 0.25, 3.0
    F = np.zeros((3, n))
    F[0] = E0
    p = one_d(n, np.full(n, E0), F, bc=("fixed", "outflow"),
              bc_value={(0, 0): (Eb, Eb, 0.0, 0.0, 1.0)})
    o = oracle.Oracle(p)
    dt = o.dt()
    o.step(1, dt)
    dx = 1.0 / n
    assert o.E[0] == pytest.approx(E0 + p.chat * dt / dx * (Eb - E0), rel=1e-14)
    np.testing.assert_allclose(o.E[1:], E0, rtol=1e-14)


def test_lte_boundary_closed_form_flux_into_a_static_interior():
    """E = a T_b^4 in the ghosts, F = 0 interior: the HLL flux through the
    boundary face is chat (E_b - E_1) / (2 sqrt 3) for E and
    chat (E_b + E_1) / 6 for F_x (f = 0: speeds -/+ chat / sqrt 3, D = I/3)."""
    n = 10
    E1, Tb = 1.0, 1.3
    p = one_d(n, np.full(n, E1), np.zeros((3, n)), bc=("lte", "outflow"),
              bc_value={(0, 0): (0.0, 0.0, 0.0, 0.0, Tb)}, chat=2.0)
    o = oracle.Oracle(p)
    dt = o.dt()
    o.step(1, dt)
    Eb = Tb ** 4
    lam = dt * n
    assert o.E[0] == pytest.approx(E1 + lam * p.chat * (Eb - E1) / (2 * math.sqrt(3)), rel=1e-14)
    assert o.F[0, 0] == pytest.approx(lam * (p.chat * (Eb + E1) / 6 - p.chat * E1 / 3), rel=1e-13)
    np.testing.assert_allclose(o.E[1:], E1, rtol=1e-14)


@pytest.mark.parametrize("bc", ["fixed", "lte"])
def test_boundary_state_equal_to_the_edge_cell_reproduces_outflow(bc):
    """Ghosts that hold the edge cell's own state (E, F, e) make the first
    step identical to the outflow (zero-gradient) boundary: pins that LTE
    copies F and that both take the edge density and e = C_v T_b."""
    p = W.random_smooth("cartesian", (20, 1, 1), 1, seed=29, chat=2.0, c=4.0)
    p.T[0] = 0.8
    p.T[-1] = 1.1
    p.E[0] = 0.8 ** 4 * p.a_rad
    p.E[-1] = 1.1 ** 4 * p.a_rad
    ref = oracle.Oracle(p).step(1)
    q = p.copy()
    q.bc_lo = (bc, "outflow", "outflow")
    q.bc_hi = (bc, "outflow", "outflow")
    q.bc_value = {(0, 0): (p.E[0], p.F[0, 0], p.F[1, 0], p.F[2, 0], 0.8),
                  (0, 1): (p.E[-1], p.F[0, -1], p.F[1, -1], p.F[2, -1], 1.1)}
    o = oracle.Oracle(q).step(1)
    np.testing.assert_allclose(o.E, ref.E, rtol=1e-15)
    np.testing.assert_allclose(o.F, ref.F, rtol=1e-15, atol=1e-300)
    np.testing.assert_allclose(o.e, ref.e, rtol=1e-15)
