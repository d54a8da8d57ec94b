"""Pins of the oracle's CFL step (Sect. 2.4, item 10 of the step list) and of
the optical depth of Sect. 2.6 that limits the signal speeds (tau_cell =
rho chi dx with dx the cell's largest width, the mean of the two cells at a
face).  The expected values are closed forms worked out by hand for small
grids, and a brute force written from the definition of the widths.  CPU
only."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _problem(geometry, n, xfaces, ndim, chat=1.0, cfl=0.4, bc="periodic"):
    return W._blank("pin", ndim, n, geometry, bc, xfaces, chat=chat, cfl=cfl, ncomp=3)


def _fill(p, E=None, rho=None):
    p.rho = np.ones(p.N) if rho is None else rho
    p.v = np.zeros((3, p.N))
    p.T = np.ones(p.N)
    p.E = np.ones(p.N) if E is None else E
    p.F = np.zeros((3, p.N))
    return p


# ---------------------------------------------------------------------------
# CFL step
# ---------------------------------------------------------------------------

def test_cfl_step_of_the_gaussian_pulse_is_cfl_dx_over_chat():
    # 512 cells on [0, 1], chat = 100, CFL 0.4: dt = 0.4 / (512 * 100)
    p = W.pulse_1d()
    assert oracle.Oracle(p).dt() == pytest.approx(0.4 / (512 * 100.0), rel=1e-14)


def test_cfl_step_on_a_uniform_3d_box_sums_the_three_directions():
    # cells of 1/8 x 1/4 x 1/2: sum chat / h = chat (8 + 4 + 2)
    xf = [W.uniform_faces(8, 0, 1), W.uniform_faces(4, 0, 1), W.uniform_faces(2, 0, 1)]
    p = _fill(_problem("cartesian", (8, 4, 2), xf, 3, chat=3.0, cfl=0.5))
    assert oracle.Oracle(p).dt() == pytest.approx(0.5 / (3.0 * 14.0), rel=1e-14)


def test_cfl_step_on_a_stretched_cylindrical_grid():
    # R faces 1, 2, 4 (widths 1 and 2, centres 1.5 and 3), phi in four steps of
    # pi/8, z in two steps of 1/2.  The inner ring has the smallest widths:
    # h = (1, 1.5 pi/8, 1/2), so sum chat / h = chat (1 + 16 / (3 pi) + 2).
    xf = [np.array([1.0, 2.0, 4.0]), W.uniform_faces(4, 0.0, math.pi / 2),
          W.uniform_faces(2, 0.0, 1.0)]
    p = _fill(_problem("cylindrical", (2, 4, 2), xf, 3, chat=2.0, cfl=0.4, bc="outflow"))
    want = 0.4 / (2.0 * (3.0 + 16.0 / (3.0 * math.pi)))
    assert oracle.Oracle(p).dt() == pytest.approx(want, rel=1e-14)
    # in 2D (R, phi) the z width does not enter
    p2 = _fill(_problem("cylindrical", (2, 4, 1), [xf[0], xf[1], W.uniform_faces(1, 0, 1)], 2,
                        chat=2.0, cfl=0.4, bc="outflow"))
    want2 = 0.4 / (2.0 * (1.0 + 16.0 / (3.0 * math.pi)))
    assert oracle.Oracle(p2).dt() == pytest.approx(want2, rel=1e-14)


def test_cfl_step_on_a_log_r_spherical_grid():
    # r faces 1, 2, 4; theta from pi/6 to 5 pi/6 in steps of pi/6 (centres
    # pi/4 .. 3 pi/4, the smallest sin theta_c = sqrt(2)/2 next to the axis);
    # phi in two steps of pi/4.  Smallest widths in the inner shell next to the
    # axis: h = (1, 1.5 pi/6, 1.5 sin(pi/4) pi/4), so
    # sum chat / h = chat (1 + 4/pi + 16 / (3 sqrt(2) pi)).
    xf = [W.log_faces(2, 1.0, 4.0), W.uniform_faces(4, math.pi / 6, 5 * math.pi / 6),
          W.uniform_faces(2, 0.0, math.pi / 2)]
    p = _fill(_problem("spherical", (2, 4, 2), xf, 3, chat=5.0, cfl=0.3, bc="outflow"))
    want = 0.3 / (5.0 * (1.0 + 4.0 / math.pi + 16.0 / (3.0 * math.sqrt(2.0) * math.pi)))
    assert oracle.Oracle(p).dt() == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("geometry", ["cartesian", "cylindrical", "spherical"])
def test_cfl_step_matches_a_brute_force_over_the_cell_widths(geometry):
    # widths by definition: (dx0, dx1, dx2) Cartesian, (dR, R dphi, dz)
    # cylindrical, (dr, r dtheta, r sin(theta) dphi) spherical, at the centre
    rng = np.random.default_rng(7)
    n = (5, 6, 4)
    x0 = np.cumsum(np.r_[1.0, rng.uniform(0.1, 1.0, n[0])])
    if geometry == "spherical":
        x1 = np.sort(np.r_[0.2, rng.uniform(0.2, math.pi - 0.2, n[1] - 1), math.pi - 0.2])
    else:
        x1 = np.cumsum(np.r_[0.0, rng.uniform(0.05, 0.5, n[1])])
    x2 = np.cumsum(np.r_[0.0, rng.uniform(0.05, 0.5, n[2])])
    p = _fill(_problem(geometry, n, [x0, x1, x2], 3, chat=7.0, cfl=0.45, bc="outflow"))
    c0, c1 = 0.5 * (x0[1:] + x0[:-1]), 0.5 * (x1[1:] + x1[:-1])
    worst = 0.0
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                h0, h1, h2 = x0[i + 1] - x0[i], x1[j + 1] - x1[j], x2[k + 1] - x2[k]
                if geometry == "cylindrical":
                    h1 *= c0[i]
                elif geometry == "spherical":
                    h1 *= c0[i]
                    h2 *= c0[i] * math.sin(c1[j])
                worst = max(worst, 7.0 / h0 + 7.0 / h1 + 7.0 / h2)
    assert oracle.Oracle(p).dt() == pytest.approx(0.45 / worst, rel=1e-14)


# ---------------------------------------------------------------------------
# optical depth of the thick-limit correction (Sect. 2.6)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1])
def test_thick_limit_uses_the_widest_side_and_the_mean_of_the_two_cells(axis):
    """One step of a checkerboard in E and rho along `axis` on cells of
    1/8 x 1/2 (x narrow, y wide), with pure scattering (kappa_P = 0, so the
    coupling leaves E alone) and F = 0.

    The van Leer slopes vanish at every extremum, so the face states are the
    cell values, f = 0 and lambda = -/+ 1/sqrt(3).  With F = 0 only the
    dissipative term of HLL carries E: with S_L = -b, S_R = b the face flux
    is -b (E_R - E_L) / 2, and the update of E_i = 1 + a (-1)^i is
        E_i - 2 a b dt / h_axis (-1)^i.
    b = min(chat / sqrt(3), 4 chat / (3 tau)), tau = (tau_L + tau_R) / 2,
    tau_cell = rho (kappa_R + sigma) max(dx, dy).  Here rho = 1, 3 alternate,
    kappa_R = 1, sigma = 3 and max(dx, dy) = 1/2: tau = 4 and b = chat / 3.
    Other readings give other b: the width along the face normal in x
    (1/8: tau = 1, b = chat / sqrt(3)), the larger of the two cells
    (tau = 6, b = 2 chat / 9), the smaller (tau = 2, b = chat / sqrt(3)) or
    sigma left out of chi (tau = 1)."""
    n = (8, 4, 1) if axis == 0 else (4, 8, 1)
    ext = [(0.0, n[0] * (0.125 if axis == 0 else 0.5)), (0.0, n[1] * (0.5 if axis == 0 else 0.125))]
    # x narrow (1/8) and y wide (1/2) when axis = 0; transposed when axis = 1
    xf = [W.uniform_faces(n[0], *ext[0]), W.uniform_faces(n[1], *ext[1]),
          W.uniform_faces(1, 0.0, 1.0)]
    p = _problem("cartesian", n, xf, 2, chat=1.0)
    p.ncomp = 2
    p.opacity = {"kind": "const", "kappa_p": 0.0, "kappa_r": 1.0, "sigma": 3.0}
    idx = np.indices((n[1], n[0]))  # (y, x)
    sgn = np.where(idx[1 - axis].ravel() % 2 == 0, 1.0, -1.0)
    a = 0.5
    rho = np.where(sgn > 0, 1.0, 3.0)
    _fill(p, E=1.0 + a * sgn, rho=rho)
    o = oracle.Oracle(p)
    h_axis = 0.125
    dt = 0.1 * h_axis
    o.step(1, dt)
    b = 1.0 / 3.0
    want = 1.0 + a * sgn - 2.0 * a * b * dt / h_axis * sgn
    np.testing.assert_allclose(o.E, want, rtol=1e-14, atol=0)
    # the alternative readings differ from it by far more than rounding
    for b_alt in (1.0 / math.sqrt(3.0), 2.0 / 9.0):
        alt = 1.0 + a * sgn - 2.0 * a * b_alt * dt / h_axis * sgn
        assert np.max(np.abs(alt - want)) > 1e-3
