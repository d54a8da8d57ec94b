"""The shadow test of Sect. 3 on the oracle (half the paper's resolution,
70 x 20, ten light-crossing times): what the paper states about its two
panels, and the Beer-Lambert attenuation of the unshadowed beam.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

NX, NY = 70, 20


def run(coupling):
    p = W.shadow((NX, NY), coupling)
    o = oracle.Oracle(p)
    dt = o.dt()
    o.step(int(10 * 1.0 / (p.chat * dt)), dt)  # ten crossings of the 1 cm box
    return p, o.E.reshape(NY, NX) / p.bc_value[(0, 0)][0]


@pytest.fixture(scope="module")
def panels():
    return {c: run(c) for c in ("absorb", "once")}


def column(x):
    return int((x + 0.5) * NX)


def test_unshadowed_beam_follows_beer_lambert(panels):
    """Above the shadow the f = 1 beam crosses gas of kappa rho = 0.1 / cm:
    E(x) = E_b exp(-0.1 (x + 1/2)) at steady state."""
    p, E = panels["absorb"]
    xc = W.cell_centres(p.xfaces[0])
    exact = np.exp(-0.1 * (xc + 0.5))
    np.testing.assert_allclose(E[-1, 5:], exact[5:], rtol=2e-3)


def test_absorption_only_gives_a_shadow_with_a_one_cell_edge(panels):
    """Sect. 3: without emission the shadow behind the spheroid is sharp,
    its edge confined to a single cell."""
    _, E = panels["absorb"]
    for x in (0.2, 0.3, 0.4):
        col = E[:, column(x)]
        level = col[-1]
        mid = np.sum((col > 0.1 * level) & (col < 0.9 * level))
        assert mid <= 1, (x, col)
        assert col[0] < 1e-6 * level


def test_emission_fills_and_blurs_the_shadow_and_overshoots(panels):
    """Sect. 3: with emission and absorption the shadow is more diffuse,
    holds more radiation, and E overshoots at the edge of the beam."""
    _, Ea = panels["absorb"]
    _, Ef = panels["once"]
    c = column(0.4)
    a, f = Ea[:, c], Ef[:, c]
    assert f[0] > 1e3 * a[0]
    level = f[-1]
    assert np.sum((f > 0.1 * level) & (f < 0.9 * level)) >= 2
    assert f.max() > 1.01 * level
