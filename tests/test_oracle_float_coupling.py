"""The oracle's host emulation of the split form's coupling products in float
(the linearised solve of Sect. 2.8 with a T^3, the determinant, its
reciprocal and the increments rounded to float; the emission residual
E* - a T^4 in double).  It is off by default, and on the hot-sphere box its
effect on one step is far below the float rounding of the stored state, so
the products the split form keeps in float are not where its error comes
from.  CPU only."""
import numpy as np

import oracle
import workloads as W
from helpers import rounded


def _box(mode):
    p = rounded(W.hot_sphere_3d(ns=(36, 24, 20), nsteps=1), np.float32)
    p.implicit_mode = mode
    p.newton_rtol = 1e-7 if mode == "newton" else 1e-12
    return p


def test_emulation_is_off_by_default_and_changes_nothing_then():
    p = _box("once")
    a = oracle.Oracle(p)
    q = p.copy()
    q.float_coupling = False
    b = oracle.Oracle(q)
    dt = a.dt()
    a.step(2, dt)
    b.step(2, dt)
    np.testing.assert_array_equal(a.E, b.E)
    np.testing.assert_array_equal(a.e, b.e)


def test_float_products_move_one_step_far_less_than_float_storage():
    for mode in ("once", "newton"):
        p = _box(mode)
        ref = p.copy()
        ref.newton_rtol = 1e-12
        o = oracle.Oracle(ref)
        dt = o.dt()
        o.step(1, dt)
        q = p.copy()
        q.float_coupling = True
        f = oracle.Oracle(q)
        f.step(1, dt)
        dE = np.abs(f.E - o.E) / o.E
        de = np.abs(f.e - o.e) / o.e
        # the products change the step (the emulation is active) ...
        assert np.max(dE) > 0.0
        # ... by less than 1e-8 relative in E per cell (storing E in float
        # costs 6e-8) and 1e-10 normwise.  The gas energy takes -(c/chat) dE,
        # and dE in float carries 6e-8 |dE|, which where the coupling moves
        # much energy against e (the edge of the hot sphere) is the same
        # amount that adding a float dE to a float e loses anyway; normwise
        # it stays below 1e-8.
        assert np.max(dE) <= 1e-8, (mode, np.max(dE))
        assert np.linalg.norm(f.E - o.E) / np.linalg.norm(o.E) <= 1e-10
        assert np.linalg.norm(f.e - o.e) / np.linalg.norm(o.e) <= 1e-8, (mode, np.max(de))
