"""Batched grids (rad_batch_*): many independent uneven grids advanced by one
persistent launch per step, replayed from a CUDA graph.  Each member must
end where the same grid ends when stepped alone with rad_step: in both
precisions, in Newton mode with the learned guess, for every launch shape,
with and without the graph, across odd step counts and member steps
interleaved with batch steps.  The tile code is the same, but it is compiled
into a different kernel, where the compiler may fuse a different set of
multiply-adds, so the two agree to rounding (per cell: 1e-13 in FP64, 1e-5
for FP32 transport) rather than bit for bit; launch shapes and graph replay
of the same batch kernel agree bit for bit.  The FP64 batch is also held to
the oracle bound."""
import numpy as np
import pytest

import workloads as W
from helpers import errors, rounded, run_oracle

pytestmark = pytest.mark.gpu

FIELDS = ("E", "F", "e", "m")


def uneven_problems(seed0=300, newton=False):
    """Seven 2D turbulent boxes of uneven, tile-ragged sizes (one smaller
    than a tile, one a single row of tiles, several not multiples of the tile
    width), periodic or outflow, optical depths from thin to thick."""
    sizes = [(200, 130), (64, 64), (33, 17), (129, 257), (5, 3), (300, 40), (96, 80)]
    kscale = [1.0, 1e-2, 30.0, 0.3, 1.0, 1e2, 3.0]
    out = []
    for i, (n, k) in enumerate(zip(sizes, kscale)):
        p = W.turbulent_2d(n, nsteps=10, seed_base=seed0 + 4 * i, nonequilibrium=True,
                           kappa_scale=k)
        if i % 3 == 1:
            p.bc_lo = p.bc_hi = ("outflow",) * 3
        if newton:
            p.implicit_mode = "newton"
        out.append(rounded(p, np.float32))
    return out


def members(probs, precision, **kw):
    import paper_2606_26268_b300 as R
    return [R.from_problem(p, precision=precision, **kw) for p in probs]


def state(r):
    return {k: np.asarray(r.read(k)).copy() for k in FIELDS}


def assert_same(a, b, what=""):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), (what, k, np.max(np.abs(a[k] - b[k])))


def assert_close(a, b, what=""):
    """Per-cell agreement to rounding: |dE|/E, |dF|/E, |de|/e, |dm|/(|m| + E)."""
    E = np.abs(a["E"].astype(np.float64))
    tol = 1e-13 if a["E"].dtype == np.float64 else 1e-5
    d = {"E": np.max(np.abs(a["E"] - b["E"]) / E),
         "F": np.max(np.abs(a["F"] - b["F"]) / E),
         "e": np.max(np.abs(a["e"] - b["e"]) / np.abs(a["e"])),
         "m": np.max(np.abs(a["m"] - b["m"]) / (np.abs(a["m"]) + E))}
    assert max(d.values()) <= tol, (what, d)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_batch_equals_grids_stepped_alone(precision):
    import paper_2606_26268_b300 as R
    probs = uneven_problems()
    alone = members(probs, precision)
    inb = members(probs, precision)
    batch = R.RadBatch(inb)
    for r in alone:
        r.step(7)
        assert r.sync() == 0
    batch.step(7)                  # odd count: the members' buffers swap
    assert batch.sync() == 0
    for ra, rb in zip(alone, inb):
        assert_close(state(ra), state(rb), "after 7")
    for r in alone:
        r.step(4)
    batch.step(4)                  # replays from the other parity
    for ra, rb in zip(alone, inb):
        assert_close(state(ra), state(rb), "after 11")
    st = batch.stats()
    assert st["steps"] == 11
    fix = sum(r.stats()["fix"] for r in alone)
    assert abs(st["fix"] - fix) <= max(2, fix // 1000), (st["fix"], fix)
    batch.close()


def test_fp64_batch_within_the_oracle_bound():
    import paper_2606_26268_b300 as R
    probs = uneven_problems(seed0=500)
    inb = members(probs, "fp64")
    batch = R.RadBatch(inb)
    dts = [r.dt() for r in inb]
    batch.step(5)
    assert batch.sync() == 0
    for p, r, dt in zip(probs, inb, dts):
        o = run_oracle(p, 5, dt=dt)
        g = {k: np.asarray(r.read(k), dtype=np.float64) for k in ("E", "F", "e", "m")}
        err = errors(g, o, p.ncomp, p.chat, p.c / p.chat, 5)
        assert max(err.values()) <= 1e-11, (p.name, err)
    batch.close()


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_batch_newton_with_learned_guess_equals_grids_alone(precision):
    """Newton mode with the learned guess: the batched queue pass finishes
    every queued cell of every grid as the single-grid queue pass does, with
    the same iteration counts."""
    import paper_2606_26268_b300 as R
    probs = uneven_problems(seed0=700, newton=True)
    kw = dict(use_mlp=1, mlp_gate=1e-3)
    alone = members(probs, precision, **kw)
    inb = members(probs, precision, **kw)
    alone[0].mlp_init(5)
    w = alone[0].mlp_get()
    for r in alone:
        r.mlp_set(w)
    batch = R.RadBatch(inb)
    batch.mlp_set(w)
    for r in alone:
        r.step(3)
        assert r.sync() == 0
    batch.step(3)
    assert batch.sync() == 0
    for ra, rb in zip(alone, inb):
        assert_close(state(ra), state(rb), "newton")
    st = batch.stats()
    iters = sum(r.stats()["iters"] for r in alone)
    assert iters > 0
    assert abs(st["iters"] - iters) <= max(2, iters // 1000), (st["iters"], iters)
    batch.close()


def test_batch_launch_shapes_graph_and_tuner():
    """Every CTA shape and march length, with and without the graph, gives the
    same state (bit for bit within one shape, whose kernel is the same; to
    rounding across shapes); the tuner does not advance the state or change
    the counters."""
    import paper_2606_26268_b300 as R
    probs = uneven_problems(seed0=900)
    ref = {}
    nvar = None
    for graph in (True, False):
        for v in range(3):
            for chunk in (0, 7, 16):
                inb = members(probs, "split")
                batch = R.RadBatch(inb, use_graph=graph)
                nvar = batch.get_launch()[2]
                batch.set_launch(v, chunk)
                batch.step(3)
                out = [state(r) for r in inb]
                batch.close()
                if v not in ref:
                    ref[v] = out
                for a, b in zip(ref[v], out):
                    assert_same(a, b, (graph, v, chunk))
                for a, b in zip(ref[0], out):
                    assert_close(a, b, (graph, v, chunk))
    assert nvar == 8
    inb = members(probs, "split")
    batch = R.RadBatch(inb)
    batch.step(2)
    before = [state(r) for r in inb]
    st0 = batch.stats()
    v, c, ms = batch.tune(2)
    assert 0 <= v < 8 and c > 0 and ms > 0
    assert batch.stats() == st0
    for a, r in zip(before, inb):
        assert_same(a, state(r), "tune")
    # the tuned configuration continues the same trajectory
    batch.step(1)
    for a, r in zip(ref[0], inb):
        assert_close(a, state(r), "tuned step")
    batch.close()


def test_member_steps_interleaved_with_batch_steps():
    import paper_2606_26268_b300 as R
    probs = uneven_problems(seed0=1100)
    alone = members(probs, "split")
    inb = members(probs, "split")
    batch = R.RadBatch(inb)
    for r in alone:
        r.step(4)
    batch.step(2)
    inb[2].step(1)        # one member alone, then the others catch up
    for i, r in enumerate(inb):
        if i != 2:
            r.step(1)
    batch.step(1)
    for ra, rb in zip(alone, inb):
        assert_close(state(ra), state(rb), "interleaved")
    # new radiation state on one member between batch steps
    E = np.asarray(alone[1].read("E")).copy() * 1.5
    F = np.asarray(alone[1].read("F")).copy()
    for r in (alone[1], inb[1]):
        r.set_rad(E, F)
    for r in alone:
        r.step(2)
    batch.step(2)
    for ra, rb in zip(alone, inb):
        assert_close(state(ra), state(rb), "after set_rad")
    batch.close()


def test_batch_per_member_step_lengths():
    import paper_2606_26268_b300 as R
    probs = uneven_problems(seed0=1300)
    alone = members(probs, "split")
    inb = members(probs, "split")
    dts = [0.5 * r.dt() for r in alone]
    for r, dt in zip(alone, dts):
        r.step(3, dt)
    batch = R.RadBatch(inb)
    batch.step(3, dts)
    for ra, rb in zip(alone, inb):
        assert_close(state(ra), state(rb), "dt")
    batch.close()


def test_batch_3d():
    import paper_2606_26268_b300 as R
    probs = []
    for i, n in enumerate([(40, 33, 20), (17, 9, 70), (64, 64, 8)]):
        p = W.random_smooth("cartesian", n, 3, seed=40 + i, bc="periodic", ncomp=3)
        probs.append(rounded(p, np.float32))
    for precision in ("split", "fp64"):
        alone = members(probs, precision)
        inb = members(probs, precision)
        batch = R.RadBatch(inb)
        assert batch.get_launch()[2] == 2
        for r in alone:
            r.step(3)
        batch.step(3)
        assert batch.sync() == 0
        for ra, rb in zip(alone, inb):
            assert_close(state(ra), state(rb), precision)
        batch.close()


def test_batch_rejects_mixed_or_unsupported_members():
    import paper_2606_26268_b300 as R
    probs = uneven_problems()[:2]
    a = members(probs[:1], "split")[0]
    b = members(probs[1:], "fp64")[0]
    with pytest.raises(R.RadError) as e:
        R.RadBatch([a, b])
    assert e.value.status == R.RAD_EUNSUPPORTED
    with pytest.raises(R.RadError) as e:
        R.RadBatch([a, a])
    assert e.value.status == R.RAD_EINVAL
    sph = R.from_problem(W.random_smooth("spherical", (16, 12, 1), 2, seed=3), "split")
    with pytest.raises(R.RadError) as e:
        R.RadBatch([sph])
    assert e.value.status == R.RAD_EUNSUPPORTED
