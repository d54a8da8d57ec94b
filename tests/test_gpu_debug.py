"""The debug build (librad_debug.so, device-side index checks on the stores
of the step kernels and the gas step): on tiny grids, the steps report no
failed check and match the FP64 oracle as the release build does; a check
run on an index outside the padded arrays reports RAD_EBOUNDS through
rad_sync and skips the access, and the context stays usable.  The checks run
in a child process with RAD_DEBUG=1, which makes the package load the debug
build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import paper_2606_26268_b300 as R
import workloads as W
from helpers import errors, rounded, run_gpu, run_oracle
assert R.LIB_PATH.endswith("librad_debug.so"), R.LIB_PATH
out = {}
# tiny grids cell by cell against the oracle: 1D 16 cells, 3D 8^3 (and a
# ragged 3D box over several tiles), FP64 and split, single solve and Newton
cases = [("1d", W.random_smooth("cartesian", (16, 1, 1), 1, seed=71, bc="outflow", ncomp=1)),
         ("3d8", W.random_smooth("cartesian", (8, 8, 8), 3, seed=72, bc="periodic", ncomp=3,
                                 fmax=0.8)),
         ("3d", W.random_smooth("cartesian", (37, 21, 19), 3, seed=73, bc="outflow", ncomp=3,
                                fmax=0.8))]
for name, p in cases:
    for prec in ("fp64", "split"):
        for mode in ("once", "newton"):
            q = rounded(p, np.float32) if prec == "split" else p
            q.implicit_mode = mode
            g = run_gpu(q, 3, prec)
            o = run_oracle(q, 3, dt=g["dt"])
            err = errors(g, o, q.ncomp, q.chat, q.c / q.chat, 3)
            nE = float(np.linalg.norm(g["E"] - o["E"]) / np.linalg.norm(o["E"]))
            out["%s_%s_%s" % (name, prec, mode)] = {"status": int(g["status"]), "E": float(err["E"]),
                                                    "normE": nE}
# the gas step (evolved gas, two-stage RK2) on a small box
p = W.random_smooth("cartesian", (24, 20, 18), 3, seed=74, bc="periodic", ncomp=3, fmax=0.5)
p.hydro = True
p.integrator = "rk2"
q = rounded(p, np.float32)
g = run_gpu(q, 2, "split")
out["hydro_split"] = {"status": int(g["status"])}
# the index check itself: out of range (past the end, negative), then in range
q = rounded(W.random_smooth("cartesian", (12, 10, 9), 3, seed=75, bc="periodic", ncomp=3),
            np.float32)
r = R.from_problem(q, "split")
E0 = np.asarray(r.read("E")).copy()
out["check_far"] = [int(r.debug_check_index(1 << 40)), int(r.sync())]
out["check_neg"] = [int(r.debug_check_index(-1)), int(r.sync())]
out["check_in"] = [int(r.debug_check_index(0)), int(r.sync())]
out["state_kept"] = bool(np.array_equal(np.asarray(r.read("E")), E0))
r.step(2)
out["after"] = int(r.sync())
r.close()
print("RESULT " + json.dumps(out))
"""


def test_debug_build_reports_no_failed_check_and_catches_one_out_of_range():
    from paper_2606_26268_b300 import build
    build.build(debug=True)
    env = dict(os.environ, RAD_DEBUG="1")
    res = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env,
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    line = [x for x in res.stdout.splitlines() if x.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    R_OK, R_EBOUNDS = 0, 8
    for key, v in out.items():
        if key.endswith(("_once", "_newton")):
            assert v["status"] == R_OK, (key, v)
            if "_fp64_" in key:
                assert v["E"] <= 1e-11, (key, v)
            else:
                assert v["normE"] <= 1e-5, (key, v)
    assert out["hydro_split"]["status"] == R_OK
    assert out["check_far"] == [R_OK, R_EBOUNDS]
    assert out["check_neg"] == [R_OK, R_EBOUNDS]
    assert out["check_in"] == [R_OK, R_OK]
    assert out["state_kept"]
    assert out["after"] == R_OK
