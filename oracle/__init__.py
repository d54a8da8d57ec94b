"""FP64 CPU oracle of the M1 radiation step (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package; the CUDA library never imports it.  The arithmetic lives in
m1_oracle.c (plain FP64 C, built without FMA contraction); this module only
marshals arrays and converts the workload's primitive gas inputs (rho, v, T)
into the conserved state (m = rho v, e = C_v T with C_v = rho / (mu (Gamma-1))).
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, Optional

import numpy as np

from . import build as _build

_GEOM = {"cartesian": 0, "cylindrical": 1, "spherical": 2}
_BC = {"outflow": 0, "periodic": 1, "reflective": 2, "fixed": 3, "lte": 4}
_OPAC = {"const": 0, "powerlaw": 1, "table": 2}
_MODE = {"once": 0, "newton": 1, "absorb": 2}
_RECON = {"plm": 0, "limo3": 1}
_FIX = {"fpreserve": 0, "pluto": 1, "clip": 2}
_RIEMANN = {"hll": 0, "lf": 1}
STAT_NAMES = ["fix", "efloor", "fclip", "iters", "itmax", "fallback", "noconv", "spare"]

_dp = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("geom", C.c_int),
                ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3), ("xf", _dp * 3),
                ("chat", C.c_double), ("c", C.c_double), ("a_rad", C.c_double),
                ("gamma_gas", C.c_double), ("mu", C.c_double), ("cfl", C.c_double),
                ("e_floor", C.c_double), ("opac_kind", C.c_int), ("kappa_p", C.c_double),
                ("kappa_r", C.c_double), ("sigma", C.c_double), ("k0", C.c_double),
                ("a_rho", C.c_double), ("b_T", C.c_double), ("kmin", C.c_double),
                ("kmax", C.c_double), ("sigma_ratio", C.c_double), ("nrho", C.c_int),
                ("nT", C.c_int), ("lrho0", C.c_double), ("lrho1", C.c_double),
                ("lT0", C.c_double), ("lT1", C.c_double), ("ltable", _dp),
                ("implicit_mode", C.c_int), ("newton_rtol", C.c_double),
                ("newton_maxit", C.c_int), ("nthreads", C.c_int), ("integrator", C.c_int),
                ("qirr", _dp), ("recon", C.c_int), ("face_fix", C.c_int), ("riemann", C.c_int),
                ("bc_val", C.c_double * 30), ("hydro", C.c_int), ("float_coupling", C.c_int)]


class _State(C.Structure):
    _fields_ = [(k, _dp) for k in ("E", "F0", "F1", "F2", "rho", "e", "m0", "m1", "m2")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_xi.restype = C.c_double
        L.orc_xi.argtypes = [C.c_double]
        L.orc_vanleer.restype = C.c_double
        L.orc_vanleer.argtypes = [C.c_double, C.c_double]
        L.orc_closure.argtypes = [C.c_double, _dp, _dp, _dp]
        L.orc_phys_flux.argtypes = [C.c_double, C.c_double, _dp, C.c_int, _dp]
        L.orc_lambda.argtypes = [C.c_double, _dp, C.c_int, _dp, _dp]
        L.orc_fix_face.restype = C.c_int
        L.orc_fix_face.argtypes = [C.c_double, _dp, C.c_double, _dp]
        L.orc_hll.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp]
        L.orc_lf.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp]
        L.orc_limo3.restype = C.c_double
        L.orc_limo3.argtypes = [C.c_double, C.c_double]
        L.orc_fix_face_mode.restype = C.c_int
        L.orc_fix_face_mode.argtypes = [C.c_int, _dp, _dp, C.c_double, _dp]
        L.orc_opacity.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, _dp, _dp, _dp]
        L.orc_dt.restype = C.c_double
        L.orc_dt.argtypes = [C.POINTER(_Problem)]
        L.orc_dt_gas.restype = C.c_double
        L.orc_dt_gas.argtypes = [C.POINTER(_Problem)] + [_dp] * 5
        L.hydro_face_flux.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_int * 3,
                                      C.c_int, _dp]
        L.orc_solve2x2.argtypes = [C.c_double] * 7 + [_dp, _dp]
        L.orc_solve2x2_irr.argtypes = [C.c_double] * 8 + [_dp, _dp]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.POINTER(_State),
                               C.c_double, C.c_int, C.POINTER(C.c_int64)]
        L.orc_step_cells.restype = C.c_int
        L.orc_step_cells.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_double,
                                     C.c_longlong, C.POINTER(C.c_longlong), _dp]
        L.orc_couple_cells.restype = C.c_int
        L.orc_couple_cells.argtypes = [C.POINTER(_Problem), C.c_double, C.c_longlong, _dp, _dp,
                                       _dp, _dp, _dp, _dp, _dp, C.POINTER(C.c_int),
                                       C.POINTER(C.c_int)]
        L.orc_face_flux_states.argtypes = [C.c_double, C.c_int, C.c_double, _dp, C.c_double, _dp,
                                           C.c_double, _dp]
        L.orc_max_threads.restype = C.c_int
        L.orc_face_states.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_int, C.c_int,
                                      C.c_int, C.c_int, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _vec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


# ---------------------------------------------------------------------------
# pointwise pieces (for the pin tests)
# ---------------------------------------------------------------------------

def xi(f: float) -> float:
    return lib().orc_xi(float(f))


def vanleer(dl: float, dr: float) -> float:
    return lib().orc_vanleer(float(dl), float(dr))


def closure(E: float, F) -> tuple:
    F = _vec(F)
    D = np.zeros(9)
    f = np.zeros(1)
    lib().orc_closure(float(E), _ptr(F), _ptr(D), _ptr(f))
    return D.reshape(3, 3), float(f[0])


def phys_flux(chat: float, E: float, F, d: int) -> np.ndarray:
    F = _vec(F)
    out = np.zeros(4)
    lib().orc_phys_flux(float(chat), float(E), _ptr(F), int(d), _ptr(out))
    return out


def eigen(E: float, F, d: int) -> tuple:
    F = _vec(F)
    lm = C.c_double()
    lp = C.c_double()
    lib().orc_lambda(float(E), _ptr(F), int(d), C.byref(lm), C.byref(lp))
    return lm.value, lp.value


def fix_face(Ef: float, Ff, Ec: float, Fc) -> tuple:
    Ff = _vec(Ff).copy()
    Fc = _vec(Fc)
    r = lib().orc_fix_face(float(Ef), _ptr(Ff), float(Ec), _ptr(Fc))
    return Ff, bool(r)


def hll(sl, sr, uL, uR, fL, fR) -> np.ndarray:
    out = np.zeros(4)
    lib().orc_hll(float(sl), float(sr), _ptr(_vec(uL)), _ptr(_vec(uR)), _ptr(_vec(fL)),
                  _ptr(_vec(fR)), _ptr(out))
    return out


def lf(sl, sr, uL, uR, fL, fR) -> np.ndarray:
    out = np.zeros(4)
    lib().orc_lf(float(sl), float(sr), _ptr(_vec(uL)), _ptr(_vec(uR)), _ptr(_vec(fL)),
                 _ptr(_vec(fR)), _ptr(out))
    return out


def limo3(dn: float, dt: float) -> float:
    """LimO3 increment phi(dn/dt) dt / 2 towards the face on the dt side."""
    return lib().orc_limo3(float(dn), float(dt))


def fix_face_mode(mode: str, Ef: float, Ff, Ec: float, Fc) -> tuple:
    """The f <= 1 treatment `mode` of one face state: (Ef, Ff, changed)."""
    E = np.array([float(Ef)])
    Ff = _vec(Ff).copy()
    r = lib().orc_fix_face_mode(_FIX[mode], _ptr(E), _ptr(Ff), float(Ec), _ptr(_vec(Fc)))
    return float(E[0]), Ff, bool(r)


def face_flux_states(chat, d, EL, FL, ER, FR, tau=-1.0) -> np.ndarray:
    out = np.zeros(4)
    lib().orc_face_flux_states(float(chat), int(d), float(EL), _ptr(_vec(FL)), float(ER),
                               _ptr(_vec(FR)), float(tau), _ptr(out))
    return out


def solve2x2(Estar, Tn, Tk, Cv, g, gr, a, sq=None) -> tuple:
    """The 2x2 coupling solve (Eq. implicit_matrix); sq = dt (-div F_irr) adds
    the irradiation term of Sect. 2.9 to the gas row."""
    E = C.c_double()
    T = C.c_double()
    if sq is None:
        lib().orc_solve2x2(float(Estar), float(Tn), float(Tk), float(Cv), float(g), float(gr),
                           float(a), C.byref(E), C.byref(T))
    else:
        lib().orc_solve2x2_irr(float(Estar), float(Tn), float(Tk), float(Cv), float(g),
                               float(gr), float(a), float(sq), C.byref(E), C.byref(T))
    return E.value, T.value


# ---------------------------------------------------------------------------
# whole problems
# ---------------------------------------------------------------------------

class Oracle:
    """Holds a problem in the oracle's layout and advances it."""

    def __init__(self, prob, nthreads: int = 0):
        self.prob = prob
        p = _Problem()
        p.ndim = prob.ndim
        for d in range(3):
            p.n[d] = int(prob.n[d])
            p.bc_lo[d] = _BC[prob.bc_lo[d]]
            p.bc_hi[d] = _BC[prob.bc_hi[d]]
        p.geom = _GEOM[prob.geometry]
        self._xf = [_vec(x) for x in prob.xfaces]
        for d in range(3):
            assert self._xf[d].size == prob.n[d] + 1
            p.xf[d] = _ptr(self._xf[d])
        p.chat = prob.chat
        p.c = prob.c
        p.a_rad = prob.a_rad
        p.gamma_gas = prob.gamma_gas
        p.mu = prob.mu
        p.cfl = prob.cfl
        p.e_floor = prob.e_floor
        op = prob.opacity
        p.opac_kind = _OPAC[op["kind"]]
        p.kappa_p = op.get("kappa_p", 0.0)
        p.kappa_r = op.get("kappa_r", 0.0)
        p.sigma = op.get("sigma", 0.0)
        p.k0 = op.get("k0", 0.0)
        p.a_rho = op.get("a_rho", 0.0)
        p.b_T = op.get("b_T", 0.0)
        p.kmin = op.get("kmin", 0.0)
        p.kmax = op.get("kmax", 1e300)
        p.sigma_ratio = op.get("sigma_ratio", 0.0)
        self._table = _vec(np.asarray(op.get("table", np.zeros(4))).astype(np.float64))
        p.nrho = op.get("nrho", 2)
        p.nT = op.get("nT", 2)
        p.lrho0 = op.get("lrho0", 0.0)
        p.lrho1 = op.get("lrho1", 1.0)
        p.lT0 = op.get("lT0", 0.0)
        p.lT1 = op.get("lT1", 1.0)
        p.ltable = _ptr(self._table)
        p.implicit_mode = _MODE[prob.implicit_mode]
        p.newton_rtol = prob.newton_rtol
        p.newton_maxit = prob.newton_maxit
        p.nthreads = int(nthreads)
        p.integrator = {"euler": 0, "rk2": 1}[getattr(prob, "integrator", "euler")]
        q = getattr(prob, "qirr", None)
        self._qirr = None if q is None else _vec(q).copy()
        p.qirr = _ptr(self._qirr) if self._qirr is not None else None
        p.recon = _RECON[getattr(prob, "recon", "plm")]
        p.face_fix = _FIX[getattr(prob, "face_fix", "fpreserve")]
        p.riemann = _RIEMANN[getattr(prob, "riemann", "hll")]
        p.hydro = int(bool(getattr(prob, "hydro", False)))
        # host emulation of the split form's float coupling products (for
        # measuring their share of its error; never the reference)
        p.float_coupling = int(bool(getattr(prob, "float_coupling", False)))
        for (d, side), v in getattr(prob, "bc_value", {}).items():
            for q in range(5):
                p.bc_val[10 * d + 5 * side + q] = float(v[q])
        self._p = p
        self.stats = np.zeros(8, dtype=np.int64)
        self.set_state_from_problem()

    # state -----------------------------------------------------------------
    def heat_capacity(self, rho):
        return rho / (self.prob.mu * (self.prob.gamma_gas - 1.0))

    def set_state_from_problem(self):
        pr = self.prob
        N = pr.N
        self.E = _vec(pr.E).copy()
        F = np.zeros((3, N)) if pr.F is None else np.asarray(pr.F, dtype=np.float64)
        self.F = np.ascontiguousarray(F).copy()
        self.rho = _vec(pr.rho).copy()
        v = np.zeros((3, N)) if pr.v is None else np.asarray(pr.v, dtype=np.float64)
        self.m = np.ascontiguousarray(self.rho[None, :] * v)
        self.e = self.heat_capacity(self.rho) * _vec(pr.T)
        self._work = [np.zeros(N) for _ in range(9)]

    def set_state(self, E, F, rho, e, m):
        self.E = _vec(E).copy()
        self.F = np.ascontiguousarray(np.asarray(F, dtype=np.float64)).copy()
        self.rho = _vec(rho).copy()
        self.e = _vec(e).copy()
        self.m = np.ascontiguousarray(np.asarray(m, dtype=np.float64)).copy()
        N = self.E.size
        if len(self._work) != 9 or self._work[0].size != N:
            self._work = [np.zeros(N) for _ in range(9)]

    def _state(self):
        return _State(_ptr(self.E), _ptr(self.F[0]), _ptr(self.F[1]), _ptr(self.F[2]),
                      _ptr(self.rho), _ptr(self.e), _ptr(self.m[0]), _ptr(self.m[1]),
                      _ptr(self.m[2]))

    def temperature(self):
        return self.e / self.heat_capacity(self.rho)

    # stepping --------------------------------------------------------------
    def dt(self) -> float:
        """The CFL step: radiation alone, or with the gas signal speeds when
        the gas is evolved."""
        if self._p.hydro:
            return lib().orc_dt_gas(C.byref(self._p), _ptr(self.rho), _ptr(self.e),
                                    _ptr(self.m[0]), _ptr(self.m[1]), _ptr(self.m[2]))
        return lib().orc_dt(C.byref(self._p))

    def step(self, nsteps: int = 1, dt: Optional[float] = None):
        dt = self.dt() if dt is None else float(dt)
        s = self._state()
        ws = _State(*[_ptr(a) for a in self._work])
        st = np.zeros(8, dtype=np.int64)
        lib().orc_step(C.byref(self._p), C.byref(s), C.byref(ws), dt, int(nsteps),
                       st.ctypes.data_as(C.POINTER(C.c_int64)))
        for q in range(8):
            if q == 4:
                self.stats[q] = max(self.stats[q], st[q])
            else:
                self.stats[q] += st[q]
        return self

    def step_cells(self, cells, dt: Optional[float] = None) -> Dict[str, np.ndarray]:
        """One step of the listed cells from the current state (state unchanged)."""
        dt = self.dt() if dt is None else float(dt)
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
        out = np.zeros((cells.size, 9))
        s = self._state()
        lib().orc_step_cells(C.byref(self._p), C.byref(s), dt, cells.size,
                             cells.ctypes.data_as(C.POINTER(C.c_longlong)), _ptr(out))
        return {"E": out[:, 0], "F": out[:, 1:4].T, "e": out[:, 4], "m": out[:, 5:8].T,
                "T": out[:, 8]}

    def couple_cells(self, dt, rho, Tn, kp, Estar, T0=None):
        rho, Tn, kp, Estar = (_vec(a) for a in (rho, Tn, kp, Estar))
        n = rho.size
        T0a = _vec(T0) if T0 is not None else np.zeros(n)
        E = np.zeros(n)
        T = np.zeros(n)
        it = np.zeros(n, dtype=np.int32)
        stt = np.zeros(n, dtype=np.int32)
        lib().orc_couple_cells(C.byref(self._p), float(dt), n, _ptr(rho), _ptr(Tn), _ptr(kp),
                               _ptr(Estar), _ptr(T0a), _ptr(E), _ptr(T),
                               it.ctypes.data_as(C.POINTER(C.c_int)),
                               stt.ctypes.data_as(C.POINTER(C.c_int)))
        return E, T, it, stt

    def face_states(self, i: int, j: int, k: int, d: int) -> tuple:
        """Raw and fixed (EL, FL, ER, FR) at the lower face of cell (i,j,k) along d."""
        out = np.zeros(16)
        s = self._state()
        lib().orc_face_states(C.byref(self._p), C.byref(s), int(i), int(j), int(k), int(d),
                              _ptr(out))
        return out[:8].copy(), out[8:].copy()

    def opacity(self, rho, T) -> tuple:
        kp = C.c_double()
        kr = C.c_double()
        sg = C.c_double()
        lib().orc_opacity(C.byref(self._p), float(rho), float(T), C.byref(kp), C.byref(kr),
                          C.byref(sg))
        return kp.value, kr.value, sg.value


def max_threads() -> int:
    return lib().orc_max_threads()
