"""B300-native M1 radiation step (transport + implicit coupling).

Python binding of the C ABI in include/rad.h (librad.so, hand-written sm_103a
CUDA).  This module only marshals arguments: every step of the method runs in
the library's kernels.  PyTorch supplies device memory (the workspace) and the
stream.  There is no CPU fallback: importing the binding without the built
library raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RAD_DEBUG=1: the debug build (device-side index checks, RAD_EBOUNDS)
LIB_PATH = os.path.join(_HERE, "_lib", "librad_debug.so" if os.environ.get("RAD_DEBUG") == "1"
                        else "librad.so")

RAD_OK, RAD_EINVAL, RAD_ENOMEM, RAD_ECUDA, RAD_ENONPHYS, RAD_ENOCONV, RAD_ETIMEOUT, \
    RAD_EUNSUPPORTED, RAD_EBOUNDS = range(9)
RAD_CARTESIAN, RAD_CYLINDRICAL, RAD_SPHERICAL = range(3)
RAD_BC_OUTFLOW, RAD_BC_PERIODIC, RAD_BC_REFLECTIVE, RAD_BC_FIXED, RAD_BC_LTE = range(5)
RAD_OPAC_CONST, RAD_OPAC_POWERLAW, RAD_OPAC_TABLE = range(3)
RAD_FP64, RAD_FP32_SPLIT = range(2)
RAD_LINEARIZED_ONCE, RAD_NEWTON, RAD_ABSORPTION_ONLY = range(3)
RAD_PLM, RAD_LIMO3 = range(2)
RAD_FIX_FPRESERVE, RAD_FIX_PLUTO, RAD_FIX_CLIP = range(3)
RAD_HLL, RAD_LF = range(2)
RAD_EULER, RAD_RK2 = range(2)
RAD_FIELD_E, RAD_FIELD_F, RAD_FIELD_EINT, RAD_FIELD_M, RAD_FIELD_T, RAD_FIELD_RHO = range(6)

GEOMETRY = {"cartesian": RAD_CARTESIAN, "cylindrical": RAD_CYLINDRICAL,
            "spherical": RAD_SPHERICAL}
BC = {"outflow": RAD_BC_OUTFLOW, "periodic": RAD_BC_PERIODIC, "reflective": RAD_BC_REFLECTIVE,
      "fixed": RAD_BC_FIXED, "lte": RAD_BC_LTE}
OPACITY = {"const": RAD_OPAC_CONST, "powerlaw": RAD_OPAC_POWERLAW, "table": RAD_OPAC_TABLE}
PRECISION = {"fp64": RAD_FP64, "split": RAD_FP32_SPLIT}
IMPLICIT = {"once": RAD_LINEARIZED_ONCE, "newton": RAD_NEWTON, "absorb": RAD_ABSORPTION_ONLY}
RECON = {"plm": RAD_PLM, "limo3": RAD_LIMO3}
FACE_FIX = {"fpreserve": RAD_FIX_FPRESERVE, "pluto": RAD_FIX_PLUTO, "clip": RAD_FIX_CLIP}
RIEMANN = {"hll": RAD_HLL, "lf": RAD_LF}
INTEGRATOR = {"euler": RAD_EULER, "rk2": RAD_RK2}
FIELDS = {"E": RAD_FIELD_E, "F": RAD_FIELD_F, "e": RAD_FIELD_EINT, "m": RAD_FIELD_M,
          "T": RAD_FIELD_T, "rho": RAD_FIELD_RHO}


class rad_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("xface", C.c_void_p * 3),
                ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3), ("bc_value", C.c_double * 30)]


class rad_opacity(C.Structure):
    _fields_ = [("kind", C.c_int), ("kappa_p", C.c_double), ("kappa_r", C.c_double),
                ("sigma", C.c_double), ("k0", C.c_double), ("a_rho", C.c_double),
                ("b_T", C.c_double), ("kmin", C.c_double), ("kmax", C.c_double),
                ("sigma_ratio", C.c_double), ("nrho", C.c_int), ("nT", C.c_int),
                ("lrho0", C.c_double), ("lrho1", C.c_double), ("lT0", C.c_double),
                ("lT1", C.c_double), ("table_log10_kappa", C.c_void_p)]


class rad_params(C.Structure):
    _fields_ = [("chat", C.c_double), ("c", C.c_double), ("a_rad", C.c_double),
                ("gamma_gas", C.c_double), ("mu", C.c_double), ("cfl", C.c_double),
                ("e_floor", C.c_double), ("precision", C.c_int), ("implicit_mode", C.c_int),
                ("newton_rtol", C.c_double), ("newton_maxit", C.c_int), ("ncomp", C.c_int),
                ("use_mlp", C.c_int), ("mlp_gate", C.c_double), ("integrator", C.c_int),
                ("irradiation", C.c_int), ("reconstruction", C.c_int), ("face_fix", C.c_int),
                ("riemann", C.c_int), ("hydro", C.c_int)]


class rad_stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("fix", "efloor", "fclip", "iters", "itmax",
                                          "fallback", "noconv", "steps")]


EXPORTS = ["rad_default_params", "rad_create", "rad_workspace_size", "rad_bind_workspace",
           "rad_alloc_workspace", "rad_set_stream", "rad_set_gas", "rad_set_rad",
           "rad_set_irradiation", "rad_step",
           "rad_read", "rad_set_gas_host_async", "rad_set_rad_host_async",
           "rad_read_host_async", "rad_sync", "rad_dt", "rad_get_stats", "rad_reset_stats",
           "rad_launches_per_step", "rad_profile_begin", "rad_profile_end",
           "rad_set_launch", "rad_get_launch", "rad_set_wait_limit", "rad_debug_check_index",
           "rad_tune",
           "rad_mlp_nparam", "rad_mlp_set", "rad_mlp_get", "rad_mlp_init", "rad_mlp_train",
           "rad_mlp_grad", "rad_mlp_predict", "rad_mlp_predict_tc", "rad_log_bind",
           "rad_log_count",
           "rad_mlp_grad_noalloc",
           "rad_batch_create", "rad_batch_workspace_size", "rad_batch_bind_workspace",
           "rad_batch_alloc_workspace", "rad_batch_set_stream", "rad_batch_set_graph",
           "rad_batch_step", "rad_batch_sync", "rad_batch_get_stats", "rad_batch_reset_stats",
           "rad_batch_launches_per_step", "rad_batch_set_launch", "rad_batch_get_launch",
           "rad_batch_tune", "rad_batch_mlp_set", "rad_batch_destroy",
           "rad_destroy", "rad_strerror"]

_lib = None


def lib() -> C.CDLL:
    """Loads librad.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librad.so is missing (%s): build it with "
                           "`python -m paper_2606_26268_b300.build`" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp = C.c_void_p
    L.rad_default_params.argtypes = [P(rad_params)]
    L.rad_create.argtypes = [P(rad_grid), C.c_int, P(rad_opacity), P(rad_params), P(vp)]
    L.rad_workspace_size.argtypes = [vp, P(C.c_size_t)]
    L.rad_bind_workspace.argtypes = [vp, vp, C.c_size_t]
    L.rad_alloc_workspace.argtypes = [vp]
    L.rad_set_stream.argtypes = [vp, vp]
    L.rad_set_gas.argtypes = [vp, vp, vp, vp, C.c_int]
    L.rad_set_rad.argtypes = [vp, vp, vp, C.c_int]
    L.rad_set_irradiation.argtypes = [vp, vp, C.c_int]
    L.rad_step.argtypes = [vp, C.c_double, C.c_int]
    L.rad_read.argtypes = [vp, C.c_int, vp, C.c_size_t, C.c_int]
    L.rad_sync.argtypes = [vp]
    L.rad_set_gas_host_async.argtypes = [vp, vp, vp, vp]
    L.rad_set_rad_host_async.argtypes = [vp, vp, vp]
    L.rad_read_host_async.argtypes = [vp, C.c_int, vp, C.c_size_t]
    L.rad_dt.argtypes = [vp, P(C.c_double)]
    L.rad_get_stats.argtypes = [vp, P(rad_stats)]
    L.rad_reset_stats.argtypes = [vp]
    L.rad_launches_per_step.argtypes = [vp]
    L.rad_launches_per_step.restype = C.c_int
    L.rad_profile_begin.argtypes = [vp, C.c_int]
    L.rad_profile_end.argtypes = [vp, P(C.c_float), P(C.c_float), P(C.c_int)]
    L.rad_set_launch.argtypes = [vp, C.c_int, C.c_int]
    L.rad_set_wait_limit.argtypes = [vp, C.c_uint]
    L.rad_debug_check_index.argtypes = [vp, C.c_longlong]
    L.rad_get_launch.argtypes = [vp, P(C.c_int), P(C.c_int), P(C.c_int)]
    L.rad_tune.argtypes = [vp, C.c_int, P(C.c_int), P(C.c_int), P(C.c_float)]
    L.rad_mlp_nparam.argtypes = []
    L.rad_mlp_nparam.restype = C.c_int
    fp = P(C.c_float)
    L.rad_mlp_set.argtypes = [vp, vp, C.c_size_t]
    L.rad_mlp_get.argtypes = [vp, vp, C.c_size_t]
    L.rad_mlp_init.argtypes = [vp, C.c_uint64]
    L.rad_mlp_train.argtypes = [vp, vp, C.c_size_t, C.c_int, C.c_int, C.c_float, C.c_uint64, fp]
    L.rad_mlp_grad.argtypes = [vp, vp, C.c_size_t, vp, fp]
    L.rad_mlp_predict.argtypes = [vp, vp, C.c_size_t, vp]
    L.rad_mlp_predict_tc.argtypes = [vp, vp, C.c_size_t, vp]
    L.rad_log_bind.argtypes = [vp, vp, C.c_size_t, C.c_longlong]
    L.rad_log_count.argtypes = [vp, P(C.c_size_t)]
    L.rad_mlp_grad_noalloc.argtypes = [vp, vp, C.c_size_t, vp, vp, vp]
    ip = P(C.c_int)
    L.rad_batch_create.argtypes = [P(vp), C.c_int, P(vp)]
    L.rad_batch_workspace_size.argtypes = [vp, P(C.c_size_t)]
    L.rad_batch_bind_workspace.argtypes = [vp, vp, C.c_size_t]
    L.rad_batch_alloc_workspace.argtypes = [vp]
    L.rad_batch_set_stream.argtypes = [vp, vp]
    L.rad_batch_set_graph.argtypes = [vp, C.c_int]
    L.rad_batch_step.argtypes = [vp, vp, C.c_int]
    L.rad_batch_sync.argtypes = [vp]
    L.rad_batch_get_stats.argtypes = [vp, P(rad_stats)]
    L.rad_batch_reset_stats.argtypes = [vp]
    L.rad_batch_launches_per_step.argtypes = [vp]
    L.rad_batch_launches_per_step.restype = C.c_int
    L.rad_batch_set_launch.argtypes = [vp, C.c_int, C.c_int]
    L.rad_batch_get_launch.argtypes = [vp, ip, ip, ip, ip]
    L.rad_batch_tune.argtypes = [vp, C.c_int, ip, ip, P(C.c_float)]
    L.rad_batch_mlp_set.argtypes = [vp, vp, C.c_size_t]
    L.rad_batch_destroy.argtypes = [vp]
    L.rad_batch_destroy.restype = None
    L.rad_destroy.argtypes = [vp]
    L.rad_destroy.restype = None
    L.rad_strerror.argtypes = [C.c_int]
    L.rad_strerror.restype = C.c_char_p
    _lib = L
    return L


class RadError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().rad_strerror(status).decode()
        super().__init__("%s failed: %s (status %d)" % (where, msg, status))


def check(status: int, where: str) -> None:
    if status != RAD_OK:
        raise RadError(status, where)


NOALLOC_MAX_RECORDS = 16384


def mlp_grad_noalloc(params, records, grad_out, loss_out, stream=None) -> int:
    """rad_mlp_grad_noalloc on device tensors (float32, contiguous): params
    (8577), records (n, 4), grad_out (8577), loss_out (1).  Enqueued on
    `stream` (a torch stream; default: the current one); returns the status."""
    import torch
    for t in (params, records, grad_out, loss_out):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib().rad_mlp_grad_noalloc(C.c_void_p(params.data_ptr()),
                                      C.c_void_p(records.data_ptr()), records.shape[0],
                                      C.c_void_p(grad_out.data_ptr()),
                                      C.c_void_p(loss_out.data_ptr()), C.c_void_p(s.cuda_stream))


def default_params() -> rad_params:
    p = rad_params()
    check(lib().rad_default_params(C.byref(p)), "rad_default_params")
    return p


class Rad:
    """One radiation problem on one GPU.

    grid: dict(ndim, n=(n0,n1,n2), xfaces=[3 arrays], bc_lo=(...), bc_hi=(...),
    bc_value={(d, side): (E, F0, F1, F2, T_b)}) with bc names 'outflow' |
    'periodic' | 'reflective' | 'fixed' | 'lte'; opacity: dict with 'kind'
    and the fields of rad_opacity; params: rad_params field values, with
    precision 'fp64' | 'split', implicit_mode 'once' | 'newton' | 'absorb',
    reconstruction 'plm' | 'limo3', face_fix 'fpreserve' | 'pluto' | 'clip',
    riemann 'hll' | 'lf'.
    """

    def __init__(self, grid: dict, geometry: str, opacity: dict, params: dict,
                 device: Optional[object] = None, workspace: str = "torch"):
        import torch
        self.torch = torch
        L = lib()
        g = rad_grid()
        g.ndim = int(grid["ndim"])
        self._xf = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in grid["xfaces"]]
        for d in range(3):
            g.n[d] = int(grid["n"][d])
            g.xface[d] = self._xf[d].ctypes.data
            g.bc_lo[d] = BC[grid["bc_lo"][d]]
            g.bc_hi[d] = BC[grid["bc_hi"][d]]
        for (d, side), v in grid.get("bc_value", {}).items():
            for q in range(5):
                g.bc_value[10 * d + 5 * side + q] = float(v[q])
        o = rad_opacity()
        o.kind = OPACITY[opacity["kind"]]
        for k in ("kappa_p", "kappa_r", "sigma", "k0", "a_rho", "b_T", "kmin", "sigma_ratio",
                  "lrho0", "lT0"):
            setattr(o, k, float(opacity.get(k, 0.0)))
        o.kmax = float(opacity.get("kmax", 1e300))
        o.lrho1 = float(opacity.get("lrho1", 1.0))
        o.lT1 = float(opacity.get("lT1", 1.0))
        o.nrho = int(opacity.get("nrho", 2))
        o.nT = int(opacity.get("nT", 2))
        self._table = None
        if opacity["kind"] == "table":
            self._table = np.ascontiguousarray(np.asarray(opacity["table"], dtype=np.float32))
            o.table_log10_kappa = self._table.ctypes.data
        p = default_params()
        for k, v in params.items():
            if k == "precision":
                v = PRECISION[v] if isinstance(v, str) else v
            elif k == "implicit_mode":
                v = IMPLICIT[v] if isinstance(v, str) else v
            elif k == "integrator":
                v = INTEGRATOR[v] if isinstance(v, str) else v
            elif k == "reconstruction":
                v = RECON[v] if isinstance(v, str) else v
            elif k == "face_fix":
                v = FACE_FIX[v] if isinstance(v, str) else v
            elif k == "riemann":
                v = RIEMANN[v] if isinstance(v, str) else v
            setattr(p, k, v)
        self.params = p
        self.ncomp = int(p.ncomp)
        self.N = int(np.prod([int(x) for x in grid["n"]]))
        self._inflight = []
        self.dtype = np.float64 if p.precision == RAD_FP64 else np.float32
        ctx = C.c_void_p()
        check(L.rad_create(C.byref(g), GEOMETRY[geometry], C.byref(o), C.byref(p),
                           C.byref(ctx)), "rad_create")
        self.ctx = ctx
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = C.c_size_t()
        check(L.rad_workspace_size(ctx, C.byref(nbytes)), "rad_workspace_size")
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            check(L.rad_set_stream(ctx, C.c_void_p(self.stream.cuda_stream)), "rad_set_stream")
            if workspace == "torch":
                self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8,
                                       device=self.device)
                base = self._ws.data_ptr()
                aligned = (base + 255) // 256 * 256
                check(L.rad_bind_workspace(ctx, C.c_void_p(aligned), self.workspace_bytes),
                      "rad_bind_workspace")
            else:
                self._ws = None
                check(L.rad_alloc_workspace(ctx), "rad_alloc_workspace")

    # -- marshalling ---------------------------------------------------------
    def _arg(self, a, count):
        torch = self.torch
        if isinstance(a, torch.Tensor):
            assert a.is_cuda and a.is_contiguous() and a.numel() == count, "bad device tensor"
            assert a.dtype == (torch.float64 if self.dtype == np.float64 else torch.float32)
            return C.c_void_p(a.data_ptr()), 1, a
        arr = np.ascontiguousarray(np.asarray(a, dtype=self.dtype)).reshape(-1)
        assert arr.size == count, "expected %d values, got %d" % (count, arr.size)
        return C.c_void_p(arr.ctypes.data), 0, arr

    def set_gas(self, rho, v, T):
        r, dr, kr = self._arg(rho, self.N)
        vv, dv, kv = self._arg(v, self.N * self.ncomp)
        t, dt_, kt = self._arg(T, self.N)
        assert dr == dv == dt_, "all host or all device"
        check(lib().rad_set_gas(self.ctx, r, vv, t, dr), "rad_set_gas")

    def set_rad(self, E, F):
        e, de, ke = self._arg(E, self.N)
        f, df, kf = self._arg(F, self.N * self.ncomp)
        assert de == df, "all host or all device"
        check(lib().rad_set_rad(self.ctx, e, f, de), "rad_set_rad")

    def set_irradiation(self, q):
        """q = -div F_irr per cell (Sect. 2.9); needs irradiation=1 at creation."""
        qq, dq, kq = self._arg(q, self.N)
        check(lib().rad_set_irradiation(self.ctx, qq, dq), "rad_set_irradiation")

    def step(self, nsteps: int = 1, dt: Optional[float] = None):
        check(lib().rad_step(self.ctx, float(dt) if dt else 0.0, int(nsteps)), "rad_step")

    def dt(self) -> float:
        v = C.c_double()
        check(lib().rad_dt(self.ctx, C.byref(v)), "rad_dt")
        return v.value

    def read(self, field: str, out=None, host: bool = True):
        """Field as a numpy array (host=True) or into/as a device tensor."""
        fid = FIELDS[field]
        count = self.N * (self.ncomp if field in ("F", "m") else 1)
        itemsize = np.dtype(self.dtype).itemsize
        if host:
            arr = np.empty(count, dtype=self.dtype) if out is None else out
            check(lib().rad_read(self.ctx, fid, C.c_void_p(arr.ctypes.data), count * itemsize, 0),
                  "rad_read")
            return arr.reshape(self.ncomp, self.N) if field in ("F", "m") else arr
        torch = self.torch
        t = out if out is not None else torch.empty(
            count, dtype=torch.float64 if self.dtype == np.float64 else torch.float32,
            device=self.device)
        check(lib().rad_read(self.ctx, fid, C.c_void_p(t.data_ptr()), count * itemsize, 1),
              "rad_read")
        return t

    def _host(self, a, count):
        assert isinstance(a, np.ndarray) and a.dtype == self.dtype and a.flags.c_contiguous
        assert a.size == count, "expected %d values, got %d" % (count, a.size)
        self._inflight.append(a)  # kept alive until sync()
        return C.c_void_p(a.ctypes.data)

    def set_gas_async(self, rho, v, T):
        """Asynchronous rad_set_gas from host arrays (pinned for overlap);
        the arrays must stay unchanged until sync()."""
        check(lib().rad_set_gas_host_async(self.ctx, self._host(rho, self.N),
                                           self._host(v, self.N * self.ncomp),
                                           self._host(T, self.N)), "rad_set_gas_host_async")

    def set_rad_async(self, E, F):
        check(lib().rad_set_rad_host_async(self.ctx, self._host(E, self.N),
                                           self._host(F, self.N * self.ncomp)),
              "rad_set_rad_host_async")

    def read_async(self, field: str, out):
        """Enqueues the read-back of a field into the host array `out`,
        valid after sync()."""
        count = self.N * (self.ncomp if field in ("F", "m") else 1)
        ptr = self._host(out, count)
        check(lib().rad_read_host_async(self.ctx, FIELDS[field], ptr,
                                        count * np.dtype(self.dtype).itemsize),
              "rad_read_host_async")

    def sync(self) -> int:
        st = lib().rad_sync(self.ctx)
        self._inflight = []
        return st

    def stats(self) -> dict:
        s = rad_stats()
        check(lib().rad_get_stats(self.ctx, C.byref(s)), "rad_get_stats")
        return {k: int(getattr(s, k)) for k, _ in rad_stats._fields_}

    def reset_stats(self):
        check(lib().rad_reset_stats(self.ctx), "rad_reset_stats")

    def set_launch(self, variant: int, chunk: int = 0):
        check(lib().rad_set_launch(self.ctx, int(variant), int(chunk)), "rad_set_launch")

    def debug_check_index(self, index: int) -> int:
        """rad_debug_check_index (the debug build's index check on cell
        `index` of the padded layout); returns the status code."""
        return lib().rad_debug_check_index(self.ctx, int(index))

    def set_wait_limit(self, polls: int):
        """Bound of the staged-plane waits (0: the default)."""
        check(lib().rad_set_wait_limit(self.ctx, int(polls)), "rad_set_wait_limit")

    def get_launch(self) -> tuple:
        v, c, n = C.c_int(), C.c_int(), C.c_int()
        check(lib().rad_get_launch(self.ctx, C.byref(v), C.byref(c), C.byref(n)), "rad_get_launch")
        return v.value, c.value, n.value

    def tune(self, reps: int = 3) -> tuple:
        """Picks the fastest launch shape on the current state (state unchanged)."""
        v, c, t = C.c_int(), C.c_int(), C.c_float()
        check(lib().rad_tune(self.ctx, int(reps), C.byref(v), C.byref(c), C.byref(t)), "rad_tune")
        return v.value, c.value, t.value

    # -- learned starting guess ------------------------------------------------
    def mlp_nparam(self) -> int:
        return lib().rad_mlp_nparam()

    def mlp_set(self, params):
        arr = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        check(lib().rad_mlp_set(self.ctx, C.c_void_p(arr.ctypes.data), arr.size), "rad_mlp_set")

    def mlp_get(self) -> np.ndarray:
        arr = np.empty(self.mlp_nparam(), dtype=np.float32)
        check(lib().rad_mlp_get(self.ctx, C.c_void_p(arr.ctypes.data), arr.size), "rad_mlp_get")
        return arr

    def mlp_init(self, seed: int = 0):
        check(lib().rad_mlp_init(self.ctx, int(seed)), "rad_mlp_init")

    def mlp_train(self, records, epochs: int, batch: int = 1024, lr: float = 1e-3,
                  seed: int = 0) -> float:
        """records: a (n, 4) float32 device tensor of (x1, x2, target, gate)."""
        assert records.is_cuda and records.dtype == self.torch.float32 and records.is_contiguous()
        loss = C.c_float()
        check(lib().rad_mlp_train(self.ctx, C.c_void_p(records.data_ptr()), records.shape[0],
                                  int(epochs), int(batch), float(lr), int(seed), C.byref(loss)),
              "rad_mlp_train")
        return loss.value

    def mlp_grad(self, records):
        assert records.is_cuda and records.dtype == self.torch.float32 and records.is_contiguous()
        g = np.empty(self.mlp_nparam(), dtype=np.float32)
        loss = C.c_float()
        check(lib().rad_mlp_grad(self.ctx, C.c_void_p(records.data_ptr()), records.shape[0],
                                 C.c_void_p(g.ctypes.data), C.byref(loss)), "rad_mlp_grad")
        return loss.value, g

    def mlp_predict(self, records, tensor_cores: bool = False):
        """Network output for a (n, 4) float32 device tensor of records; on the
        tensor cores (as the queue pass) when tensor_cores is true."""
        out = self.torch.empty(records.shape[0], dtype=self.torch.float32, device=records.device)
        fn = lib().rad_mlp_predict_tc if tensor_cores else lib().rad_mlp_predict
        check(fn(self.ctx, C.c_void_p(records.data_ptr()), records.shape[0],
                 C.c_void_p(out.data_ptr())), "rad_mlp_predict")
        return out

    def log_bind(self, records, stride: int = 1):
        """records: (capacity, 4) float32 device tensor, or None to unbind."""
        if records is None:
            check(lib().rad_log_bind(self.ctx, None, 0, 1), "rad_log_bind")
            self._log = None
            return
        self._log = records
        check(lib().rad_log_bind(self.ctx, C.c_void_p(records.data_ptr()), records.shape[0],
                                 int(stride)), "rad_log_bind")

    def log_count(self) -> int:
        n = C.c_size_t()
        check(lib().rad_log_count(self.ctx, C.byref(n)), "rad_log_count")
        return n.value

    def launches_per_step(self) -> int:
        return lib().rad_launches_per_step(self.ctx)

    def profile_begin(self, max_steps: int):
        """Time the step kernel and the queue pass of the next max_steps steps."""
        check(lib().rad_profile_begin(self.ctx, int(max_steps)), "rad_profile_begin")

    def profile_end(self) -> tuple:
        """(summed step-kernel ms, summed queue-pass ms, steps timed)."""
        a, b, n = C.c_float(), C.c_float(), C.c_int()
        check(lib().rad_profile_end(self.ctx, C.byref(a), C.byref(b), C.byref(n)),
              "rad_profile_end")
        return a.value, b.value, n.value

    def close(self):
        if getattr(self, "ctx", None):
            lib().rad_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RadBatch:
    """Many independent grids (Rad members of one kind) advanced together:
    one persistent launch per step over a shared tile work list, replayed
    from a captured CUDA graph.  The members stay usable for set_gas,
    set_rad and read; they must outlive the batch."""

    def __init__(self, members, use_graph: bool = True):
        import torch
        self.torch = torch
        L = lib()
        self.members = list(members)
        assert self.members, "empty batch"
        self.device = self.members[0].device
        arr = (C.c_void_p * len(self.members))(*[m.ctx for m in self.members])
        b = C.c_void_p()
        check(L.rad_batch_create(arr, len(self.members), C.byref(b)), "rad_batch_create")
        self.b = b
        nbytes = C.c_size_t()
        check(L.rad_batch_workspace_size(b, C.byref(nbytes)), "rad_batch_workspace_size")
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            check(L.rad_batch_set_stream(b, C.c_void_p(self.stream.cuda_stream)),
                  "rad_batch_set_stream")
            self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8,
                                   device=self.device)
            aligned = (self._ws.data_ptr() + 255) // 256 * 256
            check(L.rad_batch_bind_workspace(b, C.c_void_p(aligned), self.workspace_bytes),
                  "rad_batch_bind_workspace")
        check(L.rad_batch_set_graph(b, int(bool(use_graph))), "rad_batch_set_graph")

    def step(self, nsteps: int = 1, dt=None):
        """dt: None (each member's CFL step) or one step length per member."""
        if dt is None:
            check(lib().rad_batch_step(self.b, None, int(nsteps)), "rad_batch_step")
            return
        d = np.ascontiguousarray(np.asarray(dt, dtype=np.float64)).reshape(-1)
        assert d.size == len(self.members)
        check(lib().rad_batch_step(self.b, C.c_void_p(d.ctypes.data), int(nsteps)),
              "rad_batch_step")

    def set_graph(self, use_graph: bool):
        check(lib().rad_batch_set_graph(self.b, int(bool(use_graph))), "rad_batch_set_graph")

    def sync(self) -> int:
        return lib().rad_batch_sync(self.b)

    def stats(self) -> dict:
        s = rad_stats()
        check(lib().rad_batch_get_stats(self.b, C.byref(s)), "rad_batch_get_stats")
        return {k: int(getattr(s, k)) for k, _ in rad_stats._fields_}

    def reset_stats(self):
        check(lib().rad_batch_reset_stats(self.b), "rad_batch_reset_stats")

    def launches_per_step(self) -> int:
        return lib().rad_batch_launches_per_step(self.b)

    def set_launch(self, variant: int, chunk: int = 0):
        check(lib().rad_batch_set_launch(self.b, int(variant), int(chunk)), "rad_batch_set_launch")

    def get_launch(self) -> tuple:
        v, c, n, k = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        check(lib().rad_batch_get_launch(self.b, C.byref(v), C.byref(c), C.byref(n), C.byref(k)),
              "rad_batch_get_launch")
        return v.value, c.value, n.value, k.value

    def tune(self, reps: int = 3) -> tuple:
        v, c, t = C.c_int(), C.c_int(), C.c_float()
        check(lib().rad_batch_tune(self.b, int(reps), C.byref(v), C.byref(c), C.byref(t)),
              "rad_batch_tune")
        return v.value, c.value, t.value

    def mlp_set(self, params):
        arr = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        check(lib().rad_batch_mlp_set(self.b, C.c_void_p(arr.ctypes.data), arr.size),
              "rad_batch_mlp_set")

    def close(self):
        if getattr(self, "b", None):
            lib().rad_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_problem(prob, precision: str = "fp64", device=None, **overrides) -> "Rad":
    """Builds a Rad from any object with the attributes of a problem
    description (ndim, n, geometry, bc_lo, bc_hi, xfaces, chat, c, a_rad,
    gamma_gas, mu, cfl, e_floor, opacity, implicit_mode, newton_rtol,
    newton_maxit, ncomp) and uploads its fields (rho, v, T, E, F)."""
    params = dict(chat=prob.chat, c=prob.c, a_rad=prob.a_rad, gamma_gas=prob.gamma_gas,
                  mu=prob.mu, cfl=prob.cfl, e_floor=prob.e_floor, precision=precision,
                  implicit_mode=prob.implicit_mode, newton_rtol=prob.newton_rtol,
                  newton_maxit=prob.newton_maxit, ncomp=prob.ncomp,
                  integrator=getattr(prob, "integrator", "euler"),
                  irradiation=int(getattr(prob, "qirr", None) is not None),
                  reconstruction=getattr(prob, "recon", "plm"),
                  face_fix=getattr(prob, "face_fix", "fpreserve"),
                  riemann=getattr(prob, "riemann", "hll"),
                  hydro=int(bool(getattr(prob, "hydro", False))))
    params.update(overrides)
    grid = dict(ndim=prob.ndim, n=prob.n, xfaces=prob.xfaces, bc_lo=prob.bc_lo, bc_hi=prob.bc_hi,
                bc_value=dict(getattr(prob, "bc_value", {})))
    r = Rad(grid, prob.geometry, prob.opacity, params, device=device)
    nc = prob.ncomp
    r.set_gas(prob.rho, np.asarray(prob.v)[:nc], prob.T)
    r.set_rad(prob.E, np.asarray(prob.F)[:nc])
    if getattr(prob, "qirr", None) is not None:
        r.set_irradiation(prob.qirr)
    return r
