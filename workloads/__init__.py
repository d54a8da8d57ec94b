"""Seeded synthetic inputs for the M1 radiation step.

This module only builds inputs: grids, gas fields (rho, v, T), radiation
fields (E, F), opacity descriptions and physical constants.  It contains none
of the method's arithmetic, and both the CUDA library's tests/benchmark and
the CPU oracle consume it.

Random fields use numpy's PCG64 generator with the seeds listed per workload.
A "Gaussian random field with spectrum k^-11/3" is white noise filtered in
Fourier space so that |g_hat(k)|^2 ~ |k|^-11/3, with the k = 0 mode zeroed and
the result normalised to zero mean and unit variance.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

GEOMETRIES = ("cartesian", "cylindrical", "spherical")
BCS = ("outflow", "periodic")


@dataclasses.dataclass
class Problem:
    """A radiation-step problem: grid, constants, opacity model and fields.

    Fields are flat float64 arrays of N = n0*n1*n2 cells, x fastest.  `v` and
    `F` are (3, N); components beyond `ncomp` are zero.
    """
    name: str
    ndim: int
    n: Tuple[int, int, int]
    geometry: str
    bc_lo: Tuple[str, str, str]
    bc_hi: Tuple[str, str, str]
    xfaces: List[np.ndarray]
    chat: float
    c: float
    a_rad: float = 1.0
    gamma_gas: float = 5.0 / 3.0
    mu: float = 1.0
    cfl: float = 0.4
    e_floor: float = 1e-30
    opacity: Dict = dataclasses.field(default_factory=lambda: {"kind": "const", "kappa_p": 0.0,
                                                               "kappa_r": 0.0, "sigma": 0.0})
    implicit_mode: str = "once"
    integrator: str = "euler"     # "euler" or "rk2" (two-stage, Sect. 2.4)
    qirr: Optional[np.ndarray] = None  # -div F_irr per cell (Sect. 2.9), or None
    # options of Sect. 2.5: "plm" | "limo3"; "fpreserve" | "pluto" | "clip";
    # "hll" | "lf"
    recon: str = "plm"
    face_fix: str = "fpreserve"
    riemann: str = "hll"
    # boundary states of "fixed" and "lte" sides: {(d, side): (E, F0, F1, F2, T)},
    # side 0 = lower, 1 = upper ("lte" uses T only)
    bc_value: Dict = dataclasses.field(default_factory=dict)
    # evolve the gas with a hydrodynamic step before the radiation transport
    # (Cartesian grids)
    hydro: bool = False
    newton_rtol: float = 1e-12
    newton_maxit: int = 50
    ncomp: int = 3
    rho: Optional[np.ndarray] = None
    v: Optional[np.ndarray] = None
    T: Optional[np.ndarray] = None
    E: Optional[np.ndarray] = None
    F: Optional[np.ndarray] = None
    nsteps: int = 1
    precision: str = "fp64"

    @property
    def N(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def copy(self) -> "Problem":
        p = dataclasses.replace(self)
        for k in ("rho", "v", "T", "E", "F"):
            a = getattr(self, k)
            setattr(p, k, None if a is None else a.copy())
        p.xfaces = [x.copy() for x in self.xfaces]
        p.opacity = dict(self.opacity)
        p.bc_value = dict(self.bc_value)
        return p


# ---------------------------------------------------------------------------
# grids
# ---------------------------------------------------------------------------

def uniform_faces(n: int, lo: float, hi: float) -> np.ndarray:
    return np.linspace(lo, hi, n + 1, dtype=np.float64)


def log_faces(n: int, lo: float, hi: float) -> np.ndarray:
    return np.exp(np.linspace(math.log(lo), math.log(hi), n + 1, dtype=np.float64))


def default_extent(geometry: str, d: int) -> Tuple[float, float]:
    """Extent of an inactive direction: unit length, or the full angle."""
    if geometry == "cylindrical" and d == 1:
        return (0.0, 2.0 * math.pi)
    if geometry == "spherical" and d == 1:
        return (0.0, math.pi)
    if geometry == "spherical" and d == 2:
        return (0.0, 2.0 * math.pi)
    return (0.0, 1.0)


def make_faces(geometry: str, n: Sequence[int], extents: Sequence[Optional[Tuple[float, float]]],
               log_r: bool = False) -> List[np.ndarray]:
    out = []
    for d in range(3):
        ext = extents[d] if d < len(extents) and extents[d] is not None else default_extent(geometry, d)
        if d == 0 and log_r:
            out.append(log_faces(n[d], ext[0], ext[1]))
        else:
            out.append(uniform_faces(n[d], ext[0], ext[1]))
    return out


def cell_centres(xf: np.ndarray) -> np.ndarray:
    return 0.5 * (xf[:-1] + xf[1:])


def mesh(p: Problem) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Cell-centre coordinates broadcast to flat N arrays (x fastest)."""
    c = [cell_centres(p.xfaces[d]) for d in range(3)]
    z, y, x = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


# ---------------------------------------------------------------------------
# random fields
# ---------------------------------------------------------------------------

def gaussian_random_field(shape: Sequence[int], seed: int, slope: float = -11.0 / 3.0) -> np.ndarray:
    """Unit-variance Gaussian random field with |g_hat(k)|^2 ~ |k|^slope.

    `shape` is given slowest-first (numpy order); the result is flat, x
    fastest.  Periodic by construction.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(int(s) for s in shape)
    noise = rng.standard_normal(shape)
    spec = np.fft.rfftn(noise)
    ks = [np.fft.fftfreq(s) * s for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1]) * shape[-1]]
    grids = np.meshgrid(*ks, indexing="ij")
    k2 = sum(g * g for g in grids)
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # |k|^(slope/2) on the amplitude
    g = np.fft.irfftn(spec * amp, s=shape, axes=tuple(range(len(shape))))
    g -= g.mean()
    g /= g.std()
    return g.ravel().astype(np.float64)


def lognormal_density(shape, seed: int, sigma_ln: float = 1.0) -> np.ndarray:
    """rho = exp(sigma g - sigma^2/2): log-normal with mean 1 and log-std sigma."""
    g = gaussian_random_field(shape, seed)
    return np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)


def random_velocity(shape, seeds: Sequence[int], vrms: float, ncomp: int) -> np.ndarray:
    """Velocity with each of the first len(seeds) components a random field,
    scaled so that the rms of |v| is vrms."""
    N = int(np.prod(shape))
    v = np.zeros((3, N))
    for q, s in enumerate(seeds):
        v[q] = gaussian_random_field(shape, s)
    rms = math.sqrt(float(np.mean(np.sum(v * v, axis=0))))
    if rms > 0:
        v *= vrms / rms
    return v


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def _blank(name, ndim, n, geometry, bc, xfaces, chat, c=None, ncomp=3, **kw) -> Problem:
    bc3 = tuple(bc) if isinstance(bc, (tuple, list)) else (bc, bc, bc)
    return Problem(name=name, ndim=ndim, n=tuple(int(x) for x in n), geometry=geometry,
                   bc_lo=bc3, bc_hi=bc3, xfaces=xfaces, chat=float(chat),
                   c=float(chat if c is None else c), ncomp=ncomp, **kw)


def pulse_1d(n: int = 512, nsteps: int = 200) -> Problem:
    """1D Cartesian Gaussian pulse in a static gas: rho = 1, v = 0, T = 1,
    kappa_a rho = 1, no scattering, E = 1e-4 + exp(-(x-0.5)^2/(2 0.05^2)),
    F = 0, chat = c = 100, CFL 0.4, outflow, FP64."""
    xf = make_faces("cartesian", (n, 1, 1), [(0.0, 1.0)])
    p = _blank("pulse1d_%d" % n, 1, (n, 1, 1), "cartesian", "outflow", xf, chat=100.0, ncomp=1,
               opacity={"kind": "const", "kappa_p": 1.0, "kappa_r": 1.0, "sigma": 0.0},
               nsteps=nsteps)
    x, _, _ = mesh(p)
    p.rho = np.ones(p.N)
    p.v = np.zeros((3, p.N))
    p.T = np.ones(p.N)
    p.E = 1e-4 + np.exp(-(x - 0.5) ** 2 / (2 * 0.05 ** 2))
    p.F = np.zeros((3, p.N))
    return p


def turbulent_2d(n: Tuple[int, int] = (1024, 1024), nsteps: int = 100, seed_base: int = 1,
                 nonequilibrium: bool = False, kappa_scale: float = 1.0) -> Problem:
    """2D periodic box: log-normal density (sigma_ln = 1, k^-11/3, seed 1),
    random velocity with rms 0.1 (seeds 2, 3), kappa_a = kappa0 rho,
    sigma = 0.3 kappa_a, kappa0 chosen so that the median cell optical depth
    rho (kappa_a + sigma) dx is 1 (times kappa_scale), T = 1, E = T^4 (a_R = 1),
    F = 0, chat = c = 50.  With nonequilibrium=True, E = (1 + 0.5 g4)^4
    clipped at 1e-4 (seed 4) instead."""
    nx, ny = n
    xf = make_faces("cartesian", (nx, ny, 1), [(0.0, 1.0), (0.0, 1.0)])
    p = _blank("turb2d_%dx%d%s" % (nx, ny, "_neq" if nonequilibrium else ""), 2, (nx, ny, 1),
               "cartesian", "periodic", xf, chat=50.0, ncomp=2, nsteps=nsteps)
    shape = (ny, nx)
    p.rho = lognormal_density(shape, seed_base + 0, 1.0)
    p.v = random_velocity(shape, [seed_base + 1, seed_base + 2], 0.1, 2)
    dx = 1.0 / max(nx, ny)
    kappa0 = kappa_scale / (1.3 * float(np.median(p.rho * p.rho)) * dx)
    p.opacity = {"kind": "powerlaw", "k0": kappa0, "a_rho": 1.0, "b_T": 0.0, "kmin": 0.0,
                 "kmax": 1e300, "sigma_ratio": 0.3}
    p.T = np.ones(p.N)
    if nonequilibrium:
        g4 = gaussian_random_field(shape, seed_base + 3)
        p.E = np.maximum((1.0 + 0.5 * g4) ** 4, 1e-4)
    else:
        p.E = np.ones(p.N)
    p.F = np.zeros((3, p.N))
    return p


def hot_sphere_3d(n: int = 256, nsteps: int = 100, ns: Optional[Tuple[int, int, int]] = None) -> Problem:
    """3D periodic box: the 2D recipe in 3D (density seed 5, velocity seeds
    6-8), hot sphere |x - 1/2| < 0.1 at T = 10, T = 1 elsewhere, E = T^4,
    F = 0, Kramers-like kappa = clip(rho T^-3.5, 1e-4, 1e4), no scattering,
    chat = c = 30."""
    nx, ny, nz = ns if ns is not None else (n, n, n)
    xf = make_faces("cartesian", (nx, ny, nz), [(0.0, 1.0)] * 3)
    p = _blank("hotsphere3d_%dx%dx%d" % (nx, ny, nz), 3, (nx, ny, nz), "cartesian", "periodic",
               xf, chat=30.0, ncomp=3, nsteps=nsteps)
    shape = (nz, ny, nx)
    p.rho = lognormal_density(shape, 5, 1.0)
    p.v = random_velocity(shape, [6, 7, 8], 0.1, 3)
    x, y, z = mesh(p)
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    p.T = np.where(r < 0.1, 10.0, 1.0)
    p.E = p.T ** 4
    p.F = np.zeros((3, p.N))
    p.opacity = {"kind": "powerlaw", "k0": 1.0, "a_rho": 1.0, "b_T": -3.5, "kmin": 1e-4,
                 "kmax": 1e4, "sigma_ratio": 0.0}
    return p


def opacity_table(nrho: int = 128, nT: int = 128, seed: int = 10, kK: float = 1e6,
                  kes: float = 0.35) -> Dict:
    """Synthetic 2D opacity table over log10 rho in [-12, 0] and log10 T in
    [0, 6]: kappa = (kK rho T^-3.5 + kes) (1 + 0.01 eps), eps ~ N(0, 1) per
    node (seed 10); stored as float32 log10 kappa, rho fastest."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lr = np.linspace(-12.0, 0.0, nrho)
    lt = np.linspace(0.0, 6.0, nT)
    LT, LR = np.meshgrid(lt, lr, indexing="ij")
    kap = (kK * 10.0 ** LR * 10.0 ** (-3.5 * LT) + kes) * (1.0 + 0.01 * rng.standard_normal(LT.shape))
    return {"kind": "table", "nrho": nrho, "nT": nT, "lrho0": -12.0, "lrho1": 0.0, "lT0": 0.0,
            "lT1": 6.0, "table": np.log10(kap).astype(np.float32).ravel(), "sigma_ratio": 0.0}


def disk_spherical(n: Tuple[int, int, int] = (192, 128, 256), nsteps: int = 50) -> Problem:
    """3D spherical (r, theta, phi): r log-spaced on [1, 100], theta in
    [pi/6, 5pi/6], phi in [0, 2pi) periodic, outflow in r and theta.
    rho = r^-1.5 exp(-cos^2 theta / (2 0.1^2)) exp(0.3 g - 0.045) (seed 9),
    v_phi = (r sin theta)^-1/2, T = 1000 r^-1/2, E = a_R T^4, F = 0, tabulated
    opacity, chat = c = 20.  a_R = 1e-12 in these code units, so that the
    radiation energy is 1e-3 of the gas energy in the midplane at r = 1, as in
    a protoplanetary disk (with a_R = 1 and T = 1000 the radiation would
    exceed the gas energy by 1e9, and its pressure would drive the gas
    internal energy negative within a few steps)."""
    nr, nth, nph = n
    xf = [log_faces(nr, 1.0, 100.0), uniform_faces(nth, math.pi / 6, 5 * math.pi / 6),
          uniform_faces(nph, 0.0, 2 * math.pi)]
    p = _blank("disk_sph_%dx%dx%d" % n, 3, n, "spherical",
               ("outflow", "outflow", "periodic"), xf, chat=20.0, ncomp=3, nsteps=nsteps)
    r, th, _ = mesh(p)
    g = gaussian_random_field((nph, nth, nr), 9)
    p.rho = r ** -1.5 * np.exp(-np.cos(th) ** 2 / (2 * 0.1 ** 2)) * np.exp(0.3 * g - 0.045)
    p.v = np.zeros((3, p.N))
    p.v[2] = (r * np.sin(th)) ** -0.5
    p.T = 1000.0 * r ** -0.5
    p.a_rad = 1e-12
    p.E = p.a_rad * p.T ** 4
    p.F = np.zeros((3, p.N))
    p.opacity = opacity_table()
    return p


def batched_2d(count: int = 64, seed: int = 11, kappa_seed: int = 12, nsteps: int = 100,
               lo: int = 64, hi: int = 512) -> List[Problem]:
    """`count` independent 2D periodic instances of the turbulent recipe with
    sizes log-uniform in [lo, hi] rounded to 16 (seed 11) and kappa0 scale
    log-uniform in [1e-2, 1e2] (seed 12); instance i uses seeds 100 + 4 i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), count))
    sizes = np.clip((np.round(sizes / 16.0) * 16).astype(int), lo, hi)
    krng = np.random.Generator(np.random.PCG64(kappa_seed))
    kscale = 10.0 ** krng.uniform(-2.0, 2.0, count)
    out = []
    for i in range(count):
        p = turbulent_2d((int(sizes[i]), int(sizes[i])), nsteps=nsteps, seed_base=100 + 4 * i,
                         kappa_scale=float(kscale[i]))
        p.name = "batch%02d_%d" % (i, sizes[i])
        out.append(p)
    return out


# ---------------------------------------------------------------------------
# test problems (Sect. 3 of the paper)
# ---------------------------------------------------------------------------

def shock_tube(which: int, n: int, t_end: float = 20.0) -> Problem:
    """Optically thin 1D Riemann problems on x in [-20, 20] (Sect. 3.1).
    The caller fills the left/right states.  Zero opacity, outflow."""
    xf = make_faces("cartesian", (n, 1, 1), [(-20.0, 20.0)])
    p = _blank("tube%d_%d" % (which, n), 1, (n, 1, 1), "cartesian", "outflow", xf, chat=1.0,
               ncomp=3)
    p.rho = np.ones(p.N)
    p.v = np.zeros((3, p.N))
    p.T = np.full(p.N, 1e-3)
    p.E = np.ones(p.N)
    p.F = np.zeros((3, p.N))
    p.opacity = {"kind": "const", "kappa_p": 0.0, "kappa_r": 0.0, "sigma": 0.0}
    return p


# cgs constants for the shadow test
C_LIGHT = 2.99792458e10
A_RAD = 7.5657e-15
KB_OVER_MU = 8.314462618e7   # k_B / m_u in erg / (g K)


def shadow(n: Tuple[int, int] = (140, 40), coupling: str = "absorb") -> Problem:
    """The shadow test of Sect. 3 (cgs): box x in [-0.5, 0.5], y in [0, 0.3]
    cm, spheroid of rho_1 = 1e3 at the origin in a background rho_0 = 1,
    rho = rho_0 + (rho_1 - rho_0) / (1 + e^D), D = 10 ((x/0.1)^2 +
    (y/0.06)^2 - 1); T = 290 K everywhere with E = a T^4 and F = v = 0;
    Kramers kappa = 0.1 (rho/rho_0) (T/290)^-3.5 cm^2/g, no scattering.  A
    beam at T_r = 1740 K with F_x = E enters through the left side (fixed
    boundary state, ghost gas at 290 K); the lower side y = 0 is reflective,
    the right and upper sides are outflow.  chat = c; mu = 1 and Gamma = 5/3
    (the paper gives neither).  coupling "absorb" drops the emission by the
    gas (the paper's first panel), "once" keeps the full coupling."""
    nx, ny = n
    xf = [uniform_faces(nx, -0.5, 0.5), uniform_faces(ny, 0.0, 0.3), uniform_faces(1, 0.0, 1.0)]
    p = _blank("shadow_%dx%d" % (nx, ny), 2, (nx, ny, 1), "cartesian", "outflow", xf,
               chat=C_LIGHT, ncomp=2, implicit_mode=coupling)
    p.bc_lo = ("fixed", "reflective", "outflow")
    p.bc_hi = ("outflow", "outflow", "outflow")
    p.a_rad = A_RAD
    p.mu = 1.0 / KB_OVER_MU
    p.gamma_gas = 5.0 / 3.0
    Eb = A_RAD * 1740.0 ** 4
    p.bc_value = {(0, 0): (Eb, Eb, 0.0, 0.0, 290.0)}
    x, y, _ = mesh(p)
    D = 10.0 * ((x / 0.1) ** 2 + (y / 0.06) ** 2 - 1.0)
    p.rho = 1.0 + (1e3 - 1.0) / (1.0 + np.exp(np.minimum(D, 700.0)))
    p.v = np.zeros((3, p.N))
    p.T = np.full(p.N, 290.0)
    p.E = A_RAD * p.T ** 4
    p.F = np.zeros((3, p.N))
    p.opacity = {"kind": "powerlaw", "k0": 0.1 * 290.0 ** 3.5, "a_rho": 1.0, "b_T": -3.5,
                 "kmin": 0.0, "kmax": 1e300, "sigma_ratio": 0.0}
    return p


def pulse_3d_rhd(n: int = 256, nsteps: int = 20) -> Problem:
    """The paper's performance workload (Sect. 4): the Cartesian pulse test
    of Sect. 3 with the gas evolved and the two-stage step.  Box [-50, 50]^3,
    rho = 1, v = 0, gas at T0, E = a T_r^4 with T_r = T0 (1 + 100 e^(-r^2/w^2)),
    w = 5, F = 0, no absorption, scattering only (optically thin), Gamma =
    5/3, chat = c = 1 (velocity unit c), CFL 0.4, outflow.  The paper's T0
    and units leave the radiation and gas energies unspecified; here T0 =
    1e-6 (sound speed ~1e-3 c) and a_R = 1e8 put the pulse's peak energy at
    1e-2 of the gas energy, so that the gas stays nearly static as in the
    paper's run, and keep E^2 inside FP32's normal range."""
    xf = make_faces("cartesian", (n, n, n), [(-50.0, 50.0)] * 3)
    p = _blank("rhd_pulse3d_%d" % n, 3, (n, n, n), "cartesian", "outflow", xf, chat=1.0,
               ncomp=3, nsteps=nsteps, integrator="rk2", hydro=True)
    T0 = 1e-6
    p.a_rad = 1e8
    x, y, z = mesh(p)
    r2 = x * x + y * y + z * z
    p.rho = np.ones(p.N)
    p.v = np.zeros((3, p.N))
    p.T = np.full(p.N, T0)
    p.E = p.a_rad * (T0 * (1.0 + 100.0 * np.exp(-r2 / 25.0))) ** 4
    p.F = np.zeros((3, p.N))
    p.opacity = {"kind": "const", "kappa_p": 0.0, "kappa_r": 0.0, "sigma": 1e-6}
    return p


def beam_2d(n: int = 300, recon: str = "plm", face_fix: str = "fpreserve") -> Tuple[Problem, np.ndarray]:
    """The free-streaming beam of Sect. 3: square [0, 5]^2, E = 1e4, F = 0, no
    opacity, outflow, chat = c = 1, CFL 0.4, HLL.  The beam region x in
    [0.5, 0.6], y in [0.3, 0.44] holds E = 1e12 and F = E (1, 1) / sqrt(2)
    (f = 1 along the diagonal); the caller re-imposes it after every step.
    Returns the problem and the boolean mask of the beam region."""
    xf = make_faces("cartesian", (n, n, 1), [(0.0, 5.0), (0.0, 5.0)])
    p = _blank("beam_%d" % n, 2, (n, n, 1), "cartesian", "outflow", xf, chat=1.0, ncomp=2,
               recon=recon, face_fix=face_fix)
    x, y, _ = mesh(p)
    mask = (x >= 0.5) & (x <= 0.6) & (y >= 0.3) & (y <= 0.44)
    # the paper's beam does not touch the gas; a heavy gas keeps the momentum
    # that the |F| <= E clip after the transport hands to it negligible
    p.rho = np.full(p.N, 1e20)
    p.v = np.zeros((3, p.N))
    p.T = np.ones(p.N)
    p.E = np.where(mask, 1e12, 1e4)
    p.F = np.zeros((3, p.N))
    p.F[0] = p.F[1] = np.where(mask, 1e12 / math.sqrt(2.0), 0.0)
    p.opacity = {"kind": "const", "kappa_p": 0.0, "kappa_r": 0.0, "sigma": 0.0}
    return p, mask


def radiative_shock(n: int = 1000, v_kms: float = 6.0, chat_over_c: float = 1e-3) -> Problem:
    """The radiative shocks of Sect. 3 (cgs): x in [0, 7e10] cm, rho =
    7.78e-10, T = 10 K with E = a T^4, mu = 1, Gamma = 7/5, absorption
    kappa = 0.39 cm^2/g, no scattering, gas moving at -v (6 km/s:
    subcritical, 20 km/s: supercritical) towards the reflective wall at x = 0,
    outflow at the far side, HLL, PLM f-preserving, RK2, chat = c x
    chat_over_c."""
    xf = [uniform_faces(n, 0.0, 7e10), uniform_faces(1, 0.0, 1.0), uniform_faces(1, 0.0, 1.0)]
    p = _blank("radshock_%d_v%g" % (n, v_kms), 1, (n, 1, 1), "cartesian", "outflow", xf,
               chat=C_LIGHT * chat_over_c, c=C_LIGHT, ncomp=1, integrator="rk2", hydro=True)
    p.bc_lo = ("reflective", "outflow", "outflow")
    p.a_rad = A_RAD
    p.mu = 1.0 / KB_OVER_MU
    p.gamma_gas = 7.0 / 5.0
    p.rho = np.full(p.N, 7.78e-10)
    p.v = np.zeros((3, p.N))
    p.v[0] = -v_kms * 1e5
    p.T = np.full(p.N, 10.0)
    p.E = A_RAD * p.T ** 4
    p.F = np.zeros((3, p.N))
    p.opacity = {"kind": "const", "kappa_p": 0.39, "kappa_r": 0.39, "sigma": 0.0}
    return p


def uniform_state(geometry: str, n: Tuple[int, int, int], ndim: int, log_r: bool = False,
                  extents=None, E: float = 2.0, kappa: float = 0.5) -> Problem:
    """A uniform isotropic state (E const, F = 0) in equilibrium with the gas
    (E = a T^4) on any geometry: it must stay uniform."""
    if extents is None:
        if geometry == "cartesian":
            extents = [(0.0, 1.0)] * 3
        elif geometry == "cylindrical":
            extents = [(0.5, 2.0), (0.0, 2.0 * math.pi), (0.0, 1.0)]
        else:
            extents = [(1.0, 10.0), (0.3, math.pi - 0.3), (0.0, 2.0 * math.pi)]
    nn = tuple(n[d] if d < ndim else 1 for d in range(3))
    ext = [extents[d] if d < ndim else default_extent(geometry, d) for d in range(3)]
    xf = make_faces(geometry, nn, ext, log_r=log_r)
    p = _blank("uniform_%s_%dd" % (geometry, ndim), ndim, nn, geometry, "outflow", xf, chat=1.0,
               ncomp=3)
    p.rho = np.ones(p.N)
    p.v = np.zeros((3, p.N))
    p.T = np.full(p.N, E ** 0.25)
    p.E = np.full(p.N, E)
    p.F = np.zeros((3, p.N))
    p.opacity = {"kind": "const", "kappa_p": kappa, "kappa_r": kappa, "sigma": 0.0}
    return p


def random_smooth(geometry: str, n: Tuple[int, int, int], ndim: int, seed: int,
                  bc: str = "outflow", opacity: Optional[Dict] = None, log_r: bool = False,
                  chat: float = 3.0, c: Optional[float] = None, fmax: float = 0.9,
                  ncomp: int = 3, extents=None) -> Problem:
    """Generic seeded test state: smooth positive E with large contrasts,
    random F with |F| <= fmax E, random rho, v, T.  Used by parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if extents is None:
        if geometry == "cartesian":
            extents = [(0.0, 1.0), (0.0, 0.8), (0.0, 0.6)]
        elif geometry == "cylindrical":
            extents = [(0.5, 2.0), (0.0, 1.0), (0.0, 1.0)]
        else:
            extents = [(1.0, 4.0), (0.4, math.pi - 0.4), (0.0, 1.2)]
    nn = tuple(n[d] if d < ndim else 1 for d in range(3))
    ext = [extents[d] if d < ndim else default_extent(geometry, d) for d in range(3)]
    xf = make_faces(geometry, nn, ext, log_r=log_r)
    bc3 = tuple(bc if d < ndim else "outflow" for d in range(3))
    p = Problem(name="rand_%s_%dd_s%d" % (geometry, ndim, seed), ndim=ndim, n=nn,
                geometry=geometry, bc_lo=bc3, bc_hi=bc3, xfaces=xf, chat=float(chat),
                c=float(chat if c is None else c), ncomp=ncomp)
    N = p.N
    shape = tuple(reversed(nn))
    g1 = rng.standard_normal(shape)
    # smooth by a few passes of neighbour averaging (periodic) to get structure
    for _ in range(3):
        acc = g1.copy()
        for ax in range(len(shape)):
            if shape[ax] > 1:
                acc += np.roll(g1, 1, axis=ax) + np.roll(g1, -1, axis=ax)
        g1 = acc / (1 + 2 * sum(1 for s in shape if s > 1))
    g1 = (g1 - g1.mean()) / (g1.std() + 1e-300)
    p.E = np.exp(1.5 * g1).ravel()
    u = rng.standard_normal((3, N))
    u[ncomp:] = 0.0
    nu = np.sqrt(np.sum(u * u, axis=0)) + 1e-300
    frac = fmax * rng.uniform(0.0, 1.0, N)
    p.F = u / nu * frac * p.E
    p.rho = np.exp(0.5 * rng.standard_normal(N))
    p.v = 0.1 * rng.standard_normal((3, N))
    p.v[ncomp:] = 0.0
    p.T = np.exp(0.3 * rng.standard_normal(N)) * np.mean(p.E) ** 0.25
    p.opacity = opacity if opacity is not None else {"kind": "const", "kappa_p": 0.7,
                                                     "kappa_r": 0.9, "sigma": 0.4}
    return p
