/*
 * m1_oracle.c -- plain, slow, FP64 CPU oracle of one radiation step of the
 * gray M1 module of Scepi & Lesur, "A nonrelativistic radiative transfer
 * module for Idefix" (arxiv 2606.26268).
 *
 * TEST INFRASTRUCTURE ONLY.  The CUDA path is checked against this file: only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (one explicit Euler step, Sect. 2.4 "Integration scheme",
 * items 1-10, followed literally and cell by cell):
 *   1. boundary values by index mapping (outflow = copy of the nearest
 *      interior cell, periodic = wrap, reflective = mirror with the normal
 *      flux negated) or from a boundary state (fixed injection, LTE);
 *   3. PLM reconstruction with the van Leer limiter, or LimO3 (Sect. 2.5);
 *   4. the f-preserving face fix, Eq. (f_reconstruct), or the flat
 *      ("PLUTO") or clipping treatment of f_face > 1 (Sect. 2.5);
 *   5. signal speeds lambda_{1,3}, Sect. 2.6, with the optically thick
 *      correction of the same section;
 *   6. the HLL flux, or the Lax-Friedrichs-Rusanov flux (Sect. 2.5);
 *   7. finite-volume flux divergence with Cartesian, cylindrical or spherical
 *      metric (orthonormal components);
 *   0. with `hydro`: a hydrodynamic step of the gas first (Sect. 2.4 orders
 *      the substep as gas, radiation transport, radiation sources): PLM on
 *      primitive variables, HLL with the Davis speeds, Cartesian divergence;
 *      the radiation transport then takes its optical depths, and the
 *      coupling its gas, from the gas after that step;
 *   8. the implicit matter-radiation coupling of Sect. 2.8, Eqs.
 *      (source_discrete2) and (implicit_matrix), optionally iterated to
 *      convergence (Newton mode) or reduced to absorption only (the shadow
 *      test of Sect. 3), and the gas energy / momentum from the rescaled
 *      conservation laws of Sect. 2.7;
 *  10. the CFL time step.
 * Primitive and conservative radiation variables are identical (Sect. 2.4),
 * so items 2 and 9 are the identity.
 *
 * Readings where the paper is silent (each is restated in the design notes):
 *   - f-fix: keep the reconstructed face flux iff f_face <= 1 and
 *     f_face > f_center (the inequality of Eq. f_reconstruct), else
 *     F_face = F_center * (E_face / E_center).
 *   - PLM on stretched grids: one-sided differences divided by centre
 *     distances, van Leer harmonic mean, face = u_c + s (x_face - x_c),
 *     cell centre = midpoint of its faces.
 *   - tau at a face: mean of rho*chi*dx of the two adjacent cells, dx = the
 *     largest physical width of the cell over the active directions.
 *   - transport is unsplit (every direction sees U^n).
 *   - dt = cfl / max_cells sum_d (chat / h_d).
 *   - metric terms: well-balanced finite-volume forms, angular-momentum
 *     conserving form for the phi component.  An inactive direction is one
 *     cell whose two faces carry the cell's own physical flux.
 *   - C_v = rho / (mu (Gamma - 1)) per unit volume; e = C_v T.
 *   - opacities frozen at (rho, T^n) for the whole step.
 *   - E floor after transport and after the coupling; |F| <= E clip after
 *     the coupling; gas bookkeeping uses the final E and F.
 *   - LimO3: the limiter of orc_limo3 on index-space differences, without
 *     the smooth-extremum switch of its authors.
 *   - PLUTO treatment and clipping act on one face state at a time;
 *     LF-Rusanov takes S = max(|S_L|, |S_R|) after the thick-limit bound.
 *   - absorption only: E^{n+1} = E* / (1 + g_r), gas energy by
 *     conservation, F as in every mode.
 *   - fixed and LTE ghosts carry the edge cell's density and the side's
 *     boundary temperature T_b (e = C_v T_b); fixed ghosts E and F of the
 *     boundary state, LTE ghosts E = a T_b^4 and the edge cell's F.
 * Parity status: every step above is pinned by the oracle tests (closed
 * forms, invariants, brute force and printed values of the paper); the whole
 * step has no printed reference values, so end-to-end parity of full configs
 * rests on those pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_CART = 0, ORC_CYL = 1, ORC_SPH = 2 };
enum { ORC_BC_OUTFLOW = 0, ORC_BC_PERIODIC = 1, ORC_BC_REFLECT = 2, ORC_BC_FIXED = 3, ORC_BC_LTE = 4 };
enum { ORC_OPAC_CONST = 0, ORC_OPAC_POWERLAW = 1, ORC_OPAC_TABLE = 2 };
enum { ORC_ONCE = 0, ORC_NEWTON = 1, ORC_ABSORB = 2 };
enum { ORC_PLM = 0, ORC_LIMO3 = 1 };
enum { ORC_FIX_FPRESERVE = 0, ORC_FIX_PLUTO = 1, ORC_FIX_CLIP = 2 };
enum { ORC_HLL = 0, ORC_LF = 1 };
enum { ORC_EULER = 0, ORC_RK2 = 1 };

/* Problem description.  Face coordinates xf[d] hold n[d]+1 values; for an
 * inactive direction n[d] = 1 and xf[d] gives its extent. */
typedef struct {
  int ndim;
  int n[3];
  int geom;
  int bc_lo[3], bc_hi[3];
  const double *xf[3];
  /* physics, code units */
  double chat, c, a_rad, gamma_gas, mu, cfl, e_floor;
  /* opacity */
  int opac_kind;
  double kappa_p, kappa_r, sigma;             /* CONST, per unit mass */
  double k0, a_rho, b_T, kmin, kmax;          /* POWERLAW */
  double sigma_ratio;                         /* POWERLAW and TABLE */
  int nrho, nT;
  double lrho0, lrho1, lT0, lT1;
  const double *ltable;                       /* log10 kappa, [iT][irho] */
  /* implicit step */
  int implicit_mode;
  double newton_rtol;
  int newton_maxit;
  int nthreads;
  /* time integration: ORC_EULER (one transport + coupling step) or ORC_RK2
   * (two such stages, then the average of the conserved variables) */
  int integrator;
  /* irradiation (Sect. 2.9): energy deposited per unit volume and time,
   * -div F_irr, per cell (NULL: none) */
  const double *qirr;
  /* options of Sect. 2.5: reconstruction (ORC_PLM, ORC_LIMO3), the f <= 1
   * treatment of face states (ORC_FIX_*) and the Riemann solver (ORC_HLL,
   * ORC_LF) */
  int recon, face_fix, riemann;
  /* boundary states of the ORC_BC_FIXED and ORC_BC_LTE sides:
   * bc_val[d][side] = (E, F0, F1, F2, T), side 0 = lower, 1 = upper; FIXED
   * uses E, F and T, LTE only T (E = a T^4, F copied from the edge cell) */
  double bc_val[3][2][5];
  /* 1: the gas is evolved too (Cartesian grids): a hydrodynamic step before
   * the radiation transport in every (sub)step, Sect. 2.4 */
  int hydro;
  /* 1: a host emulation, not the definition: the coupling with the products
   * that the CUDA library's split precision forms in float rounded to float
   * (see couple_float), so that their share of the split form's error can be
   * measured apart from the FP32 transport.  0 (the default): FP64 as
   * defined. */
  int float_coupling;
} orc_problem;

/* State: SoA arrays of N = n0 n1 n2 cells, x fastest.  Three flux and three
 * momentum components are always carried. */
typedef struct {
  double *E, *F0, *F1, *F2, *rho, *e, *m0, *m1, *m2;
} orc_state;

/* Counters, summed over cells and steps. */
enum {
  ORC_ST_FIX = 0,      /* face states where the f-fix recomputed F */
  ORC_ST_EFLOOR = 1,   /* E floor applications */
  ORC_ST_FCLIP = 2,    /* |F| <= E clips after the coupling */
  ORC_ST_ITERS = 3,    /* coupling iterations (sum) */
  ORC_ST_ITMAX = 4,    /* coupling iterations of one cell, both attempts (max) */
  ORC_ST_FALLBACK = 5, /* Newton restarts from T^n */
  ORC_ST_NOCONV = 6,   /* cells that did not converge */
  ORC_NSTATS = 8
};

/* ------------------------------------------------------------------------ */
/* Closure and signal speeds (Sect. 2.1, Sect. 2.6)                          */
/* ------------------------------------------------------------------------ */

/* Levermore Eddington factor xi(f), Sect. 2.1. */
double orc_xi(double f) {
  return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
}

static double norm3(const double F[3]) {
  return sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
}

/* Eddington tensor D (row-major 3x3) and reduced flux f of a state (E, F),
 * Sect. 2.1: D = (1-xi)/2 delta + (3 xi - 1)/2 n n, n = F/|F|, f = |F|/E
 * capped at 1. */
void orc_closure(double E, const double F[3], double D[9], double *f_out) {
  double nF = norm3(F);
  double f = nF / E;
  if (f > 1.0) f = 1.0;
  double xi = orc_xi(f);
  double nvec[3] = {0.0, 0.0, 0.0};
  if (nF > 0.0) {
    nvec[0] = F[0] / nF;
    nvec[1] = F[1] / nF;
    nvec[2] = F[2] / nF;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      D[3 * i + j] = (i == j ? 0.5 * (1.0 - xi) : 0.0) + 0.5 * (3.0 * xi - 1.0) * nvec[i] * nvec[j];
  if (f_out) *f_out = f;
}

/* Physical flux of (E, F) along direction d: (chat F_d, chat D_{d j} E). */
void orc_phys_flux(double chat, double E, const double F[3], int d, double out[4]) {
  double D[9];
  orc_closure(E, F, D, NULL);
  out[0] = chat * F[d];
  for (int j = 0; j < 3; ++j) out[1 + j] = chat * D[3 * d + j] * E;
}

/* Eigenvalues lambda_{1,3} (units of chat) along direction d, Sect. 2.6:
 * lambda = (f cos(theta) +/- zeta) / sqrt(4 - 3 f^2), theta = angle between F
 * and the direction.  zeta^2 is clamped at zero against rounding. */
void orc_lambda(double E, const double F[3], int d, double *lm, double *lp) {
  double nF = norm3(F);
  double f = nF / E;
  if (f > 1.0) f = 1.0;
  double cth = (nF > 0.0) ? F[d] / nF : 0.0;
  double s = sqrt(4.0 - 3.0 * f * f);
  double z2 = (2.0 / 3.0) * (4.0 - 3.0 * f * f - s) + 2.0 * cth * cth * (2.0 - f * f - s);
  if (z2 < 0.0) z2 = 0.0;
  double z = sqrt(z2);
  *lp = (f * cth + z) / s;
  *lm = (f * cth - z) / s;
}

/* ------------------------------------------------------------------------ */
/* Reconstruction (Sect. 2.5)                                                */
/* ------------------------------------------------------------------------ */

/* van Leer limited slope from left and right one-sided slopes. */
double orc_vanleer(double dl, double dr) {
  if (dl * dr > 0.0) return 2.0 * dl * dr / (dl + dr);
  return 0.0;
}

/* LimO3, the compact third-order limited reconstruction that Sect. 2.5
 * offers beside PLM (Cada & Torrilhon 2009).  The face value on the side of
 * the difference dt (the other one-sided difference being dn) is
 *   u + phi(theta) dt / 2,   theta = dn / dt,
 *   phi = max(0, min(phi3, max(-theta/2, min(2 theta, phi3, 3/2)))),
 * phi3 = (2 + theta) / 3 being the unlimited third-order value (exact for
 * parabolas on a uniform grid).  The caps 2 theta and 3/2 for theta > 0 and
 * -theta/2 for theta < 0 keep the face between the neighbouring values
 * (total-variation bounds of the form 0 <= phi <= min(2 theta, M),
 * phi <= (2 - M) |theta| with M = 3/2).  Returns phi(theta) dt / 2 (zero
 * when dt = 0). */
double orc_limo3(double dn, double dt) {
  if (dt == 0.0) return 0.0;
  double th = dn / dt;
  double p3 = (2.0 + th) / 3.0;
  double a = 2.0 * th;
  if (p3 < a) a = p3;
  if (1.5 < a) a = 1.5;
  if (-0.5 * th > a) a = -0.5 * th;
  if (p3 < a) a = p3;
  if (a < 0.0) a = 0.0;
  return 0.5 * a * dt;
}

/* f-preserving face fix, Eq. (f_reconstruct).  (Ef, Ff) is the reconstructed
 * face state, (Ec, Fc) the centre of the cell it was reconstructed from.
 * Returns 1 when F was recomputed. */
int orc_fix_face(double Ef, double Ff[3], double Ec, const double Fc[3]) {
  double rf = norm3(Ff) / Ef;
  double rc = norm3(Fc) / Ec;
  if (rf <= 1.0 && rf > rc) return 0;
  double scale = Ef / Ec;
  Ff[0] = Fc[0] * scale;
  Ff[1] = Fc[1] * scale;
  Ff[2] = Fc[2] * scale;
  return 1;
}

/* The f <= 1 treatment of a face state chosen by `mode` (Sect. 2.5):
 *   ORC_FIX_FPRESERVE  Eq. (f_reconstruct), orc_fix_face;
 *   ORC_FIX_PLUTO      the flat state (E_c, F_c) of the cell wherever the
 *                      reconstruction has |F_f| > E_f ("PLUTO
 *                      reconstruction"; one face state at a time);
 *   ORC_FIX_CLIP       F_f rescaled to |F_f| = E_f wherever |F_f| > E_f
 *                      (the plain limiter that Sect. 3's beam test shows to
 *                      fail).
 * Returns 1 when the state was changed. */
int orc_fix_face_mode(int mode, double *Ef, double Ff[3], double Ec, const double Fc[3]) {
  if (mode == ORC_FIX_FPRESERVE) return orc_fix_face(*Ef, Ff, Ec, Fc);
  double nf = norm3(Ff);
  if (nf <= *Ef) return 0;
  if (mode == ORC_FIX_PLUTO) {
    *Ef = Ec;
    Ff[0] = Fc[0];
    Ff[1] = Fc[1];
    Ff[2] = Fc[2];
  } else {
    double r = *Ef / nf;
    Ff[0] *= r;
    Ff[1] *= r;
    Ff[2] *= r;
  }
  return 1;
}

/* HLL flux from left/right states and their physical fluxes with signal
 * speeds sl <= sr. */
void orc_hll(double sl, double sr, const double uL[4], const double uR[4], const double fL[4],
             const double fR[4], double out[4]) {
  if (sl >= 0.0) {
    for (int q = 0; q < 4; ++q) out[q] = fL[q];
  } else if (sr <= 0.0) {
    for (int q = 0; q < 4; ++q) out[q] = fR[q];
  } else {
    for (int q = 0; q < 4; ++q)
      out[q] = (sr * fL[q] - sl * fR[q] + sl * sr * (uR[q] - uL[q])) / (sr - sl);
  }
}

/* Lax-Friedrichs-Rusanov flux (Sect. 2.5 lists it beside HLL) with the
 * local speed S = max(|S_L|, |S_R|) of the same (thick-limited) signal
 * speeds: (F_L + F_R) / 2 - S (U_R - U_L) / 2. */
void orc_lf(double sl, double sr, const double uL[4], const double uR[4], const double fL[4],
            const double fR[4], double out[4]) {
  double S = fabs(sl) > fabs(sr) ? fabs(sl) : fabs(sr);
  for (int q = 0; q < 4; ++q) out[q] = 0.5 * (fL[q] + fR[q]) - 0.5 * S * (uR[q] - uL[q]);
}

/* ------------------------------------------------------------------------ */
/* Opacities                                                                 */
/* ------------------------------------------------------------------------ */

/* Absorption (Planck, Rosseland) and scattering opacities per unit mass at
 * (rho, T): constant, a clipped power law (the Kramers-like form of
 * Sect. 3.3 is k0 rho T^-3.5), or a table bilinear in log space. */
void orc_opacity(const orc_problem *p, double rho, double T, double *kp, double *kr,
                 double *sg) {
  if (p->opac_kind == ORC_OPAC_CONST) {
    *kp = p->kappa_p;
    *kr = p->kappa_r;
    *sg = p->sigma;
    return;
  }
  double k;
  if (p->opac_kind == ORC_OPAC_POWERLAW) {
    k = p->k0 * pow(rho, p->a_rho) * pow(T, p->b_T);
    if (k < p->kmin) k = p->kmin;
    if (k > p->kmax) k = p->kmax;
  } else {
    /* bilinear interpolation of log10 kappa in (log10 rho, log10 T), clamped
     * at the table edges */
    double xr = (log10(rho) - p->lrho0) / (p->lrho1 - p->lrho0) * (p->nrho - 1);
    double xt = (log10(T) - p->lT0) / (p->lT1 - p->lT0) * (p->nT - 1);
    if (xr < 0.0) xr = 0.0;
    if (xr > p->nrho - 1) xr = p->nrho - 1;
    if (xt < 0.0) xt = 0.0;
    if (xt > p->nT - 1) xt = p->nT - 1;
    int ir = (int)floor(xr), it = (int)floor(xt);
    if (ir > p->nrho - 2) ir = p->nrho - 2;
    if (it > p->nT - 2) it = p->nT - 2;
    double wr = xr - ir, wt = xt - it;
    const double *t = p->ltable;
    double l00 = t[it * p->nrho + ir], l10 = t[it * p->nrho + ir + 1];
    double l01 = t[(it + 1) * p->nrho + ir], l11 = t[(it + 1) * p->nrho + ir + 1];
    double lk = (1.0 - wr) * (1.0 - wt) * l00 + wr * (1.0 - wt) * l10 + (1.0 - wr) * wt * l01 +
                wr * wt * l11;
    k = pow(10.0, lk);
  }
  *kp = k;
  *kr = k;
  *sg = p->sigma_ratio * k;
}

/* ------------------------------------------------------------------------ */
/* Grid geometry                                                             */
/* ------------------------------------------------------------------------ */

/* The interior cell that ghost index i along d copies: the wrapped cell
 * (periodic), the mirror image (reflective) or the edge cell (outflow; also
 * the cell whose density and geometry the ghosts of the fixed and LTE sides
 * take).  Interior indices map to themselves. */
static int map_index(const orc_problem *p, int d, int i) {
  int n = p->n[d];
  if (i >= 0 && i < n) return i;
  int bc = (i < 0) ? p->bc_lo[d] : p->bc_hi[d];
  if (bc == ORC_BC_PERIODIC) return ((i % n) + n) % n;
  if (bc == ORC_BC_REFLECT) {
    int m = (i < 0) ? -1 - i : 2 * n - 1 - i;
    return m < 0 ? 0 : (m >= n ? n - 1 : m);
  }
  return (i < 0) ? 0 : n - 1;
}

/* Centre coordinate of cell i along d, for i in [-2, n+1].  Ghost centres
 * are shifted by the period (periodic) or mirror the cells inside (every
 * other boundary). */
static double centre(const orc_problem *p, int d, int i) {
  int n = p->n[d];
  const double *x = p->xf[d];
  if (i >= 0 && i < n) return 0.5 * (x[i] + x[i + 1]);
  double L = x[n] - x[0];
  if (i < 0) {
    if (p->bc_lo[d] == ORC_BC_PERIODIC) return centre(p, d, i + n) - L;
    return 2.0 * x[0] - centre(p, d, -1 - i);
  }
  if (p->bc_hi[d] == ORC_BC_PERIODIC) return centre(p, d, i - n) + L;
  return 2.0 * x[n] - centre(p, d, 2 * n - 1 - i);
}

static size_t lin(const orc_problem *p, int i, int j, int k) {
  return (size_t)i + (size_t)p->n[0] * ((size_t)j + (size_t)p->n[1] * (size_t)k);
}

/* Physical widths h_d of cell (i,j,k) (used by tau and the CFL condition). */
static void widths(const orc_problem *p, int i, int j, int k, double h[3]) {
  const double *x0 = p->xf[0], *x1 = p->xf[1], *x2 = p->xf[2];
  double d0 = x0[i + 1] - x0[i], d1 = x1[j + 1] - x1[j], d2 = x2[k + 1] - x2[k];
  if (p->geom == ORC_CART) {
    h[0] = d0; h[1] = d1; h[2] = d2;
  } else if (p->geom == ORC_CYL) {
    double Rc = 0.5 * (x0[i] + x0[i + 1]);
    h[0] = d0; h[1] = Rc * d1; h[2] = d2;
  } else {
    double rc = 0.5 * (x0[i] + x0[i + 1]);
    double thc = 0.5 * (x1[j] + x1[j + 1]);
    h[0] = d0; h[1] = rc * d1; h[2] = rc * sin(thc) * d2;
  }
}

static double max_active_width(const orc_problem *p, int i, int j, int k) {
  double h[3];
  widths(p, i, j, k, h);
  double m = h[0];
  for (int d = 1; d < p->ndim; ++d)
    if (h[d] > m) m = h[d];
  return m;
}

/* Time step from the CFL condition (Sect. 2.4 item 10): cfl over the largest
 * sum over active directions of chat / h_d. */
double orc_dt(const orc_problem *p) {
  double worst = 0.0;
  for (int k = 0; k < p->n[2]; ++k)
    for (int j = 0; j < p->n[1]; ++j)
      for (int i = 0; i < p->n[0]; ++i) {
        double h[3];
        widths(p, i, j, k, h);
        double s = 0.0;
        for (int d = 0; d < p->ndim; ++d) s += p->chat / h[d];
        if (s > worst) worst = s;
      }
  return p->cfl / worst;
}

/* Time step with the gas (hydro): cfl over the largest sum over active
 * directions of max(chat, |v_d| + c_s) / h_d, c_s = sqrt(Gamma p / rho). */
double orc_dt_gas(const orc_problem *p, const double *rho, const double *e, const double *m0,
                  const double *m1, const double *m2) {
  double worst = 0.0;
  const double *m[3] = {m0, m1, m2};
  for (int k = 0; k < p->n[2]; ++k)
    for (int j = 0; j < p->n[1]; ++j)
      for (int i = 0; i < p->n[0]; ++i) {
        size_t c = lin(p, i, j, k);
        double h[3];
        widths(p, i, j, k, h);
        double cs = sqrt(p->gamma_gas * (p->gamma_gas - 1.0) * e[c] / rho[c]);
        double sum = 0.0;
        for (int d = 0; d < p->ndim; ++d) {
          double v = fabs(m[d][c] / rho[c]) + cs;
          sum += (v > p->chat ? v : p->chat) / h[d];
        }
        if (sum > worst) worst = sum;
      }
  return p->cfl / worst;
}

/* Cell volume and face areas (lower/upper face along each direction). */
static void vol_area(const orc_problem *p, int i, int j, int k, double *V, double Alo[3],
                     double Ahi[3]) {
  const double *x0 = p->xf[0], *x1 = p->xf[1], *x2 = p->xf[2];
  double a0 = x0[i], b0 = x0[i + 1], a1 = x1[j], b1 = x1[j + 1], a2 = x2[k], b2 = x2[k + 1];
  if (p->geom == ORC_CART) {
    *V = (b0 - a0) * (b1 - a1) * (b2 - a2);
    Alo[0] = Ahi[0] = (b1 - a1) * (b2 - a2);
    Alo[1] = Ahi[1] = (b0 - a0) * (b2 - a2);
    Alo[2] = Ahi[2] = (b0 - a0) * (b1 - a1);
  } else if (p->geom == ORC_CYL) { /* (R, phi, z) */
    *V = 0.5 * (b0 * b0 - a0 * a0) * (b1 - a1) * (b2 - a2);
    Alo[0] = a0 * (b1 - a1) * (b2 - a2);
    Ahi[0] = b0 * (b1 - a1) * (b2 - a2);
    Alo[1] = Ahi[1] = (b0 - a0) * (b2 - a2);
    Alo[2] = Ahi[2] = 0.5 * (b0 * b0 - a0 * a0) * (b1 - a1);
  } else { /* (r, theta, phi) */
    double dcos = cos(a1) - cos(b1);
    *V = (b0 * b0 * b0 - a0 * a0 * a0) / 3.0 * dcos * (b2 - a2);
    Alo[0] = a0 * a0 * dcos * (b2 - a2);
    Ahi[0] = b0 * b0 * dcos * (b2 - a2);
    Alo[1] = 0.5 * (b0 * b0 - a0 * a0) * sin(a1) * (b2 - a2);
    Ahi[1] = 0.5 * (b0 * b0 - a0 * a0) * sin(b1) * (b2 - a2);
    Alo[2] = Ahi[2] = 0.5 * (b0 * b0 - a0 * a0) * (b1 - a1);
  }
}

/* ------------------------------------------------------------------------ */
/* One face                                                                  */
/* ------------------------------------------------------------------------ */

static void load_u(const orc_state *s, size_t c, double *E, double F[3]) {
  *E = s->E[c];
  F[0] = s->F0[c];
  F[1] = s->F1[c];
  F[2] = s->F2[c];
}

static double temperature(const orc_problem *p, double rho, double e) {
  double Cv = rho / (p->mu * (p->gamma_gas - 1.0));
  return e / Cv;
}

/* Values of the cell with index a (a[d] may be a ghost index along d; the
 * other two are interior): u = (E, F0, F1, F2), rho and e.  Boundary
 * conditions (Sect. 3 uses all of them):
 *   periodic, outflow   the wrapped or edge cell;
 *   reflective          the mirror cell with the normal flux F_d negated;
 *   fixed (injection)   E and F of the side's boundary state, the edge
 *                       cell's rho and e = C_v T_b;
 *   LTE                 E = a T_b^4, F of the edge cell (zero gradient), the
 *                       edge cell's rho and e = C_v T_b. */
static void cell_values(const orc_problem *p, const orc_state *s, const int a[3], int d,
                        double u[4], double *rho, double *e) {
  int b[3] = {a[0], a[1], a[2]};
  int i = a[d], n = p->n[d];
  b[d] = map_index(p, d, i);
  size_t c = lin(p, b[0], b[1], b[2]);
  load_u(s, c, &u[0], u + 1);
  *rho = s->rho[c];
  *e = s->e[c];
  if (i >= 0 && i < n) return;
  int side = (i < 0) ? 0 : 1;
  int bc = side ? p->bc_hi[d] : p->bc_lo[d];
  const double *v = p->bc_val[d][side];
  double Cv = *rho / (p->mu * (p->gamma_gas - 1.0));
  if (bc == ORC_BC_REFLECT) {
    u[1 + d] = -u[1 + d];
  } else if (bc == ORC_BC_FIXED) {
    u[0] = v[0];
    u[1] = v[1];
    u[2] = v[2];
    u[3] = v[3];
    *e = Cv * v[4];
  } else if (bc == ORC_BC_LTE) {
    u[0] = p->a_rad * v[4] * v[4] * v[4] * v[4];
    *e = Cv * v[4];
  }
}

/* rho * chi * dx of the cell with index a (a[d] possibly a ghost index),
 * with chi = kappa_R + sigma at (rho, T^n); a ghost takes the width of the
 * cell it maps to. */
static double tau_cell(const orc_problem *p, const orc_state *s, const int a[3], int d) {
  double u[4], rho, e;
  cell_values(p, s, a, d, u, &rho, &e);
  int b[3] = {a[0], a[1], a[2]};
  b[d] = map_index(p, d, a[d]);
  double T = temperature(p, rho, e);
  double kp, kr, sg;
  orc_opacity(p, rho, T, &kp, &kr, &sg);
  return rho * (kr + sg) * max_active_width(p, b[0], b[1], b[2]);
}

/* ------------------------------------------------------------------------ */
/* Hydrodynamics (the gas step that precedes the radiation transport in each */
/* substep, Sect. 2.4; a standard Godunov step: PLM on primitive variables, */
/* HLL with the Davis signal speeds, Cartesian flux divergence)              */
/* ------------------------------------------------------------------------ */

/* Primitive gas state w = (rho, v0, v1, v2, p) of the cell with index a
 * (a[d] possibly a ghost index along d), p = (Gamma - 1) e.  Ghost gas as in
 * cell_values: wrapped or edge cells, mirrored with v_d negated
 * (reflective), at rest with T = T_b and the edge density (fixed, LTE). */
static void gas_prim(const orc_problem *p, const orc_state *s, const int a[3], int d,
                     double w[5]) {
  double u[4], rho, e;
  cell_values(p, s, a, d, u, &rho, &e);
  int b[3] = {a[0], a[1], a[2]};
  int i = a[d], n = p->n[d];
  b[d] = map_index(p, d, i);
  size_t c = lin(p, b[0], b[1], b[2]);
  double m[3] = {s->m0[c], s->m1[c], s->m2[c]};
  if (i < 0 || i >= n) {
    int bc = (i < 0) ? p->bc_lo[d] : p->bc_hi[d];
    if (bc == ORC_BC_REFLECT) m[d] = -m[d];
    if (bc == ORC_BC_FIXED || bc == ORC_BC_LTE) m[0] = m[1] = m[2] = 0.0;
  }
  w[0] = rho;
  w[1] = m[0] / rho;
  w[2] = m[1] / rho;
  w[3] = m[2] / rho;
  w[4] = (p->gamma_gas - 1.0) * e;
}

/* Conserved state (rho, m0, m1, m2, E_gas) and physical flux along d of a
 * primitive state. */
static void gas_flux(const orc_problem *p, const double w[5], int d, double U[5], double f[5]) {
  double rho = w[0], pr = w[4];
  double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  double Eg = pr / (p->gamma_gas - 1.0) + 0.5 * rho * v2;
  double vd = w[1 + d];
  U[0] = rho;
  U[1] = rho * w[1];
  U[2] = rho * w[2];
  U[3] = rho * w[3];
  U[4] = Eg;
  f[0] = rho * vd;
  f[1] = rho * vd * w[1];
  f[2] = rho * vd * w[2];
  f[3] = rho * vd * w[3];
  f[1 + d] += pr;
  f[4] = (Eg + pr) * vd;
}

/* HLL flux of the gas through the lower face of cell idx along d: PLM (van
 * Leer, the same limited slopes as the radiation) of the primitive
 * variables, signal speeds S_L = min(v_L - c_L, v_R - c_R) and
 * S_R = max(v_L + c_L, v_R + c_R) with c = sqrt(Gamma p / rho). */
void hydro_face_flux(const orc_problem *p, const orc_state *s, const int idx[3], int d,
                     double out[5]) {
  int a[3] = {idx[0], idx[1], idx[2]};
  int i = idx[d];
  double w[4][5];
  for (int q = 0; q < 4; ++q) {
    a[d] = i - 2 + q;
    gas_prim(p, s, a, d, w[q]);
  }
  double xm2 = centre(p, d, i - 2), xm1 = centre(p, d, i - 1), x0 = centre(p, d, i),
         xp1 = centre(p, d, i + 1);
  double xf = p->xf[d][i];
  double wl[5], wr[5];
  for (int q = 0; q < 5; ++q) {
    double s0 = orc_vanleer((w[1][q] - w[0][q]) / (xm1 - xm2), (w[2][q] - w[1][q]) / (x0 - xm1));
    double s1 = orc_vanleer((w[2][q] - w[1][q]) / (x0 - xm1), (w[3][q] - w[2][q]) / (xp1 - x0));
    wl[q] = w[1][q] + s0 * (xf - xm1);
    wr[q] = w[2][q] + s1 * (xf - x0);
  }
  double UL[5], UR[5], fL[5], fR[5];
  gas_flux(p, wl, d, UL, fL);
  gas_flux(p, wr, d, UR, fR);
  double cl = sqrt(p->gamma_gas * wl[4] / wl[0]), cr = sqrt(p->gamma_gas * wr[4] / wr[0]);
  double sl = wl[1 + d] - cl, sr = wr[1 + d] + cr;
  if (wr[1 + d] - cr < sl) sl = wr[1 + d] - cr;
  if (wl[1 + d] + cl > sr) sr = wl[1 + d] + cl;
  for (int q = 0; q < 5; ++q) {
    if (sl >= 0.0)
      out[q] = fL[q];
    else if (sr <= 0.0)
      out[q] = fR[q];
    else
      out[q] = (sr * fL[q] - sl * fR[q] + sl * sr * (UR[q] - UL[q])) / (sr - sl);
  }
}

/* The gas after the hydrodynamic step of length dt of cell (i,j,k):
 * g = (rho, m0, m1, m2, e) from the Cartesian flux divergence of the
 * conserved (rho, m, E_gas). */
static void hydro_cell(const orc_problem *p, const orc_state *s, double dt, int i, int j, int k,
                       double g[5]) {
  int idx[3] = {i, j, k};
  size_t c = lin(p, i, j, k);
  double rho = s->rho[c];
  double m[3] = {s->m0[c], s->m1[c], s->m2[c]};
  double U[5] = {rho, m[0], m[1], m[2],
                 s->e[c] + 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho};
  for (int d = 0; d < p->ndim; ++d) {
    double flo[5], fhi[5];
    hydro_face_flux(p, s, idx, d, flo);
    int up[3] = {i, j, k};
    up[d] += 1;
    hydro_face_flux(p, s, up, d, fhi);
    double h = p->xf[d][idx[d] + 1] - p->xf[d][idx[d]];
    for (int q = 0; q < 5; ++q) U[q] -= dt * (fhi[q] - flo[q]) / h;
  }
  g[0] = U[0];
  g[1] = U[1];
  g[2] = U[2];
  g[3] = U[3];
  g[4] = U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
}

/* Right face state (side = +1) or left face state (side = -1) of cell ic
 * along d, the other two indices of the cell being those of idx. */
static void face_state(const orc_problem *p, const orc_state *s, const int idx[3], int d, int ic,
                       int side, double *Ef, double Ff[3], double *Ec, double Fc[3]) {
  int a[3] = {idx[0], idx[1], idx[2]};
  double u[3][4];
  for (int q = -1; q <= 1; ++q) {
    a[d] = ic + q;
    double rho, e;
    cell_values(p, s, a, d, u[q + 1], &rho, &e);
  }
  double xm = centre(p, d, ic - 1), x0 = centre(p, d, ic), xp = centre(p, d, ic + 1);
  /* face coordinate: the ghost cells -1 and n are only asked for the face
   * they share with the domain, so the index stays in [0, n] */
  double xface = (side > 0) ? p->xf[d][ic + 1] : p->xf[d][ic];
  double uf[4];
  for (int q = 0; q < 4; ++q) {
    if (p->recon == ORC_LIMO3) {
      /* index-space differences (the limiter is defined on a uniform grid) */
      double dm = u[1][q] - u[0][q], dp = u[2][q] - u[1][q];
      uf[q] = (side > 0) ? u[1][q] + orc_limo3(dm, dp) : u[1][q] - orc_limo3(dp, dm);
    } else {
      double dl = (u[1][q] - u[0][q]) / (x0 - xm);
      double dr = (u[2][q] - u[1][q]) / (xp - x0);
      uf[q] = u[1][q] + orc_vanleer(dl, dr) * (xface - x0);
    }
  }
  *Ef = uf[0];
  Ff[0] = uf[1];
  Ff[1] = uf[2];
  Ff[2] = uf[3];
  *Ec = u[1][0];
  Fc[0] = u[1][1];
  Fc[1] = u[1][2];
  Fc[2] = u[1][3];
}

/* Riemann flux (HLL, or LF-Rusanov) through the lower face (between cells
 * i_d - 1 and i_d) of the cell idx along active direction d.  Returns the
 * number of face states the f <= 1 treatment changed. */
static int face_flux(const orc_problem *p, const orc_state *s, const int idx[3], int d,
                     double out[4]) {
  int i = idx[d];
  double EL, FL[3], EcL, FcL[3], ER, FR[3], EcR, FcR[3];
  face_state(p, s, idx, d, i - 1, +1, &EL, FL, &EcL, FcL);
  face_state(p, s, idx, d, i, -1, &ER, FR, &EcR, FcR);
  int nfix = orc_fix_face_mode(p->face_fix, &EL, FL, EcL, FcL) +
             orc_fix_face_mode(p->face_fix, &ER, FR, EcR, FcR);

  double fL[4], fR[4];
  orc_phys_flux(p->chat, EL, FL, d, fL);
  orc_phys_flux(p->chat, ER, FR, d, fR);
  double lmL, lpL, lmR, lpR;
  orc_lambda(EL, FL, d, &lmL, &lpL);
  orc_lambda(ER, FR, d, &lmR, &lpR);
  double sl = p->chat * (lmL < lmR ? lmL : lmR);
  double sr = p->chat * (lpL > lpR ? lpL : lpR);

  /* optically thick correction (Sect. 2.6), tau = mean of the two cells */
  int a[3] = {idx[0], idx[1], idx[2]};
  a[d] = i - 1;
  double tL = tau_cell(p, s, a, d);
  a[d] = i;
  double tR = tau_cell(p, s, a, d);
  double tau = 0.5 * (tL + tR);
  if (tau > 0.0) {
    double bound = 4.0 * p->chat / (3.0 * tau);
    if (sl < -bound) sl = -bound;
    if (sr > bound) sr = bound;
  }
  double uL[4] = {EL, FL[0], FL[1], FL[2]}, uR[4] = {ER, FR[0], FR[1], FR[2]};
  if (p->riemann == ORC_LF)
    orc_lf(sl, sr, uL, uR, fL, fR, out);
  else
    orc_hll(sl, sr, uL, uR, fL, fR, out);
  return nfix;
}

/* ------------------------------------------------------------------------ */
/* Implicit coupling (Sect. 2.8) and gas bookkeeping (Sect. 2.7)             */
/* ------------------------------------------------------------------------ */

/* Solves the 2x2 system of Eq. (implicit_matrix) with T^4 linearised about
 * Tk.  sq = dt * (-div F_irr) is the irradiation term of Sect. 2.9 added to
 * the gas row of the right-hand side (S_1); it enters T's numerator with the
 * factor (1 + g_r) of the elimination.  Written out by Cramer's rule; the determinant
 *   (1+g_r)(C_v + 4 g a Tk^3) - (4 g_r a Tk^3) g
 * simplifies exactly to (1+g_r) C_v + 4 g a Tk^3, and the T numerator to
 * (1+g_r) C_v T^n + 3 g a Tk^4 + g E*, which are used as such.  Tn enters only
 * through C_v T^n on the right-hand side. */
void orc_solve2x2_irr(double Estar, double Tn, double Tk, double Cv, double g, double gr,
                      double a, double sq, double *Enew, double *Tnew) {
  double aT3 = a * Tk * Tk * Tk;
  double aT4 = aT3 * Tk;
  double det = (1.0 + gr) * Cv + 4.0 * g * aT3;
  double T = ((1.0 + gr) * (Cv * Tn + sq) + 3.0 * g * aT4 + g * Estar) / det;
  double E = (Estar + gr * aT3 * (4.0 * T - 3.0 * Tk)) / (1.0 + gr);
  *Enew = E;
  *Tnew = T;
}

void orc_solve2x2(double Estar, double Tn, double Tk, double Cv, double g, double gr, double a,
                  double *Enew, double *Tnew) {
  orc_solve2x2_irr(Estar, Tn, Tk, Cv, g, gr, a, 0.0, Enew, Tnew);
}

/* The coupling step of one cell.  In ORC_ONCE mode this is the paper's
 * single solve about T^n; in ORC_NEWTON mode the same solve is repeated about
 * the latest temperature until |T_{k+1} - T_k| <= rtol T_{k+1} (Newton's
 * method on C_v (T - T^n) + g/(1+g_r) (a T^4 - E*) = 0).  T0 is the starting
 * point of the iteration (T^n when no other guess is given). */
/* The coupling of Sect. 2.8 in the precision of the CUDA library's split
 * form (a host emulation for measuring error shares; never the reference):
 * the products see float-rounded inputs; the emission term a T^4 and the
 * residual D = E* - a T^4 are formed in double from the float temperature;
 * the other products of the linearised solve (a T^3, the determinant, its
 * reciprocal, the increments of T and E) in float.  The increments are
 * added to the unrounded E* and T^n, so that the rounding of the stored
 * state (float in the split form) is left out and only the products' share
 * is measured.  Newton mode takes the single solve first and keeps it if it
 * passes the convergence test (in float); otherwise it iterates from T^n
 * with the residual and the numerator in double, the determinant and its
 * reciprocal in float.  No irradiation, no absorption-only mode. */
static void couple_float(const orc_problem *p, double dt, double rho, double Tn, double kp,
                         double Estar, double *Enew, double *Tnew, int64_t st[ORC_NSTATS]) {
  const float cvfac = (float)(1.0 / (p->mu * (p->gamma_gas - 1.0)));
  const float rf = (float)rho, kf = (float)kp, Ef = (float)Estar, Tf = (float)Tn;
  const float af = (float)p->a_rad, rtol = (float)p->newton_rtol;
  const float Cv = rf * cvfac;
  const float gr = (float)(dt * p->chat) * kf * rf;
  const float g = (float)(dt * p->c) * kf * rf;
  const float c1 = (1.0f + gr) * Cv;
  /* single linearised solve about T^n */
  const double T2 = (double)Tf * (double)Tf;
  const float D = (float)fma(-(p->a_rad * T2), T2, (double)Ef);
  const float aT3 = af * Tf * Tf * Tf;
  const float det = c1 + 4.0f * g * aT3;
  const float q = D * (1.0f / det);
  const float dT = g * q;
  const float dE = -gr * Cv * q;
  const float T1 = Tf + dT;
  st[ORC_ST_ITERS] += 1;
  if (st[ORC_ST_ITMAX] < 1) st[ORC_ST_ITMAX] = 1;
  if (p->implicit_mode == ORC_ONCE || fabsf(dT) <= rtol * T1) {
    *Enew = Estar + (double)dE;
    *Tnew = Tn + (double)dT;
    return;
  }
  /* Newton from T^n, the single solve above counted as the first iterate
   * of a separate pass (as the library's queue pass does) */
  const double Tnd = (double)Tf, c1d = (double)c1;
  double Tk = Tnd, Tnext = Tnd, aT3d = 0.0, Dd = 0.0;
  float detf = 1.0f;
  int it, ok = 0;
  for (it = 1; it <= p->newton_maxit; ++it) {
    aT3d = p->a_rad * Tk * Tk * Tk;
    Dd = (double)Ef - aT3d * Tk;
    detf = c1 + 4.0f * g * (float)aT3d;
    const double num = c1d * (Tnd - Tk) + (double)g * Dd;
    const double dTd = num * (double)(1.0f / detf);
    Tnext = Tk + dTd;  /* Tk starts from the float T^n, as in the library */
    if (!(Tnext > 0.0)) break;
    if (fabsf((float)dTd) <= rtol * (float)Tnext) {
      ok = 1;
      break;
    }
    Tk = Tnext;
  }
  const int used = ok ? it : (it > p->newton_maxit ? p->newton_maxit : it);
  st[ORC_ST_ITERS] += used;
  if (st[ORC_ST_ITMAX] < used + 1) st[ORC_ST_ITMAX] = used + 1;
  if (!ok) st[ORC_ST_NOCONV] += 1;
  const float inner = (float)(4.0 * aT3d * ((double)Cv * (Tnd - Tk)) - (double)Cv * Dd);
  *Enew = Estar + (double)(gr * inner * (1.0f / detf));
  *Tnew = Tn + (Tnext - Tnd);
}

static void couple(const orc_problem *p, double dt, double rho, double Tn, double T0, double kp,
                   double Estar, double sq, double *Enew, double *Tnew,
                   int64_t st[ORC_NSTATS]) {
  if (p->float_coupling && p->implicit_mode != ORC_ABSORB && sq == 0.0) {
    couple_float(p, dt, rho, Tn, kp, Estar, Enew, Tnew, st);
    return;
  }
  double Cv = rho / (p->mu * (p->gamma_gas - 1.0));
  double g = dt * p->c * kp * rho;
  double gr = dt * p->chat * kp * rho;
  if (p->implicit_mode == ORC_ABSORB) {
    /* absorption only (the first shadow test of Sect. 3): no emission by
     * the gas, E^{n+1} = E* / (1 + g_r); the gas energy follows from the
     * conservation of Sect. 2.7 in the caller.  Tnew is T^n here. */
    *Enew = Estar / (1.0 + gr);
    *Tnew = Tn;
    st[ORC_ST_ITERS] += 1;
    if (st[ORC_ST_ITMAX] < 1) st[ORC_ST_ITMAX] = 1;
    return;
  }
  if (p->implicit_mode == ORC_ONCE) {
    orc_solve2x2_irr(Estar, Tn, Tn, Cv, g, gr, p->a_rad, sq, Enew, Tnew);
    st[ORC_ST_ITERS] += 1;
    if (st[ORC_ST_ITMAX] < 1) st[ORC_ST_ITMAX] = 1;
    return;
  }
  int total = 0; /* iterations of this cell over both attempts */
  for (int attempt = 0; attempt < 2; ++attempt) {
    double Tk = (attempt == 0) ? T0 : Tn;
    double E = Estar, T = Tk;
    int it, ok = 0;
    for (it = 1; it <= p->newton_maxit; ++it) {
      orc_solve2x2_irr(Estar, Tn, Tk, Cv, g, gr, p->a_rad, sq, &E, &T);
      if (!(T > 0.0)) break;
      if (fabs(T - Tk) <= p->newton_rtol * T) {
        ok = 1;
        break;
      }
      Tk = T;
    }
    int used = ok ? it : (it > p->newton_maxit ? p->newton_maxit : it);
    st[ORC_ST_ITERS] += used;
    total += used;
    if (st[ORC_ST_ITMAX] < total) st[ORC_ST_ITMAX] = total;
    if (ok) {
      *Enew = E;
      *Tnew = T;
      return;
    }
    if (attempt == 0) st[ORC_ST_FALLBACK] += 1;
    else {
      st[ORC_ST_NOCONV] += 1;
      *Enew = E;
      *Tnew = T;
    }
  }
}

/* One full step of one cell, reading the old state `s` and writing the new
 * values into out[9] = (E, F0, F1, F2, e, m0, m1, m2, T).  T0 is the start of
 * the Newton iteration (<= 0: T^n). */
static void cell_step(const orc_problem *p, const orc_state *s, double dt, int i, int j, int k,
                      double T0, double out[9], int64_t st[ORC_NSTATS]) {
  int idx[3] = {i, j, k};
  size_t c = lin(p, i, j, k);
  double E0, F0v[3];
  load_u(s, c, &E0, F0v);

  /* items 3-7: face fluxes and their divergence */
  double V, Alo[3], Ahi[3];
  vol_area(p, i, j, k, &V, Alo, Ahi);
  const double *x0 = p->xf[0], *x1 = p->xf[1];
  double dE = 0.0, dF[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < 3; ++d) {
    double flo[4], fhi[4];
    if (d < p->ndim) {
      st[ORC_ST_FIX] += face_flux(p, s, idx, d, flo);
      int up[3] = {i, j, k};
      up[d] += 1; /* upper face of this cell = lower face of index i_d + 1 */
      st[ORC_ST_FIX] += face_flux(p, s, up, d, fhi);
    } else {
      /* inactive direction: one cell whose faces carry its own flux */
      orc_phys_flux(p->chat, E0, F0v, d, flo);
      orc_phys_flux(p->chat, E0, F0v, d, fhi);
    }
    /* weights of the angular-momentum-conserving phi component */
    double wlo[3] = {1, 1, 1}, whi[3] = {1, 1, 1}, wc[3] = {1, 1, 1};
    if (p->geom == ORC_CYL && d == 0) {
      wlo[1] = x0[i];
      whi[1] = x0[i + 1];
      wc[1] = 0.5 * (x0[i] + x0[i + 1]);
    }
    if (p->geom == ORC_SPH && d == 0) {
      double a = x0[i], b = x0[i + 1];
      wlo[2] = a;
      whi[2] = b;
      wc[2] = 2.0 * (b * b * b - a * a * a) / (3.0 * (b * b - a * a));
    }
    if (p->geom == ORC_SPH && d == 1) {
      wlo[2] = sin(x1[j]);
      whi[2] = sin(x1[j + 1]);
      wc[2] = sin(0.5 * (x1[j] + x1[j + 1]));
    }
    dE -= (Ahi[d] * fhi[0] - Alo[d] * flo[0]) / V;
    for (int q = 0; q < 3; ++q)
      dF[q] -= (whi[q] * Ahi[d] * fhi[1 + q] - wlo[q] * Alo[d] * flo[1 + q]) / (wc[q] * V);
  }
  /* geometric sources from the cell-centred pressure tensor of U^n */
  if (p->geom != ORC_CART) {
    double D[9];
    orc_closure(E0, F0v, D, NULL);
    double P[9];
    for (int q = 0; q < 9; ++q) P[q] = D[q] * E0;
    if (p->geom == ORC_CYL) {
      double Rc = 0.5 * (x0[i] + x0[i + 1]);
      dF[0] += p->chat * P[4] / Rc; /* P_phiphi / R */
    } else {
      double a = x0[i], b = x0[i + 1];
      double rt = 2.0 * (b * b * b - a * a * a) / (3.0 * (b * b - a * a));
      double cott = (sin(x1[j + 1]) - sin(x1[j])) / (cos(x1[j]) - cos(x1[j + 1]));
      dF[0] += p->chat * (P[4] + P[8]) / rt;          /* (P_thth + P_phph) / r */
      dF[1] += p->chat * (-P[1] + cott * P[8]) / rt;  /* -P_rth / r + cot P_phph / r */
    }
  }
  double Es = E0 + dt * dE;
  double Fs[3] = {F0v[0] + dt * dF[0], F0v[1] + dt * dF[1], F0v[2] + dt * dF[2]};
  if (Es < p->e_floor) {
    Es = p->e_floor;
    st[ORC_ST_EFLOOR] += 1;
  }

  /* item 8: local sources */
  double rho = s->rho[c];
  double e0 = s->e[c];
  double m0[3] = {s->m0[c], s->m1[c], s->m2[c]};
  double Tn = temperature(p, rho, e0);
  double kp, kr, sg;
  orc_opacity(p, rho, Tn, &kp, &kr, &sg);
  double En, Tnew;
  const double sq = p->qirr ? dt * p->qirr[c] : 0.0;
  couple(p, dt, rho, Tn, T0 > 0.0 ? T0 : Tn, kp, Es, sq, &En, &Tnew, st);
  if (En < p->e_floor) {
    En = p->e_floor;
    st[ORC_ST_EFLOOR] += 1;
  }
  /* Eq. (source_discrete2): F^{n+1} (1 + dt chat chi rho) = F* */
  double sc = 1.0 + dt * p->chat * (kr + sg) * rho;
  double Fn[3] = {Fs[0] / sc, Fs[1] / sc, Fs[2] / sc};
  double nF = norm3(Fn);
  if (nF > En) {
    double r = En / nF;
    Fn[0] *= r;
    Fn[1] *= r;
    Fn[2] *= r;
    st[ORC_ST_FCLIP] += 1;
  }
  /* Sect. 2.7: E_gas + (c/chat) E_r and m + F/chat are conserved by the
   * coupling; the internal energy absorbs the kinetic-energy change. */
  double ke0 = (m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2]) / (2.0 * rho);
  double Egas = e0 + ke0 - (p->c / p->chat) * (En - Es) + sq;
  double mn[3];
  for (int q = 0; q < 3; ++q) mn[q] = m0[q] - (Fn[q] - Fs[q]) / p->chat;
  double ke1 = (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) / (2.0 * rho);
  out[0] = En;
  out[1] = Fn[0];
  out[2] = Fn[1];
  out[3] = Fn[2];
  out[4] = Egas - ke1;
  out[5] = mn[0];
  out[6] = mn[1];
  out[7] = mn[2];
  /* the coupling's T^{n+1}; absorption only: the temperature of the
   * updated gas energy */
  out[8] = (p->implicit_mode == ORC_ABSORB) ? out[4] / (rho / (p->mu * (p->gamma_gas - 1.0)))
                                            : Tnew;
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */

static void set_threads(const orc_problem *p) {
#ifdef _OPENMP
  if (p->nthreads > 0) omp_set_num_threads(p->nthreads);
#else
  (void)p;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* One Euler step of every cell (transport from `s`, then the local
 * coupling) into `w`; counters accumulated into tot. */
static void euler_pass(const orc_problem *p, const orc_state *s, orc_state *w, double dt,
                       int64_t tot[ORC_NSTATS]) {
  size_t N = (size_t)p->n[0] * p->n[1] * p->n[2];
  /* with hydro: the hydrodynamic step first (all cells), then the radiation
   * transport of E, F from s with the optical depths, the coupling and the
   * bookkeeping on the gas after the hydro step (Sect. 2.4) */
  orc_state r = *s;
  double *gbuf = NULL;
  if (p->hydro) {
    gbuf = (double *)malloc(5 * N * sizeof(double));
    if (!gbuf) return;
    r.rho = gbuf;
    r.m0 = gbuf + N;
    r.m1 = gbuf + 2 * N;
    r.m2 = gbuf + 3 * N;
    r.e = gbuf + 4 * N;
#pragma omp parallel for schedule(static)
    for (long long cc = 0; cc < (long long)N; ++cc) {
      int i = (int)(cc % p->n[0]);
      int j = (int)((cc / p->n[0]) % p->n[1]);
      int k = (int)(cc / ((long long)p->n[0] * p->n[1]));
      double g[5];
      hydro_cell(p, s, dt, i, j, k, g);
      r.rho[cc] = g[0];
      r.m0[cc] = g[1];
      r.m1[cc] = g[2];
      r.m2[cc] = g[3];
      r.e[cc] = g[4];
    }
    s = &r;
  }
#pragma omp parallel
  {
    int64_t loc[ORC_NSTATS] = {0};
#pragma omp for schedule(static)
    for (long long cc = 0; cc < (long long)N; ++cc) {
      int i = (int)(cc % p->n[0]);
      int j = (int)((cc / p->n[0]) % p->n[1]);
      int k = (int)(cc / ((long long)p->n[0] * p->n[1]));
      double o[9];
      cell_step(p, s, dt, i, j, k, -1.0, o, loc);
      w->E[cc] = o[0];
      w->F0[cc] = o[1];
      w->F1[cc] = o[2];
      w->F2[cc] = o[3];
      w->e[cc] = o[4];
      w->m0[cc] = o[5];
      w->m1[cc] = o[6];
      w->m2[cc] = o[7];
    }
#pragma omp critical
    {
      for (int q = 0; q < ORC_NSTATS; ++q) {
        if (q == ORC_ST_ITMAX) {
          if (loc[q] > tot[q]) tot[q] = loc[q];
        } else {
          tot[q] += loc[q];
        }
      }
    }
  }
  if (gbuf) {
    memcpy(w->rho, gbuf, N * sizeof(double));
    free(gbuf);
  }
}

static void copy_state(const orc_state *from, orc_state *to, size_t N, int with_rho) {
  if (with_rho) memcpy(to->rho, from->rho, N * sizeof(double));
  memcpy(to->E, from->E, N * sizeof(double));
  memcpy(to->F0, from->F0, N * sizeof(double));
  memcpy(to->F1, from->F1, N * sizeof(double));
  memcpy(to->F2, from->F2, N * sizeof(double));
  memcpy(to->e, from->e, N * sizeof(double));
  memcpy(to->m0, from->m0, N * sizeof(double));
  memcpy(to->m1, from->m1, N * sizeof(double));
  memcpy(to->m2, from->m2, N * sizeof(double));
}

/* s <- (s + u) / 2 for the conserved variables rho, E_r, F_r, m and the
 * total gas energy E_gas = e + |m|^2 / (2 rho); e is recovered from the
 * averaged E_gas, m and rho (the second stage of the RK2 / IMEX1 step). */
static void average_into(orc_state *s, const orc_state *u, size_t N) {
#pragma omp parallel for schedule(static)
  for (long long c = 0; c < (long long)N; ++c) {
    double rn = s->rho[c], ru = u->rho[c];
    double kn = (s->m0[c] * s->m0[c] + s->m1[c] * s->m1[c] + s->m2[c] * s->m2[c]) / (2.0 * rn);
    double ku = (u->m0[c] * u->m0[c] + u->m1[c] * u->m1[c] + u->m2[c] * u->m2[c]) / (2.0 * ru);
    double eg = 0.5 * ((s->e[c] + kn) + (u->e[c] + ku));
    double rho = (rn == ru) ? rn : 0.5 * (rn + ru);
    s->rho[c] = rho;
    s->E[c] = 0.5 * (s->E[c] + u->E[c]);
    s->F0[c] = 0.5 * (s->F0[c] + u->F0[c]);
    s->F1[c] = 0.5 * (s->F1[c] + u->F1[c]);
    s->F2[c] = 0.5 * (s->F2[c] + u->F2[c]);
    s->m0[c] = 0.5 * (s->m0[c] + u->m0[c]);
    s->m1[c] = 0.5 * (s->m1[c] + u->m1[c]);
    s->m2[c] = 0.5 * (s->m2[c] + u->m2[c]);
    double k = (s->m0[c] * s->m0[c] + s->m1[c] * s->m1[c] + s->m2[c] * s->m2[c]) / (2.0 * rho);
    s->e[c] = eg - k;
  }
}

/* Advances `s` by nsteps steps of size dt, using `w` (same shape) as the
 * second buffer; on return the result is in `s`.  stats[ORC_NSTATS] is
 * accumulated.
 *   ORC_EULER: transport then coupling (Sect. 2.4).
 *   ORC_RK2:   the same split applied in each stage of the two-stage scheme
 *              (Sect. 2.4): U1 = step(U^n), U2 = step(U1),
 *              U^{n+1} = (U^n + U2) / 2 for the conserved variables. */
int orc_step(const orc_problem *p, orc_state *s, orc_state *w, double dt, int nsteps,
             int64_t *stats) {
  set_threads(p);
  size_t N = (size_t)p->n[0] * p->n[1] * p->n[2];
  orc_state u = {0};
  double *block = NULL;
  if (p->integrator == ORC_RK2) {
    block = (double *)malloc(9 * N * sizeof(double));
    if (!block) return -1;
    u.E = block;
    u.F0 = block + N;
    u.F1 = block + 2 * N;
    u.F2 = block + 3 * N;
    u.e = block + 4 * N;
    u.m0 = block + 5 * N;
    u.m1 = block + 6 * N;
    u.m2 = block + 7 * N;
    u.rho = p->hydro ? block + 8 * N : s->rho;
  }
  /* without hydro rho is constant and shared; with it each state has its own */
  if (!p->hydro) w->rho = s->rho;
  for (int step = 0; step < nsteps; ++step) {
    int64_t tot[ORC_NSTATS] = {0};
    if (p->integrator == ORC_RK2) {
      euler_pass(p, s, w, dt, tot);   /* stage 1: U1 in w */
      euler_pass(p, w, &u, dt, tot);  /* stage 2: U2 in u */
      average_into(s, &u, N);
    } else {
      euler_pass(p, s, w, dt, tot);
      copy_state(w, s, N, p->hydro);
    }
    if (stats) {
      for (int q = 0; q < ORC_NSTATS; ++q) {
        if (q == ORC_ST_ITMAX) {
          if (tot[q] > stats[q]) stats[q] = tot[q];
        } else {
          stats[q] += tot[q];
        }
      }
    }
  }
  free(block);
  return 0;
}

/* One step for a list of cells only (each computed from its own stencil of
 * the old state): out has 9 values per cell, see cell_step. */
int orc_step_cells(const orc_problem *p, const orc_state *s, double dt, long long ncells,
                   const long long *cells, double *out) {
  if (p->hydro) return -2; /* needs the hydro step of the neighbours: use orc_step */
  set_threads(p);
#pragma omp parallel for schedule(dynamic, 64)
  for (long long q = 0; q < ncells; ++q) {
    long long cc = cells[q];
    int i = (int)(cc % p->n[0]);
    int j = (int)((cc / p->n[0]) % p->n[1]);
    int k = (int)(cc / ((long long)p->n[0] * p->n[1]));
    int64_t st[ORC_NSTATS] = {0};
    cell_step(p, s, dt, i, j, k, -1.0, out + 9 * q, st);
  }
  return 0;
}

/* The coupling step alone for arrays of cells (tests of Sect. 2.8):
 * inputs rho, Tn, kp, Estar, T0 (<= 0: T^n); outputs Enew, Tnew, iters. */
int orc_couple_cells(const orc_problem *p, double dt, long long n, const double *rho,
                     const double *Tn, const double *kp, const double *Estar, const double *T0,
                     double *Enew, double *Tnew, int *iters, int *status) {
  for (long long q = 0; q < n; ++q) {
    int64_t st[ORC_NSTATS] = {0};
    double t0 = (T0 && T0[q] > 0.0) ? T0[q] : Tn[q];
    couple(p, dt, rho[q], Tn[q], t0, kp[q], Estar[q], 0.0, &Enew[q], &Tnew[q], st);
    if (iters) iters[q] = (int)st[ORC_ST_ITERS];
    if (status) status[q] = st[ORC_ST_NOCONV] ? 2 : (st[ORC_ST_FALLBACK] ? 1 : 0);
  }
  return 0;
}

/* HLL face flux between two given states (tests): (EL, FL) and (ER, FR) are
 * face states already fixed; tau < 0 disables the thick correction. */
void orc_face_flux_states(double chat, int d, double EL, const double FL[3], double ER,
                          const double FR[3], double tau, double out[4]) {
  double fL[4], fR[4], lmL, lpL, lmR, lpR;
  orc_phys_flux(chat, EL, FL, d, fL);
  orc_phys_flux(chat, ER, FR, d, fR);
  orc_lambda(EL, FL, d, &lmL, &lpL);
  orc_lambda(ER, FR, d, &lmR, &lpR);
  double sl = chat * (lmL < lmR ? lmL : lmR);
  double sr = chat * (lpL > lpR ? lpL : lpR);
  if (tau > 0.0) {
    double bound = 4.0 * chat / (3.0 * tau);
    if (sl < -bound) sl = -bound;
    if (sr > bound) sr = bound;
  }
  double uL[4] = {EL, FL[0], FL[1], FL[2]}, uR[4] = {ER, FR[0], FR[1], FR[2]};
  orc_hll(sl, sr, uL, uR, fL, fR, out);
}

/* Reconstructed face states at the lower face of cell (i,j,k) along d,
 * before (raw) and after (fixed) the f-fix: out = (EL, FL0..2, ER, FR0..2)
 * raw, then the same fixed (16 values).  For the tests of Sect. 2.5. */
void orc_face_states(const orc_problem *p, const orc_state *s, int i, int j, int k, int d,
                     double out[16]) {
  int idx[3] = {i, j, k};
  double EL, FL[3], EcL, FcL[3], ER, FR[3], EcR, FcR[3];
  face_state(p, s, idx, d, idx[d] - 1, +1, &EL, FL, &EcL, FcL);
  face_state(p, s, idx, d, idx[d], -1, &ER, FR, &EcR, FcR);
  double raw[8] = {EL, FL[0], FL[1], FL[2], ER, FR[0], FR[1], FR[2]};
  orc_fix_face_mode(p->face_fix, &EL, FL, EcL, FcL);
  orc_fix_face_mode(p->face_fix, &ER, FR, EcR, FcR);
  double fixed[8] = {EL, FL[0], FL[1], FL[2], ER, FR[0], FR[1], FR[2]};
  for (int q = 0; q < 8; ++q) {
    out[q] = raw[q];
    out[8 + q] = fixed[q];
  }
}
