// rad_api.cu -- host side of the C ABI declared in include/rad.h: argument
// validation, geometry tables, workspace layout, host<->device transfers
// (pack/unpack kernels between the caller's flat arrays and the padded
// ghost-layer layout) and the step dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "ctx_internal.h"
#include "hydro.cuh"

using namespace m1;


static const char* kMsg[] = {"ok",
                             "invalid argument",
                             "workspace missing or too small / out of memory",
                             "CUDA runtime error",
                             "non-physical input or state",
                             "coupling iteration did not converge",
                             "bounded device wait ran out",
                             "unsupported request",
                             "device-side index check failed (debug build)"};

extern "C" const char* rad_strerror(rad_status s) {
  int i = int(s);
  if (i < 0 || i > 8) return "unknown status";
  return kMsg[i];
}

extern "C" rad_status rad_default_params(rad_params* p) {
  if (!p) return RAD_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->chat = 1.0;
  p->c = 1.0;
  p->a_rad = 1.0;
  p->gamma_gas = 5.0 / 3.0;
  p->mu = 1.0;
  p->cfl = 0.4;
  p->e_floor = 1e-30;
  p->precision = RAD_FP64;
  p->implicit_mode = RAD_LINEARIZED_ONCE;
  p->newton_rtol = 1e-12;
  p->newton_maxit = 50;
  p->ncomp = 3;
  p->use_mlp = 0;
  p->mlp_gate = 1e-2;
  p->integrator = RAD_EULER;
  p->irradiation = 0;
  p->reconstruction = RAD_PLM;
  p->face_fix = RAD_FIX_FPRESERVE;
  p->riemann = RAD_HLL;
  p->hydro = 0;
  return RAD_OK;
}

static_assert(int(BC_OUTFLOW) == int(RAD_BC_OUTFLOW) && int(BC_PERIODIC) == int(RAD_BC_PERIODIC) &&
                  int(BC_REFLECT) == int(RAD_BC_REFLECTIVE) && int(BC_FIXED) == int(RAD_BC_FIXED) &&
                  int(BC_LTE) == int(RAD_BC_LTE),
              "device boundary kinds follow rad_bc");

// ---------------------------------------------------------------------------
// geometry tables
// ---------------------------------------------------------------------------

static int map_index(int i, int n, int lo_periodic, int hi_periodic) {
  if (i < 0) return lo_periodic ? ((i % n) + n) % n : 0;
  if (i >= n) return hi_periodic ? i % n : n - 1;
  return i;
}

// Centre of cell i (ghosts: mirrored for outflow, shifted by the period).
static double centre_ext(const std::vector<double>& x, int n, int i, int lo_p, int hi_p) {
  if (i >= 0 && i < n) return 0.5 * (x[i] + x[i + 1]);
  double L = x[n] - x[0];
  if (i < 0) return lo_p ? centre_ext(x, n, i + n, lo_p, hi_p) - L
                         : 2.0 * x[0] - centre_ext(x, n, -1 - i, lo_p, hi_p);
  return hi_p ? centre_ext(x, n, i - n, lo_p, hi_p) + L
              : 2.0 * x[n] - centre_ext(x, n, 2 * n - 1 - i, lo_p, hi_p);
}

static void build_tables(rad_ctx* c) {
  for (int d = 0; d < 3; ++d) {
    const int n = c->n[d];
    const int g = d < c->ndim ? 2 : 0;
    const int len = n + 2 * g;
    c->len[d] = len;
    const std::vector<double>& x = c->xf[d];
    const int lp = c->bc_lo[d] == RAD_BC_PERIODIC, hp = c->bc_hi[d] == RAD_BC_PERIODIC;
    std::vector<double>& T = c->tab64[d];
    T.assign(size_t(TAB_N) * len, 0.0);
    auto at = [&](int slot, int ip) -> double& { return T[size_t(slot) * len + ip]; };
    for (int ip = 0; ip < len; ++ip) {
      const int i = ip - g;
      const int mi = map_index(i, n, lp, hp);
      const double xc = centre_ext(x, n, i, lp, hp);
      if (ip + 1 < len) at(TAB_IDXC, ip) = 1.0 / (centre_ext(x, n, i + 1, lp, hp) - xc);
      if (i >= 0 && i <= n) at(TAB_HLO, ip) = x[i] - xc;
      if (i + 1 >= 0 && i + 1 <= n) at(TAB_HHI, ip) = x[i + 1] - xc;
      const double a = x[mi], b = x[mi + 1];
      at(TAB_WID, ip) = b - a;
      if (d == 0) at(TAB_RC, ip) = 0.5 * (a + b);
      if (d == 1 && c->geom == RAD_SPHERICAL) at(TAB_RC, ip) = std::sin(0.5 * (a + b));
      if (i < 0 || i >= n) continue;
      // interior: area/volume factors
      if (c->geom == RAD_CARTESIAN || (c->geom == RAD_CYLINDRICAL && d != 0) ||
          (c->geom == RAD_SPHERICAL && d == 2)) {
        at(TAB_ALO, ip) = at(TAB_AHI, ip) = 1.0 / (b - a);
      } else if (c->geom == RAD_CYLINDRICAL) {  // d == 0, radius R
        double den = b * b - a * a;
        at(TAB_ALO, ip) = 2.0 * a / den;
        at(TAB_AHI, ip) = 2.0 * b / den;
        double invRc = 2.0 / (a + b);
        at(TAB_MET, ip) = invRc;
        at(TAB_AMLO, ip) = at(TAB_ALO, ip) * a * invRc;
        at(TAB_AMHI, ip) = at(TAB_AHI, ip) * b * invRc;
      } else if (d == 0) {  // spherical radius
        double den = b * b * b - a * a * a;
        at(TAB_ALO, ip) = 3.0 * a * a / den;
        at(TAB_AHI, ip) = 3.0 * b * b / den;
        double invrt = 3.0 * (b * b - a * a) / (2.0 * den);
        at(TAB_MET, ip) = invrt;
        at(TAB_AMLO, ip) = at(TAB_ALO, ip) * a * invrt;
        at(TAB_AMHI, ip) = at(TAB_AHI, ip) * b * invrt;
      } else {  // spherical theta
        double dcos = std::cos(a) - std::cos(b);
        double sc = std::sin(0.5 * (a + b));
        at(TAB_ALO, ip) = std::sin(a) / dcos;
        at(TAB_AHI, ip) = std::sin(b) / dcos;
        at(TAB_MET, ip) = (std::sin(b) - std::sin(a)) / dcos;
        at(TAB_AMLO, ip) = at(TAB_ALO, ip) * std::sin(a) / sc;
        at(TAB_AMHI, ip) = at(TAB_AHI, ip) * std::sin(b) / sc;
        at(TAB_PHF, ip) = (b - a) / dcos;
      }
    }
    c->tab32[d].resize(T.size());
    for (size_t k = 0; k < T.size(); ++k) c->tab32[d][k] = float(T[k]);
  }
}

// dt = cfl / max over cells of sum_d chat / h_d (Sect. 2.4 item 10).
static double cfl_dt(const rad_ctx* c) {
  const std::vector<double>*x = c->xf;
  double worst = 0.0;
  for (int k = 0; k < c->n[2]; ++k) {
    double w2 = x[2][k + 1] - x[2][k];
    for (int j = 0; j < c->n[1]; ++j) {
      double w1 = x[1][j + 1] - x[1][j];
      double sth = std::sin(0.5 * (x[1][j] + x[1][j + 1]));
      for (int i = 0; i < c->n[0]; ++i) {
        double w0 = x[0][i + 1] - x[0][i];
        double rc = 0.5 * (x[0][i] + x[0][i + 1]);
        double h[3] = {w0, w1, w2};
        if (c->geom == RAD_CYLINDRICAL) h[1] = rc * w1;
        if (c->geom == RAD_SPHERICAL) {
          h[1] = rc * w1;
          h[2] = rc * sth * w2;
        }
        double s = 0.0;
        for (int d = 0; d < c->ndim; ++d) s += c->par.chat / h[d];
        worst = std::max(worst, s);
      }
    }
  }
  return c->par.cfl / worst;
}

// ---------------------------------------------------------------------------
// creation and workspace
// ---------------------------------------------------------------------------

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// float4 records (the learned guess's training and prediction sets, the log
// of converged solves) are read and written as 16-byte vectors: a pointer
// off that boundary is refused on the host instead of faulting on the device.
static bool misaligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

extern "C" rad_status rad_create(const rad_grid* grid, int geometry, const rad_opacity* opacity,
                                 const rad_params* params, rad_ctx** out) {
  NvtxRange nvtx_range("rad_create");
  if (!grid || !opacity || !params || !out) return RAD_EINVAL;
  if (grid->ndim < 1 || grid->ndim > 3) return RAD_EINVAL;
  if (geometry < 0 || geometry > 2) return RAD_EINVAL;
  const rad_params& p = *params;
  if (!finite_pos(p.chat) || !(p.c >= p.chat) || !std::isfinite(p.c) || !finite_pos(p.a_rad) ||
      !(p.gamma_gas > 1.0) || !finite_pos(p.mu) || !(p.cfl > 0.0 && p.cfl <= 1.0) ||
      !finite_pos(p.e_floor))
    return RAD_EINVAL;
  if (p.precision != RAD_FP64 && p.precision != RAD_FP32_SPLIT) return RAD_EINVAL;
  if (p.implicit_mode != RAD_LINEARIZED_ONCE && p.implicit_mode != RAD_NEWTON &&
      p.implicit_mode != RAD_ABSORPTION_ONLY)
    return RAD_EINVAL;
  if (p.reconstruction < RAD_PLM || p.reconstruction > RAD_LIMO3) return RAD_EINVAL;
  if (p.face_fix < RAD_FIX_FPRESERVE || p.face_fix > RAD_FIX_CLIP) return RAD_EINVAL;
  if (p.riemann < RAD_HLL || p.riemann > RAD_LF) return RAD_EINVAL;
  if (p.hydro != 0 && p.hydro != 1) return RAD_EINVAL;
  if (p.hydro && geometry != RAD_CARTESIAN) return RAD_EUNSUPPORTED;
  if (p.implicit_mode == RAD_NEWTON && (!(p.newton_rtol > 0.0) || p.newton_maxit < 1))
    return RAD_EINVAL;
  if (p.ncomp < 1 || p.ncomp > 3) return RAD_EINVAL;
  if (p.use_mlp && (p.implicit_mode != RAD_NEWTON || !(p.mlp_gate >= 0.0))) return RAD_EINVAL;
  if (p.integrator != RAD_EULER && p.integrator != RAD_RK2) return RAD_EINVAL;
  if (p.irradiation != 0 && p.irradiation != 1) return RAD_EINVAL;
  size_t N = 1;
  for (int d = 0; d < 3; ++d) {
    int n = grid->n[d];
    if (n < 1 || (d >= grid->ndim && n != 1) || !grid->xface[d]) return RAD_EINVAL;
    if (n > (1 << 24)) return RAD_EINVAL;
    for (int i = 0; i < n; ++i)
      if (!(grid->xface[d][i + 1] > grid->xface[d][i]) || !std::isfinite(grid->xface[d][i + 1]))
        return RAD_EINVAL;
    if (d < grid->ndim) {
      int lo = grid->bc_lo[d], hi = grid->bc_hi[d];
      if (lo < RAD_BC_OUTFLOW || lo > RAD_BC_LTE || hi < RAD_BC_OUTFLOW || hi > RAD_BC_LTE)
        return RAD_EINVAL;
      if ((lo == RAD_BC_PERIODIC) != (hi == RAD_BC_PERIODIC)) return RAD_EINVAL;
      for (int side = 0; side < 2; ++side) {
        const int bc = side ? hi : lo;
        const double* v = grid->bc_value[d][side];
        if ((bc == RAD_BC_FIXED || bc == RAD_BC_LTE) && !(v[4] > 0.0 && std::isfinite(v[4])))
          return RAD_EINVAL;
        if (bc == RAD_BC_FIXED &&
            !(v[0] > 0.0 && std::isfinite(v[0]) &&
              v[1] * v[1] + v[2] * v[2] + v[3] * v[3] <= v[0] * v[0] * (1.0 + 1e-12)))
          return RAD_EINVAL;
        if (bc == RAD_BC_FIXED)
          for (int q = p.ncomp; q < 3; ++q)
            if (v[1 + q] != 0.0) return RAD_EINVAL;  // components the caller does not carry
      }
    }
    N *= size_t(n);
  }
  if (N > (size_t(1) << 34)) return RAD_EINVAL;
  if (geometry != RAD_CARTESIAN && grid->xface[0][0] < 0.0) return RAD_EINVAL;
  if (geometry == RAD_SPHERICAL && (grid->xface[1][0] < 0.0 || grid->xface[1][grid->n[1]] > M_PI + 1e-12))
    return RAD_EINVAL;
  const rad_opacity& o = *opacity;
  if (o.kind < 0 || o.kind > 2) return RAD_EINVAL;
  if (o.kind == RAD_OPAC_CONST && !(o.kappa_p >= 0 && o.kappa_r >= 0 && o.sigma >= 0))
    return RAD_EINVAL;
  if (o.kind == RAD_OPAC_POWERLAW &&
      !(o.k0 >= 0 && o.kmin >= 0 && o.kmax >= o.kmin && o.sigma_ratio >= 0))
    return RAD_EINVAL;
  if (o.kind == RAD_OPAC_TABLE &&
      (o.nrho < 2 || o.nT < 2 || !o.table_log10_kappa || !(o.lrho1 > o.lrho0) ||
       !(o.lT1 > o.lT0) || !(o.sigma_ratio >= 0)))
    return RAD_EINVAL;

  rad_ctx* c = new (std::nothrow) rad_ctx();
  if (!c) return RAD_ENOMEM;
  c->ndim = grid->ndim;
  c->geom = geometry;
  for (int d = 0; d < 3; ++d) {
    c->n[d] = grid->n[d];
    c->bc_lo[d] = d < grid->ndim ? grid->bc_lo[d] : 0;
    c->bc_hi[d] = d < grid->ndim ? grid->bc_hi[d] : 0;
    for (int side = 0; side < 2; ++side)
      for (int q = 0; q < 5; ++q) c->bc_val[d][side][q] = grid->bc_value[d][side][q];
    c->xf[d].assign(grid->xface[d], grid->xface[d] + grid->n[d] + 1);
  }
  c->opac = o;
  if (o.kind == RAD_OPAC_TABLE) {
    c->table32.assign(o.table_log10_kappa, o.table_log10_kappa + size_t(o.nrho) * o.nT);
    c->table64.assign(c->table32.begin(), c->table32.end());
  } else {
    c->table32.assign(4, 0.f);
    c->table64.assign(4, 0.0);
  }
  c->opac.table_log10_kappa = nullptr;
  c->par = p;
  c->N = N;
  c->nc = (geometry == RAD_CARTESIAN) ? std::max(p.ncomp, grid->ndim) : 3;
  c->esize = p.precision == RAD_FP64 ? 8 : 4;
  build_tables(c);
  c->dt_cfl = cfl_dt(c);
  c->uniform = geometry == RAD_CARTESIAN;
  for (int d = 0; d < c->ndim && c->uniform; ++d) {
    const std::vector<double>& x = c->xf[d];
    double w0 = x[1] - x[0];
    for (int i = 1; i < c->n[d]; ++i)
      if (std::fabs((x[i + 1] - x[i]) - w0) > 1e-12 * w0) {
        c->uniform = false;
        break;
      }
  }
  // the general form of the step kernel carries the face options, the
  // absorption-only coupling and the irradiation deposit (register-tiled
  // shapes only); the default form compiles them out
  c->general = p.reconstruction != RAD_PLM || p.face_fix != RAD_FIX_FPRESERVE ||
               p.riemann != RAD_HLL || p.irradiation || p.implicit_mode == RAD_ABSORPTION_ONLY ||
               p.hydro;
  if (p.hydro) {
    c->hydro_fn = select_hydro(p.precision == RAD_FP32_SPLIT, c->ndim, c->nc, c->uniform);
    c->gas_cfl_fn = select_gas_cfl(p.precision == RAD_FP32_SPLIT, c->ndim, c->nc);
    if (!c->hydro_fn || !c->gas_cfl_fn) {
      delete c;
      return RAD_EUNSUPPORTED;
    }
  }
  const bool options =
      p.reconstruction != RAD_PLM || p.face_fix != RAD_FIX_FPRESERVE || p.riemann != RAD_HLL;
  // directions 1 and 2 evenly spaced (a grid stretched in its first
  // direction only, such as a log-spaced radius)
  bool even_yz = c->ndim == 3;
  for (int d = 1; d < 3 && even_yz; ++d) {
    const std::vector<double>& x = c->xf[d];
    const double w0 = x[1] - x[0];
    for (int i = 1; i < c->n[d]; ++i)
      if (std::fabs((x[i + 1] - x[i]) - w0) > 1e-12 * w0) {
        even_yz = false;
        break;
      }
  }
  c->launch = select_launch(p.precision == RAD_FP32_SPLIT, c->ndim, geometry, c->nc,
                            (c->uniform ? 1 : 0) | (even_yz ? 2 : 0), c->general, options);
  c->qpass = select_queue_pass(p.precision == RAD_FP32_SPLIT, c->ndim, c->nc);
  if (!c->launch.fn) {
    delete c;
    return RAD_EUNSUPPORTED;
  }
  // padded layout
  StepDims& D = c->dims;
  D.ndim = c->ndim;
  for (int d = 0; d < 3; ++d) {
    D.n[d] = c->n[d];
    D.g[d] = d < c->ndim ? 2 : 0;
    D.pn[d] = c->n[d] + 2 * D.g[d];
    D.bc_lo[d] = c->bc_lo[d];
    D.bc_hi[d] = c->bc_hi[d];
  }
  const int align_elems = int(16 / c->esize);
  D.pn[0] = (D.pn[0] + align_elems - 1) / align_elems * align_elems;
  D.sy = D.pn[0];
  D.sz = (long long)D.pn[0] * D.pn[1];
  c->pcells = size_t(D.pn[0]) * D.pn[1] * D.pn[2];
  // workspace offsets (256-byte aligned pieces)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o2 = off;
    off += (bytes + 255) / 256 * 256;
    return o2;
  };
  const size_t arr = c->pcells * c->esize;
  c->nbuf = p.integrator == RAD_RK2 ? 3 : 2;
  for (int b = 0; b < 3; ++b)
    for (int k = 0; k < 8; ++k) {
      int comp = (k >= 1 && k <= 3) ? k - 1 : (k >= 5 ? k - 5 : 0);
      bool used = b < c->nbuf && ((k == 0 || k == 4) || comp < c->nc);
      c->off_state[b][k] = used ? take(arr) : size_t(-1);
    }
  c->off_rho = take(arr);
  if (p.hydro) {
    for (int b = 0; b < c->nbuf; ++b) c->off_rho_buf[b] = b == 0 ? c->off_rho : take(arr);
    c->off_gas_e = take(arr);
    for (int q = 0; q < c->nc; ++q) c->off_gas_m[q] = take(arr);
    c->off_cfl = take(sizeof(unsigned long long));
  }
  if (p.irradiation) c->off_qirr = take(arr);
  const size_t tsz = c->esize;
  for (int d = 0; d < 3; ++d) c->off_tab_dir[d] = take(size_t(TAB_N) * c->len[d] * tsz);
  c->off_op32 = take(c->table32.size() * 4);
  c->off_op64 = take(c->table64.size() * 8);
  c->off_stats = take(sizeof(unsigned long long) * ST_N);
  c->off_status = take(sizeof(int) * 4);
  c->off_stage = take(3 * N * c->esize);
  const size_t np = size_t(mlp_nparam()) * sizeof(float);
  c->off_mlp = take(np);
  c->off_grad = take(np);
  c->off_m = take(np);
  c->off_v = take(np);
  c->off_loss = take(sizeof(double));
  c->off_qcount = take(sizeof(unsigned int));
  c->off_lcount = take(sizeof(unsigned int));
  c->off_queue = p.implicit_mode == RAD_NEWTON ? take(N * sizeof(long long)) : 0;
  c->total = off;
  *out = c;
  return RAD_OK;
}

extern "C" rad_status rad_workspace_size(const rad_ctx* c, size_t* bytes) {
  if (!c || !bytes) return RAD_EINVAL;
  *bytes = c->total;
  return RAD_OK;
}

static rad_status cuda_err(cudaError_t e) { return e == cudaSuccess ? RAD_OK : RAD_ECUDA; }

static rad_status upload_static(rad_ctx* c) {
  cudaError_t e;
  for (int d = 0; d < 3; ++d) {
    const void* src = c->esize == 8 ? (const void*)c->tab64[d].data() : (const void*)c->tab32[d].data();
    e = cudaMemcpyAsync(c->ws + c->off_tab_dir[d], src, size_t(TAB_N) * c->len[d] * c->esize,
                        cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return RAD_ECUDA;
  }
  e = cudaMemcpyAsync(c->ws + c->off_op32, c->table32.data(), c->table32.size() * 4,
                      cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return RAD_ECUDA;
  e = cudaMemcpyAsync(c->ws + c->off_op64, c->table64.data(), c->table64.size() * 8,
                      cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return RAD_ECUDA;
  e = cudaMemsetAsync(c->ws + c->off_stats, 0, sizeof(unsigned long long) * ST_N + 256, c->stream);
  if (e != cudaSuccess) return RAD_ECUDA;
  e = cudaMemsetAsync(c->ws + c->off_status, 0, sizeof(int) * 4, c->stream);
  if (e != cudaSuccess) return RAD_ECUDA;
  if (c->off_qirr != size_t(-1)) {
    e = cudaMemsetAsync(c->ws + c->off_qirr, 0, c->pcells * c->esize, c->stream);
    if (e != cudaSuccess) return RAD_ECUDA;
  }
  const size_t np = size_t(mlp_nparam()) * sizeof(float);
  e = cudaMemsetAsync(c->ws + c->off_mlp, 0, c->off_qcount - c->off_mlp, c->stream);
  if (e != cudaSuccess) return RAD_ECUDA;
  (void)np;
  c->mlp_ready = false;
  c->adam_step = 0;
  return cuda_err(cudaStreamSynchronize(c->stream));
}

extern "C" rad_status rad_bind_workspace(rad_ctx* c, void* ptr, size_t bytes) {
  if (!c || !ptr) return RAD_EINVAL;
  if (reinterpret_cast<uintptr_t>(ptr) % 256) return RAD_EINVAL;
  if (bytes < c->total) return RAD_ENOMEM;
  if (c->ws_owned) {
    cudaFree(c->ws);
    c->ws_owned = false;
  }
  c->ws = static_cast<char*>(ptr);
  c->ws_bytes = bytes;
  c->have_gas = c->have_rad = false;
  c->tma.clear();
  return upload_static(c);
}

extern "C" rad_status rad_alloc_workspace(rad_ctx* c) {
  if (!c) return RAD_EINVAL;
  void* p = nullptr;
  if (cudaMalloc(&p, c->total) != cudaSuccess) return RAD_ENOMEM;
  rad_status s = rad_bind_workspace(c, p, c->total);
  if (s != RAD_OK) {
    cudaFree(p);
    return s;
  }
  c->ws_owned = true;
  return RAD_OK;
}

extern "C" rad_status rad_set_stream(rad_ctx* c, void* stream) {
  if (!c) return RAD_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  return RAD_OK;
}

static void* state_ptr(rad_ctx* c, int b, int k);
static void* rho_ptr(rad_ctx* c, int b);

template <class P>
static cudaError_t enqueue_gas_cfl(rad_ctx* c) {
  using S = typename P::S;
  using T = typename P::T;
  GasCflArgs<P> g{};
  g.dim = c->dims;
  for (int d = 0; d < 3; ++d) {
    g.geo.tab[d] = reinterpret_cast<const T*>(c->ws + c->off_tab_dir[d]);
    g.geo.len[d] = c->len[d];
  }
  g.rho = static_cast<const S*>(rho_ptr(c, c->cur));
  g.e = static_cast<const S*>(state_ptr(c, c->cur, 4));
  for (int q = 0; q < 3; ++q)
    g.m[q] = q < c->nc ? static_cast<const S*>(state_ptr(c, c->cur, 5 + q)) : nullptr;
  g.chat = c->par.chat;
  g.gamma = c->par.gamma_gas;
  g.out = reinterpret_cast<unsigned long long*>(c->ws + c->off_cfl);
  return c->gas_cfl_fn(&g, c->stream);
}

// The CFL step: the radiation's (fixed by the grid), or with evolved gas the
// step of the current state, max(chat, |v_d| + c_s) per direction (reduced
// on the device; the call waits for it).
static rad_status current_dt(rad_ctx* c, double* dt) {
  if (!c->par.hydro) {
    *dt = c->dt_cfl;
    return RAD_OK;
  }
  if (!c->ws || !c->have_gas) return RAD_EINVAL;
  unsigned long long bits = 0;
  if (cudaMemsetAsync(c->ws + c->off_cfl, 0, sizeof(bits), c->stream) != cudaSuccess)
    return RAD_ECUDA;
  cudaError_t e = c->esize == 8 ? enqueue_gas_cfl<Fp64>(c) : enqueue_gas_cfl<Split>(c);
  if (e != cudaSuccess ||
      cudaMemcpyAsync(&bits, c->ws + c->off_cfl, sizeof(bits), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  double rate;
  std::memcpy(&rate, &bits, sizeof(rate));
  if (!(rate > 0.0) || !std::isfinite(rate)) return RAD_ENONPHYS;
  *dt = c->par.cfl / rate;
  return RAD_OK;
}

extern "C" rad_status rad_dt(const rad_ctx* c, double* dt) {
  if (!c || !dt) return RAD_EINVAL;
  return current_dt(const_cast<rad_ctx*>(c), dt);
}

// ---------------------------------------------------------------------------
// pack / unpack kernels
// ---------------------------------------------------------------------------

enum { PK_COPY = 0, PK_MOM = 1, PK_EINT = 2 };

// What a packed array holds, for the ghost rules of the boundary kinds.
enum { FK_RHO = 0, FK_E = 1, FK_F = 2, FK_M = 3, FK_EINT = 4, FK_OTHER = 5 };

// Boundary states of the FIXED and LTE sides: (E, F0, F1, F2, T_b) per
// direction and side, and a_R for the LTE energy a_R T_b^4.
struct GhostVals {
  double v[3][2][5];
  double a_rad;
};

// Fills every padded cell (ghosts included) of dst from the flat array src
// (x fastest); PK_MOM multiplies by rho (flat), PK_EINT by rho * cvfac.  A
// ghost takes the wrapped (periodic), mirrored (reflective) or edge cell
// (the other kinds); reflective sides negate the normal component (comp ==
// direction) of F and m; FIXED and LTE sides substitute their boundary
// state: E (FIXED: E_b, LTE: a_R T_b^4), F (FIXED: F_b), m (zero) and
// e = rho cvfac T_b.  Caller values that are not finite, and E, rho or T
// that are not positive, set STATUS_NONPHYS in *bad.
template <class S>
__global__ void pack_kernel(S* __restrict__ dst, const S* __restrict__ src,
                            const S* __restrict__ rho, StepDims D, int mode, double cvfac,
                            int field, int comp, GhostVals gv, int* __restrict__ bad) {
  const long long total = (long long)D.pn[0] * D.pn[1] * D.pn[2];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    int c[3];
    long long r = p;
    c[0] = int(r % D.pn[0]);
    r /= D.pn[0];
    c[1] = int(r % D.pn[1]);
    c[2] = int(r / D.pn[1]);
    long long lin = 0, mul = 1;
    double sign = 1.0;
    int over = -1;             // direction whose boundary state replaces the value
    int over_side = 0;
    for (int d = 0; d < 3; ++d) {
      int i = c[d] - D.g[d];
      const int n = D.n[d];
      if (i < 0 || i >= n) {
        const int side = i < 0 ? 0 : 1;
        const int bc = side ? D.bc_hi[d] : D.bc_lo[d];
        if (bc == BC_PERIODIC) {
          i = ((i % n) + n) % n;
        } else if (bc == BC_REFLECT) {
          i = min(max(side ? 2 * n - 1 - i : -1 - i, 0), n - 1);
          if ((field == FK_F || field == FK_M) && comp == d) sign = -sign;
        } else {
          i = side ? n - 1 : 0;
          if (bc == BC_FIXED || bc == BC_LTE) {
            over = d;
            over_side = side;
          }
        }
      }
      lin += (long long)i * mul;
      mul *= n;
    }
    double v = double(src[lin]);
    {
      const bool positive = field == FK_E || field == FK_RHO || field == FK_EINT;
      if (!isfinite(v) || (positive && !(v > 0.0))) atomicOr(bad, STATUS_NONPHYS);
    }
    if (mode == PK_MOM) v = v * double(rho[lin]);
    if (mode == PK_EINT) v = v * double(rho[lin]) * cvfac;
    if (over >= 0) {
      const int bc = over_side ? D.bc_hi[over] : D.bc_lo[over];
      const double* b = gv.v[over][over_side];
      if (field == FK_E) v = bc == BC_FIXED ? b[0] : gv.a_rad * b[4] * b[4] * b[4] * b[4];
      if (field == FK_F && bc == BC_FIXED) v = b[1 + comp];
      if (field == FK_M) v = 0.0;
      if (field == FK_EINT) v = b[4] * double(rho[lin]) * cvfac;
    }
    dst[p] = S(sign * v);
  }
}

enum { UN_COPY = 0, UN_TEMP = 1 };

template <class S>
__global__ void unpack_kernel(S* __restrict__ dst, const S* __restrict__ src,
                              const S* __restrict__ rho, StepDims D, int mode, double cvfac) {
  const long long N = (long long)D.n[0] * D.n[1] * D.n[2];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
       q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    int i = int(r % D.n[0]);
    r /= D.n[0];
    int j = int(r % D.n[1]);
    int k = int(r / D.n[1]);
    long long p = (long long)(i + D.g[0]) + D.sy * (j + D.g[1]) + D.sz * (k + D.g[2]);
    S v = src[p];
    if (mode == UN_TEMP) v = S(double(v) / (double(rho[p]) * cvfac));
    dst[q] = v;
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return int(std::min<long long>(std::max<long long>(b, 1), 148 * 32));
}

template <class S>
static rad_status pack(rad_ctx* c, S* dst, const S* src, const S* rho, int mode, int field,
                       int comp = 0) {
  double cvfac = 1.0 / (c->par.mu * (c->par.gamma_gas - 1.0));
  GhostVals gv;
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side)
      for (int q = 0; q < 5; ++q) gv.v[d][side][q] = c->bc_val[d][side][q];
  gv.a_rad = c->par.a_rad;
  pack_kernel<S><<<grid_for((long long)c->pcells), 256, 0, c->stream>>>(
      dst, src, rho, c->dims, mode, cvfac, field, comp, gv,
      reinterpret_cast<int*>(c->ws + c->off_status) + 1);
  return cuda_err(cudaGetLastError());
}

// The input word (status slot 1) that pack_kernel sets for non-physical
// caller values: read and cleared once the uploads have finished.
static rad_status take_input_status(rad_ctx* c) {
  int st = 0;
  int* w = reinterpret_cast<int*>(c->ws + c->off_status) + 1;
  if (cudaMemcpyAsync(&st, w, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (!st) return RAD_OK;
  if (cudaMemsetAsync(w, 0, sizeof(int), c->stream) != cudaSuccess) return RAD_ECUDA;
  return RAD_ENONPHYS;
}

// End of a synchronous upload: wait, then report non-physical input.
static rad_status finish_upload(rad_ctx* c, bool wait) {
  if (!wait) return cuda_err(cudaGetLastError());
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RAD_ECUDA;
  return take_input_status(c);
}

static void* state_ptr(rad_ctx* c, int b, int k) {
  size_t o = c->off_state[b][k];
  return o == size_t(-1) ? nullptr : c->ws + o;
}

// Density of state buffer b: one shared array, or one per buffer when the
// gas is evolved.
static void* rho_ptr(rad_ctx* c, int b) {
  return c->ws + (c->par.hydro ? c->off_rho_buf[b] : c->off_rho);
}

// Copies `count` values from the caller (host or device) to a device flat
// array and returns it: the staging area for host input, else the pointer.
static const void* stage_in(rad_ctx* c, const void* src, size_t count, int slot, int on_device,
                            rad_status* st) {
  *st = RAD_OK;
  if (on_device) return src;
  char* dst = c->ws + c->off_stage + size_t(slot) * c->N * c->esize;
  if (cudaMemcpyAsync(dst, src, count * c->esize, cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess)
    *st = RAD_ECUDA;
  return dst;
}

template <class S>
static rad_status set_gas_t(rad_ctx* c, const void* rho, const void* v, const void* T, int dev,
                           bool wait = true) {
  rad_status st;
  // rho first (flat copy kept in stage slot 0 while m and e are built)
  const S* r = static_cast<const S*>(stage_in(c, rho, c->N, 0, dev, &st));
  if (st) return st;
  for (int b = 0; b < (c->par.hydro ? c->nbuf : 1); ++b)
    if ((st = pack<S>(c, static_cast<S*>(rho_ptr(c, b)), r, r, PK_COPY, FK_RHO))) return st;
  // v: ncomp arrays (host input goes through stage slot 1 one component at a
  // time); internal components beyond ncomp are zero
  for (int comp = 0; comp < c->nc; ++comp) {
    const S* src = nullptr;
    if (comp < c->par.ncomp) {
      if (dev) {
        src = static_cast<const S*>(v) + comp * c->N;
      } else {
        char* slot = c->ws + c->off_stage + c->N * c->esize;
        if (cudaMemcpyAsync(slot, static_cast<const char*>(v) + comp * c->N * c->esize,
                            c->N * c->esize, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
          return RAD_ECUDA;
        src = reinterpret_cast<const S*>(slot);
      }
    }
    for (int b = 0; b < c->nbuf; ++b) {
      S* dst = static_cast<S*>(state_ptr(c, b, 5 + comp));
      if (src) {
        if ((st = pack<S>(c, dst, src, r, PK_MOM, FK_M, comp))) return st;
      } else if (cudaMemsetAsync(dst, 0, c->pcells * c->esize, c->stream) != cudaSuccess) {
        return RAD_ECUDA;
      }
    }
  }
  const S* t = static_cast<const S*>(stage_in(c, T, c->N, 2, dev, &st));
  if (st) return st;
  for (int b = 0; b < c->nbuf; ++b)
    if ((st = pack<S>(c, static_cast<S*>(state_ptr(c, b, 4)), t, r, PK_EINT, FK_EINT))) return st;
  c->have_gas = true;
  return finish_upload(c, wait);
}

extern "C" rad_status rad_set_gas(rad_ctx* c, const void* rho, const void* v, const void* T,
                                  int on_device) {
  NvtxRange nvtx_range("rad_set_gas");
  if (!c || !rho || !v || !T) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  return c->esize == 8 ? set_gas_t<double>(c, rho, v, T, on_device)
                       : set_gas_t<float>(c, rho, v, T, on_device);
}

template <class S>
static rad_status set_rad_t(rad_ctx* c, const void* E, const void* F, int dev, bool wait = true) {
  rad_status st;
  const S* e = static_cast<const S*>(stage_in(c, E, c->N, 0, dev, &st));
  if (st) return st;
  for (int b = 0; b < c->nbuf; ++b)
    if ((st = pack<S>(c, static_cast<S*>(state_ptr(c, b, 0)), e, e, PK_COPY, FK_E))) return st;
  for (int comp = 0; comp < c->nc; ++comp) {
    for (int b = 0; b < c->nbuf; ++b) {
      S* dst = static_cast<S*>(state_ptr(c, b, 1 + comp));
      if (comp < c->par.ncomp) {
        const S* src;
        if (dev) {
          src = static_cast<const S*>(F) + comp * c->N;
        } else {
          char* slot = c->ws + c->off_stage + c->N * c->esize;
          if (b == 0 && cudaMemcpyAsync(slot, static_cast<const char*>(F) + comp * c->N * c->esize,
                                        c->N * c->esize, cudaMemcpyHostToDevice,
                                        c->stream) != cudaSuccess)
            return RAD_ECUDA;
          src = reinterpret_cast<const S*>(slot);
        }
        if ((st = pack<S>(c, dst, src, src, PK_COPY, FK_F, comp))) return st;
      } else if (cudaMemsetAsync(dst, 0, c->pcells * c->esize, c->stream) != cudaSuccess) {
        return RAD_ECUDA;
      }
    }
  }
  c->have_rad = true;
  return finish_upload(c, wait);
}

template <class S>
static rad_status set_irr_t(rad_ctx* c, const void* q, int dev) {
  rad_status st;
  const S* src = static_cast<const S*>(stage_in(c, q, c->N, 0, dev, &st));
  if (st) return st;
  if ((st = pack<S>(c, reinterpret_cast<S*>(c->ws + c->off_qirr), src, src, PK_COPY, FK_OTHER))) return st;
  return finish_upload(c, true);
}

extern "C" rad_status rad_set_irradiation(rad_ctx* c, const void* q, int on_device) {
  if (!c || !q || c->off_qirr == size_t(-1)) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  return c->esize == 8 ? set_irr_t<double>(c, q, on_device) : set_irr_t<float>(c, q, on_device);
}

extern "C" rad_status rad_set_rad(rad_ctx* c, const void* E, const void* F, int on_device) {
  NvtxRange nvtx_range("rad_set_rad");
  if (!c || !E || !F) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  return c->esize == 8 ? set_rad_t<double>(c, E, F, on_device)
                       : set_rad_t<float>(c, E, F, on_device);
}

// ---------------------------------------------------------------------------
// stepping
// ---------------------------------------------------------------------------

template <class S>
static void fill_fields(rad_ctx* c, int b, Fields<S>& f) {
  f.E = static_cast<S*>(state_ptr(c, b, 0));
  for (int q = 0; q < 3; ++q) {
    f.F[q] = static_cast<S*>(state_ptr(c, b, 1 + q));
    f.m[q] = static_cast<S*>(state_ptr(c, b, 5 + q));
  }
  f.e = static_cast<S*>(state_ptr(c, b, 4));
}

template <class P>
static void fill_args(rad_ctx* c, StepArgs<P>& a, double dt, int in_buf, int out_buf) {
  using S = typename P::S;
  using T = typename P::T;
  a.dim = c->dims;
  fill_fields<S>(c, in_buf, a.in);
  fill_fields<S>(c, out_buf, a.out);
  a.stash = a.out;
  a.average = 0;
  a.qirr = c->off_qirr != size_t(-1) ? reinterpret_cast<const S*>(c->ws + c->off_qirr) : nullptr;
  a.rho = static_cast<const S*>(rho_ptr(c, in_buf));
  a.rho_avg = nullptr;
  a.hydro = c->par.hydro;
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) a.bcT[d][side] = c->bc_val[d][side][4];
  for (int d = 0; d < 3; ++d) {
    a.geo.tab[d] = reinterpret_cast<const T*>(c->ws + c->off_tab_dir[d]);
    a.geo.len[d] = c->len[d];
  }
  const rad_opacity& o = c->opac;
  OpacityDev& od = a.opac;
  od.kind = o.kind;
  od.kappa_p = o.kappa_p;
  od.kappa_r = o.kappa_r;
  od.sigma = o.sigma;
  od.k0 = o.k0;
  od.a_rho = o.a_rho;
  od.b_T = o.b_T;
  od.kmin = o.kmin;
  od.kmax = o.kmax;
  od.sigma_ratio = o.sigma_ratio;
  od.nrho = o.nrho;
  od.nT = o.nT;
  od.lrho0 = o.lrho0;
  od.lT0 = o.lT0;
  od.sr = o.kind == RAD_OPAC_TABLE ? (o.nrho - 1) / (o.lrho1 - o.lrho0) : 0.0;
  od.sT = o.kind == RAD_OPAC_TABLE ? (o.nT - 1) / (o.lT1 - o.lT0) : 0.0;
  od.tab64 = reinterpret_cast<const double*>(c->ws + c->off_op64);
  od.tab32 = reinterpret_cast<const float*>(c->ws + c->off_op32);
  od.linear_rho = (o.kind == RAD_OPAC_POWERLAW && o.a_rho == 1.0 && o.b_T == 0.0);
  od.f_kp = float(o.kappa_p);
  od.f_chi0 = float(o.kappa_r + o.sigma);
  od.f_k0 = float(o.k0);
  od.f_a = float(o.a_rho);
  od.f_b = float(o.b_T);
  od.f_kmin = float(o.kmin);
  od.f_kmax = o.kmax > 3.0e38 ? 3.0e38f : float(o.kmax);
  od.f_s1 = float(1.0 + o.sigma_ratio);
  od.f_lrho0 = float(o.lrho0);
  od.f_lT0 = float(o.lT0);
  od.f_sr = float(od.sr);
  od.f_sT = float(od.sT);
  {
    const double lcv = std::log2(1.0 / (c->par.mu * (c->par.gamma_gas - 1.0)));
    od.f_lcv = float(lcv);
    od.f_blcv = float(o.b_T * lcv);
    od.f_amb = float(o.a_rho - o.b_T);
  }
  CoupleParams& cp = a.cp;
  cp.dt = dt;
  cp.chat = c->par.chat;
  cp.c = c->par.c;
  cp.a_rad = c->par.a_rad;
  cp.cvfac = 1.0 / (c->par.mu * (c->par.gamma_gas - 1.0));
  cp.rtol = c->par.newton_rtol;
  cp.maxit = c->par.newton_maxit;
  cp.newton = c->par.implicit_mode == RAD_NEWTON;
  cp.absorb = c->par.implicit_mode == RAD_ABSORPTION_ONLY;
  a.scheme.recon = c->par.reconstruction;
  a.scheme.ffix = c->par.face_fix;
  a.scheme.riemann = c->par.riemann;
  cp.f_dtchat = float(dt * c->par.chat);
  cp.f_dtc = float(dt * c->par.c);
  cp.f_cvfac = float(cp.cvfac);
  cp.f_a = float(c->par.a_rad);
  cp.f_a_lo = float(c->par.a_rad - double(cp.f_a));
  cp.f_rtol = float(c->par.newton_rtol);
  cp.a_is_one = c->par.a_rad == 1.0;
  a.chat = T(c->par.chat);
  a.dt = T(dt);
  a.efloor = T(c->par.e_floor);
  a.ratio = T(c->par.c / c->par.chat);
  a.inv_chat = T(1.0 / c->par.chat);
  a.stats = reinterpret_cast<unsigned long long*>(c->ws + c->off_stats);
  a.status = reinterpret_cast<int*>(c->ws + c->off_status);
  a.wait_polls = c->wait_polls;
  a.chunk = 0;
  double hmax = 0.0;
  for (int d = 0; d < 3; ++d) {
    double w = c->xf[d][1] - c->xf[d][0];
    a.uni_inv[d] = T(1.0 / w);
    if (d < c->ndim) hmax = std::max(hmax, w);
  }
  a.uni_h = T(hmax);
  const bool q = c->par.implicit_mode == RAD_NEWTON;
  a.queue = q ? reinterpret_cast<long long*>(c->ws + c->off_queue) : nullptr;
  a.queue_count = reinterpret_cast<unsigned int*>(c->ws + c->off_qcount);
  a.queue_cap = q ? (unsigned int)std::min<size_t>(c->N, 0xffffffffu) : 0u;
  a.mlp_gate = float(c->par.mlp_gate);
  a.mlp_w = (c->par.use_mlp && c->mlp_ready) ? reinterpret_cast<const float*>(c->ws + c->off_mlp)
                                             : nullptr;
  a.log = c->log_buf;
  a.log_count = reinterpret_cast<unsigned int*>(c->ws + c->off_lcount);
  a.log_cap = c->log_buf ? c->log_cap : 0u;
  a.log_stride = c->log_stride;
}

// ---------------------------------------------------------------------------
// tensor maps of the TMA-staged step (split precision, 3D Cartesian)
// ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); nullptr if the driver does not provide it.
static EncodeTiledFn encode_tiled() {
  static std::mutex mu;
  static bool looked = false;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// The six tensor maps (E, F0..F2, rho, e of the current input buffer) of a
// TMA-staged variant; nullptr if the variant is not TMA-staged here or the
// maps cannot be encoded.  Each map views one padded field array as a 3D
// tensor (pn0, pn1, pn2) with boxes of bx x by x 1 elements; reads outside
// the array are zero-filled.
static const void* tma_maps(rad_ctx* c, int variant, int in_buf, int rho_buf = -1) {
  if (variant < 0 || variant >= kMaxVariants) return nullptr;
  const int bx = c->launch.tma_box[variant][0], by = c->launch.tma_box[variant][1];
  if (bx <= 0 || c->esize != 4 || c->ndim != 3 || c->nc != 3 || !c->ws) return nullptr;
  // the staged kernels index cells with 32 bits
  if ((long long)c->dims.pn[0] * c->dims.pn[1] * c->dims.pn[2] >= (1ll << 31)) return nullptr;
  for (const TmaSet& t : c->tma)
    if (t.bx == bx && t.by == by) return rho_buf < 0 ? t.maps[in_buf] : t.gas[in_buf][rho_buf];
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return nullptr;
  TmaSet t;
  t.bx = bx;
  t.by = by;
  const StepDims& D = c->dims;
  const cuuint64_t dims[3] = {cuuint64_t(D.pn[0]), cuuint64_t(D.pn[1]), cuuint64_t(D.pn[2])};
  const cuuint64_t strides[2] = {cuuint64_t(D.pn[0]) * 4, cuuint64_t(D.pn[0]) * D.pn[1] * 4};
  const cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  auto encode = [&](CUtensorMap* m, void* ptr) {
    if (!ptr || reinterpret_cast<uintptr_t>(ptr) % 16) return false;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
  };
  for (int b = 0; b < c->nbuf; ++b) {
    void* fields[6] = {state_ptr(c, b, 0), state_ptr(c, b, 1), state_ptr(c, b, 2),
                       state_ptr(c, b, 3), rho_ptr(c, b), state_ptr(c, b, 4)};
    for (int f = 0; f < 6; ++f)
      if (!encode(&t.maps[b][f], fields[f])) return nullptr;
    if (c->par.hydro)
      for (int rb = 0; rb < c->nbuf; ++rb) {
        void* gf[6] = {fields[0], fields[1], fields[2], fields[3], rho_ptr(c, rb),
                       c->ws + c->off_gas_e};
        for (int f = 0; f < 6; ++f)
          if (!encode(&t.gas[b][rb][f], gf[f])) return nullptr;
      }
  }
  c->tma.push_back(t);
  return rho_buf < 0 ? c->tma.back().maps[in_buf] : c->tma.back().gas[in_buf][rho_buf];
}

size_t ctx_args_size(const rad_ctx* c) {
  return c->esize == 8 ? sizeof(StepArgs<Fp64>) : sizeof(StepArgs<Split>);
}

void ctx_fill_args(rad_ctx* c, void* out, double dt, int in_buf) {
  if (c->esize == 8) {
    StepArgs<Fp64> a{};
    fill_args<Fp64>(c, a, dt, in_buf, 1 - in_buf);
    std::memcpy(out, &a, sizeof(a));
  } else {
    StepArgs<Split> a{};
    fill_args<Split>(c, a, dt, in_buf, 1 - in_buf);
    std::memcpy(out, &a, sizeof(a));
  }
}

// The buffer a step or a trial step may write without touching the state.
static int spare_buffer(const rad_ctx* c) { return (c->cur + 1) % c->nbuf; }

// One transport + coupling pass from buffer in_buf into out_buf: the queue
// reset, the step kernel and (RAD_NEWTON) the queue pass, timed when
// profiling is on.  stash_buf >= 0: the last stage of the two-stage step,
// whose result is averaged in place with the U^n held by out_buf; queued
// cells then leave (E*, F*) in stash_buf.
// The gas step of a pass (evolved gas): from the gas of state buffer in_buf
// to rho* in the density of buffer rho_buf and e*, m* in the gas arrays.
template <class P>
static cudaError_t enqueue_gas(rad_ctx* c, double dt, int in_buf, int rho_buf) {
  using S = typename P::S;
  using T = typename P::T;
  HydroArgs<P> h{};
  h.dim = c->dims;
  for (int d = 0; d < 3; ++d) {
    h.geo.tab[d] = reinterpret_cast<const T*>(c->ws + c->off_tab_dir[d]);
    h.geo.len[d] = c->len[d];
    for (int side = 0; side < 2; ++side) h.bcT[d][side] = T(c->bc_val[d][side][4]);
  }
  h.rho = static_cast<const S*>(rho_ptr(c, in_buf));
  h.e = static_cast<const S*>(state_ptr(c, in_buf, 4));
  h.status = reinterpret_cast<int*>(c->ws + c->off_status);
  h.rho_out = static_cast<S*>(rho_ptr(c, rho_buf));
  h.e_out = reinterpret_cast<S*>(c->ws + c->off_gas_e);
  for (int q = 0; q < 3; ++q) {
    h.m[q] = q < c->nc ? static_cast<const S*>(state_ptr(c, in_buf, 5 + q)) : nullptr;
    h.m_out[q] = q < c->nc ? reinterpret_cast<S*>(c->ws + c->off_gas_m[q]) : nullptr;
  }
  h.dt = T(dt);
  h.gamma = T(c->par.gamma_gas);
  h.inv_gm1 = T(1.0 / (c->par.gamma_gas - 1.0));
  h.cvfac = T(1.0 / (c->par.mu * (c->par.gamma_gas - 1.0)));
  for (int d = 0; d < 3; ++d) h.uni_inv[d] = T(1.0 / (c->xf[d][1] - c->xf[d][0]));
  return c->hydro_fn(&h, c->stream);
}

// The radiation step of a pass with evolved gas reads its gas (rho*, e*, m*)
// from the gas step's output instead of the input buffer.
template <class P>
static void gas_inputs(rad_ctx* c, StepArgs<P>& a, int rho_buf) {
  using S = typename P::S;
  a.rho = static_cast<const S*>(rho_ptr(c, rho_buf));
  a.in.e = reinterpret_cast<S*>(c->ws + c->off_gas_e);
  for (int q = 0; q < c->nc; ++q) a.in.m[q] = reinterpret_cast<S*>(c->ws + c->off_gas_m[q]);
}

static rad_status enqueue_pass(rad_ctx* c, double dt, int in_buf, int out_buf,
                               int stash_buf = -1) {
  const bool queue = c->par.implicit_mode == RAD_NEWTON;
  const bool staged = c->launch.tma_box[c->variant][0] > 0;
  const int rho_buf = stash_buf >= 0 ? stash_buf : out_buf;
  const void* maps =
      staged ? tma_maps(c, c->variant, in_buf, c->par.hydro ? rho_buf : -1) : nullptr;
  if (staged && !maps) return RAD_EUNSUPPORTED;
  if (queue && cudaMemsetAsync(c->ws + c->off_qcount, 0, sizeof(unsigned int), c->stream) !=
                   cudaSuccess)
    return RAD_ECUDA;
  cudaError_t e = cudaSuccess;
  // evolved gas: the gas step writes rho* to the output buffer's density, or
  // (last stage of the two-stage step, whose output buffer still holds U^n)
  // to the stash buffer's
  if (c->par.hydro)
    e = c->esize == 8 ? enqueue_gas<Fp64>(c, dt, in_buf, rho_buf)
                      : enqueue_gas<Split>(c, dt, in_buf, rho_buf);
  if (e != cudaSuccess) return RAD_ECUDA;
  cudaEvent_t* ev = c->prof_n < c->prof_cap ? &c->prof_ev[3 * size_t(c->prof_n++)] : nullptr;
  if (ev) cudaEventRecord(ev[0], c->stream);
  if (c->esize == 8) {
    StepArgs<Fp64> a{};
    fill_args<Fp64>(c, a, dt, in_buf, out_buf);
    if (stash_buf >= 0) {
      fill_fields<double>(c, stash_buf, a.stash);
      a.average = 1;
    }
    if (c->par.hydro) {
      gas_inputs<Fp64>(c, a, rho_buf);
      if (stash_buf >= 0) a.rho_avg = static_cast<double*>(rho_ptr(c, out_buf));
    }
    e = c->launch.fn(&a, maps, c->stream, c->variant, c->chunk);
    if (ev) cudaEventRecord(ev[1], c->stream);
    if (e == cudaSuccess && queue) e = c->qpass(&a, c->stream);
  } else {
    StepArgs<Split> a{};
    fill_args<Split>(c, a, dt, in_buf, out_buf);
    if (stash_buf >= 0) {
      fill_fields<float>(c, stash_buf, a.stash);
      a.average = 1;
    }
    if (c->par.hydro) {
      gas_inputs<Split>(c, a, rho_buf);
      if (stash_buf >= 0) a.rho_avg = static_cast<float*>(rho_ptr(c, out_buf));
    }
    e = c->launch.fn(&a, maps, c->stream, c->variant, c->chunk);
    if (ev) cudaEventRecord(ev[1], c->stream);
    if (e == cudaSuccess && queue) e = c->qpass(&a, c->stream);
  }
  if (ev) cudaEventRecord(ev[2], c->stream);
  return cuda_err(e);
}

extern "C" rad_status rad_step(rad_ctx* c, double dt, int nsteps) {
  NvtxRange nvtx_range("rad_step");
  if (!c || nsteps < 0) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  if (!c->have_gas || !c->have_rad) return RAD_EINVAL;
  const bool auto_dt = !(dt > 0.0);
  if (auto_dt) dt = c->dt_cfl;
  if (!std::isfinite(dt)) return RAD_EINVAL;
  for (int s = 0; s < nsteps; ++s) {
    rad_status st;
    // evolved gas: the CFL step of the current state, every step
    if (auto_dt && c->par.hydro && (st = current_dt(c, &dt)) != RAD_OK) return st;
    if (c->par.integrator == RAD_RK2) {
      // stage 1 into b1; stage 2 from b1 straight into the average with U^n
      const int b1 = (c->cur + 1) % 3, b2 = (c->cur + 2) % 3;
      if ((st = enqueue_pass(c, dt, c->cur, b1)) != RAD_OK) return st;
      if ((st = enqueue_pass(c, dt, b1, c->cur, b2)) != RAD_OK) return st;
    } else {
      if ((st = enqueue_pass(c, dt, c->cur, 1 - c->cur)) != RAD_OK) return st;
      c->cur = 1 - c->cur;
    }
    ++c->steps;
  }
  return RAD_OK;
}

static void profile_release(rad_ctx* c) {
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  c->prof_ev.clear();
  c->prof_cap = c->prof_n = 0;
}

extern "C" rad_status rad_profile_begin(rad_ctx* c, int max_steps) {
  if (!c || max_steps < 1 || max_steps > (1 << 20)) return RAD_EINVAL;
  profile_release(c);
  c->prof_ev.assign(3 * size_t(max_steps), nullptr);
  for (cudaEvent_t& e : c->prof_ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
      profile_release(c);
      return RAD_ECUDA;
    }
  c->prof_cap = max_steps;
  return RAD_OK;
}

extern "C" rad_status rad_profile_end(rad_ctx* c, float* step_ms, float* queue_ms, int* nsteps) {
  if (!c) return RAD_EINVAL;
  const int n = c->prof_n;
  float ts = 0.f, tq = 0.f;
  rad_status st = RAD_OK;
  if (n > 0 && cudaEventSynchronize(c->prof_ev[3 * size_t(n - 1) + 2]) != cudaSuccess) st = RAD_ECUDA;
  for (int i = 0; i < n && st == RAD_OK; ++i) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, c->prof_ev[3 * i], c->prof_ev[3 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, c->prof_ev[3 * i + 1], c->prof_ev[3 * i + 2]) != cudaSuccess)
      st = RAD_ECUDA;
    ts += a;
    tq += b;
  }
  profile_release(c);
  if (st != RAD_OK) return st;
  if (step_ms) *step_ms = ts;
  if (queue_ms) *queue_ms = tq;
  if (nsteps) *nsteps = n;
  return RAD_OK;
}

extern "C" int rad_launches_per_step(const rad_ctx* c) {
  if (!c) return 0;
  const int pass = (c->par.implicit_mode == RAD_NEWTON ? 2 : 1) + (c->par.hydro ? 1 : 0);
  return c->par.integrator == RAD_RK2 ? 2 * pass : pass;
}

// ---------------------------------------------------------------------------
// learned starting guess: parameters, training, logging
// ---------------------------------------------------------------------------

extern "C" int rad_mlp_nparam(void) { return mlp_nparam(); }

extern "C" rad_status rad_mlp_set(rad_ctx* c, const float* host, size_t n) {
  if (!c || !host || n != size_t(mlp_nparam())) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  if (cudaMemcpyAsync(c->ws + c->off_mlp, host, n * sizeof(float), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->ws + c->off_m, 0, 2 * (c->off_v - c->off_m), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  c->mlp_ready = true;
  c->adam_step = 0;
  return RAD_OK;
}

extern "C" rad_status rad_mlp_get(rad_ctx* c, float* host, size_t n) {
  if (!c || !host || n != size_t(mlp_nparam())) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  if (cudaMemcpyAsync(host, c->ws + c->off_mlp, n * sizeof(float), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  return RAD_OK;
}

static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Glorot-uniform weights and zero biases from a seeded splitmix64 stream.
extern "C" rad_status rad_mlp_init(rad_ctx* c, uint64_t seed) {
  if (!c) return RAD_EINVAL;
  const int H = 64;
  std::vector<float> w(mlp_nparam(), 0.f);
  uint64_t st = seed;
  auto uni = [&](double lim) {
    double u = (splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
    return float((2.0 * u - 1.0) * lim);
  };
  size_t k = 0;
  const int fan[4][2] = {{2, H}, {H, H}, {H, H}, {H, 1}};
  for (int layer = 0; layer < 4; ++layer) {
    int fin = fan[layer][0], fout = fan[layer][1];
    double lim = std::sqrt(6.0 / (fin + fout));
    for (int i = 0; i < fin * fout; ++i) w[k++] = uni(lim);
    k += fout;  // biases stay zero
  }
  return rad_mlp_set(c, w.data(), w.size());
}

extern "C" rad_status rad_mlp_grad(rad_ctx* c, const float* dev_records, size_t n,
                                   float* host_grad, float* host_loss) {
  if (!c || !dev_records || n == 0 || n > (size_t(1) << 31) || misaligned16(dev_records))
    return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  float* w = reinterpret_cast<float*>(c->ws + c->off_mlp);
  float* g = reinterpret_cast<float*>(c->ws + c->off_grad);
  double* loss = reinterpret_cast<double*>(c->ws + c->off_loss);
  const size_t np = size_t(mlp_nparam());
  if (cudaMemsetAsync(g, 0, np * sizeof(float), c->stream) != cudaSuccess ||
      cudaMemsetAsync(loss, 0, sizeof(double), c->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (mlp_grad_launch(w, reinterpret_cast<const float4*>(dev_records), (long long)n, 1, 0, 0,
                      int(n), g, loss, c->stream) != cudaSuccess)
    return RAD_ECUDA;
  double l = 0.0;
  if ((host_grad && cudaMemcpyAsync(host_grad, g, np * sizeof(float), cudaMemcpyDeviceToHost,
                                    c->stream) != cudaSuccess) ||
      cudaMemcpyAsync(&l, loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(g, 0, np * sizeof(float), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (host_loss) *host_loss = float(l / double(n));
  return RAD_OK;
}

extern "C" rad_status rad_mlp_train(rad_ctx* c, const float* dev_records, size_t n, int epochs,
                                    int batch, float lr, uint64_t seed, float* final_loss) {
  NvtxRange nvtx_range("rad_mlp_train");
  if (!c || !dev_records || n == 0 || epochs < 0 || batch < 1 || !(lr > 0.f) ||
      n > (size_t(1) << 40) || misaligned16(dev_records))
    return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  if (!c->mlp_ready) {
    rad_status s = rad_mlp_init(c, seed ^ 0x5bd1e995ull);
    if (s != RAD_OK) return s;
  }
  float* w = reinterpret_cast<float*>(c->ws + c->off_mlp);
  float* g = reinterpret_cast<float*>(c->ws + c->off_grad);
  float* m = reinterpret_cast<float*>(c->ws + c->off_m);
  float* v = reinterpret_cast<float*>(c->ws + c->off_v);
  double* loss = reinterpret_cast<double*>(c->ws + c->off_loss);
  const float4* rec = reinterpret_cast<const float4*>(dev_records);
  uint64_t st = seed;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    // a random affine permutation k -> (a k + b) mod n of the records
    unsigned long long a_perm, b_perm;
    do {
      a_perm = (splitmix64(st) % n) | 1ull;
    } while (std::gcd(a_perm, (unsigned long long)n) != 1ull);
    b_perm = splitmix64(st) % n;
    if (cudaMemsetAsync(loss, 0, sizeof(double), c->stream) != cudaSuccess) return RAD_ECUDA;
    for (size_t b0 = 0; b0 < n; b0 += size_t(batch)) {
      int bs = int(std::min<size_t>(size_t(batch), n - b0));
      if (mlp_grad_launch(w, rec, (long long)n, a_perm, b_perm, (long long)b0, bs, g, loss,
                          c->stream) != cudaSuccess ||
          mlp_adam_launch(w, g, m, v, lr, ++c->adam_step, c->stream) != cudaSuccess)
        return RAD_ECUDA;
    }
    if (cudaMemcpyAsync(&last, loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return RAD_ECUDA;
  }
  c->mlp_ready = true;
  if (final_loss) *final_loss = float(last / double(n));
  return RAD_OK;
}

extern "C" rad_status rad_mlp_predict(rad_ctx* c, const float* dev_records, size_t n,
                                      float* dev_out) {
  if (!c || !dev_records || !dev_out || n == 0 || misaligned16(dev_records)) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  return cuda_err(mlp_predict_launch(reinterpret_cast<const float*>(c->ws + c->off_mlp),
                                     reinterpret_cast<const float4*>(dev_records), (long long)n,
                                     dev_out, c->stream));
}

extern "C" rad_status rad_mlp_predict_tc(rad_ctx* c, const float* dev_records, size_t n,
                                         float* dev_out) {
  if (!c || !dev_records || !dev_out || n == 0 || misaligned16(dev_records)) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  return cuda_err(mlp_predict_tc_launch(reinterpret_cast<const float*>(c->ws + c->off_mlp),
                                        reinterpret_cast<const float4*>(dev_records), (long long)n,
                                        dev_out, reinterpret_cast<int*>(c->ws + c->off_status),
                                        c->stream));
}

extern "C" rad_status rad_log_bind(rad_ctx* c, float* dev_records, size_t capacity,
                                   long long stride) {
  if (!c || (dev_records && (capacity == 0 || stride < 1 || misaligned16(dev_records))) ||
      capacity > 0xffffffffull)
    return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  c->log_buf = dev_records;
  c->log_cap = (unsigned int)capacity;
  c->log_stride = stride < 1 ? 1 : stride;
  return cuda_err(cudaMemsetAsync(c->ws + c->off_lcount, 0, sizeof(unsigned int), c->stream));
}

extern "C" rad_status rad_log_count(rad_ctx* c, size_t* n) {
  if (!c || !n) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  unsigned int k = 0;
  if (cudaMemcpyAsync(&k, c->ws + c->off_lcount, sizeof(k), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  *n = std::min<size_t>(k, c->log_cap);
  return RAD_OK;
}

// ---------------------------------------------------------------------------
// launch shape selection and autotuning
// ---------------------------------------------------------------------------

extern "C" rad_status rad_set_launch(rad_ctx* c, int variant, int chunk) {
  if (!c || variant < 0 || variant >= c->launch.variants || chunk < 0) return RAD_EINVAL;
  c->variant = variant;
  c->chunk = chunk;
  return RAD_OK;
}

// One index check of the debug build on E of the current state.
__global__ void debug_check_kernel(float* E32, double* E64, long long i, long long n,
                                   int* status) {
  if (index_ok(i, n, status)) {
    if (E32) E32[i] = E32[i];
    if (E64) E64[i] = E64[i];
  }
}

extern "C" rad_status rad_debug_check_index(rad_ctx* c, long long index) {
  if (!c) return RAD_EINVAL;
#ifdef RAD_DEBUG_CHECKS
  if (!c->ws) return RAD_ENOMEM;
  void* E = state_ptr(c, c->cur, 0);
  debug_check_kernel<<<1, 1, 0, c->stream>>>(c->esize == 4 ? static_cast<float*>(E) : nullptr,
                                             c->esize == 8 ? static_cast<double*>(E) : nullptr,
                                             index, padded_cells(c->dims),
                                             reinterpret_cast<int*>(c->ws + c->off_status));
  return cudaGetLastError() == cudaSuccess ? RAD_OK : RAD_ECUDA;
#else
  (void)index;
  return RAD_EUNSUPPORTED;
#endif
}

extern "C" rad_status rad_set_wait_limit(rad_ctx* c, unsigned int polls) {
  if (!c) return RAD_EINVAL;
  c->wait_polls = polls;
  return RAD_OK;
}

extern "C" rad_status rad_get_launch(const rad_ctx* c, int* variant, int* chunk, int* nvariants) {
  if (!c) return RAD_EINVAL;
  if (variant) *variant = c->variant;
  if (chunk) *chunk = c->chunk;
  if (nvariants) *nvariants = c->launch.variants;
  return RAD_OK;
}

// Times one step per (shape, chunk) candidate on the current state without
// advancing it (the step is recomputed from the same input buffer), keeps
// the fastest, and restores the counters and the status word.
extern "C" rad_status rad_tune(rad_ctx* c, int reps, int* variant, int* chunk, float* ms) {
  NvtxRange nvtx_range("rad_tune");
  if (!c || reps < 1) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  if (!c->have_gas || !c->have_rad) return RAD_EINVAL;
  unsigned long long saved[ST_N + 1];
  int saved_status = 0;
  if (cudaMemcpyAsync(saved, c->ws + c->off_stats, sizeof(unsigned long long) * ST_N,
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(&saved_status, c->ws + c->off_status, sizeof(int), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  std::vector<int> chunks;
  if (c->ndim == 3) {
    // and the march length of every march count up to 40: the CTAs of the
    // last marches, launched last, are the short ones, and the length sets
    // how much of the GPU the last wave leaves idle
    chunks = {8, 16, 32, 64, 128};
    for (int nb = 2; nb <= 40 && nb <= c->n[2]; ++nb) chunks.push_back((c->n[2] + nb - 1) / nb);
    std::sort(chunks.begin(), chunks.end());
    chunks.erase(std::unique(chunks.begin(), chunks.end()), chunks.end());
  }
  else if (c->ndim == 2) chunks = {8, 16, 32, 64, 128, 256};
  else chunks = {1};
  const int nmarch = c->ndim == 3 ? c->n[2] : (c->ndim == 2 ? c->n[1] : 1);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return RAD_ECUDA;
  float best = 1e30f;
  int bv = 0, bc = 0;
  rad_status st = RAD_OK;
  StepArgs<Fp64> a64{};
  StepArgs<Split> a32{};
  if (c->esize == 8)
    fill_args<Fp64>(c, a64, c->dt_cfl, c->cur, spare_buffer(c));
  else
    fill_args<Split>(c, a32, c->dt_cfl, c->cur, spare_buffer(c));
  const void* args = c->esize == 8 ? (const void*)&a64 : (const void*)&a32;
  for (int v = 0; v < c->launch.variants && st == RAD_OK; ++v) {
    const bool staged = c->launch.tma_box[v][0] > 0;
    const void* maps = staged ? tma_maps(c, v, c->cur) : nullptr;
    if (staged && !maps) continue;  // TMA maps unavailable: skip the staged shapes
    for (size_t k = 0; k < chunks.size(); ++k) {
      int ch = chunks[k];
      if (k > 0 && ch >= 2 * nmarch) break;
      if (c->launch.fn(args, maps, c->stream, v, ch) != cudaSuccess) {
        st = RAD_ECUDA;
        break;
      }
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < reps; ++r) c->launch.fn(args, maps, c->stream, v, ch);
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = RAD_ECUDA;
        break;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      t /= reps;
      if (t < best) {
        best = t;
        bv = v;
        bc = ch;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaMemcpyAsync(c->ws + c->off_stats, saved, sizeof(unsigned long long) * ST_N,
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->ws + c->off_status, &saved_status, sizeof(int), cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (st != RAD_OK) return st;
  c->variant = bv;
  c->chunk = c->ndim == 1 ? 0 : bc;
  if (variant) *variant = bv;
  if (chunk) *chunk = c->chunk;
  if (ms) *ms = best;
  return RAD_OK;
}

// ---------------------------------------------------------------------------
// reads, status, counters
// ---------------------------------------------------------------------------

static rad_status take_status(rad_ctx* c) {
  // slot 0: the kernels' word; slot 1: non-physical values of asynchronous
  // uploads (the synchronous ones report them themselves)
  int w[2] = {0, 0};
  if (cudaMemcpyAsync(w, c->ws + c->off_status, sizeof(w), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RAD_ECUDA;
  const int st = w[0] | w[1];
  if (st) cudaMemsetAsync(c->ws + c->off_status, 0, sizeof(w), c->stream);
  if (st & STATUS_BOUNDS) return RAD_EBOUNDS;
  if (st & STATUS_TIMEOUT) return RAD_ETIMEOUT;
  if (st & STATUS_NONPHYS) return RAD_ENONPHYS;
  if (st & STATUS_NOCONV) return RAD_ENOCONV;
  return RAD_OK;
}

extern "C" rad_status rad_sync(rad_ctx* c) {
  if (!c) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RAD_ECUDA;
  for (cudaStream_t s : {c->up, c->down})
    if (s && cudaStreamSynchronize(s) != cudaSuccess) return RAD_ECUDA;
  return take_status(c);
}

template <class S>
static rad_status read_t(rad_ctx* c, int field, void* dst, int dev) {
  const double cvfac = 1.0 / (c->par.mu * (c->par.gamma_gas - 1.0));
  const S* rho = static_cast<const S*>(rho_ptr(c, c->cur));
  int ncomp = (field == RAD_FIELD_F || field == RAD_FIELD_M) ? c->par.ncomp : 1;
  for (int comp = 0; comp < ncomp; ++comp) {
    const S* src;
    int mode = UN_COPY;
    switch (field) {
      case RAD_FIELD_E: src = static_cast<const S*>(state_ptr(c, c->cur, 0)); break;
      case RAD_FIELD_F: src = static_cast<const S*>(state_ptr(c, c->cur, 1 + comp)); break;
      case RAD_FIELD_EINT: src = static_cast<const S*>(state_ptr(c, c->cur, 4)); break;
      case RAD_FIELD_M: src = static_cast<const S*>(state_ptr(c, c->cur, 5 + comp)); break;
      case RAD_FIELD_T:
        src = static_cast<const S*>(state_ptr(c, c->cur, 4));
        mode = UN_TEMP;
        break;
      default: src = rho; break;
    }
    S* out = dev ? static_cast<S*>(dst) + comp * c->N
                 : reinterpret_cast<S*>(c->ws + c->off_stage);
    unpack_kernel<S><<<grid_for((long long)c->N), 256, 0, c->stream>>>(out, src, rho, c->dims, mode,
                                                                   cvfac);
    if (cudaGetLastError() != cudaSuccess) return RAD_ECUDA;
    if (!dev) {
      if (cudaMemcpyAsync(static_cast<char*>(dst) + comp * c->N * c->esize, out, c->N * c->esize,
                          cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return RAD_ECUDA;
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RAD_ECUDA;
    }
  }
  return RAD_OK;
}

extern "C" rad_status rad_read(rad_ctx* c, int field, void* dst, size_t bytes, int on_device) {
  NvtxRange nvtx_range("rad_read");
  if (!c || !dst || field < 0 || field > 5) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  int ncomp = (field == RAD_FIELD_F || field == RAD_FIELD_M) ? c->par.ncomp : 1;
  if (bytes < size_t(ncomp) * c->N * c->esize) return RAD_EINVAL;
  if (!c->have_gas || !c->have_rad) return RAD_EINVAL;
  rad_status s = c->esize == 8 ? read_t<double>(c, field, dst, on_device)
                               : read_t<float>(c, field, dst, on_device);
  if (s != RAD_OK) return s;
  if (on_device) return RAD_OK;
  return take_status(c);
}

// ---------------------------------------------------------------------------
// asynchronous host transfers
// ---------------------------------------------------------------------------

// Input slots: rho, v (nc), T, E, F (nc); output slots: E, F (nc), e, m (nc),
// T, rho.  Each slot holds N values.
static int async_in_slot(const rad_ctx* c, int which) {  // 0 rho, 1 v, 2 T, 3 E, 4 F
  const int nc = c->par.ncomp;
  const int base[5] = {0, 1, 1 + nc, 2 + nc, 3 + nc};
  return base[which];
}
static int async_out_slot(const rad_ctx* c, int field) {
  const int nc = c->par.ncomp;
  const int in = 3 + 2 * nc;
  switch (field) {
    case RAD_FIELD_E: return in;
    case RAD_FIELD_F: return in + 1;
    case RAD_FIELD_EINT: return in + 1 + nc;
    case RAD_FIELD_M: return in + 2 + nc;
    case RAD_FIELD_T: return in + 2 + 2 * nc;
    default: return in + 3 + 2 * nc;  // rho
  }
}

static rad_status async_setup(rad_ctx* c) {
  if (c->astage) return RAD_OK;
  const size_t slots = size_t(async_out_slot(c, RAD_FIELD_RHO)) + 1;
  if (cudaMalloc(&c->astage, slots * c->N * c->esize) != cudaSuccess) {
    c->astage = nullptr;
    return RAD_ENOMEM;
  }
  bool ok = cudaStreamCreateWithFlags(&c->up, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->down, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_up, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_packed[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_packed[1], cudaEventDisableTiming) == cudaSuccess;
  for (int f = 0; f < 6 && ok; ++f)
    ok = cudaEventCreateWithFlags(&c->ev_unpacked[f], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_down[f], cudaEventDisableTiming) == cudaSuccess;
  return ok ? RAD_OK : RAD_ECUDA;
}

static void async_release(rad_ctx* c) {
  for (cudaStream_t s : {c->up, c->down})
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  for (cudaEvent_t e : {c->ev_up, c->ev_packed[0], c->ev_packed[1]})
    if (e) cudaEventDestroy(e);
  for (int f = 0; f < 6; ++f) {
    if (c->ev_unpacked[f]) cudaEventDestroy(c->ev_unpacked[f]);
    if (c->ev_down[f]) cudaEventDestroy(c->ev_down[f]);
  }
  if (c->astage) cudaFree(c->astage);
  c->astage = nullptr;
}

// Uploads `count` values per array into input slots on the upload stream,
// once the previous packs of the same slots (gas: 0, radiation: 1) are done
// with them.
static rad_status async_upload(rad_ctx* c, const void* const* src, const size_t* count,
                               const int* slot, int n, int kind) {
  if (cudaStreamWaitEvent(c->up, c->ev_packed[kind], 0) != cudaSuccess) return RAD_ECUDA;
  for (int i = 0; i < n; ++i)
    if (cudaMemcpyAsync(c->astage + size_t(slot[i]) * c->N * c->esize, src[i], count[i] * c->esize,
                        cudaMemcpyHostToDevice, c->up) != cudaSuccess)
      return RAD_ECUDA;
  if (cudaEventRecord(c->ev_up, c->up) != cudaSuccess ||
      cudaStreamWaitEvent(c->stream, c->ev_up, 0) != cudaSuccess)
    return RAD_ECUDA;
  return RAD_OK;
}

extern "C" rad_status rad_set_gas_host_async(rad_ctx* c, const void* rho, const void* v,
                                             const void* T) {
  NvtxRange nvtx_range("rad_set_gas_host_async");
  if (!c || !rho || !v || !T) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  rad_status st = async_setup(c);
  if (st != RAD_OK) return st;
  const void* src[3] = {rho, v, T};
  const size_t count[3] = {c->N, size_t(c->par.ncomp) * c->N, c->N};
  const int slot[3] = {async_in_slot(c, 0), async_in_slot(c, 1), async_in_slot(c, 2)};
  if ((st = async_upload(c, src, count, slot, 3, 0)) != RAD_OK) return st;
  char* base = c->astage;
  const size_t w = c->N * c->esize;
  st = c->esize == 8 ? set_gas_t<double>(c, base + slot[0] * w, base + slot[1] * w,
                                         base + slot[2] * w, 1, false)
                     : set_gas_t<float>(c, base + slot[0] * w, base + slot[1] * w,
                                        base + slot[2] * w, 1, false);
  if (st != RAD_OK) return st;
  return cuda_err(cudaEventRecord(c->ev_packed[0], c->stream));
}

extern "C" rad_status rad_set_rad_host_async(rad_ctx* c, const void* E, const void* F) {
  NvtxRange nvtx_range("rad_set_rad_host_async");
  if (!c || !E || !F) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  rad_status st = async_setup(c);
  if (st != RAD_OK) return st;
  const void* src[2] = {E, F};
  const size_t count[2] = {c->N, size_t(c->par.ncomp) * c->N};
  const int slot[2] = {async_in_slot(c, 3), async_in_slot(c, 4)};
  if ((st = async_upload(c, src, count, slot, 2, 1)) != RAD_OK) return st;
  const size_t w = c->N * c->esize;
  st = c->esize == 8 ? set_rad_t<double>(c, c->astage + slot[0] * w, c->astage + slot[1] * w, 1,
                                         false)
                     : set_rad_t<float>(c, c->astage + slot[0] * w, c->astage + slot[1] * w, 1,
                                        false);
  if (st != RAD_OK) return st;
  return cuda_err(cudaEventRecord(c->ev_packed[1], c->stream));
}

extern "C" rad_status rad_read_host_async(rad_ctx* c, int field, void* dst, size_t bytes) {
  NvtxRange nvtx_range("rad_read_host_async");
  if (!c || !dst || field < 0 || field > 5) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  const int ncomp = (field == RAD_FIELD_F || field == RAD_FIELD_M) ? c->par.ncomp : 1;
  if (bytes < size_t(ncomp) * c->N * c->esize) return RAD_EINVAL;
  if (!c->have_gas || !c->have_rad) return RAD_EINVAL;
  rad_status st = async_setup(c);
  if (st != RAD_OK) return st;
  // the field's output slots are free once its previous read-back is done
  if (cudaStreamWaitEvent(c->stream, c->ev_down[field], 0) != cudaSuccess) return RAD_ECUDA;
  char* out = c->astage + size_t(async_out_slot(c, field)) * c->N * c->esize;
  st = c->esize == 8 ? read_t<double>(c, field, out, 1) : read_t<float>(c, field, out, 1);
  if (st != RAD_OK) return st;
  if (cudaEventRecord(c->ev_unpacked[field], c->stream) != cudaSuccess ||
      cudaStreamWaitEvent(c->down, c->ev_unpacked[field], 0) != cudaSuccess ||
      cudaMemcpyAsync(dst, out, size_t(ncomp) * c->N * c->esize, cudaMemcpyDeviceToHost,
                      c->down) != cudaSuccess ||
      cudaEventRecord(c->ev_down[field], c->down) != cudaSuccess)
    return RAD_ECUDA;
  return RAD_OK;
}

extern "C" rad_status rad_get_stats(rad_ctx* c, rad_stats* out) {
  if (!c || !out) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  unsigned long long v[ST_N] = {};
  if (cudaMemcpyAsync(v, c->ws + c->off_stats, sizeof(v), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return RAD_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RAD_ECUDA;
  out->fix = v[ST_FIX];
  out->efloor = v[ST_EFLOOR];
  out->fclip = v[ST_FCLIP];
  out->iters = v[ST_ITERS];
  out->itmax = v[ST_ITMAX];
  out->fallback = v[ST_FALLBACK];
  out->noconv = v[ST_NOCONV];
  out->steps = c->steps;
  return RAD_OK;
}

extern "C" rad_status rad_reset_stats(rad_ctx* c) {
  if (!c) return RAD_EINVAL;
  if (!c->ws) return RAD_ENOMEM;
  c->steps = 0;
  return cuda_err(
      cudaMemsetAsync(c->ws + c->off_stats, 0, sizeof(unsigned long long) * ST_N, c->stream));
}

extern "C" void rad_destroy(rad_ctx* c) {
  if (!c) return;
  profile_release(c);
  async_release(c);
  if (c->ws_owned && c->ws) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->ws);
  }
  delete c;
}
