// ctx_internal.h -- the context behind the opaque rad_ctx handle, shared by
// the single-grid host code (rad_api.cu) and the batched host code
// (batch_api.cu).  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "m1_internal.h"
#include "hydro_launch.h"
#include "mlp_launch.h"
#include "rad.h"
#include "step_launch.h"

// NVTX range over one host entry point (header-only NVTX v3: a no-op unless a
// profiler is attached), so that profiles show the library's calls.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Tensor maps of the TMA-staged step for one box shape: per state buffer (up to 3),
// E, F0..F2, rho and e (the order of the kernel's TmaMaps).
struct TmaSet {
  int bx = 0, by = 0;
  CUtensorMap maps[3][6];
  // evolved gas: E, F0..F2 of the input buffer, rho* of a buffer's density
  // and e* of the gas arrays, per (input buffer, density buffer)
  CUtensorMap gas[3][3][6];
};

struct rad_ctx {
  // description
  int ndim = 1, n[3] = {1, 1, 1}, geom = 0;
  int bc_lo[3] = {0, 0, 0}, bc_hi[3] = {0, 0, 0};
  double bc_val[3][2][5] = {};  // boundary states of FIXED / LTE sides (rad_grid.bc_value)
  std::vector<double> xf[3];
  rad_opacity opac{};
  std::vector<float> table32;
  std::vector<double> table64;
  rad_params par{};
  int nc = 3;            // flux/momentum components carried internally
  double dt_cfl = 0.0;
  // layout
  m1::StepDims dims{};
  size_t pcells = 0;     // padded cells per array
  size_t N = 0;          // interior cells
  size_t esize = 8;      // bytes per stored value
  std::vector<double> tab64[3];
  std::vector<float> tab32[3];
  int len[3] = {1, 1, 1};
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  size_t off_state[3][8] = {};  // E, F0..F2, e, m0..m2 per buffer (the third for RAD_RK2)
  int nbuf = 2;                 // state buffers: 2, or 3 for RAD_RK2
  size_t off_rho = 0, off_tab = 0, off_tab_dir[3] = {}, off_op32 = 0, off_op64 = 0;
  size_t off_stats = 0, off_status = 0, off_stage = 0;
  size_t off_qirr = size_t(-1);  // irradiation deposit (padded), if params.irradiation
  // evolved gas (params.hydro): a density per state buffer, and the gas after
  // the gas step (rho* goes to a state buffer's density, e* and m* here)
  size_t off_rho_buf[3] = {};
  size_t off_gas_e = 0, off_gas_m[3] = {};
  m1::HydroFn hydro_fn = nullptr, gas_cfl_fn = nullptr;
  size_t off_cfl = 0;  // reduction word of the gas CFL rate
  size_t total = 0;
  cudaStream_t stream = nullptr;
  // asynchronous host transfers (rad_*_host_async): an upload and a
  // read-back stream, their events and a staging area of their own
  // (input slots rho, v, T, E, F; output slots per field), allocated on
  // first use
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t ev_up = nullptr, ev_packed[2] = {}, ev_unpacked[6] = {}, ev_down[6] = {};
  char* astage = nullptr;
  int cur = 0;
  bool have_gas = false, have_rad = false;
  uint64_t steps = 0;
  LaunchEntry launch{nullptr, 0};
  int variant = 0, chunk = 0;   // CTA shape and march length (0 = defaults)
  unsigned int wait_polls = 0;  // bound of the staged-plane waits (0 = default)
  bool uniform = false;         // Cartesian with a constant width along each direction
  bool general = false;         // general form of the step kernel (options, absorption, irradiation)
  // learned guess
  m1::QueueFn qpass = nullptr;
  size_t off_mlp = 0, off_grad = 0, off_m = 0, off_v = 0, off_loss = 0, off_queue = 0;
  size_t off_qcount = 0, off_lcount = 0;
  bool mlp_ready = false;
  int adam_step = 0;
  float* log_buf = nullptr;
  unsigned int log_cap = 0;
  long long log_stride = 1;
  // tensor maps of the TMA-staged variants, built on first use per box shape
  std::vector<TmaSet> tma;
  // kernel timing: 3 events per profiled step (step kernel start, step kernel
  // end = queue pass start, queue pass end)
  std::vector<cudaEvent_t> prof_ev;
  int prof_cap = 0, prof_n = 0;
};

// Size of the step-kernel argument block of this context (StepArgs of its
// precision policy) and its filling for one step of length dt that reads
// state buffer `in_buf` and writes the other one.
size_t ctx_args_size(const rad_ctx* c);
void ctx_fill_args(rad_ctx* c, void* out, double dt, int in_buf);
