// batch_api.cu -- host side of the batched entry points (rad_batch_*):
// validation of the member grids, the tile work list, the per-grid argument
// blocks in device memory, capture of whole step sequences into CUDA graphs,
// the autotuner of the persistent launch, and the batch counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "batch_launch.h"
#include "ctx_internal.h"

using namespace m1;

namespace {

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  int nsteps = 0, phase = 0;
  uint64_t key = 0;  // launch configuration the graph was captured with
};

}  // namespace

struct rad_batch {
  std::vector<rad_ctx*> g;  // member grids (not owned)
  int count = 0;
  bool split = false, newton = false, mlp = false;
  int ndim = 2, nc = 2;
  bool uniform = false;
  BatchEntry ent{};
  size_t args_size = 0;
  int sms = 148;
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0, total = 0;
  bool ws_owned = false;
  size_t off_args[2] = {}, off_items = 0, off_ctl = 0, off_stats = 0, off_status = 0;
  size_t off_qcounts = 0, off_mlp = 0;
  size_t max_items = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream that graphs are captured on
  // launch
  int variant = 0, chunk = 0, blocks = 0, nitems = 0;
  bool items_dirty = true, args_dirty = true;
  uint64_t config_key = 1;  // bumped whenever the captured launches change
  // argument blocks: [parity][grid]; parity p reads buffer cur0[i] ^ p
  std::vector<char> host_args;
  std::vector<int> cur0;
  std::vector<char*> ws0;  // members' workspaces the blocks point into
  std::vector<double> dt_args;
  int phase = 0;  // steps taken since the arguments were written, mod 2
  bool mlp_ready = false;
  bool use_graph = true;
  GraphSlot graphs[4];
  int next_slot = 0;
  uint64_t steps = 0;
};

namespace {

rad_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? RAD_OK : RAD_ECUDA; }

int march_axis(const rad_batch* b) { return b->ndim == 3 ? 2 : 1; }

int default_chunk(const rad_batch* b) { return b->ndim == 3 ? 32 : 64; }

// Chunk (cells marched per CTA) of grid i under the batch's setting.
int grid_chunk(const rad_batch* b, int i, int chunk) {
  const int nm = b->g[i]->n[march_axis(b)];
  const int c = chunk > 0 ? chunk : default_chunk(b);
  return std::min(c, nm);
}

// Tiles of grid i for CTA shape (tx, ty) and march length c.
size_t tiles_of(const rad_batch* b, int i, int tx, int ty, int c) {
  const rad_ctx* m = b->g[i];
  size_t nbx = size_t((m->n[0] + tx - 2) / (tx - 1));
  if (b->ndim == 3) {
    size_t nby = size_t((m->n[1] + ty - 2) / (ty - 1));
    return nbx * nby * size_t((m->n[2] + c - 1) / c);
  }
  return nbx * size_t((m->n[1] + c - 1) / c);
}

// Work list: grids in decreasing size (largest first), each grid's tiles in
// march-block-major order.
void build_items(rad_batch* b, std::vector<int4>& items) {
  const int tx = b->ent.tx[b->variant], ty = b->ent.ty[b->variant];
  std::vector<int> order(b->count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->g[x]->N > b->g[y]->N; });
  items.clear();
  for (int i : order) {
    const rad_ctx* m = b->g[i];
    const int c = grid_chunk(b, i, b->chunk);
    const int nbx = (m->n[0] + tx - 2) / (tx - 1);
    if (b->ndim == 3) {
      const int nby = (m->n[1] + ty - 2) / (ty - 1);
      const int nbz = (m->n[2] + c - 1) / c;
      for (int bz = 0; bz < nbz; ++bz)
        for (int by = 0; by < nby; ++by)
          for (int bx = 0; bx < nbx; ++bx) items.push_back(make_int4(i, bx, by, bz));
    } else {
      const int nby = (m->n[1] + c - 1) / c;
      for (int by = 0; by < nby; ++by)
        for (int bx = 0; bx < nbx; ++bx) items.push_back(make_int4(i, bx, by, 0));
    }
  }
}

// Points the batch-level fields of one argument block at the batch's own
// counters, queue lengths and network parameters.
template <class P>
void patch_args(rad_batch* b, void* blk, int i) {
  StepArgs<P>& a = *static_cast<StepArgs<P>*>(blk);
  a.chunk = grid_chunk(b, i, b->chunk);
  a.stats = reinterpret_cast<unsigned long long*>(b->ws + b->off_stats);
  a.status = reinterpret_cast<int*>(b->ws + b->off_status);
  a.wait_polls = 0;
  a.queue_count = reinterpret_cast<unsigned int*>(b->ws + b->off_qcounts) + i;
  a.mlp_w = (b->mlp && b->mlp_ready) ? reinterpret_cast<const float*>(b->ws + b->off_mlp)
                                     : nullptr;
  a.log = nullptr;
  a.log_count = nullptr;
  a.log_cap = 0u;
}

rad_status upload_args(rad_batch* b, const std::vector<double>& dt) {
  const size_t sz = b->args_size;
  b->host_args.assign(2 * size_t(b->count) * sz, 0);
  b->cur0.resize(b->count);
  for (int p = 0; p < 2; ++p)
    for (int i = 0; i < b->count; ++i) {
      rad_ctx* m = b->g[i];
      void* blk = b->host_args.data() + (size_t(p) * b->count + i) * sz;
      ctx_fill_args(m, blk, dt[i], m->cur ^ p);
      if (b->split)
        patch_args<Split>(b, blk, i);
      else
        patch_args<Fp64>(b, blk, i);
    }
  b->ws0.resize(b->count);
  for (int i = 0; i < b->count; ++i) {
    b->cur0[i] = b->g[i]->cur;
    b->ws0[i] = b->g[i]->ws;
  }
  for (int p = 0; p < 2; ++p)
    if (cudaMemcpyAsync(b->ws + b->off_args[p], b->host_args.data() + size_t(p) * b->count * sz,
                        size_t(b->count) * sz, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return RAD_ECUDA;
  b->dt_args = dt;
  b->phase = 0;
  b->args_dirty = false;
  return RAD_OK;
}

rad_status upload_items(rad_batch* b) {
  std::vector<int4> items;
  build_items(b, items);
  if (items.size() > b->max_items) return RAD_EINVAL;
  b->nitems = int(items.size());
  if (cudaMemcpyAsync(b->ws + b->off_items, items.data(), items.size() * sizeof(int4),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RAD_ECUDA;
  int per_sm = 0;
  if (b->ent.occupancy(b->variant, &per_sm) != cudaSuccess || per_sm < 1) return RAD_ECUDA;
  b->blocks = std::max(1, std::min(per_sm * b->sms, b->nitems));
  b->items_dirty = false;
  ++b->config_key;
  return RAD_OK;
}

void drop_graphs(rad_batch* b) {
  for (GraphSlot& s : b->graphs) {
    if (s.exec) cudaGraphExecDestroy(s.exec);
    s = GraphSlot{};
  }
}

// Enqueues one step of every grid reading parity p of the argument blocks.
rad_status enqueue_step(rad_batch* b, int p, cudaStream_t s) {
  unsigned int* qc = reinterpret_cast<unsigned int*>(b->ws + b->off_qcounts);
  const void* args = b->ws + b->off_args[p];
  if (b->newton && cudaMemsetAsync(qc, 0, sizeof(unsigned int) * b->count, s) != cudaSuccess)
    return RAD_ECUDA;
  if (b->ent.step(args, reinterpret_cast<const int4*>(b->ws + b->off_items), b->nitems,
                  reinterpret_cast<unsigned int*>(b->ws + b->off_ctl), b->variant, b->blocks,
                  s) != cudaSuccess)
    return RAD_ECUDA;
  if (b->newton && b->ent.qpass(args, b->count, qc, b->mlp && b->mlp_ready, s) != cudaSuccess)
    return RAD_ECUDA;
  return RAD_OK;
}

// Brings the work list and the argument blocks up to date with the members'
// buffers and the requested time steps.
rad_status refresh(rad_batch* b, const std::vector<double>& dt) {
  rad_status st;
  if (b->items_dirty && (st = upload_items(b)) != RAD_OK) return st;
  bool stale = b->args_dirty || dt != b->dt_args;
  for (int i = 0; i < b->count && !stale; ++i)
    stale = b->g[i]->cur != (b->cur0[i] ^ b->phase) || b->g[i]->ws != b->ws0[i];
  if (stale && (st = upload_args(b, dt)) != RAD_OK) return st;
  return RAD_OK;
}

rad_status graph_for(rad_batch* b, int nsteps, cudaGraphExec_t* out) {
  for (GraphSlot& s : b->graphs)
    if (s.exec && s.nsteps == nsteps && s.phase == b->phase && s.key == b->config_key) {
      *out = s.exec;
      return RAD_OK;
    }
  if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return RAD_ECUDA;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return RAD_ECUDA;
  rad_status st = RAD_OK;
  for (int k = 0; k < nsteps && st == RAD_OK; ++k) st = enqueue_step(b, (b->phase + k) & 1, b->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (st != RAD_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return RAD_ECUDA;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return RAD_ECUDA;
  GraphSlot& s = b->graphs[b->next_slot];
  b->next_slot = (b->next_slot + 1) % 4;
  if (s.exec) cudaGraphExecDestroy(s.exec);
  s.exec = exec;
  s.nsteps = nsteps;
  s.phase = b->phase;
  s.key = b->config_key;
  *out = exec;
  return RAD_OK;
}

std::vector<double> step_sizes(const rad_batch* b, const double* dt) {
  std::vector<double> v(b->count);
  for (int i = 0; i < b->count; ++i)
    v[i] = (dt && dt[i] > 0.0) ? dt[i] : b->g[i]->dt_cfl;
  return v;
}

}  // namespace

extern "C" rad_status rad_batch_create(rad_ctx* const* members, int count, rad_batch** out) {
  if (!members || !out || count < 1 || count > kBatchMaxGrids) return RAD_EINVAL;
  const rad_ctx* m0 = members[0];
  if (!m0) return RAD_EINVAL;
  for (int i = 0; i < count; ++i) {
    const rad_ctx* m = members[i];
    if (!m) return RAD_EINVAL;
    for (int j = 0; j < i; ++j)
      if (members[j] == m) return RAD_EINVAL;  // a grid appears once
    if (m->geom != RAD_CARTESIAN || m->ndim != m0->ndim || m->esize != m0->esize ||
        m->nc != m0->nc || m->uniform != m0->uniform ||
        m->par.implicit_mode != m0->par.implicit_mode || m->par.use_mlp != m0->par.use_mlp ||
        m->par.integrator != RAD_EULER || m->general)
      return RAD_EUNSUPPORTED;  // the batched kernel runs the default form only
  }
  BatchEntry ent = select_batch(m0->esize == 4, m0->ndim, m0->nc, m0->uniform);
  if (!ent.step) return RAD_EUNSUPPORTED;
  rad_batch* b = new (std::nothrow) rad_batch();
  if (!b) return RAD_ENOMEM;
  b->g.assign(members, members + count);
  b->count = count;
  b->split = m0->esize == 4;
  b->newton = m0->par.implicit_mode == RAD_NEWTON;
  b->mlp = m0->par.use_mlp != 0;
  b->ndim = m0->ndim;
  b->nc = m0->nc;
  b->uniform = m0->uniform;
  b->ent = ent;
  b->args_size = ctx_args_size(m0);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
    b->sms = sms;
  // bound on the work list over every shape and any march length >= 1
  for (int i = 0; i < count; ++i) {
    size_t worst = 0;
    for (int v = 0; v < ent.variants; ++v) worst = std::max(worst, tiles_of(b, i, ent.tx[v], ent.ty[v], 1));
    b->max_items += worst;
  }
  if (b->max_items > size_t(1) << 31) {
    delete b;
    return RAD_EINVAL;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  b->off_args[0] = take(size_t(count) * b->args_size);
  b->off_args[1] = take(size_t(count) * b->args_size);
  b->off_items = take(b->max_items * sizeof(int4));
  b->off_ctl = take(2 * sizeof(unsigned int));
  b->off_stats = take(sizeof(unsigned long long) * ST_N);
  b->off_status = take(sizeof(int) * 4);
  b->off_qcounts = take(sizeof(unsigned int) * count);
  b->off_mlp = take(size_t(mlp_nparam()) * sizeof(float));
  b->total = off;
  *out = b;
  return RAD_OK;
}

extern "C" rad_status rad_batch_workspace_size(const rad_batch* b, size_t* bytes) {
  if (!b || !bytes) return RAD_EINVAL;
  *bytes = b->total;
  return RAD_OK;
}

extern "C" rad_status rad_batch_bind_workspace(rad_batch* b, void* ptr, size_t bytes) {
  if (!b || !ptr) return RAD_EINVAL;
  if (reinterpret_cast<uintptr_t>(ptr) % 256) return RAD_EINVAL;
  if (bytes < b->total) return RAD_ENOMEM;
  drop_graphs(b);
  if (b->ws_owned) {
    cudaFree(b->ws);
    b->ws_owned = false;
  }
  b->ws = static_cast<char*>(ptr);
  b->ws_bytes = bytes;
  b->items_dirty = b->args_dirty = true;
  b->mlp_ready = false;
  ++b->config_key;
  if (cudaMemsetAsync(b->ws + b->off_ctl, 0, b->off_mlp - b->off_ctl, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RAD_ECUDA;
  return RAD_OK;
}

extern "C" rad_status rad_batch_alloc_workspace(rad_batch* b) {
  if (!b) return RAD_EINVAL;
  void* p = nullptr;
  if (cudaMalloc(&p, b->total) != cudaSuccess) return RAD_ENOMEM;
  rad_status s = rad_batch_bind_workspace(b, p, b->total);
  if (s != RAD_OK) {
    cudaFree(p);
    return s;
  }
  b->ws_owned = true;
  return RAD_OK;
}

extern "C" rad_status rad_batch_set_stream(rad_batch* b, void* stream) {
  if (!b) return RAD_EINVAL;
  b->stream = static_cast<cudaStream_t>(stream);
  for (rad_ctx* m : b->g) m->stream = b->stream;
  return RAD_OK;
}

extern "C" rad_status rad_batch_set_graph(rad_batch* b, int use_graph) {
  if (!b) return RAD_EINVAL;
  b->use_graph = use_graph != 0;
  return RAD_OK;
}

extern "C" rad_status rad_batch_step(rad_batch* b, const double* dt, int nsteps) {
  NvtxRange nvtx_range("rad_batch_step");
  if (!b || nsteps < 0) return RAD_EINVAL;
  if (!b->ws) return RAD_ENOMEM;
  for (const rad_ctx* m : b->g) {
    if (!m->ws) return RAD_ENOMEM;
    if (!m->have_gas || !m->have_rad) return RAD_EINVAL;
  }
  if (nsteps == 0) return RAD_OK;
  std::vector<double> dts = step_sizes(b, dt);
  for (double v : dts)
    if (!std::isfinite(v) || !(v > 0.0)) return RAD_EINVAL;
  rad_status st = refresh(b, dts);
  if (st != RAD_OK) return st;
  if (b->use_graph) {
    cudaGraphExec_t exec = nullptr;
    if ((st = graph_for(b, nsteps, &exec)) != RAD_OK) return st;
    if (cudaGraphLaunch(exec, b->stream) != cudaSuccess) return RAD_ECUDA;
  } else {
    for (int k = 0; k < nsteps; ++k)
      if ((st = enqueue_step(b, (b->phase + k) & 1, b->stream)) != RAD_OK) return st;
  }
  b->phase = (b->phase + nsteps) & 1;
  for (rad_ctx* m : b->g) {
    m->cur ^= (nsteps & 1);
    m->steps += uint64_t(nsteps);
  }
  b->steps += uint64_t(nsteps);
  return RAD_OK;
}

extern "C" rad_status rad_batch_sync(rad_batch* b) {
  if (!b) return RAD_EINVAL;
  if (!b->ws) return RAD_ENOMEM;
  int word = 0;
  if (cudaMemcpyAsync(&word, b->ws + b->off_status, sizeof(int), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (word && cudaMemsetAsync(b->ws + b->off_status, 0, sizeof(int), b->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (word & STATUS_BOUNDS) return RAD_EBOUNDS;
  if (word & STATUS_TIMEOUT) return RAD_ETIMEOUT;
  if (word & STATUS_NONPHYS) return RAD_ENONPHYS;
  if (word & STATUS_NOCONV) return RAD_ENOCONV;
  return RAD_OK;
}

extern "C" rad_status rad_batch_get_stats(rad_batch* b, rad_stats* out) {
  if (!b || !out) return RAD_EINVAL;
  if (!b->ws) return RAD_ENOMEM;
  unsigned long long v[ST_N] = {};
  if (cudaMemcpyAsync(v, b->ws + b->off_stats, sizeof(v), cudaMemcpyDeviceToHost, b->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RAD_ECUDA;
  out->fix = v[ST_FIX];
  out->efloor = v[ST_EFLOOR];
  out->fclip = v[ST_FCLIP];
  out->iters = v[ST_ITERS];
  out->itmax = v[ST_ITMAX];
  out->fallback = v[ST_FALLBACK];
  out->noconv = v[ST_NOCONV];
  out->steps = b->steps;
  return RAD_OK;
}

extern "C" rad_status rad_batch_reset_stats(rad_batch* b) {
  if (!b) return RAD_EINVAL;
  if (!b->ws) return RAD_ENOMEM;
  b->steps = 0;
  return cuda_ok(
      cudaMemsetAsync(b->ws + b->off_stats, 0, sizeof(unsigned long long) * ST_N, b->stream));
}

extern "C" int rad_batch_launches_per_step(const rad_batch* b) {
  if (!b) return 0;
  return b->newton ? 2 : 1;
}

extern "C" rad_status rad_batch_set_launch(rad_batch* b, int variant, int chunk) {
  if (!b || variant < 0 || variant >= b->ent.variants || chunk < 0) return RAD_EINVAL;
  b->variant = variant;
  b->chunk = chunk;
  b->items_dirty = b->args_dirty = true;
  return RAD_OK;
}

extern "C" rad_status rad_batch_get_launch(const rad_batch* b, int* variant, int* chunk,
                                           int* nvariants, int* blocks) {
  if (!b) return RAD_EINVAL;
  if (variant) *variant = b->variant;
  if (chunk) *chunk = b->chunk;
  if (nvariants) *nvariants = b->ent.variants;
  if (blocks) *blocks = b->blocks;
  return RAD_OK;
}

// Times the persistent step kernel for every (shape, march length) pair on
// the current state without advancing it: each trial recomputes the same
// step into the members' spare buffers.  Restores the counters and the status
// word and keeps the fastest pair.
extern "C" rad_status rad_batch_tune(rad_batch* b, int reps, int* variant, int* chunk, float* ms) {
  NvtxRange nvtx_range("rad_batch_tune");
  if (!b || reps < 1) return RAD_EINVAL;
  if (!b->ws) return RAD_ENOMEM;
  for (const rad_ctx* m : b->g)
    if (!m->ws || !m->have_gas || !m->have_rad) return RAD_EINVAL;
  unsigned long long saved[ST_N];
  int saved_status = 0;
  if (cudaMemcpyAsync(saved, b->ws + b->off_stats, sizeof(saved), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaMemcpyAsync(&saved_status, b->ws + b->off_status, sizeof(int), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RAD_ECUDA;
  std::vector<int> chunks = b->ndim == 3 ? std::vector<int>{8, 16, 32, 64}
                                         : std::vector<int>{8, 16, 32, 64, 128};
  int nmarch = 0;
  for (const rad_ctx* m : b->g) nmarch = std::max(nmarch, m->n[march_axis(b)]);
  const std::vector<double> dts = b->dt_args.empty() ? step_sizes(b, nullptr) : b->dt_args;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return RAD_ECUDA;
  }
  unsigned int* qc = reinterpret_cast<unsigned int*>(b->ws + b->off_qcounts);
  float best = 1e30f;
  int bv = b->variant, bc = b->chunk;
  rad_status st = RAD_OK;
  for (int v = 0; v < b->ent.variants && st == RAD_OK; ++v) {
    for (size_t k = 0; k < chunks.size() && st == RAD_OK; ++k) {
      const int ch = chunks[k];
      if (k > 0 && ch >= 2 * nmarch) break;
      b->variant = v;
      b->chunk = ch;
      b->items_dirty = b->args_dirty = true;
      if ((st = refresh(b, dts)) != RAD_OK) break;
      const void* args = b->ws + b->off_args[b->phase];
      auto launch = [&]() {
        if (b->newton && cudaMemsetAsync(qc, 0, sizeof(unsigned int) * b->count, b->stream) !=
                             cudaSuccess)
          return false;
        return b->ent.step(args, reinterpret_cast<const int4*>(b->ws + b->off_items), b->nitems,
                           reinterpret_cast<unsigned int*>(b->ws + b->off_ctl), b->variant,
                           b->blocks, b->stream) == cudaSuccess;
      };
      if (!launch()) {
        st = RAD_ECUDA;
        break;
      }
      cudaEventRecord(e0, b->stream);
      bool ok = true;
      for (int r = 0; r < reps && ok; ++r) ok = launch();
      cudaEventRecord(e1, b->stream);
      if (!ok || cudaEventSynchronize(e1) != cudaSuccess) {
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
  if (cudaMemcpyAsync(b->ws + b->off_stats, saved, sizeof(saved), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->ws + b->off_status, &saved_status, sizeof(int), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaMemsetAsync(qc, 0, sizeof(unsigned int) * b->count, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RAD_ECUDA;
  b->variant = bv;
  b->chunk = bc;
  b->items_dirty = b->args_dirty = true;
  if (st != RAD_OK) return st;
  if (variant) *variant = bv;
  if (chunk) *chunk = bc;
  if (ms) *ms = best;
  return RAD_OK;
}

extern "C" rad_status rad_batch_mlp_set(rad_batch* b, const float* host, size_t n) {
  if (!b || !host || n != size_t(mlp_nparam())) return RAD_EINVAL;
  if (!b->ws) return RAD_ENOMEM;
  if (!b->mlp) return RAD_EINVAL;
  if (cudaMemcpyAsync(b->ws + b->off_mlp, host, n * sizeof(float), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return RAD_ECUDA;
  if (!b->mlp_ready) {
    b->mlp_ready = true;
    b->args_dirty = true;  // the argument blocks now point at the parameters
    ++b->config_key;       // the queue pass now holds them in shared memory
  }
  return RAD_OK;
}

extern "C" void rad_batch_destroy(rad_batch* b) {
  if (!b) return;
  if (b->ws) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ws_owned && b->ws) cudaFree(b->ws);
  delete b;
}
