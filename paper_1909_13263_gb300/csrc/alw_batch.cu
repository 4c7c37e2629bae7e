// Batched solves: many independent 2D instances of uneven size advanced by one
// persistent launch per RK stage over a shared (instance, tile) work list,
// captured in a CUDA graph and replayed until every instance has reached its
// own t_final.  Instances are stacked vertically in padded arrays of one
// common pitch, so one set of TMA tensor maps serves all of them; each
// instance keeps its own device-side time, dt and alpha state.
//
// A small autotuner picks, per batch shape, the tile width (64 x 32 or 32 x 32
// tiles: the narrow ones halve the work of the smallest instances' tiles and
// double the tiles in flight, at 1.1x the halo reads per node) and the
// work-list order (and with it how neighbouring tiles share L2 and how the
// tail of the largest instances lines up) by timing reduction-only passes over
// the whole work list -- the full derivative work of a stage without any
// store, so the state of the batch is untouched -- and chooses the number of
// RK steps per graph replay from the amount of work per step.  Results are
// cached per batch shape.  The arena is laid out for 64-wide tiles, which
// covers the narrow ones, so both widths run on the same arrays.  A batch of
// several Hamiltonians runs either one launch per stage (the kernel choosing
// each tile's Hamiltonian) or one launch per Hamiltonian (a kernel specialised
// for it); the autotuner times both.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/alweno.h"
#include "alw_internal.h"
#include "alw_params2d.h"

using namespace alw;

namespace {

alw_status berr(alw_status st, const char *fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return st;
}

#define B_CUDA(call)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return berr(ALW_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define B_LAUNCH(call)                                                                                   \
  do {                                                                                                   \
    int e_ = (call);                                                                                     \
    if (e_ != 0) return berr(ALW_ECUDA, "%s: %s", #call, cudaGetErrorString((cudaError_t)e_));          \
  } while (0)

struct TuneKey {
  int sms, prec, weights, tiles_log2, max_inst_tiles_log2;
  bool operator<(const TuneKey &o) const {
    return std::tie(sms, prec, weights, tiles_log2, max_inst_tiles_log2) <
           std::tie(o.sms, o.prec, o.weights, o.tiles_log2, o.max_inst_tiles_log2);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, alw_batch_tuning> g_tune_cache;

int ilog2(long long v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

}  // namespace

struct alw_batch {
  alw_scheme scheme{};
  int prec = P_MIXED;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  struct Pending {
    alw_grid grid;
    int ham;
    double t_final;
    double *dev_phi0;  // phi0 copied to the device when the instance is added (freed by build)
    size_t n;
  };
  std::vector<Pending> pend;
  // device side (built on the first run)
  bool built = false;
  int pitch = 0;
  long long rows = 0;
  size_t arr_bytes = 0;
  void *H[2] = {nullptr, nullptr}, *Lo[2] = {nullptr, nullptr}, *D1 = nullptr, *D2 = nullptr;  // MIXED
  void *P = nullptr, *A = nullptr, *B = nullptr;                                               // FP32
  CUtensorMap maps[6];            // boxes of 64-wide tiles
  CUtensorMap maps_narrow[6];     // boxes of 32-wide tiles
  std::vector<InstDesc> h_inst;   // instance table for 64-wide tiles
  std::vector<InstDesc> h_inst_narrow;  // the same with the tile counts of 32-wide tiles
  InstDesc *d_inst = nullptr, *d_inst_narrow = nullptr;
  DevState *d_state = nullptr;
  DevState *h_state = nullptr;  // pinned mirror
  int *d_done = nullptr;
  int *h_done = nullptr;        // pinned
  int *d_tiles = nullptr;
  int ntiles_alloc = 0;
  std::vector<std::pair<void *, size_t>> allocs;
  alw_batch_tuning tuning{};
  bool tuned = false, user_tuning = false;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0, graph_ntiles = 0;
  int grid_cap = 0;
  // the uploaded work list: one group of entries per Hamiltonian, back to back in d_tiles
  struct Group {
    int off, n, kind;
  };
  std::vector<Group> groups;

  void *alloc(size_t bytes) {
    void *p = dev_alloc(bytes, stream);
    if (p) allocs.emplace_back(p, bytes);
    return p;
  }
};

namespace {

constexpr int kDefaultRun = 4;  // work-list entries a CTA takes in a row (alw_batch_tuning::run)

// Releases the device copies of phi0 held for instances not yet built into the arena.
void free_pending(alw_batch *b) {
  for (auto &pd : b->pend)
    if (pd.dev_phi0) {
      dev_free(pd.dev_phi0, pd.n * sizeof(double), b->stream);
      pd.dev_phi0 = nullptr;
    }
}

bool narrow(const alw_batch *b) { return b->tuning.tile_w == kTile2DXNarrow; }

// The instance table of the tuning's tile width.
const std::vector<InstDesc> &insts(const alw_batch *b) { return narrow(b) ? b->h_inst_narrow : b->h_inst; }

int cap_for(const alw_batch *b) {
  const int w = narrow(b) ? kTile2DXNarrow : kTile2DX;
  return b->prec == P_MIXED ? stage2d_grid_cap_mixed(b->scheme.weights, w) : stage2d_grid_cap_f32(b->scheme.weights, w);
}

Stage2DParams batch_params(const alw_batch *b, int stage, int loop_mode, int ntiles) {
  Stage2DParams q;
  memset(&q, 0, sizeof q);
  memcpy(q.maps, narrow(b) ? b->maps_narrow : b->maps, sizeof q.maps);
  q.tile_w = narrow(b) ? kTile2DXNarrow : kTile2DX;
  StageParams &p = q.p;
  p.pitch = b->pitch;
  p.dim = 2;
  p.weights = b->scheme.weights;
  p.alpha_mode = b->scheme.alpha_mode == ALW_ALPHA_DEFAULT ? ALW_ALPHA_GLOBAL_LAGGED : b->scheme.alpha_mode;
  p.loop_mode = loop_mode;
  p.stage = stage;
  p.src_of = stage == 0 ? 1 : stage;
  p.eps = b->scheme.eps;
  p.cfl = b->scheme.cfl;
  p.alpha_fixed[0] = b->scheme.alpha_fixed[0];
  p.alpha_fixed[1] = b->scheme.alpha_fixed[1];
  p.dt_slot = 2;
  if (stage == 0) {
    p.read_slot = -1;
    p.write_slot = 2;
    p.zero_slot = -1;
  } else {
    p.read_slot = stage == 1 ? 2 : stage - 2;
    p.write_slot = stage - 1;
    p.zero_slot = stage % 3;
  }
  const int which = p.src_of;
  if (b->prec == P_MIXED) {
    p.mix_hi[0] = b->H[0];
    p.mix_hi[1] = b->H[1];
    p.mix_lo[0] = b->Lo[0];
    p.mix_lo[1] = b->Lo[1];
    if (stage == 1) p.out0 = b->D1;
    if (stage == 2) p.out0 = b->D2;
    q.map_a = 0;
    q.map_b = 2;
    q.map_c = which == 1 ? -1 : (which == 2 ? 4 : 5);
  } else {
    p.out0 = stage == 1 ? b->A : (stage == 2 ? b->B : (stage == 3 ? b->P : nullptr));
    q.map_a = which == 1 ? 0 : (which == 2 ? 1 : 2);
    q.map_b = stage >= 2 ? 0 : -1;
    q.map_c = -1;
  }
  q.ntiles = ntiles;
  q.grid_ctas = b->tuning.grid_ctas;
  q.insts = narrow(b) ? b->d_inst_narrow : b->d_inst;
  q.states = b->d_state;
  q.tiles = b->d_tiles;
  q.done_count = b->d_done;
  return q;
}

int launch(const alw_batch *b, const Stage2DParams &q) {
  return b->prec == P_MIXED ? launch_stage2d_mixed(q, b->stream) : launch_stage2d_f32(q, b->stream);
}

// Work list of the instances for which `live[i]` holds, in the requested order.
std::vector<int> ordered_list(const alw_batch *b, const std::vector<char> &live, int order) {
  const std::vector<InstDesc> &I = insts(b);
  std::vector<int> ids;
  for (size_t i = 0; i < I.size(); ++i)
    if (live[i]) ids.push_back((int)i);
  if (order == ALW_ORDER_LARGEST_FIRST)
    std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return I[x].ntiles > I[y].ntiles; });
  std::vector<int> list;
  if (order == ALW_ORDER_INTERLEAVED) {
    int maxt = 0;
    for (int i : ids) maxt = std::max(maxt, I[i].ntiles);
    for (int t = 0; t < maxt; ++t)
      for (int i : ids)
        if (t < I[i].ntiles) list.push_back(i * 65536 + t);
  } else {
    for (int i : ids)
      for (int t = 0; t < I[i].ntiles; ++t) list.push_back(i * 65536 + t);
  }
  return list;
}

// The work list of the live instances in the given order, laid out over the CTAs the launches
// will use in runs of `run` entries (alw_batch_tuning::run).
std::vector<int> work_list(const alw_batch *b, const std::vector<char> &live, int order, int run) {
  std::vector<int> list = ordered_list(b, live, order);
  if (run == 1) return list;
  std::vector<int> out;
  const int G = stage2d_grid((int)list.size(), b->tuning.grid_ctas, b->grid_cap);
  if (run == 0) cta_runs(list, G, out);
  else cta_blocks(list, G, run, out);
  return out;
}

// Uploads the work list of the live instances as one group per Hamiltonian (each in the given
// order and run layout), so that every launch runs the kernel specialised for its Hamiltonian --
// or, with tuning.one_launch, as one group (kind -1) that a single launch per stage runs with the
// Hamiltonian chosen per tile.  Returns the number of entries.
alw_status upload_groups(alw_batch *b, const std::vector<char> &live, int order, int run, int *total) {
  std::vector<int> all;
  b->groups.clear();
  if (b->tuning.one_launch) {
    const std::vector<int> list = work_list(b, live, order, run);
    b->groups.push_back({0, (int)list.size(), -1});
    all = list;
  }
  for (int kind = 0; kind < 16 && !b->tuning.one_launch; ++kind) {
    std::vector<char> sel(live.size(), 0);
    bool any = false;
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i] && b->h_inst[i].ham == kind) sel[i] = 1, any = true;
    if (!any) continue;
    const std::vector<int> list = work_list(b, sel, order, run);
    b->groups.push_back({(int)all.size(), (int)list.size(), kind});
    all.insert(all.end(), list.begin(), list.end());
  }
  if ((int)all.size() > b->ntiles_alloc) return berr(ALW_EINVAL, "work list larger than allocated");
  if (!all.empty())
    B_CUDA(cudaMemcpyAsync(b->d_tiles, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  if (total) *total = (int)all.size();
  return ALW_OK;
}

// One stage (0: reduction only) over every group of the uploaded work list.
alw_status launch_groups(alw_batch *b, int stage, int loop_mode, double dt_stage, int write_slot = -2) {
  for (const auto &g : b->groups) {
    Stage2DParams q = batch_params(b, stage, loop_mode, g.n);
    q.tiles = b->d_tiles + g.off;
    q.batch_kind1 = g.kind + 1;
    q.p.dt_value = dt_stage;
    if (write_slot != -2) q.p.write_slot = write_slot;
    B_LAUNCH(launch(b, q));
  }
  return ALW_OK;
}

alw_status enqueue_steps(alw_batch *b, int loop_mode, int nsteps, double dt_stage) {
  for (int s = 0; s < nsteps; ++s)
    for (int stage = 1; stage <= 3; ++stage) {
      alw_status st = launch_groups(b, stage, loop_mode, dt_stage);
      if (st) return st;
    }
  return ALW_OK;
}

alw_status build_graph(alw_batch *b, int nsteps, int ntiles) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  B_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  alw_status st = enqueue_steps(b, LOOP_STEP_TO, nsteps, 0.0);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (st != ALW_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return berr(ALW_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return berr(ALW_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  b->graph_steps = nsteps;
  b->graph_ntiles = ntiles;
  return ALW_OK;
}

alw_status prime_alpha(alw_batch *b) { return launch_groups(b, 0, LOOP_ADVANCE, 0.0); }

// Lay out the arena, upload every instance and prepare the device tables.
alw_status build(alw_batch *b) {
  const int n = (int)b->pend.size();
  if (n == 0) return berr(ALW_EINVAL, "batch is empty");
  // geometry
  int pitch = 0;
  long long rows = 0;
  b->h_inst.assign(n, InstDesc{});
  long long total_tiles = 0;
  for (int i = 0; i < n; ++i) {
    const alw_batch::Pending &pd = b->pend[i];
    InstDesc &d = b->h_inst[i];
    d.nx = pd.grid.nx;
    d.ny = pd.grid.ny;
    d.tiles_x = (d.nx + kTile2DX - 1) / kTile2DX;
    d.tiles_y = (d.ny + kTile2DY - 1) / kTile2DY;
    d.ntiles = d.tiles_x * d.tiles_y;
    d.row_off = (int)rows;
    d.ham = pd.ham;
    d.bc = pd.grid.bc;
    const double dx = (pd.grid.xhi - pd.grid.xlo) / d.nx, dy = (pd.grid.yhi - pd.grid.ylo) / d.ny;
    d.dx = (float)dx;
    d.dy = (float)dy;
    d.rdx = (float)(1.0 / dx);
    d.rdy = (float)(1.0 / dy);
    d.xlo = (float)pd.grid.xlo;
    d.ylo = (float)pd.grid.ylo;
    d.lx = b->scheme.dt_mode == ALW_DT_DX53 ? std::pow(dx, 5.0 / 3.0) : dx;
    d.ly = b->scheme.dt_mode == ALW_DT_DX53 ? std::pow(dy, 5.0 / 3.0) : dy;
    pitch = std::max(pitch, d.tiles_x * kTile2DX + 2 * GX);
    rows += (long long)d.tiles_y * kTile2DY + 2 * GY;
  }
  // the same instances cut into 32-wide tiles (inside the same padded rows: ceil(nx / 32) * 32
  // never exceeds ceil(nx / 64) * 64)
  b->h_inst_narrow = b->h_inst;
  long long total_narrow = 0;
  for (int i = 0; i < n; ++i) {
    InstDesc &d = b->h_inst_narrow[i];
    d.tiles_x = (d.nx + kTile2DXNarrow - 1) / kTile2DXNarrow;
    d.ntiles = d.tiles_x * d.tiles_y;
    total_tiles += b->h_inst[i].ntiles;
    total_narrow += d.ntiles;
    if (d.ntiles > 65535) return berr(ALW_EINVAL, "instance %d has more than 65535 tiles", i);
  }
  total_tiles = std::max(total_tiles, total_narrow);
  if (rows > (1ll << 31)) return berr(ALW_EINVAL, "batch too tall");
  b->pitch = pitch;
  b->rows = rows;
  b->arr_bytes = (size_t)pitch * (size_t)rows * sizeof(float);
  std::vector<void **> bufs;
  if (b->prec == P_MIXED) bufs = {&b->H[0], &b->H[1], &b->Lo[0], &b->Lo[1], &b->D1, &b->D2};
  else bufs = {&b->P, &b->A, &b->B};
  for (void **p : bufs) {
    *p = b->alloc(b->arr_bytes);
    if (!*p) return berr(ALW_ENOMEM, "device allocation of %zu bytes failed", b->arr_bytes);
    B_CUDA(cudaMemsetAsync(*p, 0, b->arr_bytes, b->stream));
  }
  b->d_state = (DevState *)b->alloc(sizeof(DevState) * n);
  b->d_inst = (InstDesc *)b->alloc(sizeof(InstDesc) * n);
  b->d_inst_narrow = (InstDesc *)b->alloc(sizeof(InstDesc) * n);
  b->d_done = (int *)b->alloc(sizeof(int));
  b->ntiles_alloc = (int)total_tiles;
  b->d_tiles = (int *)b->alloc(sizeof(int) * std::max<long long>(1, total_tiles));
  if (!b->d_state || !b->d_inst || !b->d_inst_narrow || !b->d_done || !b->d_tiles)
    return berr(ALW_ENOMEM, "device allocation failed");
  if (cudaHostAlloc((void **)&b->h_state, sizeof(DevState) * n, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void **)&b->h_done, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return berr(ALW_ENOMEM, "pinned host allocation failed");
  }
  memset(b->h_state, 0, sizeof(DevState) * n);
  for (int i = 0; i < n; ++i) {
    b->h_inst[i].st = b->d_state + i;
    b->h_inst_narrow[i].st = b->d_state + i;
    b->h_state[i].t = 0.0;
    b->h_state[i].t_final = b->pend[i].t_final;
  }
  B_CUDA(cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaMemcpyAsync(b->d_inst_narrow, b->h_inst_narrow.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice,
                         b->stream));
  B_CUDA(cudaMemcpyAsync(b->d_state, b->h_state, sizeof(DevState) * n, cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaMemsetAsync(b->d_done, 0, sizeof(int), b->stream));
  // tensor maps over the whole stacked arrays
  memset(b->maps, 0, sizeof b->maps);
  memset(b->maps_narrow, 0, sizeof b->maps_narrow);
  void *bases[6];
  int nb = 0;
  if (b->prec == P_MIXED) {
    void *x[6] = {b->H[0], b->H[1], b->Lo[0], b->Lo[1], b->D1, b->D2};
    memcpy(bases, x, sizeof x);
    nb = 6;
  } else {
    void *x[3] = {b->P, b->A, b->B};
    memcpy(bases, x, sizeof x);
    nb = 3;
  }
  for (int i = 0; i < nb; ++i) {
    int r = encode_tile_map(&b->maps[i], bases[i], pitch, rows, kBox2DW);
    if (r == 0) r = encode_tile_map(&b->maps_narrow[i], bases[i], pitch, rows, kBox2DWNarrow);
    if (r) return berr(ALW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", r);
  }
  // split phi0 of every instance (on the device since it was added) into its block of rows with
  // its ghost frame; one synchronisation at the end
  alw_status st = ALW_OK;
  for (int i = 0; i < n && st == ALW_OK; ++i) {
    const InstDesc &d = b->h_inst[i];
    const size_t off = (size_t)d.row_off * pitch;  // element offset of the instance's first row
    const double *src = b->pend[i].dev_phi0;
    int le;
    if (b->prec == P_MIXED)
      le = launch_mixed_split(src, (float *)b->H[0] + off, (float *)b->Lo[0] + off, d.nx, d.ny, pitch, 2, b->stream);
    else
      le = launch_unpack(src, 0, (float *)b->P + off, 1, d.nx, d.ny, pitch, 2, b->stream);
    if (le) {
      st = berr(ALW_ECUDA, "upload kernel: %s", cudaGetErrorString((cudaError_t)le));
      break;
    }
    GhostParams g;
    memset(&g, 0, sizeof g);
    g.nx = d.nx;
    g.ny = d.ny;
    g.pitch = pitch;
    g.dim = 2;
    g.bc = d.bc;
    g.prec = b->prec;
    if (b->prec == P_MIXED) {
      g.mixed_pair = 1;
      g.a0 = (float *)b->H[0] + off;
      g.a1 = (float *)b->Lo[0] + off;
    } else {
      g.a0 = (float *)b->P + off;
    }
    le = launch_ghosts(g, b->stream);
    if (le) st = berr(ALW_ECUDA, "ghost kernel: %s", cudaGetErrorString((cudaError_t)le));
  }
  cudaStreamSynchronize(b->stream);  // the staged copies are released only after their readers
  free_pending(b);
  if (st) return st;
  std::vector<char> live(n, 1);
  b->grid_cap = cap_for(b);
  st = upload_groups(b, live, ALW_ORDER_INSTANCE, kDefaultRun, nullptr);
  if (st) return st;
  st = prime_alpha(b);
  if (st) return st;
  B_CUDA(cudaStreamSynchronize(b->stream));
  b->built = true;
  return ALW_OK;
}

// Time `passes` reduction-only sweeps over the work list (no stores; alpha goes to the unused slot 3).
alw_status trial(alw_batch *b, int passes, double *ms) {
  cudaEvent_t e0, e1;
  B_CUDA(cudaEventCreate(&e0));
  B_CUDA(cudaEventCreate(&e1));
  B_CUDA(cudaEventRecord(e0, b->stream));
  alw_status st = ALW_OK;
  for (int i = 0; i < passes && st == ALW_OK; ++i) st = launch_groups(b, 0, LOOP_ADVANCE, 0.0, 3);
  B_CUDA(cudaEventRecord(e1, b->stream));
  B_CUDA(cudaEventSynchronize(e1));
  float f = 0;
  cudaEventElapsedTime(&f, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = f;
  return st;
}

alw_status autotune(alw_batch *b) {
  long long total = 0;
  int maxt = 0;
  for (auto &d : b->h_inst) {
    total += d.ntiles;
    maxt = std::max(maxt, d.ntiles);
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TuneKey key{sms, b->prec, b->scheme.weights, ilog2(total), ilog2(maxt)};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      b->tuning = it->second;
      b->tuned = true;
      return ALW_OK;
    }
  }
  std::vector<char> live(b->h_inst.size(), 1);
  const int widths[2] = {kTile2DX, kTile2DXNarrow};
  const int orders[3] = {ALW_ORDER_INSTANCE, ALW_ORDER_LARGEST_FIRST, ALW_ORDER_INTERLEAVED};
  // one launch per stage is a choice only when the batch mixes Hamiltonians
  bool mixed_hams = false;
  for (auto &d : b->h_inst) mixed_hams |= d.ham != b->h_inst[0].ham;
  const int launches_n = mixed_hams ? 2 : 1;
  // runs of 4 entries per CTA: each CTA changes instance (and closes a run) a quarter as often
  // as with single entries while neighbouring blocks of tiles still run side by side (one
  // contiguous stretch per CTA times fast in these reduction-only trials but loses in full
  // stages, so the run length is fixed rather than tuned)
  const int runs[1] = {kDefaultRun};
  b->tuning.grid_ctas = 0;
  // successive halving: every candidate is timed once (after one warm-up pass per kernel form, which
  // also loads the form's kernels), the three fastest once more; the best two-pass total wins
  struct Cand {
    alw_batch_tuning t;
    double ms;
  };
  std::vector<Cand> cands;
  auto time_one = [&](const alw_batch_tuning &t, int passes, double *ms) -> alw_status {
    b->tuning.tile_w = t.tile_w;
    b->tuning.one_launch = t.one_launch;
    b->grid_cap = cap_for(b);
    alw_status st = upload_groups(b, live, t.order, t.run, nullptr);
    if (st) return st;
    return trial(b, passes, ms);
  };
  for (int one = 0; one < launches_n; ++one)
    for (int w : widths) {
      b->tuning.tile_w = w;
      b->tuning.one_launch = one;
      b->grid_cap = cap_for(b);
      if (b->grid_cap <= 0) continue;
      bool warm = false;
      for (int o : orders)
        for (int l : runs) {
          alw_batch_tuning t{};
          t.order = o;
          t.run = l;
          t.tile_w = w;
          t.one_launch = one;
          double ms;
          alw_status st;
          if (!warm) {
            st = time_one(t, 1, &ms);
            if (st) return st;
            warm = true;
          }
          st = time_one(t, 1, &ms);
          if (st) return st;
          cands.push_back({t, ms});
        }
    }
  if (cands.empty()) return berr(ALW_ECUDA, "stage kernel occupancy query failed");
  std::sort(cands.begin(), cands.end(), [](const Cand &x, const Cand &y) { return x.ms < y.ms; });
  alw_batch_tuning best = cands[0].t;
  double best_ms = 1e30;
  for (size_t i = 0; i < cands.size() && i < 3; ++i) {
    double ms;
    alw_status st = time_one(cands[i].t, 1, &ms);
    if (st) return st;
    if (ms + cands[i].ms < best_ms) {
      best_ms = ms + cands[i].ms;
      best = cands[i].t;
    }
  }
  best.steps_per_graph = total >= 4096 ? 2 : (total >= 512 ? 8 : 32);
  best.grid_ctas = 0;  // occupancy cap
  b->tuning = best;
  b->grid_cap = cap_for(b);
  b->tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return ALW_OK;
}

}  // namespace

extern "C" {

alw_status alw_batch_create(const alw_scheme *scheme, void *cuda_stream, alw_batch **out) {
  if (!scheme || !out) return berr(ALW_EINVAL, "NULL argument");
  *out = nullptr;
  if (scheme->precision != ALW_PREC_MIXED && scheme->precision != ALW_PREC_FP32)
    return berr(ALW_EINVAL, "batches run the float kernels: precision must be FP32 or MIXED");
  if (scheme->weights != ALW_W_ARCLEN && scheme->weights != ALW_W_JP) return berr(ALW_EINVAL, "unknown weights");
  if (scheme->alpha_mode != ALW_ALPHA_DEFAULT && scheme->alpha_mode != ALW_ALPHA_GLOBAL_LAGGED &&
      scheme->alpha_mode != ALW_ALPHA_LOCAL_LAGGED && scheme->alpha_mode != ALW_ALPHA_FIXED)
    return berr(ALW_EINVAL, "batches support the lagged and fixed alpha modes");
  if (!(scheme->eps > 0.0) || !(scheme->cfl > 0.0)) return berr(ALW_EINVAL, "eps and cfl must be > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return berr(ALW_ECUDA, "no CUDA device");
  }
  alw_batch *b = new (std::nothrow) alw_batch();
  if (!b) return berr(ALW_ENOMEM, "host allocation failed");
  b->scheme = *scheme;
  b->prec = scheme->precision == ALW_PREC_MIXED ? P_MIXED : P_F32;
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (!b->stream) {
    if (cudaStreamCreate(&b->stream) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return berr(ALW_ECUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  *out = b;
  return ALW_OK;
}

alw_status alw_batch_add(alw_batch *b, const alw_grid *grid, const alw_hamiltonian *ham, const double *host_phi0,
                         size_t n, double t_final, int32_t *id_out) {
  if (!b || !grid || !ham || !host_phi0) return berr(ALW_EINVAL, "NULL argument");
  if (b->built) return berr(ALW_EBUSY, "instances cannot be added after the batch has run");
  if (grid->dim != 2 || grid->nx < 1 || grid->ny < 1) return berr(ALW_EINVAL, "batches hold 2D grids");
  if (grid->bc != ALW_BC_PERIODIC) return berr(ALW_EINVAL, "batches hold periodic grids");
  if (n != (size_t)grid->nx * grid->ny) return berr(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)grid->nx * grid->ny);
  const long long tiles = (long long)((grid->nx + kTile2DX - 1) / kTile2DX) * ((grid->ny + kTile2DY - 1) / kTile2DY);
  if (tiles >= 65536) return berr(ALW_EINVAL, "instance too large for a batch (%lld tiles)", tiles);
  if (ham->kind != ALW_H_BURGERS2D && ham->kind != ALW_H_NEGCOS2D && ham->kind != ALW_H_SIN2D &&
      ham->kind != ALW_H_EIKONAL2D)
    return berr(ALW_EINVAL, "batches hold 2D Hamiltonians");
  if (!std::isfinite(t_final) || t_final < 0.0) return berr(ALW_EINVAL, "bad t_final");
  if (!(grid->xhi > grid->xlo) || !(grid->yhi > grid->ylo)) return berr(ALW_EINVAL, "empty extent");
  if (b->pend.size() >= 32768) return berr(ALW_EINVAL, "too many instances");
  alw_batch::Pending p;
  p.grid = *grid;
  p.ham = ham->kind;
  p.t_final = t_final;
  p.n = n;
  // copy phi0 to the device now (the caller may reuse its buffer on return)
  p.dev_phi0 = (double *)dev_alloc(n * sizeof(double), b->stream);
  if (!p.dev_phi0) return berr(ALW_ENOMEM, "device allocation of %zu bytes failed", n * sizeof(double));
  cudaError_t e = cudaMemcpyAsync(p.dev_phi0, host_phi0, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    dev_free(p.dev_phi0, n * sizeof(double), b->stream);
    return berr(ALW_ECUDA, "upload: %s", cudaGetErrorString(e));
  }
  b->pend.push_back(p);
  if (id_out) *id_out = (int32_t)(b->pend.size() - 1);
  return ALW_OK;
}

alw_status alw_batch_set_tuning(alw_batch *b, const alw_batch_tuning *t) {
  if (!b) return berr(ALW_EINVAL, "NULL argument");
  if (!t) {
    b->user_tuning = false;
    b->tuned = false;
    return ALW_OK;
  }
  if (t->order < ALW_ORDER_INSTANCE || t->order > ALW_ORDER_INTERLEAVED || t->steps_per_graph < 1 ||
      t->steps_per_graph > 256 || t->grid_ctas < 0 ||
      t->run < 0 || t->run > 64 || (t->tile_w != 0 && t->tile_w != kTile2DX && t->tile_w != kTile2DXNarrow) ||
      (t->one_launch != 0 && t->one_launch != 1))
    return berr(ALW_EINVAL, "bad tuning");
  b->tuning = *t;
  if (b->tuning.tile_w == 0) b->tuning.tile_w = kTile2DX;
  b->user_tuning = true;
  b->tuned = true;
  return ALW_OK;
}

alw_status alw_batch_get_tuning(alw_batch *b, alw_batch_tuning *t) {
  if (!b || !t) return berr(ALW_EINVAL, "NULL argument");
  *t = b->tuning;
  return ALW_OK;
}

alw_status alw_batch_build(alw_batch *b) {
  if (!b) return berr(ALW_EINVAL, "NULL argument");
  if (!b->built) {
    alw_status st = build(b);
    if (st) return st;
  }
  if (!b->tuned) return autotune(b);
  return ALW_OK;
}

alw_status alw_batch_run(alw_batch *b, int64_t *replays_out) {
  if (!b) return berr(ALW_EINVAL, "NULL argument");
  alw_status st = ALW_OK;
  if (!b->built) {
    st = build(b);
    if (st) return st;
  }
  if (!b->tuned) {
    st = autotune(b);
    if (st) return st;
  }
  const int ninst = (int)b->h_inst.size();
  b->grid_cap = cap_for(b);  // of the tuning's tile width
  if (b->grid_cap <= 0) return berr(ALW_ECUDA, "stage kernel occupancy query failed");
  // live set from the device state
  B_CUDA(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(DevState) * ninst, cudaMemcpyDeviceToHost, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  std::vector<char> live(ninst, 0);
  int nlive = 0;
  for (int i = 0; i < ninst; ++i) {
    live[i] = b->h_state[i].t < b->h_state[i].t_final && !b->h_state[i].err;
    nlive += live[i];
  }
  int64_t replays = 0;
  int stalls = 0;
  long long last_steps_sum = -1;
  while (nlive > 0) {
    int ntiles_now = 0;
    st = upload_groups(b, live, b->tuning.order, b->tuning.run, &ntiles_now);
    if (st) return st;
    st = build_graph(b, b->tuning.steps_per_graph, ntiles_now);
    if (st) return st;
    // replay until half of this work list is dead, then compact it
    for (;;) {
      B_CUDA(cudaGraphLaunch(b->graph, b->stream));
      ++replays;
      B_CUDA(cudaMemcpyAsync(b->h_state, b->d_state, sizeof(DevState) * ninst, cudaMemcpyDeviceToHost, b->stream));
      B_CUDA(cudaStreamSynchronize(b->stream));
      int live_tiles = 0, now_live = 0;
      long long steps_sum = 0;
      for (int i = 0; i < ninst; ++i) {
        const DevState &s = b->h_state[i];
        const bool l = s.t < s.t_final && !s.err;
        live[i] = l;
        now_live += l;
        if (l) live_tiles += insts(b)[i].ntiles;
        steps_sum += s.steps;
      }
      nlive = now_live;
      stalls = (steps_sum == last_steps_sum) ? stalls + 1 : 0;
      last_steps_sum = steps_sum;
      if (stalls >= 3) return berr(ALW_ETIMEOUT, "batch made no progress");
      if (nlive == 0 || 2 * live_tiles < ntiles_now) break;
    }
  }
  if (replays_out) *replays_out = replays;
  for (int i = 0; i < ninst; ++i)
    if (b->h_state[i].err)
      return berr(b->h_state[i].err & 2 ? ALW_ETIMEOUT : ALW_ENONFINITE, "instance %d: non-finite dH/dp or stalled load", i);
  return ALW_OK;
}

alw_status alw_batch_get_phi(alw_batch *b, int32_t id, double *host_out, size_t n) {
  if (!b || !host_out) return berr(ALW_EINVAL, "NULL argument");
  if (!b->built) return berr(ALW_EINVAL, "batch has not run");
  if (id < 0 || id >= (int)b->h_inst.size()) return berr(ALW_ENOTFOUND, "no instance %d", id);
  const InstDesc &d = b->h_inst[id];
  if (n != (size_t)d.nx * d.ny) return berr(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)d.nx * d.ny);
  B_CUDA(cudaMemcpyAsync(&b->h_state[id], &b->d_state[id], sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  const int cur = b->h_state[id].cur;
  const size_t off = (size_t)d.row_off * b->pitch;
  void *tmp = dev_alloc(n * sizeof(double), b->stream);
  if (!tmp) return berr(ALW_ENOMEM, "device allocation failed");
  int le;
  if (b->prec == P_MIXED)
    le = launch_mixed_join((float *)b->H[cur] + off, (float *)b->Lo[cur] + off, nullptr, (double *)tmp, d.nx, d.ny,
                           b->pitch, 2, b->stream);
  else
    le = launch_pack((float *)b->P + off, 1, tmp, 0, d.nx, d.ny, b->pitch, 2, b->stream);
  alw_status st = ALW_OK;
  if (le) st = berr(ALW_ECUDA, "gather: %s", cudaGetErrorString((cudaError_t)le));
  if (st == ALW_OK) {
    cudaError_t e = cudaMemcpyAsync(host_out, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) st = berr(ALW_ECUDA, "copy: %s", cudaGetErrorString(e));
  }
  dev_free(tmp, n * sizeof(double), b->stream);
  B_CUDA(cudaStreamSynchronize(b->stream));
  return st;
}

alw_status alw_batch_get_state(alw_batch *b, int32_t id, alw_state *state) {
  if (!b || !state) return berr(ALW_EINVAL, "NULL argument");
  if (!b->built) return berr(ALW_EINVAL, "batch has not run");
  if (id < 0 || id >= (int)b->h_inst.size()) return berr(ALW_ENOTFOUND, "no instance %d", id);
  DevState s;
  B_CUDA(cudaMemcpyAsync(&s, &b->d_state[id], sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  state->t = s.t;
  state->steps = s.steps;
  memcpy(&state->alpha[0], &s.alpha_bits[2][0], sizeof(double));
  memcpy(&state->alpha[1], &s.alpha_bits[2][1], sizeof(double));
  return ALW_OK;
}

alw_status alw_batch_memory_bytes(alw_batch *b, size_t *bytes) {
  if (!b || !bytes) return berr(ALW_EINVAL, "NULL argument");
  size_t t = 0;
  for (auto &a : b->allocs) t += a.second;
  *bytes = t;
  return ALW_OK;
}

alw_status alw_batch_destroy(alw_batch *b) {
  if (!b) return ALW_OK;
  cudaStreamSynchronize(b->stream);
  free_pending(b);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto &a : b->allocs) dev_free(a.first, a.second, b->stream);
  cudaStreamSynchronize(b->stream);
  if (b->h_state) cudaFreeHost(b->h_state);
  if (b->h_done) cudaFreeHost(b->h_done);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
  return ALW_OK;
}

}  // extern "C"
