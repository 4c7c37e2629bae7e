// Host runtime and C ABI of the WENO-L solver: buffers in the padded ghosted
// layout, the device-resident time state, CUDA graphs of RK3 steps, and the
// host loop that replays them until the device reports t >= t_final.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/alweno.h"
#include "alw_internal.h"
#include "alw_params2d.h"

using namespace alw;

namespace {

thread_local std::string g_err;

alw_status fail(alw_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define ALW_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(ALW_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define ALW_LAUNCH(call)                                                                 \
  do {                                                                                   \
    int e_ = (call);                                                                     \
    if (e_ != 0) return fail(ALW_ECUDA, "%s: %s", #call, cudaGetErrorString((cudaError_t)e_)); \
  } while (0)

std::mutex g_alloc_mu;
alw_allocator g_alloc = {nullptr, nullptr, nullptr};

void *dev_alloc_impl(size_t bytes, cudaStream_t s) {
  alw_allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  if (a.alloc) return a.alloc(bytes, (void *)s, a.ctx);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free_impl(void *p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  alw_allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  if (a.free) a.free(p, bytes, (void *)s, a.ctx);
  else cudaFreeAsync(p, s);
}

}  // namespace

void alw::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    cudaGetLastError();
  }
  return fn;
}


int alw::encode_tile_map(CUtensorMap *m, void *base, long long pitch, long long rows, int box_w) {
  auto enc = tensor_map_encoder_fn();
  if (!enc) return -1;
  const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)kBox2DH};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : (int)r;
}

void *alw::dev_alloc(size_t bytes, void *stream) { return dev_alloc_impl(bytes, reinterpret_cast<cudaStream_t>(stream)); }
void alw::dev_free(void *ptr, size_t bytes, void *stream) {
  dev_free_impl(ptr, bytes, reinterpret_cast<cudaStream_t>(stream));
}

int alw::tile_x(int prec, int dim) {
  if (dim == 1) return TX1D;
  return prec == P_F64 ? Tile<P_F64>::TX : Tile<P_F32>::TX;
}
int alw::tile_y(int prec, int dim) {
  if (dim == 1) return 1;
  return prec == P_F64 ? Tile<P_F64>::TY : Tile<P_F32>::TY;
}

struct alw_solver {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  alw_grid grid{};
  alw_hamiltonian ham{};
  alw_scheme scheme{};
  int prec = 0, dim = 2, nx = 0, ny = 1, pitch = 0, rows = 0, tiles_x = 0, tiles_y = 0;
  int alpha_mode = 0;
  double dx = 0, dy = 0, lx = 0, ly = 0;
  size_t elem = 8, arr_bytes = 0;
  void *P = nullptr, *A = nullptr, *B = nullptr;                  // F64/F32
  void *H[2] = {nullptr, nullptr}, *Lo[2] = {nullptr, nullptr};   // MIXED phi^n pairs
  void *D1 = nullptr, *D2 = nullptr;                              // MIXED increments
  DevState *st = nullptr;
  DevState *h_st = nullptr;   // pinned mirror
  double *h_tf = nullptr;     // pinned staging for t_final / dt
  std::vector<std::pair<void *, size_t>> allocs;
  cudaGraphExec_t g_step = nullptr;
  int g_step_n = 0;
  cudaGraphExec_t g_adv = nullptr;
  bool has_phi = false;
  bool use2d = false;       // persistent TMA kernel (2D float variants)
  int small_tiles = 0;      // FP64 2D: 16 x 16 tiles for grids that would not fill the GPU otherwise (1, 2)
  CUtensorMap maps[6];      // tensor maps of the padded arrays (see Stage2DParams)

  void *alloc(size_t bytes) {
    void *p = dev_alloc_impl(bytes, stream);
    if (p) allocs.emplace_back(p, bytes);
    return p;
  }
};

namespace {

bool is_1d_ham(int k) { return k == ALW_H_ADVECT1D || k == ALW_H_BURGERS1D || k == ALW_H_NEGCOS1D ||
                                      k == ALW_H_NONCONVEX1D; }

int kernel_prec(int precision) {
  return precision == ALW_PREC_FP64 ? P_F64 : precision == ALW_PREC_FP32 ? P_F32 : P_MIXED;
}

int launch_stage(const alw_solver *s, const StageParams &p) {
  if (s->use2d) {
    Stage2DParams q;
    memset(&q, 0, sizeof q);
    memcpy(q.maps, s->maps, sizeof q.maps);
    q.p = p;
    q.ntiles = s->tiles_x * s->tiles_y;
    q.insts = nullptr;
    q.tiles = nullptr;
    q.done_count = nullptr;
    InstDesc &d = q.inst0;
    d.nx = s->nx;
    d.ny = s->ny;
    d.tiles_x = s->tiles_x;
    d.tiles_y = s->tiles_y;
    d.row_off = 0;
    d.ham = s->ham.kind;
    d.bc = s->grid.bc;
    d.ntiles = q.ntiles;
    d.dx = (float)s->dx;
    d.dy = (float)s->dy;
    d.rdx = (float)(1.0 / s->dx);
    d.rdy = (float)(1.0 / s->dy);
    d.xlo = (float)s->grid.xlo;
    d.ylo = (float)s->grid.ylo;
    d.lx = s->lx;
    d.ly = s->ly;
    d.st = s->st;
    const int which = p.stage == 0 ? p.src_of : p.stage;
    if (s->prec == P_MIXED) {
      q.map_a = 0;
      q.map_b = 2;
      q.map_c = which == 1 ? -1 : (which == 2 ? 4 : 5);
      return launch_stage2d_mixed(q, s->stream);
    }
    q.map_a = which == 1 ? 0 : (which == 2 ? 1 : 2);
    q.map_b = p.stage >= 2 ? 0 : -1;
    q.map_c = -1;
    return launch_stage2d_f32(q, s->stream);
  }
  switch (s->prec) {
    case P_F64: return launch_stage_f64(p, s->stream);
    case P_F32: return launch_stage_f32(p, s->stream);
    default: return launch_stage_mixed(p, s->stream);
  }
}

bool exact_mode(int m) { return m == ALW_ALPHA_LOCAL_EXACT || m == ALW_ALPHA_GLOBAL_EXACT; }

// Parameters of stage `stage` (0 = reduction pass over the source of stage `src_of`).
StageParams make_params(const alw_solver *s, int stage, int src_of, int loop_mode) {
  StageParams p;
  memset(&p, 0, sizeof p);
  p.nx = s->nx;
  p.ny = s->ny;
  p.pitch = s->pitch;
  p.tiles_x = s->tiles_x;
  p.tiles_y = s->tiles_y;
  p.small_tiles = s->small_tiles;
  p.dim = s->dim;
  p.bc = s->grid.bc;
  p.ham = s->ham.kind;
  p.weights = s->scheme.weights;
  p.alpha_mode = s->alpha_mode;
  p.loop_mode = loop_mode;
  p.stage = stage;
  p.dx = s->dx;
  p.dy = s->dy;
  p.rdx = 1.0 / s->dx;
  p.rdy = 1.0 / s->dy;
  p.eps = s->scheme.eps;
  p.xlo = s->grid.xlo;
  p.ylo = s->dim == 2 ? s->grid.ylo : 0.0;
  p.cfl = s->scheme.cfl;
  p.lx = s->lx;
  p.ly = s->ly;
  p.alpha_fixed[0] = s->scheme.alpha_fixed[0];
  p.alpha_fixed[1] = s->scheme.alpha_fixed[1];
  p.state = s->st;
  p.dt_slot = exact_mode(s->alpha_mode) ? 3 : 2;
  const int which = stage == 0 ? src_of : stage;
  p.src_of = which;
  if (stage == 0) {
    p.read_slot = -1;
    p.write_slot = 3;
    p.zero_slot = -1;
  } else {
    p.read_slot = s->alpha_mode == ALW_ALPHA_GLOBAL_EXACT ? 3 : (stage == 1 ? 2 : stage - 2);
    p.write_slot = stage - 1;
    p.zero_slot = stage % 3;
  }
  if (s->prec == P_MIXED) {
    p.mix_hi[0] = s->H[0];
    p.mix_hi[1] = s->H[1];
    p.mix_lo[0] = s->Lo[0];
    p.mix_lo[1] = s->Lo[1];
    p.src2 = which == 1 ? nullptr : (which == 2 ? s->D1 : s->D2);
    if (stage == 1) p.out0 = s->D1;
    if (stage == 2) p.out0 = s->D2;
  } else {
    p.src0 = which == 1 ? s->P : (which == 2 ? s->A : s->B);
    p.base0 = s->P;
    if (stage == 1) p.out0 = s->A;
    if (stage == 2) p.out0 = s->B;
    if (stage == 3) p.out0 = s->P;
  }
  return p;
}

GhostParams ghost_params(const alw_solver *s, int after_stage) {
  GhostParams g;
  memset(&g, 0, sizeof g);
  g.nx = s->nx;
  g.ny = s->ny;
  g.pitch = s->pitch;
  g.dim = s->dim;
  g.bc = s->grid.bc;
  g.prec = s->prec;
  if (s->prec == P_MIXED) {
    if (after_stage == 1 || after_stage == 2) {
      g.a0 = after_stage == 1 ? s->D1 : s->D2;
      g.mixed_pair = 0;
      g.state = s->st;
      g.mix_hi[0] = s->H[0];
      g.mix_hi[1] = s->H[1];
    } else {
      g.mixed_pair = 1;
      g.state = s->st;
      g.mix_hi[0] = s->H[0];
      g.mix_hi[1] = s->H[1];
      g.mix_lo[0] = s->Lo[0];
      g.mix_lo[1] = s->Lo[1];
    }
  } else {
    g.a0 = after_stage == 1 ? s->A : (after_stage == 2 ? s->B : s->P);
  }
  return g;
}

// Enqueue one RK3 step (with the reduction passes and ghost fills the mode needs).
alw_status enqueue_step(alw_solver *s, int loop_mode) {
  const bool linx = s->grid.bc == ALW_BC_LINEXTRAP;
  for (int stage = 1; stage <= 3; ++stage) {
    const bool pre = (s->alpha_mode == ALW_ALPHA_GLOBAL_EXACT) || (s->alpha_mode == ALW_ALPHA_LOCAL_EXACT && stage == 1);
    if (pre) {
      ALW_CUDA(cudaMemsetAsync(&s->st->alpha_bits[3][0], 0, 2 * sizeof(unsigned long long), s->stream));
      ALW_LAUNCH(launch_stage(s, make_params(s, 0, stage, loop_mode)));
    }
    ALW_LAUNCH(launch_stage(s, make_params(s, stage, stage, loop_mode)));
    if (linx) ALW_LAUNCH(launch_ghosts(ghost_params(s, stage), s->stream));
  }
  return ALW_OK;
}

alw_status build_graph(alw_solver *s, int loop_mode, int nsteps, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  ALW_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  alw_status st = ALW_OK;
  for (int i = 0; i < nsteps && st == ALW_OK; ++i) st = enqueue_step(s, loop_mode);
  cudaError_t e = cudaStreamEndCapture(s->stream, &g);
  if (st != ALW_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(ALW_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ALW_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return ALW_OK;
}

alw_status read_state(alw_solver *s) {
  ALW_CUDA(cudaMemcpyAsync(s->h_st, s->st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
  ALW_CUDA(cudaStreamSynchronize(s->stream));
  return ALW_OK;
}

// Load interior values from a dense device array of doubles/floats into the current phi^n.
alw_status load_phi_dense(alw_solver *s, const void *dense, int dtype) {
  if (s->prec == P_MIXED) {
    const double *src = (const double *)dense;
    void *tmp = nullptr;
    if (dtype != 0) {  // widen floats to doubles first
      tmp = dev_alloc_impl((size_t)s->nx * s->ny * sizeof(double), s->stream);
      if (!tmp) return fail(ALW_ENOMEM, "device allocation of %zu bytes failed", (size_t)s->nx * s->ny * 8);
      // dense float -> dense double through the pack path is not available; use unpack into H[1] scratch-free:
      // convert elementwise with a padded round trip via H[1] as float and a join of (H[1], 0)
      ALW_LAUNCH(launch_unpack(dense, 1, s->H[1], 1, s->nx, s->ny, s->pitch, s->dim, s->stream));
      ALW_CUDA(cudaMemsetAsync(s->Lo[1], 0, s->arr_bytes, s->stream));
      ALW_LAUNCH(launch_mixed_join(s->H[1], s->Lo[1], nullptr, (double *)tmp, s->nx, s->ny, s->pitch, s->dim, s->stream));
      src = (const double *)tmp;
    }
    ALW_LAUNCH(launch_mixed_split(src, s->H[0], s->Lo[0], s->nx, s->ny, s->pitch, s->dim, s->stream));
    if (tmp) dev_free_impl(tmp, (size_t)s->nx * s->ny * sizeof(double), s->stream);
  } else {
    ALW_LAUNCH(launch_unpack(dense, dtype, s->P, s->prec == P_F64 ? 0 : 1, s->nx, s->ny, s->pitch, s->dim, s->stream));
  }
  return ALW_OK;
}

// Reset the device state to (t, steps, lagged alpha) with cur = 0, fill the
// ghost frame of phi^n, and wait for the stream (the pinned mirror is reused).
alw_status reset_state(alw_solver *s, double t, int64_t steps, const double *alpha) {
  ALW_CUDA(cudaStreamSynchronize(s->stream));
  memset(s->h_st, 0, sizeof(DevState));
  s->h_st->t = t;
  s->h_st->t_final = t;
  s->h_st->steps = steps;
  if (alpha) {
    memcpy(&s->h_st->alpha_bits[2][0], &alpha[0], sizeof(double));
    memcpy(&s->h_st->alpha_bits[2][1], &alpha[1], sizeof(double));
  }
  ALW_CUDA(cudaMemcpyAsync(s->st, s->h_st, sizeof(DevState), cudaMemcpyHostToDevice, s->stream));
  GhostParams g = ghost_params(s, 3);
  ALW_LAUNCH(launch_ghosts(g, s->stream));
  ALW_CUDA(cudaStreamSynchronize(s->stream));
  return ALW_OK;
}

// Reduction pass over phi^n into the lagged slot 2 (the first lagged alpha).
alw_status prime_alpha(alw_solver *s) {
  StageParams p = make_params(s, 0, 1, LOOP_ADVANCE);
  p.write_slot = 2;
  ALW_LAUNCH(launch_stage(s, p));
  return ALW_OK;
}


// 2D float tensor map over a padded array: box = one tile plus halo.
alw_status make_tensor_map(alw_solver *s, CUtensorMap *m, void *base) {
  const int r = encode_tile_map(m, base, s->pitch, s->rows);
  if (r == -1) return fail(ALW_ECUDA, "cuTensorMapEncodeTiled is not available");
  if (r != 0) return fail(ALW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", r);
  return ALW_OK;
}

alw_status check_solver(alw_solver *s) {
  if (!s) return fail(ALW_EINVAL, "solver is NULL");
  if (!s->has_phi) return fail(ALW_EINVAL, "phi0 not set");
  return ALW_OK;
}

}  // namespace

extern "C" {

const char *alw_version(void) { return "alweno 0.1 (sm_103a)"; }

const char *alw_last_error(void) { return g_err.c_str(); }

alw_status alw_set_allocator(const alw_allocator *a) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if (a && (!a->alloc || !a->free)) return fail(ALW_EINVAL, "allocator needs both alloc and free");
  if (a) g_alloc = *a;
  else g_alloc = alw_allocator{nullptr, nullptr, nullptr};
  return ALW_OK;
}

alw_status alw_create(const alw_grid *grid, const alw_hamiltonian *ham, const alw_scheme *scheme, void *cuda_stream,
                      alw_solver **out) {
  if (!grid || !ham || !scheme || !out) return fail(ALW_EINVAL, "NULL argument");
  *out = nullptr;
  if (grid->dim != 1 && grid->dim != 2) return fail(ALW_EINVAL, "dim must be 1 or 2");
  if (grid->nx < 1 || grid->ny < 1) return fail(ALW_EINVAL, "nx, ny must be >= 1");
  if (grid->dim == 1 && grid->ny != 1) return fail(ALW_EINVAL, "1D grids have ny = 1");
  if (grid->bc != ALW_BC_PERIODIC && grid->bc != ALW_BC_LINEXTRAP) return fail(ALW_EINVAL, "unknown bc %d", grid->bc);
  if (grid->bc == ALW_BC_LINEXTRAP && (grid->nx < 2 || (grid->dim == 2 && grid->ny < 2)))
    return fail(ALW_EINVAL, "linear extrapolation needs at least 2 nodes per direction");
  if ((long long)grid->nx * grid->ny > (1ll << 31)) return fail(ALW_EINVAL, "grid too large");
  if (ham->kind < ALW_H_BURGERS2D || ham->kind > ALW_H_OPTCTRL2D) return fail(ALW_EINVAL, "unknown Hamiltonian %d", ham->kind);
  if (is_1d_ham(ham->kind) != (grid->dim == 1)) return fail(ALW_EINVAL, "Hamiltonian does not match the dimension");
  if (scheme->weights != ALW_W_ARCLEN && scheme->weights != ALW_W_JP) return fail(ALW_EINVAL, "unknown weights");
  if (!(scheme->eps > 0.0) || !(scheme->cfl > 0.0)) return fail(ALW_EINVAL, "eps and cfl must be > 0");
  if (scheme->dt_mode != ALW_DT_CFL && scheme->dt_mode != ALW_DT_DX53) return fail(ALW_EINVAL, "unknown dt_mode");
  if (scheme->alpha_mode < ALW_ALPHA_DEFAULT || scheme->alpha_mode > ALW_ALPHA_FIXED)
    return fail(ALW_EINVAL, "unknown alpha_mode");
  if (scheme->precision < ALW_PREC_FP64 || scheme->precision > ALW_PREC_MIXED) return fail(ALW_EINVAL, "unknown precision");
  if (!(grid->xhi > grid->xlo) || (grid->dim == 2 && !(grid->yhi > grid->ylo))) return fail(ALW_EINVAL, "empty extent");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(ALW_ECUDA, "no CUDA device");
  }
  alw_solver *s = new (std::nothrow) alw_solver();
  if (!s) return fail(ALW_ENOMEM, "host allocation failed");
  cudaGetDevice(&s->device);
  s->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (!s->stream) {
    // the legacy default stream cannot be captured into a graph: use an own
    // stream that still orders itself after work on the legacy stream
    if (cudaStreamCreate(&s->stream) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return fail(ALW_ECUDA, "stream creation failed");
    }
    s->own_stream = true;
  }
  s->grid = *grid;
  s->ham = *ham;
  s->scheme = *scheme;
  s->dim = grid->dim;
  s->nx = grid->nx;
  s->ny = grid->dim == 2 ? grid->ny : 1;
  s->prec = kernel_prec(scheme->precision);
  s->alpha_mode = scheme->alpha_mode == ALW_ALPHA_DEFAULT
                      ? (grid->dim == 1 ? ALW_ALPHA_LOCAL_LAGGED : ALW_ALPHA_GLOBAL_LAGGED)
                      : scheme->alpha_mode;
  const bool per = grid->bc == ALW_BC_PERIODIC;
  s->dx = (grid->xhi - grid->xlo) / (per ? grid->nx : grid->nx - 1);
  s->dy = grid->dim == 2 ? (grid->yhi - grid->ylo) / (per ? grid->ny : grid->ny - 1) : s->dx;
  s->lx = scheme->dt_mode == ALW_DT_DX53 ? std::pow(s->dx, 5.0 / 3.0) : s->dx;
  s->ly = scheme->dt_mode == ALW_DT_DX53 ? std::pow(s->dy, 5.0 / 3.0) : s->dy;
  int tx = tile_x(s->prec, s->dim), ty = tile_y(s->prec, s->dim);
  if (s->dim == 2 && s->prec == P_F64) {
    // one FP64 tile keeps an SM busy for a long time: where the default tiles would not give every SM
    // two, 16 x 16 tiles spread the grid over four times as many CTAs
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long t = (long long)((s->nx + tx - 1) / tx) * ((s->ny + ty - 1) / ty);
    if (sms > 0 && t < 2LL * sms) {
      // fewer 16 x 16 tiles than SMs: 2-node segments, twice the threads per tile
      const long long t16 = (long long)((s->nx + 15) / 16) * ((s->ny + 15) / 16);
      s->small_tiles = t16 < sms ? 2 : 1;
      tx = ty = 16;
    }
  }
  s->tiles_x = (s->nx + tx - 1) / tx;
  s->tiles_y = (s->ny + ty - 1) / ty;
  s->pitch = s->tiles_x * tx + 2 * GX;
  s->rows = s->dim == 2 ? s->tiles_y * ty + 2 * GY : 1;
  s->elem = s->prec == P_F64 ? 8 : 4;
  s->use2d = s->dim == 2 && s->prec != P_F64;
  s->arr_bytes = (size_t)s->pitch * s->rows * s->elem;

  auto cleanup = [&](alw_status st) {
    alw_destroy(s);
    return st;
  };
  if (cudaHostAlloc((void **)&s->h_st, sizeof(DevState), cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void **)&s->h_tf, 2 * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(ALW_ENOMEM, "pinned host allocation failed"));
  }
  s->st = (DevState *)s->alloc(sizeof(DevState));
  if (!s->st) return cleanup(fail(ALW_ENOMEM, "device allocation failed"));
  std::vector<void **> bufs;
  if (s->prec == P_MIXED) bufs = {&s->H[0], &s->H[1], &s->Lo[0], &s->Lo[1], &s->D1, &s->D2};
  else bufs = {&s->P, &s->A, &s->B};
  for (void **b : bufs) {
    *b = s->alloc(s->arr_bytes);
    if (!*b) return cleanup(fail(ALW_ENOMEM, "device allocation of %zu bytes failed", s->arr_bytes));
    if (cudaMemsetAsync(*b, 0, s->arr_bytes, s->stream) != cudaSuccess)
      return cleanup(fail(ALW_ECUDA, "memset failed"));
  }
  if (cudaMemsetAsync(s->st, 0, sizeof(DevState), s->stream) != cudaSuccess) return cleanup(fail(ALW_ECUDA, "memset failed"));
  if (s->use2d) {
    memset(s->maps, 0, sizeof s->maps);
    void *bases[6];
    int nb;
    if (s->prec == P_MIXED) {
      void *b[6] = {s->H[0], s->H[1], s->Lo[0], s->Lo[1], s->D1, s->D2};
      memcpy(bases, b, sizeof b);
      nb = 6;
    } else {
      void *b[3] = {s->P, s->A, s->B};
      memcpy(bases, b, sizeof b);
      nb = 3;
    }
    for (int i = 0; i < nb; ++i) {
      alw_status st = make_tensor_map(s, &s->maps[i], bases[i]);
      if (st) return cleanup(st);
    }
  }
  *out = s;
  return ALW_OK;
}

alw_status alw_destroy(alw_solver *s) {
  if (!s) return ALW_OK;
  cudaStreamSynchronize(s->stream);
  if (s->g_step) cudaGraphExecDestroy(s->g_step);
  if (s->g_adv) cudaGraphExecDestroy(s->g_adv);
  for (auto &a : s->allocs) dev_free_impl(a.first, a.second, s->stream);
  cudaStreamSynchronize(s->stream);
  if (s->h_st) cudaFreeHost(s->h_st);
  if (s->h_tf) cudaFreeHost(s->h_tf);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  cudaGetLastError();
  delete s;
  return ALW_OK;
}

alw_status alw_memory_bytes(alw_solver *s, size_t *bytes) {
  if (!s || !bytes) return fail(ALW_EINVAL, "NULL argument");
  size_t b = 0;
  for (auto &a : s->allocs) b += a.second;
  *bytes = b;
  return ALW_OK;
}

alw_status alw_set_phi0_device(alw_solver *s, const void *dev_phi, int32_t dtype, size_t n) {
  if (!s || !dev_phi) return fail(ALW_EINVAL, "NULL argument");
  if (n != (size_t)s->nx * s->ny) return fail(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)s->nx * s->ny);
  if (dtype != 0 && dtype != 1) return fail(ALW_EINVAL, "dtype must be 0 (double) or 1 (float)");
  alw_status st = load_phi_dense(s, dev_phi, dtype);
  if (st) return st;
  st = reset_state(s, 0.0, 0, nullptr);
  if (st) return st;
  st = prime_alpha(s);
  if (st) return st;
  ALW_CUDA(cudaStreamSynchronize(s->stream));
  s->has_phi = true;
  return ALW_OK;
}

alw_status alw_set_phi0(alw_solver *s, const double *host_phi, size_t n) {
  if (!s || !host_phi) return fail(ALW_EINVAL, "NULL argument");
  if (n != (size_t)s->nx * s->ny) return fail(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)s->nx * s->ny);
  void *tmp = dev_alloc_impl(n * sizeof(double), s->stream);
  if (!tmp) return fail(ALW_ENOMEM, "device allocation of %zu bytes failed", n * sizeof(double));
  cudaError_t e = cudaMemcpyAsync(tmp, host_phi, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  alw_status st = e == cudaSuccess ? alw_set_phi0_device(s, tmp, 0, n) : fail(ALW_ECUDA, "copy: %s", cudaGetErrorString(e));
  dev_free_impl(tmp, n * sizeof(double), s->stream);
  if (st == ALW_OK) ALW_CUDA(cudaStreamSynchronize(s->stream));
  return st;
}

// Host-side fault injection for the no-progress check of alw_step_to: with
// ALW_TEST_FREEZE_STATE_AFTER=n (n >= 1) in the environment, the check sees the device state as it
// was at its n-th read, as if the device had stopped advancing; the device work is unchanged.
static int test_freeze_after() {
  const char *e = std::getenv("ALW_TEST_FREEZE_STATE_AFTER");
  return e ? std::atoi(e) : 0;
}

alw_status alw_step_to(alw_solver *s, double t_final, int64_t *steps_out) {
  alw_status st = check_solver(s);
  if (st) return st;
  if (!std::isfinite(t_final)) return fail(ALW_EINVAL, "t_final must be finite");
  if (!s->g_step) {
    s->g_step_n = (s->nx * (long long)s->ny >= (1 << 22)) ? 4 : 16;
    st = build_graph(s, LOOP_STEP_TO, s->g_step_n, &s->g_step);
    if (st) return st;
  }
  st = read_state(s);
  if (st) return st;
  const int64_t steps0 = s->h_st->steps;
  if (s->h_st->err) return fail(ALW_ENONFINITE, "non-finite dH/dp detected");
  s->h_tf[0] = t_final;
  ALW_CUDA(cudaMemcpyAsync(&s->st->t_final, s->h_tf, sizeof(double), cudaMemcpyHostToDevice, s->stream));
  int replays = 1, stalls = 0;
  const int freeze = test_freeze_after();
  int reads = 0;
  DevState frozen;
  for (;;) {
    if (!(s->h_st->t < t_final)) break;
    const double t_prev = s->h_st->t;
    const int64_t steps_prev = s->h_st->steps;
    for (int r = 0; r < replays; ++r) ALW_CUDA(cudaGraphLaunch(s->g_step, s->stream));
    st = read_state(s);
    if (st) return st;
    if (freeze > 0 && ++reads >= freeze) {
      if (reads == freeze) frozen = *s->h_st;
      else *s->h_st = frozen;
    }
    // the device must make progress on every replay batch; never loop on a stuck state
    if (!s->h_st->err && s->h_st->steps == steps_prev && s->h_st->t == t_prev) {
      if (++stalls >= 3) return fail(ALW_ETIMEOUT, "no progress at t = %.17g", s->h_st->t);
    } else {
      stalls = 0;
    }
    if (s->h_st->err) {
      if (steps_out) *steps_out = s->h_st->steps - steps0;
      return fail(ALW_ENONFINITE, "non-finite dH/dp detected at t = %.17g", s->h_st->t);
    }
    if (s->h_st->steps - steps0 > 2000000000ll) return fail(ALW_ETIMEOUT, "step limit reached");
    const double rem = t_final - s->h_st->t;
    double est = s->h_st->dt > 0 ? rem / s->h_st->dt : 1.0;
    if (!(est < 1e9)) est = 1e9;
    int r = (int)std::ceil(est / s->g_step_n);
    replays = r < 1 ? 1 : (r > 64 ? 64 : r);
  }
  if (steps_out) *steps_out = s->h_st->steps - steps0;
  return ALW_OK;
}

alw_status alw_advance(alw_solver *s, int64_t nsteps) {
  alw_status st = check_solver(s);
  if (st) return st;
  if (nsteps < 0) return fail(ALW_EINVAL, "nsteps < 0");
  if (!s->g_adv) {
    st = build_graph(s, LOOP_ADVANCE, 1, &s->g_adv);
    if (st) return st;
  }
  for (int64_t i = 0; i < nsteps; ++i) ALW_CUDA(cudaGraphLaunch(s->g_adv, s->stream));
  return ALW_OK;
}

alw_status alw_run_stage(alw_solver *s, int32_t stage, double dt) {
  alw_status st = check_solver(s);
  if (st) return st;
  if (stage < 1 || stage > 3) return fail(ALW_EINVAL, "stage must be 1, 2 or 3");
  if (!std::isfinite(dt)) return fail(ALW_EINVAL, "dt must be finite");
  const bool pre = (s->alpha_mode == ALW_ALPHA_GLOBAL_EXACT) || (s->alpha_mode == ALW_ALPHA_LOCAL_EXACT && stage == 1);
  if (pre) {
    ALW_CUDA(cudaMemsetAsync(&s->st->alpha_bits[3][0], 0, 2 * sizeof(unsigned long long), s->stream));
    ALW_LAUNCH(launch_stage(s, make_params(s, 0, stage, LOOP_STAGE)));
  }
  StageParams p = make_params(s, stage, stage, LOOP_STAGE);
  p.dt_value = dt;
  ALW_LAUNCH(launch_stage(s, p));
  if (s->grid.bc == ALW_BC_LINEXTRAP) ALW_LAUNCH(launch_ghosts(ghost_params(s, stage), s->stream));
  return ALW_OK;
}

alw_status alw_sync(alw_solver *s) {
  if (!s) return fail(ALW_EINVAL, "solver is NULL");
  alw_status st = read_state(s);
  if (st) return st;
  if (s->h_st->err) return fail(ALW_ENONFINITE, "non-finite dH/dp detected");
  return ALW_OK;
}

static alw_status gather_dense(alw_solver *s, int which, void *dst, int dtype) {
  // which: 0 = phi^n, 1/2 = stage state
  alw_status st = read_state(s);
  if (st) return st;
  const int cur = s->h_st->cur;
  const size_t n = (size_t)s->nx * s->ny;
  if (s->prec == P_MIXED) {
    const void *delta = which == 1 ? s->D1 : (which == 2 ? s->D2 : nullptr);
    if (dtype == 0) {
      ALW_LAUNCH(launch_mixed_join(s->H[cur], s->Lo[cur], delta, (double *)dst, s->nx, s->ny, s->pitch, s->dim, s->stream));
    } else {
      void *tmp = dev_alloc_impl(n * sizeof(double), s->stream);
      if (!tmp) return fail(ALW_ENOMEM, "device allocation failed");
      ALW_LAUNCH(launch_mixed_join(s->H[cur], s->Lo[cur], delta, (double *)tmp, s->nx, s->ny, s->pitch, s->dim, s->stream));
      // narrow doubles to floats via the padded float array H[cur^1] used as a scratch-free converter is unsafe;
      // convert directly with the unpack/pack pair on a temporary padded buffer
      void *pad = dev_alloc_impl(s->arr_bytes, s->stream);
      if (!pad) return fail(ALW_ENOMEM, "device allocation failed");
      ALW_LAUNCH(launch_unpack(tmp, 0, pad, 1, s->nx, s->ny, s->pitch, s->dim, s->stream));
      ALW_LAUNCH(launch_pack(pad, 1, dst, 1, s->nx, s->ny, s->pitch, s->dim, s->stream));
      dev_free_impl(pad, s->arr_bytes, s->stream);
      dev_free_impl(tmp, n * sizeof(double), s->stream);
    }
  } else {
    const void *src = which == 1 ? s->A : (which == 2 ? s->B : s->P);
    ALW_LAUNCH(launch_pack(src, s->prec == P_F64 ? 0 : 1, dst, dtype, s->nx, s->ny, s->pitch, s->dim, s->stream));
  }
  return ALW_OK;
}

alw_status alw_get_phi_device(alw_solver *s, void *dev_out, int32_t dtype, size_t n) {
  alw_status st = check_solver(s);
  if (st) return st;
  if (!dev_out) return fail(ALW_EINVAL, "NULL output");
  if (n != (size_t)s->nx * s->ny) return fail(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)s->nx * s->ny);
  if (dtype != 0 && dtype != 1) return fail(ALW_EINVAL, "dtype must be 0 or 1");
  return gather_dense(s, 0, dev_out, dtype);
}

static alw_status get_host(alw_solver *s, int which, double *host_out, size_t n) {
  alw_status st = check_solver(s);
  if (st) return st;
  if (!host_out) return fail(ALW_EINVAL, "NULL output");
  if (n != (size_t)s->nx * s->ny) return fail(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)s->nx * s->ny);
  void *tmp = dev_alloc_impl(n * sizeof(double), s->stream);
  if (!tmp) return fail(ALW_ENOMEM, "device allocation failed");
  st = gather_dense(s, which, tmp, 0);
  if (st == ALW_OK) {
    cudaError_t e = cudaMemcpyAsync(host_out, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) st = fail(ALW_ECUDA, "copy: %s", cudaGetErrorString(e));
  }
  dev_free_impl(tmp, n * sizeof(double), s->stream);
  ALW_CUDA(cudaStreamSynchronize(s->stream));
  return st;
}

alw_status alw_get_phi(alw_solver *s, double *host_out, size_t n) { return get_host(s, 0, host_out, n); }

alw_status alw_get_stage_phi(alw_solver *s, int32_t stage, double *host_out, size_t n) {
  if (stage != 1 && stage != 2) return fail(ALW_EINVAL, "stage must be 1 or 2");
  return get_host(s, stage, host_out, n);
}

alw_status alw_get_state(alw_solver *s, alw_state *state) {
  alw_status st = check_solver(s);
  if (st) return st;
  if (!state) return fail(ALW_EINVAL, "NULL output");
  st = read_state(s);
  if (st) return st;
  state->t = s->h_st->t;
  state->steps = s->h_st->steps;
  double a[2];
  memcpy(&a[0], &s->h_st->alpha_bits[2][0], sizeof(double));
  memcpy(&a[1], &s->h_st->alpha_bits[2][1], sizeof(double));
  state->alpha[0] = a[0];
  state->alpha[1] = a[1];
  return ALW_OK;
}

alw_status alw_set_state(alw_solver *s, const alw_state *state, const double *host_phi, size_t n) {
  if (!s || !state || !host_phi) return fail(ALW_EINVAL, "NULL argument");
  if (n != (size_t)s->nx * s->ny) return fail(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)s->nx * s->ny);
  void *tmp = dev_alloc_impl(n * sizeof(double), s->stream);
  if (!tmp) return fail(ALW_ENOMEM, "device allocation failed");
  ALW_CUDA(cudaMemcpyAsync(tmp, host_phi, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  alw_status st = load_phi_dense(s, tmp, 0);
  dev_free_impl(tmp, n * sizeof(double), s->stream);
  if (st) return st;
  st = reset_state(s, state->t, state->steps, state->alpha);
  if (st) return st;
  s->has_phi = true;
  return ALW_OK;
}

}  // extern "C"
