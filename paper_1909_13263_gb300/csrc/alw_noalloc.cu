// alw_step_noalloc: RK3 steps of the FP64 stage kernel without any device
// allocation.
//
// Who needs this: callers that cannot obtain device memory on demand -- for
// example a host framework whose pool allocator owns all device memory and
// forbids outside cudaMalloc, or a real-time loop that must not allocate after
// start-up because an allocation may synchronise the device or fail at an
// unpredictable moment.  They pass their own input and output arrays; the
// working storage the stage kernel needs (three padded ghosted copies of phi
// and the device-side time/alpha state) lives in one file-scope __device__
// array of fixed size that every GPU loading this library holds until the
// process exits.
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture.  CUDA loads a library's device code
// lazily by default, so that first call is also when the device code is loaded
// on the device and the array's memory is reserved there: a caller whose pool
// will own all device memory, or whose real-time phase must not reserve any,
// makes the first call before that and checks its status.  All calls on a device share the same
// array and it keeps the previous call's contents, so every call clears the
// part it uses; calls whose GPU work overlaps (different streams, or host
// threads without ordering between them) race on the array and must not be
// issued concurrently.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/alweno.h"
#include "alw_internal.h"

namespace {

using namespace alw;

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

bool is_1d(int k) { return k == ALW_H_ADVECT1D || k == ALW_H_BURGERS1D || k == ALW_H_NEGCOS1D ||
                                      k == ALW_H_NONCONVEX1D; }

alw_status err(alw_status st, const char *msg) {
  alw::set_last_error(msg);
  return st;
}

alw_status cuda_err(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return err(ALW_ECUDA, buf);
}

// Device address of the scratch array on the current device (looked up once).
alw_status scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return err(ALW_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return ALW_OK;
}

}  // namespace

extern "C" alw_status alw_step_noalloc(const alw_grid *grid, const alw_hamiltonian *ham, const alw_scheme *scheme,
                                       const double *dev_phi_in, double *dev_phi_out, double dt, int32_t nsteps,
                                       void *cuda_stream) {
  if (!grid || !ham || !scheme || !dev_phi_in || !dev_phi_out) return err(ALW_EINVAL, "NULL argument");
  if (scheme->precision != ALW_PREC_FP64) return err(ALW_EINVAL, "the no-allocation path runs the FP64 kernel only");
  if (grid->dim != 1 && grid->dim != 2) return err(ALW_EINVAL, "dim must be 1 or 2");
  if (grid->nx < 1 || grid->ny < 1 || (grid->dim == 1 && grid->ny != 1)) return err(ALW_EINVAL, "bad nx/ny");
  if (grid->bc != ALW_BC_PERIODIC && grid->bc != ALW_BC_LINEXTRAP) return err(ALW_EINVAL, "unknown bc");
  if (grid->bc == ALW_BC_LINEXTRAP && (grid->nx < 2 || (grid->dim == 2 && grid->ny < 2)))
    return err(ALW_EINVAL, "linear extrapolation needs at least 2 nodes per direction");
  if (ham->kind < ALW_H_BURGERS2D || ham->kind > ALW_H_OPTCTRL2D || is_1d(ham->kind) != (grid->dim == 1))
    return err(ALW_EINVAL, "Hamiltonian does not match the dimension");
  if (scheme->weights != ALW_W_ARCLEN && scheme->weights != ALW_W_JP) return err(ALW_EINVAL, "unknown weights");
  if (scheme->alpha_mode < ALW_ALPHA_DEFAULT || scheme->alpha_mode > ALW_ALPHA_FIXED)
    return err(ALW_EINVAL, "unknown alpha_mode");
  if (!(scheme->eps > 0.0) || !std::isfinite(dt) || dt < 0.0 || nsteps < 0) return err(ALW_EINVAL, "bad eps, dt or nsteps");
  if (!(grid->xhi > grid->xlo) || (grid->dim == 2 && !(grid->yhi > grid->ylo))) return err(ALW_EINVAL, "empty extent");

  // layout of the scratch: state, then phi^n, stage 1 and stage 2 in the padded ghosted layout;
  // sizes in 64 bits until the budget check has bounded them (nx, ny up to INT_MAX)
  const int dim = grid->dim, nx = grid->nx, ny = grid->dim == 2 ? grid->ny : 1;
  const int tx = tile_x(P_F64, dim), ty = tile_y(P_F64, dim);
  const size_t tiles_x_z = ((size_t)nx + tx - 1) / tx, tiles_y_z = ((size_t)ny + ty - 1) / ty;
  const size_t pitch_z = tiles_x_z * tx + 2 * GX;
  const size_t rows_z = dim == 2 ? tiles_y_z * ty + 2 * GY : 1;
  const size_t state_bytes = align256(sizeof(DevState));
  // the product pitch_z * rows_z is formed only after both factors are bounded, so it cannot wrap
  const bool too_big = pitch_z > kScratchBytes / sizeof(double) || rows_z > kScratchBytes / sizeof(double) ||
                       pitch_z * rows_z > kScratchBytes / sizeof(double);
  const size_t arr = too_big ? kScratchBytes : align256(pitch_z * rows_z * sizeof(double));
  const size_t need = state_bytes + 3 * arr;
  if (too_big || need > kScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof buf, "grid %d x %d needs more than the %zu bytes of working storage of the "
             "no-allocation path", nx, ny, kScratchBytes);
    return err(ALW_EBUDGET, buf);
  }
  const int tiles_x = (int)tiles_x_z, tiles_y = (int)tiles_y_z, pitch = (int)pitch_z;
  void *base = nullptr;
  alw_status st = scratch_address(&base);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char *b = static_cast<unsigned char *>(base);
  DevState *ds = reinterpret_cast<DevState *>(b);
  void *P = b + state_bytes, *A = b + state_bytes + arr, *B = b + state_bytes + 2 * arr;

  cudaError_t e = cudaMemsetAsync(base, 0, need, s);  // the previous call's contents must not leak in
  if (e != cudaSuccess) return cuda_err(e, "clearing the scratch");
  int le = launch_unpack(dev_phi_in, 0, P, 0, nx, ny, pitch, dim, s);
  if (le) return cuda_err((cudaError_t)le, "loading phi");

  GhostParams g;
  memset(&g, 0, sizeof g);
  g.nx = nx; g.ny = ny; g.pitch = pitch; g.dim = dim; g.bc = grid->bc; g.prec = P_F64;
  g.a0 = P;
  le = launch_ghosts(g, s);
  if (le) return cuda_err((cudaError_t)le, "ghost frame");

  const bool per = grid->bc == ALW_BC_PERIODIC;
  const double dx = (grid->xhi - grid->xlo) / (per ? nx : nx - 1);
  const double dy = dim == 2 ? (grid->yhi - grid->ylo) / (per ? ny : ny - 1) : dx;
  const int amode = scheme->alpha_mode == ALW_ALPHA_DEFAULT
                        ? (dim == 1 ? ALW_ALPHA_LOCAL_LAGGED : ALW_ALPHA_GLOBAL_LAGGED)
                        : scheme->alpha_mode;
  auto params = [&](int stage, int src_of) {
    StageParams p;
    memset(&p, 0, sizeof p);
    p.nx = nx; p.ny = ny; p.pitch = pitch; p.tiles_x = tiles_x; p.tiles_y = tiles_y;
    p.dim = dim; p.bc = grid->bc; p.ham = ham->kind; p.weights = scheme->weights;
    p.alpha_mode = amode; p.loop_mode = LOOP_STAGE; p.stage = stage;
    p.src_of = stage == 0 ? src_of : stage;
    p.dx = dx; p.dy = dy; p.rdx = 1.0 / dx; p.rdy = 1.0 / dy; p.eps = scheme->eps;
    p.xlo = grid->xlo; p.ylo = grid->dim == 2 ? grid->ylo : 0.0;
    p.cfl = scheme->cfl; p.lx = dx; p.ly = dy;
    p.alpha_fixed[0] = scheme->alpha_fixed[0]; p.alpha_fixed[1] = scheme->alpha_fixed[1];
    p.dt_value = dt; p.state = ds; p.dt_slot = 2;
    if (stage == 0) {
      p.read_slot = -1; p.write_slot = 3; p.zero_slot = -1;
    } else {
      p.read_slot = amode == ALW_ALPHA_GLOBAL_EXACT ? 3 : (stage == 1 ? 2 : stage - 2);
      p.write_slot = stage - 1;
      p.zero_slot = stage % 3;
    }
    const int which = p.src_of;
    p.src0 = which == 1 ? P : (which == 2 ? A : B);
    p.base0 = P;
    p.out0 = stage == 1 ? A : (stage == 2 ? B : (stage == 3 ? P : nullptr));
    return p;
  };
  // first lagged alpha: reduction over phi^n into slot 2
  StageParams prime = params(0, 1);
  prime.write_slot = 2;
  le = launch_stage_f64(prime, s);
  if (le) return cuda_err((cudaError_t)le, "alpha pass");
  for (int n = 0; n < nsteps; ++n) {
    for (int stage = 1; stage <= 3; ++stage) {
      const bool pre = amode == ALW_ALPHA_GLOBAL_EXACT || (amode == ALW_ALPHA_LOCAL_EXACT && stage == 1);
      if (pre) {
        e = cudaMemsetAsync(&ds->alpha_bits[3][0], 0, 2 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_err(e, "clearing the exact alpha slot");
        le = launch_stage_f64(params(0, stage), s);
        if (le) return cuda_err((cudaError_t)le, "alpha pass");
      }
      le = launch_stage_f64(params(stage, stage), s);
      if (le) return cuda_err((cudaError_t)le, "stage kernel");
      if (!per) {
        g.a0 = stage == 1 ? A : (stage == 2 ? B : P);
        le = launch_ghosts(g, s);
        if (le) return cuda_err((cudaError_t)le, "ghost frame");
      }
    }
  }
  le = launch_pack(P, 0, dev_phi_out, 0, nx, ny, pitch, dim, s);
  if (le) return cuda_err((cudaError_t)le, "storing phi");
  int flag = 0;
  e = cudaMemcpyAsync(&flag, &ds->err, sizeof flag, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "synchronising");
  if (flag) return err(ALW_ENONFINITE, "non-finite dH/dp detected");
  return ALW_OK;
}
