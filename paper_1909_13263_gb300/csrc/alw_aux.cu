// Auxiliary kernels: ghost frames, layout conversion between dense row-major
// arrays and the padded ghosted layout, and the double <-> (hi, lo) split.
#include <cuda_runtime.h>

#include "alw_internal.h"

namespace alw {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ size_t pidx(int i, int j, int pitch, int dim) {
  return (size_t)(j + (dim == 2 ? GY : 0)) * pitch + (i + GX);
}

// ghost value of a line at position g (g in [-3,-1] or [n, n+2]) from interior values
template <typename T, typename Get>
__device__ __forceinline__ T ghost_value(int g, int n, int bc, Get get) {
  if (bc == 0) {  // periodic
    int w = g % n;
    if (w < 0) w += n;
    return get(w);
  }
  if (g < 0) {
    const T m = T(-g);
    return (T(1) + m) * get(0) - m * get(1);
  }
  const T m = T(g - (n - 1));
  return (T(1) + m) * get(n - 1) - m * get(n - 2);
}

// One thread per (line, ghost position): rows first (x ghosts), then columns.
template <typename S>
__global__ void ghosts_plain(S *a, int nx, int ny, int pitch, int dim, int bc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = ny * 6, ncol = (dim == 2) ? nx * 6 : 0;
  if (t < nrow) {
    const int j = t / 6, k = t % 6;
    const int g = (k < 3) ? -(k + 1) : nx + (k - 3);
    auto get = [&](int i) { return a[pidx(i, j, pitch, dim)]; };
    a[pidx(g, j, pitch, dim)] = ghost_value<S>(g, nx, bc, get);
  } else if (t < nrow + ncol) {
    const int u = t - nrow;
    const int i = u / 6, k = u % 6;
    const int g = (k < 3) ? -(k + 1) : ny + (k - 3);
    auto get = [&](int j) { return a[pidx(i, j, pitch, dim)]; };
    a[pidx(i, g, pitch, dim)] = ghost_value<S>(g, ny, bc, get);
  }
}

// (hi, lo) pair: ghosts computed in double, split back into two floats.
__global__ void ghosts_pair(float *hi_, float *lo_, const DevState *st, float *const *hh, float *const *ll, int nx,
                            int ny, int pitch, int dim, int bc, float *hi0, float *lo0, float *hi1, float *lo1) {
  float *hi = hi_, *lo = lo_;
  if (st) {
    hi = st->cur ? hi1 : hi0;
    lo = st->cur ? lo1 : lo0;
  }
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = ny * 6, ncol = (dim == 2) ? nx * 6 : 0;
  int i, j, g;
  bool along_x;
  if (t < nrow) {
    j = t / 6;
    const int k = t % 6;
    g = (k < 3) ? -(k + 1) : nx + (k - 3);
    along_x = true;
    i = 0;
  } else if (t < nrow + ncol) {
    const int u = t - nrow;
    i = u / 6;
    const int k = u % 6;
    g = (k < 3) ? -(k + 1) : ny + (k - 3);
    along_x = false;
    j = 0;
  } else {
    return;
  }
  double v;
  if (along_x) {
    auto get = [&](int ii) { const size_t q = pidx(ii, j, pitch, dim); return (double)hi[q] + (double)lo[q]; };
    v = ghost_value<double>(g, nx, bc, get);
  } else {
    auto get = [&](int jj) { const size_t q = pidx(i, jj, pitch, dim); return (double)hi[q] + (double)lo[q]; };
    v = ghost_value<double>(g, ny, bc, get);
  }
  const float h = (float)v;
  const float l = (float)(v - (double)h);
  const size_t q = along_x ? pidx(g, j, pitch, dim) : pidx(i, g, pitch, dim);
  hi[q] = h;
  lo[q] = l;
}

// MIXED increment array e of a stage state phi_k = hi + e (hi = the high part of phi^n, whose ghost frame is
// already in place): the ghost of phi_k is formed in double from the interior values of hi + e and stored as
// e_ghost = ghost - hi_ghost, so that hi + e holds the extrapolated phi_k at every ghost cell (extrapolating
// e alone would leave the difference between hi's own extrapolation and hi's ghost, which carries the split
// of phi^n's ghost into hi and lo, in the ghost values).
__global__ void ghosts_incr(float *e, const DevState *st, const float *hi0, const float *hi1, int nx, int ny,
                            int pitch, int dim, int bc) {
  const float *hi = st->cur ? hi1 : hi0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nrow = ny * 6, ncol = (dim == 2) ? nx * 6 : 0;
  double v;
  size_t q;
  if (t < nrow) {
    const int j = t / 6, k = t % 6;
    const int g = (k < 3) ? -(k + 1) : nx + (k - 3);
    auto get = [&](int ii) { const size_t r = pidx(ii, j, pitch, dim); return (double)hi[r] + (double)e[r]; };
    v = ghost_value<double>(g, nx, bc, get);
    q = pidx(g, j, pitch, dim);
  } else if (t < nrow + ncol) {
    const int u = t - nrow;
    const int i = u / 6, k = u % 6;
    const int g = (k < 3) ? -(k + 1) : ny + (k - 3);
    auto get = [&](int jj) { const size_t r = pidx(i, jj, pitch, dim); return (double)hi[r] + (double)e[r]; };
    v = ghost_value<double>(g, ny, bc, get);
    q = pidx(i, g, pitch, dim);
  } else {
    return;
  }
  e[q] = (float)(v - (double)hi[q]);
}

template <typename Src, typename Dst>
__global__ void pack_kernel(const Src *pad, Dst *dst, int nx, int ny, int pitch, int dim) {
  const size_t n = (size_t)nx * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(k / nx), i = (int)(k % nx);
    dst[k] = (Dst)pad[pidx(i, j, pitch, dim)];
  }
}

template <typename Src, typename Dst>
__global__ void unpack_kernel(const Src *src, Dst *pad, int nx, int ny, int pitch, int dim) {
  const size_t n = (size_t)nx * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(k / nx), i = (int)(k % nx);
    pad[pidx(i, j, pitch, dim)] = (Dst)src[k];
  }
}

__global__ void split_kernel(const double *src, float *hi, float *lo, int nx, int ny, int pitch, int dim) {
  const size_t n = (size_t)nx * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(k / nx), i = (int)(k % nx);
    const double v = src[k];
    const float h = (float)v;
    const size_t q = pidx(i, j, pitch, dim);
    hi[q] = h;
    lo[q] = (float)(v - (double)h);
  }
}

__global__ void join_kernel(const float *hi, const float *lo, const float *delta, double *dst, int nx, int ny,
                            int pitch, int dim) {
  const size_t n = (size_t)nx * ny;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(k / nx), i = (int)(k % nx);
    const size_t q = pidx(i, j, pitch, dim);
    // phi^n = hi + lo; a MIXED stage state is hi + its increment array (which holds the low part)
    dst[k] = (double)hi[q] + (double)(delta ? delta[q] : lo[q]);
  }
}

int grid_for(size_t n) {
  size_t b = (n + kBlock - 1) / kBlock;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

}  // namespace

int launch_ghosts(const GhostParams &g, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int tasks = g.ny * 6 + (g.dim == 2 ? g.nx * 6 : 0);
  const int blocks = (tasks + kBlock - 1) / kBlock;
  if (g.prec == P_MIXED && g.mixed_pair) {
    ghosts_pair<<<blocks, kBlock, 0, s>>>(reinterpret_cast<float *>(g.a0), reinterpret_cast<float *>(g.a1), g.state,
                                          nullptr, nullptr, g.nx, g.ny, g.pitch, g.dim, g.bc,
                                          reinterpret_cast<float *>(g.mix_hi[0]), reinterpret_cast<float *>(g.mix_lo[0]),
                                          reinterpret_cast<float *>(g.mix_hi[1]), reinterpret_cast<float *>(g.mix_lo[1]));
  } else if (g.prec == P_MIXED) {
    // an increment's ghosts are formed against the current high part, whose buffer the state names
    if (!g.state || !g.mix_hi[0] || !g.mix_hi[1]) return (int)cudaErrorInvalidValue;
    ghosts_incr<<<blocks, kBlock, 0, s>>>(reinterpret_cast<float *>(g.a0), g.state,
                                          reinterpret_cast<const float *>(g.mix_hi[0]),
                                          reinterpret_cast<const float *>(g.mix_hi[1]), g.nx, g.ny, g.pitch, g.dim,
                                          g.bc);
  } else if (g.prec == P_F64) {
    ghosts_plain<double><<<blocks, kBlock, 0, s>>>(reinterpret_cast<double *>(g.a0), g.nx, g.ny, g.pitch, g.dim, g.bc);
  } else {
    ghosts_plain<float><<<blocks, kBlock, 0, s>>>(reinterpret_cast<float *>(g.a0), g.nx, g.ny, g.pitch, g.dim, g.bc);
  }
  return (int)cudaGetLastError();
}

int launch_pack(const void *padded, int prec_elem, void *dst, int dst_dtype, int nx, int ny, int pitch, int dim,
                void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int b = grid_for((size_t)nx * ny);
  if (prec_elem == 0 && dst_dtype == 0)
    pack_kernel<double, double><<<b, kBlock, 0, s>>>((const double *)padded, (double *)dst, nx, ny, pitch, dim);
  else if (prec_elem == 0)
    pack_kernel<double, float><<<b, kBlock, 0, s>>>((const double *)padded, (float *)dst, nx, ny, pitch, dim);
  else if (dst_dtype == 0)
    pack_kernel<float, double><<<b, kBlock, 0, s>>>((const float *)padded, (double *)dst, nx, ny, pitch, dim);
  else
    pack_kernel<float, float><<<b, kBlock, 0, s>>>((const float *)padded, (float *)dst, nx, ny, pitch, dim);
  return (int)cudaGetLastError();
}

int launch_unpack(const void *src, int src_dtype, void *padded, int prec_elem, int nx, int ny, int pitch, int dim,
                  void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int b = grid_for((size_t)nx * ny);
  if (prec_elem == 0 && src_dtype == 0)
    unpack_kernel<double, double><<<b, kBlock, 0, s>>>((const double *)src, (double *)padded, nx, ny, pitch, dim);
  else if (prec_elem == 0)
    unpack_kernel<float, double><<<b, kBlock, 0, s>>>((const float *)src, (double *)padded, nx, ny, pitch, dim);
  else if (src_dtype == 0)
    unpack_kernel<double, float><<<b, kBlock, 0, s>>>((const double *)src, (float *)padded, nx, ny, pitch, dim);
  else
    unpack_kernel<float, float><<<b, kBlock, 0, s>>>((const float *)src, (float *)padded, nx, ny, pitch, dim);
  return (int)cudaGetLastError();
}

int launch_mixed_split(const double *src, void *hi, void *lo, int nx, int ny, int pitch, int dim, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  split_kernel<<<grid_for((size_t)nx * ny), kBlock, 0, s>>>(src, (float *)hi, (float *)lo, nx, ny, pitch, dim);
  return (int)cudaGetLastError();
}

int launch_mixed_join(const void *hi, const void *lo, const void *delta, double *dst, int nx, int ny, int pitch,
                      int dim, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  join_kernel<<<grid_for((size_t)nx * ny), kBlock, 0, s>>>((const float *)hi, (const float *)lo,
                                                           (const float *)delta, dst, nx, ny, pitch, dim);
  return (int)cudaGetLastError();
}

}  // namespace alw
