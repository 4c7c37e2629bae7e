// Launcher of the persistent 2D float stage kernel (included once per precision TU).
#pragma once
#include <cuda_runtime.h>

#include "alw_stage2d.cuh"

namespace alw {

template <int PREC, int W, int H>
static int launch2d_one(const Stage2DParams &prm, cudaStream_t stream) {
  constexpr int NARR = (PREC == P_MIXED) ? 3 : 2;
  auto kern = stage2d_kernel<PREC, W, H>;
  const size_t smem = Geo2D::smem_bytes<NARR>();
  static int grid_cap = 0;  // CTAs that fit on the device at once (per instantiation)
  if (grid_cap == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Geo2D::NT, smem);
    if (e != cudaSuccess) return (int)e;
    grid_cap = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int tiles = prm.p.tiles_x * prm.p.tiles_y;
  const int grid = tiles < grid_cap ? tiles : grid_cap;
  kern<<<grid, Geo2D::NT, smem, stream>>>(prm);
  return (int)cudaGetLastError();
}

template <int PREC, int W>
static int launch2d_h(const Stage2DParams &prm, cudaStream_t s) {
  switch (prm.p.ham) {
    case H_BURGERS2D: return launch2d_one<PREC, W, H_BURGERS2D>(prm, s);
    case H_NEGCOS2D: return launch2d_one<PREC, W, H_NEGCOS2D>(prm, s);
    case H_SIN2D: return launch2d_one<PREC, W, H_SIN2D>(prm, s);
    case H_EIKONAL2D: return launch2d_one<PREC, W, H_EIKONAL2D>(prm, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <int PREC>
static int launch2d_impl(const Stage2DParams &prm, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  return prm.p.weights == W_JP ? launch2d_h<PREC, W_JP>(prm, s) : launch2d_h<PREC, W_ARCLEN>(prm, s);
}

}  // namespace alw
