// Launcher of the persistent 2D float stage kernel (included once per precision TU).
#pragma once
#include <cuda_runtime.h>

#include "alw_stage2d.cuh"

namespace alw {

// CTAs of one kernel instantiation that fit on the device at once (cached per instantiation).
template <int PREC, int W, int H>
static int grid_cap_of() {
  constexpr int NARR = (PREC == P_MIXED) ? 3 : 2;
  static int cap = 0;
  if (cap == 0) {
    auto kern = stage2d_kernel<PREC, W, H>;
    const size_t smem = Geo2D::smem_bytes<NARR>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Geo2D::NT, smem) != cudaSuccess) return -1;
    cap = sms * (per_sm > 0 ? per_sm : 1);
  }
  return cap;
}

template <int PREC, int W, int H>
static int launch2d_one(const Stage2DParams &prm, cudaStream_t stream) {
  constexpr int NARR = (PREC == P_MIXED) ? 3 : 2;
  const int cap = grid_cap_of<PREC, W, H>();
  if (cap < 0) return (int)cudaGetLastError();
  const int grid = stage2d_grid(prm.ntiles, prm.grid_ctas, cap);
  if (grid <= 0) return 0;
  stage2d_kernel<PREC, W, H><<<grid, Geo2D::NT, Geo2D::smem_bytes<NARR>(), stream>>>(prm);
  return (int)cudaGetLastError();
}

template <int PREC, int W>
static int launch2d_h(const Stage2DParams &prm, cudaStream_t s) {
  // a single instance's Hamiltonian, or the one every entry of a batch group shares
  switch (prm.insts ? prm.batch_kind1 - 1 : prm.inst0.ham) {
    case H_BURGERS2D: return launch2d_one<PREC, W, H_BURGERS2D>(prm, s);
    case H_NEGCOS2D: return launch2d_one<PREC, W, H_NEGCOS2D>(prm, s);
    case H_SIN2D: return launch2d_one<PREC, W, H_SIN2D>(prm, s);
    case H_EIKONAL2D: return launch2d_one<PREC, W, H_EIKONAL2D>(prm, s);
    case H_OPTCTRL2D: return launch2d_one<PREC, W, H_OPTCTRL2D>(prm, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <int PREC>
static int launch2d_impl(const Stage2DParams &prm, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  return prm.p.weights == W_JP ? launch2d_h<PREC, W_JP>(prm, s) : launch2d_h<PREC, W_ARCLEN>(prm, s);
}

template <int PREC>
static int grid_cap_impl(int weights) {
  return weights == W_JP ? grid_cap_of<PREC, W_JP, H_BURGERS2D>() : grid_cap_of<PREC, W_ARCLEN, H_BURGERS2D>();
}

}  // namespace alw
