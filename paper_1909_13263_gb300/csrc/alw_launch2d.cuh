// Launcher of the persistent 2D float stage kernel (included once per precision TU).
#pragma once
#include <cuda_runtime.h>

#include "alw_stage2d.cuh"

namespace alw {

// CTAs of one kernel instantiation that fit on the device at once (cached per instantiation).
template <int PREC, int W, int H, int TX>
static int grid_cap_of() {
  constexpr int NARR = (PREC == P_MIXED) ? 3 : 2;
  using G = Geo2D<TX>;
  static int cap = 0;
  if (cap == 0) {
    auto kern = stage2d_kernel<PREC, W, H, TX>;
    const size_t smem = G::template smem_bytes<NARR>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, smem) != cudaSuccess) return -1;
    cap = sms * (per_sm > 0 ? per_sm : 1);
  }
  return cap;
}

template <int PREC, int W, int H, int TX>
static int launch2d_one(const Stage2DParams &prm, cudaStream_t stream) {
  constexpr int NARR = (PREC == P_MIXED) ? 3 : 2;
  using G = Geo2D<TX>;
  const int cap = grid_cap_of<PREC, W, H, TX>();
  if (cap < 0) return (int)cudaGetLastError();
  const int grid = stage2d_grid(prm.ntiles, prm.grid_ctas, cap);
  if (grid <= 0) return 0;
  stage2d_kernel<PREC, W, H, TX><<<grid, G::NT, G::template smem_bytes<NARR>(), stream>>>(prm);
  return (int)cudaGetLastError();
}

template <int PREC, int W, int TX>
static int launch2d_h(const Stage2DParams &prm, cudaStream_t s) {
  // a single instance's Hamiltonian, or the one every entry of a batch group shares, or (batch_kind1
  // 0) each entry's own, dispatched in the kernel (the narrow tiles and the runtime dispatch serve
  // batches, which take the position-free Hamiltonians only)
  if (prm.insts && prm.batch_kind1 == 0) return launch2d_one<PREC, W, H_RUNTIME, TX>(prm, s);
  switch (prm.insts ? prm.batch_kind1 - 1 : prm.inst0.ham) {
    case H_BURGERS2D:
      // a grid-wide or fixed flux alpha needs only the grid maximum of the node alphas
      if (prm.p.alpha_mode != A_LOCAL_LAGGED && prm.p.alpha_mode != A_LOCAL_EXACT)
        return launch2d_one<PREC, W, H_BURGERS2D_GRID, TX>(prm, s);
      return launch2d_one<PREC, W, H_BURGERS2D, TX>(prm, s);
    case H_NEGCOS2D: return launch2d_one<PREC, W, H_NEGCOS2D, TX>(prm, s);
    case H_SIN2D: return launch2d_one<PREC, W, H_SIN2D, TX>(prm, s);
    case H_EIKONAL2D: return launch2d_one<PREC, W, H_EIKONAL2D, TX>(prm, s);
    case H_OPTCTRL2D:
      if constexpr (TX == kTile2DX) return launch2d_one<PREC, W, H_OPTCTRL2D, TX>(prm, s);
      return (int)cudaErrorInvalidValue;
    default: return (int)cudaErrorInvalidValue;
  }
}

template <int PREC, int TX>
static int launch2d_impl(const Stage2DParams &prm, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  return prm.p.weights == W_JP ? launch2d_h<PREC, W_JP, TX>(prm, s) : launch2d_h<PREC, W_ARCLEN, TX>(prm, s);
}

template <int PREC, int TX>
static int grid_cap_impl(int weights) {
  return weights == W_JP ? grid_cap_of<PREC, W_JP, H_BURGERS2D, TX>() : grid_cap_of<PREC, W_ARCLEN, H_BURGERS2D, TX>();
}

}  // namespace alw
