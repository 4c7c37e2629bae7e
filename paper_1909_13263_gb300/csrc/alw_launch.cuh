// Launcher of the stage kernel for one precision (included once per precision TU).
#pragma once
#include "alw_stage.cuh"

namespace alw {

template <int PREC, int DIM, int W, int SMALL = 0>
static int launch_one(const StageParams &p, cudaStream_t stream) {
  using Sh = Shape<PREC, DIM, SMALL>;
  auto kern = stage_kernel<PREC, DIM, W, SMALL>;
  const size_t smem = Sh::smem_bytes();
  static bool configured = false;   // attribute is per function; setting it twice is harmless
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    configured = true;
  }
  dim3 grid(p.tiles_x, p.tiles_y);
  kern<<<grid, Sh::NT, smem, stream>>>(p);
  return (int)cudaGetLastError();
}

// FP64 runs here in 1D and 2D; the float variants only in 1D (2D float stages run the persistent
// TMA kernel, so their 2D instantiations of this kernel are not built).
template <int PREC>
static int launch_stage_impl(const StageParams &p, void *stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (p.dim == 2) {
    if constexpr (PREC == P_F64) {
      if (p.small_tiles == 2)
        return p.weights == W_JP ? launch_one<PREC, 2, W_JP, 2>(p, s) : launch_one<PREC, 2, W_ARCLEN, 2>(p, s);
      if (p.small_tiles == 1)
        return p.weights == W_JP ? launch_one<PREC, 2, W_JP, 1>(p, s) : launch_one<PREC, 2, W_ARCLEN, 1>(p, s);
      return p.weights == W_JP ? launch_one<PREC, 2, W_JP>(p, s) : launch_one<PREC, 2, W_ARCLEN>(p, s);
    } else
      return (int)cudaErrorInvalidValue;
  }
  return p.weights == W_JP ? launch_one<PREC, 1, W_JP>(p, s) : launch_one<PREC, 1, W_ARCLEN>(p, s);
}

}  // namespace alw
