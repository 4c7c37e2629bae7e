// Launch parameters of the persistent 2D float stage kernel (host and device).
#pragma once
#include <cuda.h>

#include "alw_internal.h"

namespace alw {

struct alignas(64) Stage2DParams {
  CUtensorMap maps[6];  // FP32: 0 = phi^n, 1 = stage-1 state, 2 = stage-2 state;
                        // MIXED: 0/1 = hi pairs, 2/3 = lo pairs, 4 = delta_1, 5 = delta_2
  StageParams p;
  int map_a, map_b, map_c;  // FP32: source, base (-1: none); MIXED: hi base index, lo base index, delta (-1: none)
};

// TMA box of one tile with its halo (floats): 72 columns x 38 rows.
constexpr int kBox2DW = 72, kBox2DH = 38;

int launch_stage2d_f32(const Stage2DParams &prm, void *stream);
int launch_stage2d_mixed(const Stage2DParams &prm, void *stream);

}  // namespace alw
