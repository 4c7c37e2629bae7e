// Launch parameters of the persistent 2D float stage kernel (host and device).
#pragma once
#include <cuda.h>

#include <vector>

#include "alw_internal.h"

namespace alw {

// One problem instance inside the shared padded arrays.  A single solver has
// one instance at row offset 0; a batch stacks many instances vertically in
// arrays of one common pitch, each in its own block of rows.
struct InstDesc {
  int nx, ny;            // interior nodes
  int tiles_x, tiles_y;  // tile grid of this instance
  int row_off;           // padded row of this instance's first (ghost) row
  int ham, bc;           // Hamiltonian kind, boundary condition
  int ntiles;            // tiles_x * tiles_y
  float dx, dy, rdx, rdy;
  float xlo, ylo;        // coordinates of node (0, 0) (position-dependent Hamiltonians)
  double lx, ly;         // dt = cfl / (ax/lx + ay/ly)
  DevState *st;          // this instance's device-side time and alpha state
};

struct Stage2DParams {
  CUtensorMap maps[6];  // FP32: 0 = phi^n, 1 = stage-1 state, 2 = stage-2 state;
                        // MIXED: 0/1 = hi pairs, 2/3 = lo pairs, 4 = delta_1, 5 = delta_2
  StageParams p;        // stage, modes, slots, pitch and buffers (per-instance fields unused in a batch)
  int map_a, map_b, map_c;  // FP32: source, base (-1: none); MIXED: hi base index, lo base index, previous increment (-1: none)
  int ntiles;               // work-list length
  int grid_ctas;            // persistent CTAs to launch (0: as many as fit; never more than fit or ntiles)
  int tile_w;               // tile width: 64 (0 means 64) or 32; the maps' boxes and insts[].tiles_x match it
  int batch_kind1;          // batch: 1 + the Hamiltonian every listed instance has; 0: instances of any
                            // position-free 2D Hamiltonian, dispatched per tile in the kernel
  const InstDesc *insts;    // batch: instance table (nullptr: the single instance `inst0`)
  DevState *states;         // batch: state of instance i at states + i (nullptr: read insts[i].st)
  const int *tiles;         // batch: work list, entry = instance * 65536 + tile of that instance
  int *done_count;          // batch: incremented when an instance reaches its t_final (may be null)
  InstDesc inst0;
};

// TMA box of one tile with its halo (floats): 72 columns x 38 rows for the 64 x 32 tile, 40 x 38
// for the narrow 32 x 32 tile (batches may choose it).  Padded arrays are laid out for 64-wide
// tiles, which also covers the narrow ones.
constexpr int kBox2DW = 72, kBox2DH = 38;
constexpr int kTile2DX = 64, kTile2DY = 32;
constexpr int kTile2DXNarrow = 32, kBox2DWNarrow = 40;

// CTAs a launch of `ntiles` work-list entries uses: min(ntiles, grid_ctas or cap, cap).
inline int stage2d_grid(int ntiles, int grid_ctas, int cap) {
  int g = (grid_ctas > 0 && grid_ctas < cap) ? grid_ctas : cap;
  return ntiles < g ? ntiles : g;
}

// The persistent kernel hands CTA c the work-list entries c, c + G, c + 2G, ...  Reorders an
// instance-major list so that each CTA's entries form one contiguous stretch of it: a CTA then
// meets few instance boundaries (each closes a run: alpha fold, counter atomics, a fence) and
// walks neighbouring tiles of one instance in turn.
// Block-cyclic layout: CTA c takes blocks of R consecutive entries of the ordered list, the
// blocks dealt round-robin over the G CTAs (R = 1 is the list as it is).
inline void cta_blocks(const std::vector<int> &in, int G, int R, std::vector<int> &out) {
  const int n = (int)in.size();
  out.resize(n);
  if (G <= 0 || n == 0) return;
  // the kernel's k-th entry of CTA c sits at position c + k G; give it list entry
  // (k / R) G R + c R + k % R while that exists, and lay the leftovers out in order
  std::vector<char> used(n, 0);
  std::vector<int> pos(n, -1);
  for (int p = 0; p < n; ++p) {
    const int c = p % G, k = p / G;
    const long long i = (long long)(k / R) * G * R + (long long)c * R + k % R;
    if (i < n) {
      pos[p] = (int)i;
      used[i] = 1;
    }
  }
  int next = 0;
  for (int p = 0; p < n; ++p) {
    if (pos[p] < 0) {
      while (used[next]) ++next;
      pos[p] = next;
      used[next] = 1;
    }
    out[p] = in[pos[p]];
  }
}

inline void cta_runs(const std::vector<int> &in, int G, std::vector<int> &out) {
  const int n = (int)in.size();
  out.resize(n);
  if (G <= 0 || n == 0) return;
  int start = 0;
  for (int c = 0; c < G && c < n; ++c) {
    const int cnt = (n - c + G - 1) / G;  // entries c, c + G, ... below n
    for (int k = 0; k < cnt; ++k) out[c + k * G] = in[start + k];
    start += cnt;
  }
}

int launch_stage2d_f32(const Stage2DParams &prm, void *stream);
int launch_stage2d_mixed(const Stage2DParams &prm, void *stream);
// occupancy-limited CTA count of the persistent kernel (for work-list sizing), per tile width
int stage2d_grid_cap_f32(int weights, int tile_w = kTile2DX);
int stage2d_grid_cap_mixed(int weights, int tile_w = kTile2DX);
// the narrow (32-wide) tile instantiations (the two entry points above dispatch to them when
// prm.tile_w / tile_w is 32); position-free Hamiltonians only
int launch_stage2d_f32_narrow(const Stage2DParams &prm, void *stream);
int launch_stage2d_mixed_narrow(const Stage2DParams &prm, void *stream);
int stage2d_grid_cap_f32_narrow(int weights);
int stage2d_grid_cap_mixed_narrow(int weights);

// Host helpers shared by the solver and batch runtimes (alw_runtime.cu).
void *dev_alloc(size_t bytes, void *stream);
void dev_free(void *ptr, size_t bytes, void *stream);
// 2D float tensor map over a padded array of `pitch` x `rows` floats, box = one tile plus halo
// (box_w columns: kBox2DW or kBox2DWNarrow); 0 on success
int encode_tile_map(CUtensorMap *map, void *base, long long pitch, long long rows, int box_w = kBox2DW);

}  // namespace alw
