// Persistent 2D stage kernel for float arithmetic (FP32 and MIXED) on sm_103a,
// for one instance or a batch of instances stacked in shared padded arrays.
//
// Each CTA walks the work list (tile = blockIdx.x + k * gridDim.x).  Thread 0
// prepares the next tile -- decodes its instance, decides whether the instance
// still needs work, computes the instance's dt and flux alpha for this stage,
// and issues one TMA box per array (tile plus 3-node halo) into the other half
// of a double buffer on an mbarrier -- while all threads compute the current
// tile:
//   1. differences pass: Delta^+ phi along x (dX) for every cell, combining
//      the two MIXED parts (hi + lo, or hi + the previous stage's increment
//      array, which carries lo) once per cell;
//   2. both sweeps in one pass, packed two lanes per value (f32x2): each
//      thread sweeps nodes 8w..8w+7 of row `lane` along x (warp w; the odd dX
//      pitch makes these column-wise reads conflict-free) in lane .x and 8
//      consecutive nodes of one column along y in lane .y, whose differences
//      it forms itself from the tile arrays (consecutive lanes read
//      consecutive columns); phi_x^-/+ go to shared memory, phi_y^-/+ stay in
//      registers;
//   3. each thread forms, for its 8 column nodes, the Lax-Friedrichs
//      Hamiltonian and the RK combination, and stores.
// A CTA keeps running maxima of |dH/dp|, |dH/dq| over consecutive tiles of
// one instance and folds them into the instance's slot (with the number of
// tiles done) when the instance changes; the CTA that completes an instance's
// last tile closes the instance's stage (dt, time, step count, buffer flip),
// so instances advance independently.
#pragma once
#include <type_traits>

#include "alw_device.cuh"
#include "alw_params2d.h"
#include "alw_sweep32.cuh"
#include "alw_tma.cuh"

namespace alw {

// Hamiltonians of the 2D examples in float (compile-time kind).  value_sums takes the sums
// su = u^- + u^+, sv = v^- + v^+ (the Lax-Friedrichs flux evaluates H at (su/2, sv/2)); kSameAlpha
// marks Hamiltonians whose node alpha is the same in both directions.
template <int H> struct Ham2;
template <> struct Ham2<H_BURGERS2D> {
  static constexpr bool kSameAlpha = true;
  __device__ __forceinline__ static float value(float p, float q, float, float) {
    const float z = p + q + 1.0f;
    return 0.5f * z * z;
  }
  __device__ __forceinline__ static float value_sums(float su, float sv, float, float) {
    const float z = fmaf(0.5f, su + sv, 1.0f);
    return 0.5f * z * z;
  }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float, float, float &ax,
                                                    float &ay) {
    // |H_p| = |H_q| = |u + v + 1| at the four corners: the largest and the smallest corner sums are
    // max(u) + 1 + max(v) and min(u) + 1 + min(v), and |.| is largest at one of them (the same
    // values as the four corner sums, with the comparisons on the integer/logic pipe)
    const float hi = (fmaxf(um, up) + 1.0f) + fmaxf(vm, vp), lo = (fminf(um, up) + 1.0f) + fminf(vm, vp);
    ax = ay = fmaxf(fabsf(hi), fabsf(lo));
  }
};
template <> struct Ham2<H_NEGCOS2D> {
  static constexpr bool kSameAlpha = true;
  __device__ __forceinline__ static float value(float p, float q, float, float) { return -sfu_cos(p + q + 1.0f); }
  __device__ __forceinline__ static float value_sums(float su, float sv, float, float) {
    return -sfu_cos(fmaf(0.5f, su + sv, 1.0f));
  }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float, float, float &ax,
                                                    float &ay) {
    const float a = fabsf(sfu_sin(um + vm + 1.0f)), b = fabsf(sfu_sin(um + vp + 1.0f));
    const float c = fabsf(sfu_sin(up + vm + 1.0f)), d = fabsf(sfu_sin(up + vp + 1.0f));
    ax = ay = fmaxf(fmaxf(a, b), fmaxf(c, d));
  }
};
template <> struct Ham2<H_SIN2D> {
  static constexpr bool kSameAlpha = true;
  __device__ __forceinline__ static float value(float p, float q, float, float) { return sfu_sin(p + q); }
  __device__ __forceinline__ static float value_sums(float su, float sv, float, float) {
    return sfu_sin(0.5f * (su + sv));
  }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float, float, float &ax,
                                                    float &ay) {
    const float a = fabsf(sfu_cos(um + vm)), b = fabsf(sfu_cos(um + vp));
    const float c = fabsf(sfu_cos(up + vm)), d = fabsf(sfu_cos(up + vp));
    ax = ay = fmaxf(fmaxf(a, b), fmaxf(c, d));
  }
};
template <> struct Ham2<H_EIKONAL2D> {
  static constexpr bool kSameAlpha = false;
  __device__ __forceinline__ static float value_sums(float su, float sv, float x, float y) {
    return value(0.5f * su, 0.5f * sv, x, y);
  }
  __device__ __forceinline__ static float value(float p, float q, float, float) {
    const float t = fmaf(p, p, fmaf(q, q, 1.0f));   // >= 1
    return t * sfu_rsqrt(t);
  }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float, float, float &ax,
                                                    float &ay) {
    const float r00 = sfu_rsqrt(fmaf(um, um, fmaf(vm, vm, 1.0f))), r01 = sfu_rsqrt(fmaf(um, um, fmaf(vp, vp, 1.0f)));
    const float r10 = sfu_rsqrt(fmaf(up, up, fmaf(vm, vm, 1.0f))), r11 = sfu_rsqrt(fmaf(up, up, fmaf(vp, vp, 1.0f)));
    ax = fmaxf(fmaxf(fabsf(um) * r00, fabsf(um) * r01), fmaxf(fabsf(up) * r10, fabsf(up) * r11));
    ay = fmaxf(fmaxf(fabsf(vm) * r00, fabsf(vp) * r01), fmaxf(fabsf(vm) * r10, fabsf(vp) * r11));
  }
};

// Example 11 (optimal control): the only Hamiltonian that depends on the node position (x, y).
template <> struct Ham2<H_OPTCTRL2D> {
  static constexpr bool kSameAlpha = false;
  __device__ __forceinline__ static float value_sums(float su, float sv, float x, float y) {
    return value(0.5f * su, 0.5f * sv, x, y);
  }
  __device__ __forceinline__ static float value(float p, float q, float x, float y) {
    const float sx = sfu_sin(x), cx = sfu_cos(x), sy = sfu_sin(y);
    // sin(y) p + (sin(x) + sign q) q - sin^2(y)/2 - (1 - cos x), with (sign q) q = |q|
    return fmaf(sy, p, fmaf(sx, q, fabsf(q))) - fmaf(0.5f * sy, sy, 1.0f - cx);
  }
  __device__ __forceinline__ static void alpha(float, float, float vm, float vp, float x, float y, float &ax,
                                               float &ay) {
    // H_p = sin y; H_q = sin x + sign q over [min v, max v], both signs when it contains q = 0
    const float sx = sfu_sin(x), lo = fminf(vm, vp), hi = fmaxf(vm, vp);
    ax = fabsf(sfu_sin(y));
    ay = (lo <= 0.0f && hi >= 0.0f) ? fabsf(sx) + 1.0f : fabsf(sx + (lo > 0.0f ? 1.0f : -1.0f));
  }
};

// The Hamiltonian of a launch: a compile-time kind, or H_RUNTIME, for batches that run instances
// of several Hamiltonians in one launch: the kind of the tile's instance, dispatched per node (the
// branch is uniform across a tile, so warps never diverge on it).
constexpr int H_RUNTIME = -1;
// Burgers with a grid-wide or fixed flux alpha: the finish loop does not need each node's alpha, only the
// grid maximum, so it tracks the largest and the negated smallest corner sum without their + 1 and forms
// max(hi + 1, -(lo + 1)) = max(|hi + 1|, |lo + 1|) once per fold (hi >= lo)
constexpr int H_BURGERS2D_GRID = -2;
template <int H> struct HamSel {
  static constexpr bool kSameAlpha = Ham2<H>::kSameAlpha;
  static constexpr bool kGridFold = false;
  __device__ __forceinline__ explicit HamSel(int) {}
  __device__ __forceinline__ float value_sums(float su, float sv, float x, float y) const {
    return Ham2<H>::value_sums(su, sv, x, y);
  }
  __device__ __forceinline__ void alpha(float um, float up, float vm, float vp, float x, float y, float &ax,
                                        float &ay) const {
    Ham2<H>::alpha(um, up, vm, vp, x, y, ax, ay);
  }
};
// runtime kind: the position-free 2D Hamiltonians batches take
template <> struct HamSel<H_BURGERS2D_GRID> : HamSel<H_BURGERS2D> {
  static constexpr bool kGridFold = true;
  __device__ __forceinline__ explicit HamSel(int k) : HamSel<H_BURGERS2D>(k) {}
};
template <> struct HamSel<H_RUNTIME> {
  static constexpr bool kSameAlpha = false;
  static constexpr bool kGridFold = false;
  int kind;
  __device__ __forceinline__ explicit HamSel(int k) : kind(k) {}
  __device__ __forceinline__ float value_sums(float su, float sv, float x, float y) const {
    switch (kind) {
      case H_BURGERS2D: return Ham2<H_BURGERS2D>::value_sums(su, sv, x, y);
      case H_NEGCOS2D: return Ham2<H_NEGCOS2D>::value_sums(su, sv, x, y);
      case H_SIN2D: return Ham2<H_SIN2D>::value_sums(su, sv, x, y);
      default: return Ham2<H_EIKONAL2D>::value_sums(su, sv, x, y);
    }
  }
  __device__ __forceinline__ void alpha(float um, float up, float vm, float vp, float x, float y, float &ax,
                                        float &ay) const {
    switch (kind) {
      case H_BURGERS2D: Ham2<H_BURGERS2D>::alpha(um, up, vm, vp, x, y, ax, ay); break;
      case H_NEGCOS2D: Ham2<H_NEGCOS2D>::alpha(um, up, vm, vp, x, y, ax, ay); break;
      case H_SIN2D: Ham2<H_SIN2D>::alpha(um, up, vm, vp, x, y, ax, ay); break;
      default: Ham2<H_EIKONAL2D>::alpha(um, up, vm, vp, x, y, ax, ay); break;
    }
  }
};

// Tile geometry of the stage kernel for tiles TXv nodes wide and 32 high (64 or 32 wide): one thread
// per 8-node row segment and 8-node column segment, so TXv / 8 warps; the TMA box is the tile plus
// its halo (4 columns, 3 rows each side); 8 warps per SM per 32 columns of tile width.
template <int TXv>
struct Geo2D {
  static constexpr int TX = TXv, TY = kTile2DY, K = 8, NT = TX * TY / K;
  static constexpr int MINB = 512 / NT;                 // resident CTAs per SM the registers are sized for
  static constexpr int CG = TX / 32;                    // column groups of 32 in the y sweep
  static constexpr int SW = TX + 8, SH = TY + 6;        // TMA box (halo 4 columns / 3 rows each side)
  static constexpr int ARR = ((SH * SW + 31) / 32) * 32; // floats per array slot (128-byte multiple)
  static constexpr int DXW = TX + 5, DXP = TX + 9;      // x differences: width, odd pitch
  static constexpr int SUP = TX + 1;                    // phi_x^-/+ pitch in float2
  template <int NARR> static constexpr size_t smem_bytes() {
    return 128 + sizeof(float) * (size_t)(2 * NARR * ARR + TY * DXP) + sizeof(float2) * (size_t)TY * SUP;
  }
};
static_assert(Geo2D<kTile2DX>::SW == kBox2DW && Geo2D<kTile2DX>::SH == kBox2DH, "TMA box must match the tile halo");
static_assert(Geo2D<kTile2DXNarrow>::SW == kBox2DWNarrow, "TMA box must match the tile halo");

// Everything a tile needs from its instance, gathered by thread 0 into shared memory when the
// tile is prepared (one tile ahead), so that the compute phase reads no instance data from
// global memory.
struct TileInfo {
  int inst, tx0, ty0, cur, skip, last;
  float dtf, fax, fay;
  double dt;
  int nx, ny, row_off, bc, ham, ntiles, tiles_x;
  float dx, dy, rdx, rdy, xlo, ylo;
  DevState *st;
};

template <int PREC, int W, int H, int TXv>
__global__ void __launch_bounds__(Geo2D<TXv>::NT, Geo2D<TXv>::MINB)
    stage2d_kernel(const __grid_constant__ Stage2DParams prm) {
  using G = Geo2D<TXv>;
  constexpr int TX = G::TX, TY = G::TY, K = G::K, NT = G::NT;
  constexpr int SW = G::SW, SH = G::SH, ARR = G::ARR;
  constexpr int DXW = G::DXW, DXP = G::DXP, SUP = G::SUP, CG = G::CG;
  constexpr int NARR = (PREC == P_MIXED) ? 3 : 2;
  // arc length with the increment form (MIXED): try the short-interval sweep first (FP32 stores phi
  // itself, whose rounding makes second differences rough at fine grids, so it never qualifies there)
  constexpr bool SHORT = (W == W_ARCLEN && PREC == P_MIXED);
  const StageParams &p = prm.p;
  const bool batch = prm.insts != nullptr;
  if (!batch) {
    const DevState *st = prm.inst0.st;
    if (p.loop_mode == LOOP_STEP_TO && !(st->t < st->t_final)) return;
    if (st->err) return;
  }

  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // TMA destinations are kept 128-byte aligned (the launch adds 128 bytes of slack)
  unsigned char *smem = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  float *raw = reinterpret_cast<float *>(smem);            // [2][NARR][ARR]
  float *dX = raw + 2 * NARR * ARR;                        // [TY][DXP]
  float2 *su = reinterpret_cast<float2 *>(dX + TY * DXP);  // [TY][SUP] (offset is an even float count)
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ TileInfo s_info[2];
  __shared__ TileInfo s_pinfo;  // thread 0's last prepared tile (per-instance scalars reused while it repeats)
  __shared__ float s_red[2][NT / 32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ntiles = prm.ntiles;
  const bool local_alpha = (p.alpha_mode == A_LOCAL_LAGGED || p.alpha_mode == A_LOCAL_EXACT);
  const float eps = (float)p.eps;
  const uint32_t box_bytes = (uint32_t)(SH * SW * sizeof(float));

  auto desc = [&](int inst) -> const InstDesc & { return batch ? prm.insts[inst] : prm.inst0; };

  // thread 0: one TMA box per array of the tile (with halo) into buffer b
  auto issue_loads = [&](const TileInfo &info, int b) {
    const CUtensorMap *mA, *mB = nullptr, *mC = nullptr;
    if (PREC == P_MIXED) {
      mA = &prm.maps[prm.map_a + info.cur];
      mB = &prm.maps[prm.map_b + info.cur];
      if (prm.map_c >= 0) mC = &prm.maps[prm.map_c];
    } else {
      mA = &prm.maps[prm.map_a];
      if (prm.map_b >= 0) mB = &prm.maps[prm.map_b];
    }
    const int nm = 1 + (mB != nullptr) + (mC != nullptr);
    float *dst = raw + b * NARR * ARR;
    const int y = info.row_off + info.ty0;
    mbar_arrive_expect_tx(&bars[b], box_bytes * nm);
    tma_load_2d(dst, mA, info.tx0, y, &bars[b]);
    if (mB) tma_load_2d(dst + ARR, mB, info.tx0, y, &bars[b]);
    if (mC) tma_load_2d(dst + 2 * ARR, mC, info.tx0, y, &bars[b]);
  };

  // thread 0: decode work-list entry e (of list position t), gather its instance's fields and
  // stage scalars (reused while the instance repeats), issue its loads into buffer b
  auto prepare = [&](int t, int e, int b) {
    int inst = 0, tl = t;
    if (batch) {
      inst = e >> 16;
      tl = e & 0xffff;
    }
    if (inst == s_info[b].inst) {
      // the tile that last used this buffer belongs to the same instance (always so for a single
      // grid): only the tile origin changes
      TileInfo &bi = s_info[b];
      bi.tx0 = (tl % bi.tiles_x) * TX;
      bi.ty0 = (tl / bi.tiles_x) * TY;
      if (!bi.skip) issue_loads(bi, b);
      return;
    }
    TileInfo info;
    if (inst == s_pinfo.inst) {
      info = s_pinfo;
      info.tx0 = (tl % info.tiles_x) * TX;
      info.ty0 = (tl / info.tiles_x) * TY;
      s_info[b] = info;
      s_pinfo = info;
      if (!info.skip) issue_loads(info, b);
      return;
    }
    // the instance's descriptor and its state (contiguous states: no dependent load)
    const InstDesc &d = desc(inst);
    DevState *st = (batch && prm.states) ? prm.states + inst : d.st;
    info.inst = inst;
    info.nx = d.nx;
    info.ny = d.ny;
    info.row_off = d.row_off;
    info.bc = d.bc;
    info.ham = d.ham;
    info.ntiles = d.ntiles;
    info.tiles_x = d.tiles_x;
    info.dx = d.dx;
    info.dy = d.dy;
    info.rdx = d.rdx;
    info.rdy = d.rdy;
    info.xlo = d.xlo;
    info.ylo = d.ylo;
    info.st = st;
    const double lx = d.lx, ly = d.ly;
    const int s_cur = st->cur, s_err = st->err;
    const double s_t = st->t, s_tf = st->t_final, s_dt = st->dt;
    info.tx0 = (tl % info.tiles_x) * TX;
    info.ty0 = (tl / info.tiles_x) * TY;
    info.cur = (PREC == P_MIXED) ? s_cur : 0;
    info.skip = (s_err != 0) || (p.loop_mode == LOOP_STEP_TO && !(s_t < s_tf));
    double dt;
    int last = 0;
    if (p.stage == 1 && p.loop_mode != LOOP_STAGE) {
      double ax, ay;
      if (p.alpha_mode == A_FIXED) {
        ax = p.alpha_fixed[0];
        ay = p.alpha_fixed[1];
      } else {
        ax = bits_to_double(st->alpha_bits[p.dt_slot][0]);
        ay = bits_to_double(st->alpha_bits[p.dt_slot][1]);
      }
      const double den = ax / lx + ay / ly;
      dt = den > 0.0 ? p.cfl / den : (p.loop_mode == LOOP_ADVANCE ? 0.0 : INFINITY);
      if (p.loop_mode == LOOP_STEP_TO && s_t + dt >= s_tf) {
        dt = s_tf - s_t;
        last = 1;
      }
    } else if (p.loop_mode == LOOP_STAGE) {
      dt = p.dt_value;
    } else {
      dt = s_dt;
    }
    info.dt = dt;
    info.dtf = (float)dt;
    info.last = last;
    float fax = 0.0f, fay = 0.0f;
    if (p.alpha_mode == A_FIXED) {
      fax = (float)p.alpha_fixed[0];
      fay = (float)p.alpha_fixed[1];
    } else if (!local_alpha && p.read_slot >= 0) {
      fax = (float)bits_to_double(st->alpha_bits[p.read_slot][0]);
      fay = (float)bits_to_double(st->alpha_bits[p.read_slot][1]);
    }
    info.fax = fax;
    info.fay = fay;
    s_info[b] = info;
    s_pinfo = info;
    if (!info.skip) issue_loads(info, b);
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
    s_pinfo.inst = -1;
    s_info[0].inst = -1;
    s_info[1].inst = -1;
    if ((int)blockIdx.x < ntiles) prepare(blockIdx.x, batch ? prm.tiles[blockIdx.x] : 0, 0);
  }
  __syncthreads();

  uint32_t phase = 0;  // bit b: parity of the next completion of bars[b]
  int k = 0;
  // running alpha maxima and tile count of the current run of same-instance tiles
  constexpr bool GF = HamSel<H>::kGridFold;
  constexpr float A0 = GF ? -INFINITY : 0.0f;  // identity of the running maxima
  float amx = A0, amy = A0;
  float nfin = 0.0f;  // NaN once a non-finite L was met (see the finish loop)
  int run_tiles = 0;
  // thread 0: work-list entry of the tile after next, loaded one tile ahead of its use
  int e_ahead = (batch && tid == 0 && (int)(blockIdx.x + gridDim.x) < ntiles) ? prm.tiles[blockIdx.x + gridDim.x] : 0;
  // thread 0, once every thread is past the previous tile's reads of buffer buf ^ 1 and of
  // s_info[buf ^ 1]: prepare the next tile into that buffer
  auto prepare_next = [&](int next, int buf) {
    if (tid == 0 && next < ntiles) {
      fence_proxy_async_smem();
      prepare(next, e_ahead, buf ^ 1);
      const int after = next + (int)gridDim.x;
      e_ahead = (batch && after < ntiles) ? prm.tiles[after] : 0;
    }
  };
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int buf = k & 1;
    const int next = t + gridDim.x;
    const int i_inst = s_info[buf].inst, i_skip = s_info[buf].skip, i_cur = s_info[buf].cur;
    if (i_skip) {
      __syncthreads();
      prepare_next(next, buf);
      __syncthreads();
      continue;
    }
    // every thread waits for the tile's loads itself; no CTA barrier here: the buffers, the tile
    // records and the phi_x hand-off of the previous tile are rewritten only after the barrier that
    // follows the differences pass, which every thread reaches after finishing the previous tile
    const bool ok = mbar_wait_bounded(&bars[buf], (phase >> buf) & 1u);
    phase ^= 1u << buf;

    const TileInfo &d = s_info[buf];  // this tile's instance fields (shared memory)
    const int nx = d.nx, ny = d.ny, tx0 = d.tx0, ty0 = d.ty0;
    const size_t rbase = (size_t)d.row_off * p.pitch;   // element offset of the instance's rows
    const HamSel<H> ham(d.ham);
    const float dtf = s_info[buf].dtf, fax = s_info[buf].fax, fay = s_info[buf].fay;
    const float faxh = 0.5f * fax, fayh = 0.5f * fay;
    const float *A = raw + buf * NARR * ARR;
    const float *B = A + ARR;
    const float *C = A + 2 * ARR;
    // MIXED: the stage's input is A + X, the high part of phi^n plus X = its low part (stage 1) or the
    // increment array of the previous stage, which holds the low part as well (stages 2 and 3; see the
    // finish loop)
    const float *X = (PREC == P_MIXED && prm.map_c >= 0) ? C : B;

    // ---- 1. x differences in the units of the sweep (arc length: Delta^+ phi / dx^2; Jiang-Peng:
    // Delta^+ phi / dx), rows by warp, columns by lane (no division, conflict-free)
    const float rdx2 = (W == W_ARCLEN) ? d.rdx * d.rdx : d.rdx;
    {
      auto cell_diff = [&](int i0, int i1) -> float {
        if (PREC == P_MIXED) return (A[i1] - A[i0]) + (X[i1] - X[i0]);
        return A[i1] - A[i0];
      };
      // the first TX cells of every row by whole warps, the last DXW - TX cells of all rows together
      // (a third pass per row would keep only 5 of 32 lanes busy)
      static_assert(TX % 32 == 0 && DXW - TX < 32, "x-difference row split");
      for (int r = warp; r < TY; r += NT / 32) {
#pragma unroll
        for (int c = lane; c < TX; c += 32) {
          const int i0 = (r + 3) * SW + c + 1;
          dX[r * DXP + c] = cell_diff(i0, i0 + 1) * rdx2;
        }
      }
      for (int j = tid; j < TY * (DXW - TX); j += NT) {
        const int r = j / (DXW - TX), c = TX + j % (DXW - TX);
        const int i0 = (r + 3) * SW + c + 1;
        dX[r * DXP + c] = cell_diff(i0, i0 + 1) * rdx2;
      }
    }
    if (__syncthreads_or(!ok)) {
      // a tile load never completed (the differences pass above ran on whatever the buffer held):
      // flag the instance and stop; the next tile's load is issued only after this barrier, so no
      // other load is in flight
      if (tid == 0) atomicOr(&s_info[buf].st->err, 2);
      __syncthreads();
      return;
    }
    // every thread has finished the previous tile (its finish loop read buffer buf ^ 1), so the next
    // tile's load can go there; the barrier after the sweeps publishes s_info[buf ^ 1]
    prepare_next(next, buf);

    const bool edge = (tx0 < 3) || (tx0 + TX > nx - 3) || (ty0 < 3) || (ty0 + TY > ny - 3);
    const int colY = (warp % CG) * 32 + lane, segY = warp / CG;

    // ---- 2. both sweeps in one pass: each thread's row segment (x, lane .x of the packed values)
    // and column segment (y, lane .y) run the same instruction stream
    float ym[K], yp[K];
    {
      const float *vx = dX + lane * DXP + K * warp;
      // the y differences of the column segment, formed here from the tile arrays like the x
      // differences of the differences pass (in the same units); u_at is called for m = 0, 1, 2, ... in
      // order, so each position loads one new row and reuses the previous one
      const int iy = (K * segY) * SW + colY + 4;
      const float rdy2 = (W == W_ARCLEN) ? d.rdy * d.rdy : d.rdy;
      auto make_vat = [&]() {
        float pa = A[iy], px = 0.0f;
        if (PREC == P_MIXED) px = X[iy];
        return [=](int m) mutable {
          const int i1 = iy + (m + 1) * SW;
          float dy;
          if (PREC == P_MIXED) {
            const float a1 = A[i1], x1 = X[i1];
            dy = (a1 - pa) + (x1 - px);
            pa = a1;
            px = x1;
          } else {
            const float a1 = A[i1];
            dy = a1 - pa;
            pa = a1;
          }
          return make_float2(vx[m], dy * rdy2);
        };
      };
      auto emit = [&](int q, float2 dm, float2 dp) {
        su[lane * SUP + K * warp + q] = make_float2(dm.x, dp.x);
        ym[q] = dm.y;
        yp[q] = dp.y;
      };
      SweepConsts<float2> sc;
      sc.eps4 = make_float2(4.0f * eps * d.rdx * d.rdx, 4.0f * eps * d.rdy * d.rdy);
      sc.h2 = make_float2(0.5f * d.dx, 0.5f * d.dy);
      sc.h3 = make_float2(d.dx * (1.0f / 3.0f), d.dy * (1.0f / 3.0f));
      sc.mh6 = make_float2(d.dx * (-1.0f / 6.0f), d.dy * (-1.0f / 6.0f));
      // arc length, MIXED: every warp sweeps with the short-interval form first and sweeps again in
      // full when some segment of the warp does not qualify (that form then replaces all its
      // results).  Which form produced a node's values thus depends only on the data of the warp's
      // segments, whose position on the grid is fixed by the tile width -- not on the order in
      // which tiles or instances are processed, nor on history: a single solve, a batch, a server
      // round and a resumed checkpoint (all with 64-wide tiles) choose alike.
      bool full = true;
      if (SHORT) full = !sweep_stream_short<K, float2>(make_vat(), sc, emit);
      if (full) {
        if constexpr (W == W_ARCLEN) sweep_stream<K, float2>(make_vat(), sc, emit);
        else sweep_stream_jp<K, float2>(make_vat(), make_float2(eps, eps), emit);
      }
    }
    __syncthreads();

    // ---- 3. nodes (colY, K*segY + q): Lax-Friedrichs Hamiltonian, RK combination, store; one
    // unrolled loop per stage and per edge/interior tile, so that no node tests either
    auto finish = [&](auto stage_c, auto edge_c, auto hsel) {
      using HS = decltype(hsel);
      constexpr int ST = decltype(stage_c)::value;
      constexpr bool EDGE = decltype(edge_c)::value;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const float dmq = ym[q], dpq = yp[q];
        const int y = K * segY + q;
        const int gi = tx0 + colY, gj = ty0 + y;
        const bool inside = !EDGE || (gi < nx && gj < ny);
        const float2 u = su[y * SUP + colY];
        const float xn = fmaf((float)gi, d.dx, d.xlo), yn = fmaf((float)gj, d.dy, d.ylo);
        const float Hv = hsel.value_sums(u.y + u.x, dpq + dmq, xn, yn);
        float L;
        if constexpr (HS::kGridFold) {
          L = fmaf(faxh, u.y - u.x, fmaf(fayh, dpq - dmq, -Hv));
          if (inside) {
            nfin = fmaf(L, 0.0f, nfin);
            amx = fmaxf(amx, fmaxf(u.x, u.y) + fmaxf(dmq, dpq));
            amy = fmaxf(amy, -(fminf(u.x, u.y) + fminf(dmq, dpq)));
          }
        } else {
          float ax, ay;
          hsel.alpha(u.x, u.y, dmq, dpq, xn, yn, ax, ay);
          const float aX = local_alpha ? ax : fax, aY = local_alpha ? ay : fay;
          L = fmaf(aX * 0.5f, u.y - u.x, fmaf(aY * 0.5f, dpq - dmq, -Hv));
          if (inside) {
            // L depends on all four one-sided derivatives: L * 0 is NaN exactly when L is not finite
            nfin = fmaf(L, 0.0f, nfin);
            amx = fmaxf(amx, ax);
            // (with a runtime Hamiltonian the fold below does not copy amx, so amy is always kept)
            if (!HS::kSameAlpha || !HamSel<H>::kSameAlpha) amy = fmaxf(amy, ay);
          }
        }
        if (ST == 0 || !inside) continue;
        const int sidx = (y + 3) * SW + colY + 4;
        const size_t g = rbase + (size_t)(gj + GY) * p.pitch + gi + GX;
        if (PREC == P_MIXED) {
          // phi^n = hi + lo (A, B) and the stage states phi_1 = hi + e_1, phi_2 = hi + e_2, where the
          // increment arrays e_k = lo + (phi_k - phi^n) carry the low part (C = e_{k-1}):
          //   e_1 = lo + dt L,  e_2 = 3/4 lo + 1/4 (e_1 + dt L),  phi^{n+1} = hi + lo + 2/3 (e_2 + dt L - lo)
          // (Step 5's combinations with phi_k - phi^n = e_k - lo)
          if (ST == 3) {
            const float dd = (2.0f / 3.0f) * (fmaf(dtf, L, C[sidx]) - B[sidx]);
            float h, l;
            df_add(A[sidx], B[sidx], dd, h, l);
            float *oh = reinterpret_cast<float *>(p.mix_hi[i_cur ^ 1]);
            float *ol = reinterpret_cast<float *>(p.mix_lo[i_cur ^ 1]);
            if (EDGE) {
              store_node<float, 2>(oh + rbase, p.pitch, nx, ny, d.bc, gi, gj, h);
              store_node<float, 2>(ol + rbase, p.pitch, nx, ny, d.bc, gi, gj, l);
            } else {
              oh[g] = h;
              ol[g] = l;
            }
          } else {
            const float dd = (ST == 1) ? fmaf(dtf, L, B[sidx]) : fmaf(0.75f, B[sidx], 0.25f * fmaf(dtf, L, C[sidx]));
            float *o = reinterpret_cast<float *>(p.out0);
            if (EDGE) store_node<float, 2>(o + rbase, p.pitch, nx, ny, d.bc, gi, gj, dd);
            else o[g] = dd;
          }
        } else {
          const float src = A[sidx];
          float outv;
          if (ST == 1) {
            outv = fmaf(dtf, L, src);
          } else if (ST == 2) {
            outv = fmaf(0.75f, B[sidx], 0.25f * fmaf(dtf, L, src));
          } else {
            outv = fmaf(1.0f / 3.0f, B[sidx], (2.0f / 3.0f) * fmaf(dtf, L, src));
          }
          float *o = reinterpret_cast<float *>(p.out0);
          if (EDGE) store_node<float, 2>(o + rbase, p.pitch, nx, ny, d.bc, gi, gj, outv);
          else o[g] = outv;
        }
      }
    };
    // the Hamiltonian of the tile: the launch's, or with H_RUNTIME the instance's, chosen once per tile
    auto finish_h = [&](auto stage_c, auto edge_c) {
      if constexpr (H == H_RUNTIME) {
        switch (d.ham) {
          case H_BURGERS2D: finish(stage_c, edge_c, HamSel<H_BURGERS2D>(0)); break;
          case H_NEGCOS2D: finish(stage_c, edge_c, HamSel<H_NEGCOS2D>(0)); break;
          case H_SIN2D: finish(stage_c, edge_c, HamSel<H_SIN2D>(0)); break;
          default: finish(stage_c, edge_c, HamSel<H_EIKONAL2D>(0)); break;
        }
      } else {
        finish(stage_c, edge_c, ham);
      }
    };
    auto finish_stage = [&](auto stage_c) {
      if (edge) finish_h(stage_c, std::true_type{});
      else finish_h(stage_c, std::false_type{});
    };
    switch (p.stage) {
      case 0: finish_stage(std::integral_constant<int, 0>{}); break;
      case 1: finish_stage(std::integral_constant<int, 1>{}); break;
      case 2: finish_stage(std::integral_constant<int, 2>{}); break;
      default: finish_stage(std::integral_constant<int, 3>{}); break;
    }

    // ---- when the next tile of this CTA belongs to another instance (or there is none), fold the
    // run's maximum of alpha into the instance's slot and count its tiles; close the instance's stage
    ++run_tiles;
    const bool more = next < ntiles;
    if (more && !s_info[buf ^ 1].skip && s_info[buf ^ 1].inst == i_inst) {
      // no barrier: the next tile's differences pass writes only dX, which this tile read
      // before the barrier after the sweeps; su, raw[buf] and s_info[buf] are rewritten only
      // after the next tile's barrier that follows its differences pass, which every thread
      // reaches after finishing this tile
      continue;
    }
    if constexpr (GF) {
      amx = fmaxf(fmaxf(amx + 1.0f, amy - 1.0f), 0.0f);
      amy = amx;
    } else if (HamSel<H>::kSameAlpha) {
      amy = amx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, o));
      amy = fmaxf(amy, __shfl_xor_sync(0xffffffffu, amy, o));
    }
    const int anybad = __syncthreads_or(nfin != nfin ? 1 : 0);
    if (lane == 0) {
      s_red[0][warp] = amx;
      s_red[1][warp] = amy;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < NT / 32; ++w) {
        amx = fmaxf(amx, s_red[0][w]);
        amy = fmaxf(amy, s_red[1][w]);
      }
      DevState *st = d.st;
      if (anybad) atomicOr(&st->err, 1);
      if (p.write_slot >= 0) {
        atomicMax(&st->alpha_bits[p.write_slot][0], double_to_bits((double)amx));
        atomicMax(&st->alpha_bits[p.write_slot][1], double_to_bits((double)amy));
      }
      __threadfence();
      const unsigned int prev = atomicAdd(&st->counter, (unsigned int)run_tiles);
      if (prev + (unsigned int)run_tiles == (unsigned int)d.ntiles) {
        // every tile of this instance has finished this stage
        __threadfence();
        st->counter = 0;
        if (p.zero_slot >= 0) {
          st->alpha_bits[p.zero_slot][0] = 0ull;
          st->alpha_bits[p.zero_slot][1] = 0ull;
        }
        if (p.stage == 1 && p.loop_mode != LOOP_STAGE) {
          st->dt = s_info[buf].dt;
          st->last = s_info[buf].last;
        }
        if (p.stage == 3) {
          if (PREC == P_MIXED) st->cur = i_cur ^ 1;
          if (p.loop_mode != LOOP_STAGE) {
            const double tn = st->last ? st->t_final : st->t + st->dt;
            st->t = tn;
            st->steps += 1;
            if (p.loop_mode == LOOP_STEP_TO && !(tn < st->t_final) && prm.done_count) atomicAdd(prm.done_count, 1);
          }
        }
      }
    }
    amx = amy = A0;
    nfin = 0.0f;
    run_tiles = 0;
    __syncthreads();  // raw[buf], dX, su, s_info[buf] are free for the next tile
  }
}

}  // namespace alw
