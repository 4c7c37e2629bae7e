// Persistent 2D stage kernel for float arithmetic (FP32 and MIXED) on sm_103a.
//
// Each CTA walks tiles tile = blockIdx.x + k * gridDim.x.  The raw arrays of
// the next tile (phi or hi/lo/delta, with a 3-node halo; one TMA box per
// array) are loaded into the other half of a double buffer while the current
// tile is computed.  Per tile:
//   1. differences pass: Delta^+ phi along x (dX) and y (dY) for every cell,
//      combining the MIXED parts (hi + lo + delta) once per cell;
//   2. x sweep: warp w takes nodes 8w..8w+7 of every row (one row per lane;
//      the odd dX pitch makes these column-wise reads conflict-free) and
//      writes phi_x^-/+ to shared memory;
//   3. y sweep: each lane takes 8 consecutive nodes of one column, forms the
//      Lax-Friedrichs Hamiltonian and the RK combination, and stores.
// The same sweep code serves both directions.  Alpha is folded into a
// per-thread maximum and reduced once per CTA at the end.
#pragma once
#include "alw_device.cuh"
#include "alw_params2d.h"
#include "alw_sweep32.cuh"
#include "alw_tma.cuh"

namespace alw {

// Hamiltonians of the 2D examples in float (compile-time kind).
template <int H> struct Ham2;
template <> struct Ham2<H_BURGERS2D> {
  __device__ __forceinline__ static float value(float p, float q) {
    const float z = p + q + 1.0f;
    return 0.5f * z * z;
  }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float &ax, float &ay) {
    const float a = fabsf(um + vm + 1.0f), b = fabsf(um + vp + 1.0f);
    const float c = fabsf(up + vm + 1.0f), d = fabsf(up + vp + 1.0f);
    ax = ay = fmaxf(fmaxf(a, b), fmaxf(c, d));
  }
};
template <> struct Ham2<H_NEGCOS2D> {
  __device__ __forceinline__ static float value(float p, float q) { return -__cosf(p + q + 1.0f); }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float &ax, float &ay) {
    const float a = fabsf(__sinf(um + vm + 1.0f)), b = fabsf(__sinf(um + vp + 1.0f));
    const float c = fabsf(__sinf(up + vm + 1.0f)), d = fabsf(__sinf(up + vp + 1.0f));
    ax = ay = fmaxf(fmaxf(a, b), fmaxf(c, d));
  }
};
template <> struct Ham2<H_SIN2D> {
  __device__ __forceinline__ static float value(float p, float q) { return __sinf(p + q); }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float &ax, float &ay) {
    const float a = fabsf(__cosf(um + vm)), b = fabsf(__cosf(um + vp));
    const float c = fabsf(__cosf(up + vm)), d = fabsf(__cosf(up + vp));
    ax = ay = fmaxf(fmaxf(a, b), fmaxf(c, d));
  }
};
template <> struct Ham2<H_EIKONAL2D> {
  __device__ __forceinline__ static float value(float p, float q) { return sqrtf(fmaf(p, p, fmaf(q, q, 1.0f))); }
  __device__ __forceinline__ static void alpha(float um, float up, float vm, float vp, float &ax, float &ay) {
    const float r00 = rsqrtf(fmaf(um, um, fmaf(vm, vm, 1.0f))), r01 = rsqrtf(fmaf(um, um, fmaf(vp, vp, 1.0f)));
    const float r10 = rsqrtf(fmaf(up, up, fmaf(vm, vm, 1.0f))), r11 = rsqrtf(fmaf(up, up, fmaf(vp, vp, 1.0f)));
    ax = fmaxf(fmaxf(fabsf(um) * r00, fabsf(um) * r01), fmaxf(fabsf(up) * r10, fabsf(up) * r11));
    ay = fmaxf(fmaxf(fabsf(vm) * r00, fabsf(vp) * r01), fmaxf(fabsf(vm) * r10, fabsf(vp) * r11));
  }
};

struct Geo2D {
  static constexpr int TX = 64, TY = 32, K = 8, NT = 256;
  static constexpr int SW = TX + 8, SH = TY + 6;        // TMA box (halo 4 columns / 3 rows each side)
  static constexpr int ARR = ((SH * SW + 31) / 32) * 32; // floats per array slot (128-byte multiple)
  static constexpr int DXW = TX + 5, DXP = 73;          // x differences: width, odd pitch
  static constexpr int DYH = TY + 5;                    // y differences: rows
  static constexpr int SUP = TX + 1;                    // phi_x^-/+ pitch in float2
  template <int NARR> static constexpr size_t smem_bytes() {
    return 128 + sizeof(float) * (size_t)(2 * NARR * ARR + TY * DXP + DYH * TX) + sizeof(float2) * (size_t)TY * SUP;
  }
};

template <int PREC, int W, int H>
__global__ void __launch_bounds__(Geo2D::NT, 2) stage2d_kernel(const __grid_constant__ Stage2DParams prm) {
  constexpr int TX = Geo2D::TX, TY = Geo2D::TY, K = Geo2D::K, NT = Geo2D::NT;
  constexpr int SW = Geo2D::SW, SH = Geo2D::SH, ARR = Geo2D::ARR;
  constexpr int DXW = Geo2D::DXW, DXP = Geo2D::DXP, DYH = Geo2D::DYH, SUP = Geo2D::SUP;
  constexpr int NARR = (PREC == P_MIXED) ? 3 : 2;
  const StageParams &p = prm.p;
  DevState *st = p.state;
  if (p.loop_mode == LOOP_STEP_TO && !(st->t < st->t_final)) return;
  if (st->err) return;

  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // TMA destinations are kept 128-byte aligned (the launch adds 128 bytes of slack)
  unsigned char *smem = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  float *raw = reinterpret_cast<float *>(smem);          // [2][NARR][ARR]
  float *dX = raw + 2 * NARR * ARR;                      // [TY][DXP]
  float *dY = dX + TY * DXP;                             // [DYH][TX]
  float2 *su = reinterpret_cast<float2 *>(dY + DYH * TX);  // [TY][SUP] (offset is an even float count)
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ float s_red[2][NT / 32];
  __shared__ double s_dt;
  __shared__ int s_lastflag, s_last;
  __shared__ float s_fax, s_fay, s_dtf;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles = p.tiles_x * p.tiles_y;
  const int cur = (PREC == P_MIXED) ? st->cur : 0;
  const bool local_alpha = (p.alpha_mode == A_LOCAL_LAGGED || p.alpha_mode == A_LOCAL_EXACT);

  // tensor maps of this stage
  const CUtensorMap *mA, *mB = nullptr, *mC = nullptr;
  if (PREC == P_MIXED) {
    mA = &prm.maps[prm.map_a + cur];
    mB = &prm.maps[prm.map_b + cur];
    if (prm.map_c >= 0) mC = &prm.maps[prm.map_c];
  } else {
    mA = &prm.maps[prm.map_a];
    if (prm.map_b >= 0) mB = &prm.maps[prm.map_b];
  }
  const int nmaps = 1 + (mB != nullptr) + (mC != nullptr);
  const bool has_delta = (mC != nullptr);

  if (tid == 0) {
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
      const double den = ax / p.lx + ay / p.ly;
      dt = den > 0.0 ? p.cfl / den : (p.loop_mode == LOOP_ADVANCE ? 0.0 : INFINITY);
      if (p.loop_mode == LOOP_STEP_TO && st->t + dt >= st->t_final) {
        dt = st->t_final - st->t;
        last = 1;
      }
    } else if (p.loop_mode == LOOP_STAGE) {
      dt = p.dt_value;
    } else {
      dt = st->dt;
    }
    s_dt = dt;
    s_dtf = (float)dt;
    s_lastflag = last;
    float fax = 0.0f, fay = 0.0f;
    if (p.alpha_mode == A_FIXED) {
      fax = (float)p.alpha_fixed[0];
      fay = (float)p.alpha_fixed[1];
    } else if (!local_alpha && p.read_slot >= 0) {
      fax = (float)bits_to_double(st->alpha_bits[p.read_slot][0]);
      fay = (float)bits_to_double(st->alpha_bits[p.read_slot][1]);
    }
    s_fax = fax;
    s_fay = fay;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const float dtf = s_dtf, fax = s_fax, fay = s_fay;

  const uint32_t box_bytes = (uint32_t)(SH * SW * sizeof(float));
  auto issue = [&](int tile, int buf) {
    const int tx0 = (tile % p.tiles_x) * TX, ty0 = (tile / p.tiles_x) * TY;
    float *dst = raw + buf * NARR * ARR;
    mbar_arrive_expect_tx(&bars[buf], box_bytes * nmaps);
    tma_load_2d(dst, mA, tx0, ty0, &bars[buf]);
    if (mB) tma_load_2d(dst + ARR, mB, tx0, ty0, &bars[buf]);
    if (mC) tma_load_2d(dst + 2 * ARR, mC, tx0, ty0, &bars[buf]);
  };

  const float dx = (float)p.dx, dy = (float)p.dy, rdx = (float)p.rdx, rdy = (float)p.rdy, eps = (float)p.eps;
  float amx = 0.0f, amy = 0.0f;
  bool bad = false;
  int k = 0;
  int tile = blockIdx.x;
  if (tid == 0 && tile < tiles) issue(tile, 0);

  for (; tile < tiles; tile += gridDim.x, ++k) {
    const int buf = k & 1;
    const int next = tile + gridDim.x;
    if (tid == 0 && next < tiles) {
      fence_proxy_async_smem();
      issue(next, buf ^ 1);
    }
    const bool ok = mbar_wait_bounded(&bars[buf], (uint32_t)((k >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      // a tile load never completed: flag it, let the other in-flight load land, stop
      if (tid == 0) {
        atomicOr(&st->err, 2);
        if (next < tiles) mbar_wait_bounded(&bars[buf ^ 1], (uint32_t)(((k + 1) >> 1) & 1));
      }
      __syncthreads();
      return;
    }
    const int tx0 = (tile % p.tiles_x) * TX, ty0 = (tile / p.tiles_x) * TY;
    const float *A = raw + buf * NARR * ARR;
    const float *B = A + ARR;
    const float *C = A + 2 * ARR;

    // ---- 1. differences (rows by warp, columns by lane: no division, conflict-free)
    auto cell_diff = [&](int i0, int i1) -> float {
      if (PREC == P_MIXED) {
        return (A[i1] - A[i0]) + ((B[i1] - B[i0]) + (has_delta ? (C[i1] - C[i0]) : 0.0f));
      } else {
        return A[i1] - A[i0];
      }
    };
    for (int r = warp; r < TY; r += NT / 32) {
#pragma unroll
      for (int c = lane; c < DXW; c += 32) {
        const int i0 = (r + 3) * SW + c + 1;
        dX[r * DXP + c] = cell_diff(i0, i0 + 1) * rdx;
      }
    }
    for (int r = warp; r < DYH; r += NT / 32) {
#pragma unroll
      for (int c = lane; c < TX; c += 32) {
        const int i0 = r * SW + c + 4;
        dY[r * TX + c] = cell_diff(i0, i0 + SW) * rdy;
      }
    }
    __syncthreads();

    const bool edge = (tx0 < 3) || (tx0 + TX > p.nx - 3) || (ty0 < 3) || (ty0 + TY > p.ny - 3);
    const int colY = ((warp & 1) << 5) + lane, segY = warp >> 1;

    // ---- 2./3. sweeps (one code path for both directions)
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      const float *vsrc = dir == 0 ? dX + lane * DXP + K * warp : dY + (K * segY) * TX + colY;
      const int vstride = dir == 0 ? 1 : TX;
      auto v_at = [&](int m) { return vsrc[m * vstride]; };
      auto emit = [&](int q, float dmq, float dpq) {
        if (dir == 0) {
          su[lane * SUP + K * warp + q] = make_float2(dmq, dpq);
          return;
        }
        // node (colY, y) of the tile: phi_y^-/+ = (dmq, dpq)
        const int y = K * segY + q;
        const int gi = tx0 + colY, gj = ty0 + y;
        const bool inside = !edge || (gi < p.nx && gj < p.ny);
        const float2 u = su[y * SUP + colY];
        float ax, ay;
        Ham2<H>::alpha(u.x, u.y, dmq, dpq, ax, ay);
        if (inside) {
          if (!isfinite(u.x + u.y + dmq + dpq)) bad = true;
          amx = fmaxf(amx, ax);
          amy = fmaxf(amy, ay);
        }
        if (p.stage == 0 || !inside) return;
        const float aX = local_alpha ? ax : fax, aY = local_alpha ? ay : fay;
        const float Hv = Ham2<H>::value(0.5f * (u.y + u.x), 0.5f * (dpq + dmq));
        const float L = fmaf(aX * 0.5f, u.y - u.x, fmaf(aY * 0.5f, dpq - dmq, -Hv));
        const int sidx = (y + 3) * SW + colY + 4;
        const size_t g = (size_t)(gj + GY) * p.pitch + gi + GX;
        if (PREC == P_MIXED) {
          if (p.stage == 3) {
            const float d = (2.0f / 3.0f) * fmaf(dtf, L, C[sidx]);
            float h, l;
            df_add(A[sidx], B[sidx], d, h, l);
            float *oh = reinterpret_cast<float *>(p.mix_hi[cur ^ 1]);
            float *ol = reinterpret_cast<float *>(p.mix_lo[cur ^ 1]);
            if (edge) {
              store_node<float, 2>(oh, p.pitch, p.nx, p.ny, p.bc, gi, gj, h);
              store_node<float, 2>(ol, p.pitch, p.nx, p.ny, p.bc, gi, gj, l);
            } else {
              oh[g] = h;
              ol[g] = l;
            }
          } else {
            const float d = (p.stage == 1) ? dtf * L : 0.25f * fmaf(dtf, L, C[sidx]);
            float *o = reinterpret_cast<float *>(p.out0);
            if (edge) store_node<float, 2>(o, p.pitch, p.nx, p.ny, p.bc, gi, gj, d);
            else o[g] = d;
          }
        } else {
          const float src = A[sidx];
          float outv;
          if (p.stage == 1) {
            outv = fmaf(dtf, L, src);
          } else if (p.stage == 2) {
            outv = fmaf(0.75f, B[sidx], 0.25f * fmaf(dtf, L, src));
          } else {
            outv = fmaf(1.0f / 3.0f, B[sidx], (2.0f / 3.0f) * fmaf(dtf, L, src));
          }
          float *o = reinterpret_cast<float *>(p.out0);
          if (edge) store_node<float, 2>(o, p.pitch, p.nx, p.ny, p.bc, gi, gj, outv);
          else o[g] = outv;
        }
      };
      sweep_stream<K, W>(v_at, dir == 0 ? rdx : rdy, 0.5f * (dir == 0 ? dx : dy), eps, emit);
      if (dir == 0) __syncthreads();
    }
    __syncthreads();  // raw[buf], dX, dY, su are free for the next tile
  }

  // ---- grid maximum of alpha: one atomic per CTA
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, o));
    amy = fmaxf(amy, __shfl_xor_sync(0xffffffffu, amy, o));
  }
  const int anybad = __syncthreads_or(bad ? 1 : 0);
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
    if (anybad) atomicOr(&st->err, 1);
    if (p.write_slot >= 0) {
      atomicMax(&st->alpha_bits[p.write_slot][0], double_to_bits((double)amx));
      atomicMax(&st->alpha_bits[p.write_slot][1], double_to_bits((double)amy));
    }
    __threadfence();
    const unsigned int prev = atomicAdd(&st->counter, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && tid == 0) {
    __threadfence();
    st->counter = 0;
    if (p.zero_slot >= 0) {
      st->alpha_bits[p.zero_slot][0] = 0ull;
      st->alpha_bits[p.zero_slot][1] = 0ull;
    }
    if (p.stage == 1 && p.loop_mode != LOOP_STAGE) {
      st->dt = s_dt;
      st->last = s_lastflag;
    }
    if (p.stage == 3) {
      if (PREC == P_MIXED) st->cur = cur ^ 1;
      if (p.loop_mode != LOOP_STAGE) {
        st->t = st->last ? st->t_final : st->t + st->dt;
        st->steps += 1;
      }
    }
  }
}

}  // namespace alw
