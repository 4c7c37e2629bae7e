// The fused RK-stage kernel (see alw_device.cuh for the arithmetic).
#pragma once
#include "alw_device.cuh"

namespace alw {

template <int PREC> struct Types;
template <> struct Types<P_F64> { using S = double; using C = double; };
template <> struct Types<P_F32> { using S = float; using C = float; };
template <> struct Types<P_MIXED> { using S = float; using C = float; };

// SMALL (FP64 2D grids too small to fill the GPU with the default tiles): 16 x 16 tiles with 4-node
// sweep segments (SMALL = 1), or 2-node segments (SMALL = 2: twice the threads per tile, for grids
// whose 16 x 16 tiles are fewer than the SMs).
template <int PREC, int DIM, int SMALL = 0> struct Shape {
  static constexpr int TX = (DIM == 2) ? (SMALL ? 16 : Tile<PREC>::TX) : TX1D;
  static constexpr int TY = (DIM == 2) ? (SMALL ? 16 : Tile<PREC>::TY) : 1;
  static constexpr int K = (DIM == 2) ? (SMALL == 2 ? 2 : SMALL == 1 ? 4 : Tile<PREC>::K) : K1D;
  static constexpr int NT = (TX / K) * TY;          // threads per CTA
  static constexpr int SW = TX + 8;                 // smem row: GX halo on each side
  static constexpr int SH = (DIM == 2) ? TY + 6 : 1;
  static constexpr int NARR = (PREC == P_MIXED) ? 3 : 1;
  static constexpr size_t smem_bytes() {
    return (size_t)NARR * SH * SW * sizeof(typename Types<PREC>::S) +
           (DIM == 2 ? (size_t)TY * TX * 2 * sizeof(typename Types<PREC>::C) : 0);
  }
};

template <int PREC, int DIM, int WEIGHTS, int SMALL>
__global__ void __launch_bounds__(Shape<PREC, DIM, SMALL>::NT) stage_kernel(const StageParams p) {
  using S = typename Types<PREC>::S;
  using C = typename Types<PREC>::C;
  using Sh = Shape<PREC, DIM, SMALL>;
  constexpr int TX = Sh::TX, TY = Sh::TY, K = Sh::K, NT = Sh::NT, SW = Sh::SW, SH = Sh::SH;

  DevState *st = p.state;
  if (p.loop_mode == LOOP_STEP_TO && !(st->t < st->t_final)) return;
  if (st->err) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  S *s_a = reinterpret_cast<S *>(smem_raw);            // phi (or hi)
  S *s_b = s_a + SH * SW;                               // lo (MIXED)
  S *s_c = s_b + SH * SW;                               // previous stage's increment (MIXED)
  C *s_u = reinterpret_cast<C *>(smem_raw + (size_t)Sh::NARR * SH * SW * sizeof(S));
  __shared__ double s_red[2][NT / 32];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int tx0 = blockIdx.x * TX, ty0 = blockIdx.y * TY;
  const int cur = (PREC == P_MIXED) ? st->cur : 0;

  // ---- time step of this stage
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
    double den = ax / p.lx;
    if (DIM == 2) den += ay / p.ly;
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
  // ---- alpha of the flux when it is one value for the whole grid
  C fax = C(0), fay = C(0);
  const bool local_alpha = (p.alpha_mode == A_LOCAL_LAGGED || p.alpha_mode == A_LOCAL_EXACT);
  if (p.alpha_mode == A_FIXED) {
    fax = C(p.alpha_fixed[0]);
    fay = C(p.alpha_fixed[1]);
  } else if (!local_alpha && p.read_slot >= 0) {
    fax = C(bits_to_double(st->alpha_bits[p.read_slot][0]));
    fay = C(bits_to_double(st->alpha_bits[p.read_slot][1]));
  }

  // ---- load the tile and its halo (row 0 of smem = interior row ty0-3, col 0 = interior col tx0-4)
  const S *ga = reinterpret_cast<const S *>(PREC == P_MIXED ? p.mix_hi[cur] : p.src0);
  const S *gb = reinterpret_cast<const S *>(PREC == P_MIXED ? p.mix_lo[cur] : nullptr);
  const S *gc = reinterpret_cast<const S *>(p.src2);
  for (int idx = tid; idx < SH * SW; idx += NT) {
    const int r = idx / SW, c = idx - r * SW;
    const size_t g = (size_t)((DIM == 2) ? ty0 + r : 0) * p.pitch + tx0 + c;
    s_a[idx] = ga[g];
    if (PREC == P_MIXED) {
      s_b[idx] = gb[g];
      if (gc) s_c[idx] = gc[g];
    }
  }
  // MIXED: the stage's input is hi + X, X = the low part of phi^n (stage 1) or the increment array of the
  // previous stage, which holds the low part as well (stages 2 and 3; see finish_node)
  const S *s_x = gc ? s_c : s_b;
  __syncthreads();

  const C dx = C(p.dx), rdx = C(p.rdx), eps = C(p.eps);
  // Delta^+ phi between smem cells i0 and i1 (same row or column)
  auto diff = [&](int i0, int i1, C rd) -> C {
    if (PREC == P_MIXED) {
      return ((s_a[i1] - s_a[i0]) + (s_x[i1] - s_x[i0])) * rd;
    } else {
      return C(s_a[i1] - s_a[i0]) * rd;
    }
  };

  C amx = C(0), amy = C(0);
  bool bad = false;

  // RK combination, store, and alpha bookkeeping for node (lx, ly) of the tile
  auto finish_node = [&](int lxn, int lyn, C um, C up, C vm, C vp) {
    const int gi = tx0 + lxn, gj = ty0 + lyn;
    if (gi >= p.nx || gj >= p.ny) return;
    C ax, ay;
    const C xn = C(p.xlo + gi * p.dx), yn = C(p.ylo + gj * p.dy);
    node_alpha<C>(p.ham, um, up, vm, vp, xn, yn, ax, ay);
    if (!(isfinite(ax) && isfinite(ay))) bad = true;
    amx = fmax(amx, ax);
    amy = fmax(amy, ay);
    if (p.stage == 0) return;
    const C aX = local_alpha ? ax : fax, aY = local_alpha ? ay : fay;
    const C H = ham_value<C>(p.ham, C(0.5) * (up + um), C(0.5) * (vp + vm), xn, yn);
    const C L = -((H - aX * C(0.5) * (up - um)) - aY * C(0.5) * (vp - vm));
    const int sidx = ((DIM == 2) ? lyn + 3 : 0) * SW + lxn + 4;
    if (PREC == P_MIXED) {
      // phi^n = hi + lo and phi_k = hi + e_k with e_k = lo + (phi_k - phi^n):
      //   e_1 = lo + dt L,  e_2 = 3/4 lo + 1/4 (e_1 + dt L),  phi^{n+1} = hi + lo + 2/3 (e_2 + dt L - lo)
      const float dL = float(dt) * float(L);
      const float lo = float(s_b[sidx]);
      if (p.stage == 1) {
        store_node<float, DIM>(reinterpret_cast<float *>(p.out0), p.pitch, p.nx, p.ny, p.bc, gi, gj, lo + dL);
      } else if (p.stage == 2) {
        const float d = fmaf(0.75f, lo, 0.25f * (float(s_c[sidx]) + dL));
        store_node<float, DIM>(reinterpret_cast<float *>(p.out0), p.pitch, p.nx, p.ny, p.bc, gi, gj, d);
      } else {
        const float d = (2.0f / 3.0f) * ((float(s_c[sidx]) + dL) - lo);
        float h, l;
        df_add(float(s_a[sidx]), float(s_b[sidx]), d, h, l);
        store_node<float, DIM>(reinterpret_cast<float *>(p.mix_hi[cur ^ 1]), p.pitch, p.nx, p.ny, p.bc, gi, gj, h);
        store_node<float, DIM>(reinterpret_cast<float *>(p.mix_lo[cur ^ 1]), p.pitch, p.nx, p.ny, p.bc, gi, gj, l);
      }
    } else {
      const C src = C(s_a[sidx]);
      C outv;
      if (p.stage == 1) {
        outv = src + C(dt) * L;
      } else {
        const size_t g = (size_t)(gj + ((DIM == 2) ? GY : 0)) * p.pitch + gi + GX;
        const C base = C(reinterpret_cast<const S *>(p.base0)[g]);
        if (p.stage == 2) outv = C(0.75) * base + C(0.25) * (src + C(dt) * L);
        else outv = base / C(3) + C(2) * (src + C(dt) * L) / C(3);
      }
      store_node<S, DIM>(reinterpret_cast<S *>(p.out0), p.pitch, p.nx, p.ny, p.bc, gi, gj, S(outv));
    }
  };

  // ---- phase X: each thread sweeps K consecutive nodes of one row
  {
    constexpr int SEGS = TX / K;
    const int r = tid / SEGS, seg = tid - r * SEGS;
    const int srow = (DIM == 2) ? r + 3 : 0;
    const int base_i = srow * SW + seg * K + 1;     // smem index of node x = seg*K - 3
    C v[K + 5];
#pragma unroll
    for (int m = 0; m < K + 5; ++m) v[m] = diff(base_i + m, base_i + m + 1, rdx);
    C dm[K], dp[K];
    weno_sweep<C, K, WEIGHTS>(v, rdx, dx, eps, dm, dp);
    if (DIM == 2) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        s_u[2 * (r * TX + seg * K + q)] = dm[q];
        s_u[2 * (r * TX + seg * K + q) + 1] = dp[q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < K; ++q) finish_node(seg * K + q, 0, dm[q], dp[q], C(0), C(0));
    }
  }
  if (DIM == 2) {
    __syncthreads();
    // ---- phase Y: each thread sweeps K consecutive nodes of one column
    const int x = tid % TX, seg = tid / TX;
    const int col = x + 4;
    const C dy = C(p.dy), rdy = C(p.rdy);
    C v[K + 5];
#pragma unroll
    for (int m = 0; m < K + 5; ++m) v[m] = diff((seg * K + m) * SW + col, (seg * K + m + 1) * SW + col, rdy);
    C vm[K], vp[K];
    weno_sweep<C, K, WEIGHTS>(v, rdy, dy, eps, vm, vp);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int y = seg * K + q;
      finish_node(x, y, s_u[2 * (y * TX + x)], s_u[2 * (y * TX + x) + 1], vm[q], vp[q]);
    }
  }

  // ---- grid maximum of alpha: warp shuffle, then one atomicMax per CTA
  double mx = double(amx), my = double(amy);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  const int anybad = __syncthreads_or(bad ? 1 : 0);
  if ((tid & 31) == 0) {
    s_red[0][tid >> 5] = mx;
    s_red[1][tid >> 5] = my;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < NT / 32; ++w) {
      mx = fmax(mx, s_red[0][w]);
      my = fmax(my, s_red[1][w]);
    }
    if (anybad) atomicOr(&st->err, 1);
    if (p.write_slot >= 0) {
      atomicMax(&st->alpha_bits[p.write_slot][0], double_to_bits(mx));
      atomicMax(&st->alpha_bits[p.write_slot][1], double_to_bits(my));
    }
    // last-CTA epilogue: every other CTA has finished reading the state
    __threadfence();
    const unsigned int total = gridDim.x * gridDim.y;
    const unsigned int prev = atomicAdd(&st->counter, 1u);
    s_last = (prev == total - 1);
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
      st->dt = dt;
      st->last = last;
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
