// Internal host/device declarations of the WENO-L CUDA library (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>

namespace alw {

// Storage/arithmetic variants of the stage kernel.
enum Prec : int { P_F64 = 0, P_F32 = 1, P_MIXED = 2 };

// How stage kernels treat time.
enum LoopMode : int {
  LOOP_STEP_TO = 0,   // dt from the CFL rule clipped to t_final; kernels exit once t >= t_final
  LOOP_ADVANCE = 1,   // dt from the CFL rule, never clipped, never exits
  LOOP_STAGE = 2      // dt taken from DevState::dt as set by the host; t and steps untouched
};

// Device-resident solver state (one per instance).
struct DevState {
  double t;
  double t_final;
  double dt;                         // dt of the current step (written by stage 1)
  unsigned long long alpha_bits[4][2]; // grid-maximum reductions: ring slots 0..2 (stage s writes
                                       // slot s-1), slot 3 = exact pass; bit patterns of doubles >= 0
  long long steps;
  int last;                          // current step is the clipped final one
  int err;                           // bit 0: non-finite dH/dp seen
  int cur;                           // MIXED: which phi^n buffer pair is current
  unsigned int counter;              // CTA arrival counter for the last-CTA epilogue
  int pad[2];
};

// Parameters of one stage launch (plain data, passed by value).
struct StageParams {
  int nx, ny;            // interior nodes
  int pitch;             // elements per padded row
  int tiles_x, tiles_y;  // tile grid
  int dim, bc, ham, weights, alpha_mode, loop_mode;
  int stage;             // 1, 2, 3; 0 = reduction pass only
  int src_of;            // stage whose source array is read (= stage, or the stage a reduction precedes)
  int read_slot;         // slot holding the alpha this stage uses (flux/dt), -1 none
  int write_slot;        // slot this stage reduces into
  int zero_slot;         // slot the epilogue clears for a later stage, -1 none
  int dt_slot;           // slot the stage-1 dt rule reads (lagged: 2, exact: 3)
  double dx, dy, rdx, rdy, eps;
  double xlo, ylo;       // coordinates of node (0, 0) (position-dependent Hamiltonians)
  double cfl, lx, ly;    // dt = cfl / (ax/lx + ay/ly)
  double alpha_fixed[2];
  double dt_value;       // LOOP_STAGE: the dt of this stage
  int small_tiles;       // FP64 2D: 0 default tiles; 16 x 16 tiles with 4-node (1) or 2-node (2) segments
  // buffers: padded arrays whose interior origin is at row GY, column GX
  const void *src0, *src1, *src2;  // stencil source (F64/F32: src0; MIXED: hi, lo, previous increment or null)
  const void *base0, *base1;       // phi^n at the node (F64/F32: base0; MIXED: hi, lo; stage>=2)
  void *out0, *out1;               // outputs (F64/F32: out0; MIXED: increment, or hi/lo at stage 3)
  void *mix_hi[2], *mix_lo[2];     // MIXED: the two phi^n buffer pairs (selected by DevState::cur)
  DevState *state;
};

struct GhostParams {
  int nx, ny, pitch, dim, bc, prec;
  void *a0, *a1;        // arrays to fill (F64/F32: a0; MIXED hi/lo pair: a0, a1, or increment: a0 only)
  int mixed_pair;       // MIXED: 1 if (a0, a1) is a hi/lo pair, 0 if a0 is an increment array
  DevState *state;      // MIXED: the pair is mix_*[cur] when non-null; an increment's high part is mix_hi[cur]
  void *mix_hi[2], *mix_lo[2];
};

// Ghost widths of the padded layout (rows/columns before the interior).
constexpr int GX = 4;   // 3 used; 4 keeps TMA box starts 16-byte aligned
constexpr int GY = 3;

// Tile shapes per variant.
template <int PREC> struct Tile;
template <> struct Tile<P_F64> { static constexpr int TX = 32, TY = 16, K = 4; };
template <> struct Tile<P_F32> { static constexpr int TX = 64, TY = 32, K = 8; };
template <> struct Tile<P_MIXED> { static constexpr int TX = 64, TY = 32, K = 8; };
constexpr int TX1D = 256;       // 1D tile width (one row)
constexpr int K1D = 8;

int tile_x(int prec, int dim);
int tile_y(int prec, int dim);

// Set the thread-local message returned by alw_last_error().
void set_last_error(const char *msg);

// Launchers (defined per precision in alw_stage_*.cu); return cudaError_t as int.
int launch_stage_f64(const StageParams &p, void *stream);
int launch_stage_f32(const StageParams &p, void *stream);
int launch_stage_mixed(const StageParams &p, void *stream);
int launch_ghosts(const GhostParams &g, void *stream);
int launch_mixed_split(const double *src, void *hi, void *lo, int nx, int ny, int pitch, int dim, void *stream);
int launch_mixed_join(const void *hi, const void *lo, const void *delta, double *dst, int nx, int ny,
                      int pitch, int dim, void *stream);
int launch_pack(const void *padded, int prec_elem /*0 f64, 1 f32*/, void *dst, int dst_dtype, int nx, int ny,
                int pitch, int dim, void *stream);
int launch_unpack(const void *src, int src_dtype, void *padded, int prec_elem, int nx, int ny, int pitch,
                  int dim, void *stream);

}  // namespace alw
