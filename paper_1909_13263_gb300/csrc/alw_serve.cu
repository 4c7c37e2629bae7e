// Continuous-batching server for 2D HJ solves.
//
// Requests (grid, Hamiltonian, phi0, t_final) are queued by alw_server_submit.
// Two host threads share the device: a compute thread runs rounds -- a few RK3
// steps of every active instance together, one persistent launch per stage
// over the (instance, tile) work list of all of them -- and hands instances
// that reached their t_final to a copier thread, which, on its own stream and
// while rounds keep running, copies finished results out (freeing their slot
// and rows) and admits queued requests while a slot and enough of the
// device-memory budget are free (device-resident state in one arena whose size
// is the budget).  New instances join at the next round boundary.
// Requests that arrive while others are on the GPU therefore join the running
// batch; their stages interleave in the same launches.  Every instance follows
// the same arithmetic as a single solve, so a result does not depend on what
// else was resident.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/alweno.h"
#include "alw_internal.h"
#include "alw_params2d.h"

using namespace alw;

namespace {

alw_status serr(alw_status st, const char *fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return st;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator of row ranges inside the arena.
struct RowAlloc {
  std::map<long long, long long> free_;  // start -> length
  void init(long long rows) {
    free_.clear();
    if (rows > 0) free_[0] = rows;
  }
  long long take(long long n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const long long s = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[s + n] = len - n;
        return s;
      }
    }
    return -1;
  }
  void give(long long s, long long n) {
    auto it = free_.emplace(s, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  long long free_rows() const {
    long long t = 0;
    for (auto &kv : free_) t += kv.second;
    return t;
  }
};

struct Request {
  uint64_t id = 0;
  alw_grid grid{};
  int ham = 0;
  double t_final = 0;
  std::vector<double> phi0, result;
  int status = ALW_OK;
  int done = 0;
  int slot = -1;
  long long row_off = -1, rows = 0;
  int64_t steps = 0;
  int steps_cur = 0;  // MIXED: buffer pair holding the final phi
  bool primed = false;  // first lagged alpha computed (on the instance's first round)
  double t_submit = 0, t_admit = 0, t_done = 0;
};

// Instances of at most this many tiles join every round whatever the tile limit.
constexpr int kSmallTiles = 32;

}  // namespace

struct alw_server {
  alw_scheme scheme{};
  int prec = P_MIXED;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  int max_slots = 0, max_side = 0, steps_per_round = 2;
  int round_tiles = 0;  // tile limit of a round beyond its oldest instance (0: none)
  int grid_cap = 1;     // CTAs of the persistent stage kernel that fit on the device
  int pitch = 0;
  long long rows_total = 0;
  void *arr[6] = {};
  int narr = 0;
  CUtensorMap maps[6];
  RowAlloc rows;
  InstDesc *d_inst = nullptr;
  DevState *d_state = nullptr;
  DevState *h_state = nullptr;  // pinned
  int *d_tiles = nullptr;
  int tiles_cap = 0;
  double *d_stage = nullptr;    // staging for one phi (max_side^2 doubles)
  double *h_stage = nullptr;    // pinned
  std::vector<InstDesc> h_inst;
  std::vector<Request *> slot_req;
  std::vector<std::pair<void *, size_t>> allocs;
  // queue and bookkeeping
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Request *> queue;      // submitted, not yet admitted
  std::vector<Request *> ready;     // uploaded, waiting for the next round
  std::vector<Request *> finished;  // reached t_final, result not yet copied out
  std::map<uint64_t, Request *> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  int fatal = ALW_OK;
  cudaStream_t copy_stream = nullptr;  // uploads and downloads, overlapping the rounds
  std::thread worker, copier;
  alw_server_stats stats{};
};

namespace {

Stage2DParams server_params(const alw_server *s, int stage, int loop_mode, int ntiles) {
  Stage2DParams q;
  memset(&q, 0, sizeof q);
  memcpy(q.maps, s->maps, sizeof q.maps);
  StageParams &p = q.p;
  p.pitch = s->pitch;
  p.dim = 2;
  p.weights = s->scheme.weights;
  p.alpha_mode = s->scheme.alpha_mode == ALW_ALPHA_DEFAULT ? ALW_ALPHA_GLOBAL_LAGGED : s->scheme.alpha_mode;
  p.loop_mode = loop_mode;
  p.stage = stage;
  p.src_of = stage == 0 ? 1 : stage;
  p.eps = s->scheme.eps;
  p.cfl = s->scheme.cfl;
  p.alpha_fixed[0] = s->scheme.alpha_fixed[0];
  p.alpha_fixed[1] = s->scheme.alpha_fixed[1];
  p.dt_slot = 2;
  if (stage == 0) {
    p.read_slot = -1;
    p.write_slot = 2;
    p.zero_slot = -1;
  } else {
    p.read_slot = stage == 1 ? 2 : stage - 2;
    p.write_slot = stage - 1;
    p.zero_slot = stage % 3;
  }
  const int which = p.src_of;
  if (s->prec == P_MIXED) {
    p.mix_hi[0] = s->arr[0];
    p.mix_hi[1] = s->arr[1];
    p.mix_lo[0] = s->arr[2];
    p.mix_lo[1] = s->arr[3];
    if (stage == 1) p.out0 = s->arr[4];
    if (stage == 2) p.out0 = s->arr[5];
    q.map_a = 0;
    q.map_b = 2;
    q.map_c = which == 1 ? -1 : (which == 2 ? 4 : 5);
  } else {
    p.out0 = stage == 1 ? s->arr[1] : (stage == 2 ? s->arr[2] : (stage == 3 ? s->arr[0] : nullptr));
    q.map_a = which == 1 ? 0 : (which == 2 ? 1 : 2);
    q.map_b = stage >= 2 ? 0 : -1;
    q.map_c = -1;
  }
  q.ntiles = ntiles;
  q.states = s->d_state;
  q.insts = s->d_inst;
  q.tiles = s->d_tiles;
  q.done_count = nullptr;
  return q;
}

int launch(const alw_server *s, const Stage2DParams &q) {
  return s->prec == P_MIXED ? launch_stage2d_mixed(q, s->stream) : launch_stage2d_f32(q, s->stream);
}

long long rows_of(int ny) { return (long long)((ny + kTile2DY - 1) / kTile2DY) * kTile2DY + 2 * GY; }

// Upload a request into its slot and rows on the copy stream; returns a CUDA error code (0 on success).
int admit_one(alw_server *s, Request *r, int slot) {
  cudaStream_t cs = s->copy_stream;
  const int nx = r->grid.nx, ny = r->grid.ny;
  InstDesc &d = s->h_inst[slot];
  memset(&d, 0, sizeof d);
  d.nx = nx;
  d.ny = ny;
  d.tiles_x = (nx + kTile2DX - 1) / kTile2DX;
  d.tiles_y = (ny + kTile2DY - 1) / kTile2DY;
  d.ntiles = d.tiles_x * d.tiles_y;
  d.row_off = (int)r->row_off;
  d.ham = r->ham;
  d.bc = ALW_BC_PERIODIC;
  const double dx = (r->grid.xhi - r->grid.xlo) / nx, dy = (r->grid.yhi - r->grid.ylo) / ny;
  d.dx = (float)dx;
  d.dy = (float)dy;
  d.rdx = (float)(1.0 / dx);
  d.rdy = (float)(1.0 / dy);
  d.xlo = (float)r->grid.xlo;
  d.ylo = (float)r->grid.ylo;
  d.lx = s->scheme.dt_mode == ALW_DT_DX53 ? std::pow(dx, 5.0 / 3.0) : dx;
  d.ly = s->scheme.dt_mode == ALW_DT_DX53 ? std::pow(dy, 5.0 / 3.0) : dy;
  d.st = s->d_state + slot;
  const size_t n = (size_t)nx * ny;
  cudaError_t e = cudaMemcpyAsync(s->d_stage, r->phi0.data(), n * sizeof(double), cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return (int)e;
  const size_t off = (size_t)r->row_off * s->pitch;
  int le;
  if (s->prec == P_MIXED)
    le = launch_mixed_split(s->d_stage, (float *)s->arr[0] + off, (float *)s->arr[2] + off, nx, ny, s->pitch, 2, cs);
  else
    le = launch_unpack(s->d_stage, 0, (float *)s->arr[0] + off, 1, nx, ny, s->pitch, 2, cs);
  if (le) return le;
  GhostParams g;
  memset(&g, 0, sizeof g);
  g.nx = nx;
  g.ny = ny;
  g.pitch = s->pitch;
  g.dim = 2;
  g.bc = ALW_BC_PERIODIC;
  g.prec = s->prec;
  if (s->prec == P_MIXED) {
    g.mixed_pair = 1;
    g.a0 = (float *)s->arr[0] + off;
    g.a1 = (float *)s->arr[2] + off;
  } else {
    g.a0 = (float *)s->arr[0] + off;
  }
  le = launch_ghosts(g, cs);
  if (le) return le;
  DevState z;
  memset(&z, 0, sizeof z);
  z.t_final = r->t_final;
  e = cudaMemcpyAsync(s->d_state + slot, &z, sizeof(DevState), cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return (int)e;
  e = cudaMemcpyAsync(s->d_inst + slot, &d, sizeof(InstDesc), cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaStreamSynchronize(cs);  // the staging buffer and z are reused
}

// Copy a finished instance's phi into its request on the copy stream.
int retire_one(alw_server *s, Request *r, int slot, int cur) {
  cudaStream_t cs = s->copy_stream;
  const InstDesc &d = s->h_inst[slot];
  const size_t n = (size_t)d.nx * d.ny, off = (size_t)d.row_off * s->pitch;
  int le;
  if (s->prec == P_MIXED)
    le = launch_mixed_join((float *)s->arr[cur] + off, (float *)s->arr[2 + cur] + off, nullptr, s->d_stage, d.nx, d.ny,
                           s->pitch, 2, cs);
  else
    le = launch_pack((float *)s->arr[0] + off, 1, s->d_stage, 0, d.nx, d.ny, s->pitch, 2, cs);
  if (le) return le;
  r->result.resize(n);
  cudaError_t e = cudaMemcpyAsync(r->result.data(), s->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  return (int)e;
}

void set_fatal(alw_server *s, int code) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->fatal = ALW_ECUDA;
  set_last_error(cudaGetErrorString((cudaError_t)code));
  s->cv.notify_all();
  s->done_cv.notify_all();
}

// Copier thread: retires finished instances and admits queued requests, on its own stream,
// while the compute thread runs rounds.
void copier_main(alw_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request *> fin;
    Request *adm = nullptr;
    int adm_slot = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto can_admit = [&]() -> bool {
        if (s->queue.empty()) return false;
        for (int i = 0; i < s->max_slots; ++i)
          if (!s->slot_req[i]) return true;
        return false;
      };
      s->cv.wait(lk, [&] { return s->stop || s->fatal || !s->finished.empty() || can_admit(); });
      if (s->stop || s->fatal) return;
      fin.swap(s->finished);
      if (fin.empty() && can_admit()) {
        Request *r = s->queue.front();
        const long long need = rows_of(r->grid.ny);
        const long long at = s->rows.take(need);
        if (at >= 0) {  // FIFO: otherwise wait for a retirement to free rows
          int slot = 0;
          while (s->slot_req[slot]) ++slot;
          s->queue.pop_front();
          r->slot = slot;
          r->row_off = at;
          r->rows = need;
          r->t_admit = now_s();
          s->slot_req[slot] = r;
          s->stats.admitted++;
          adm = r;
          adm_slot = slot;
        } else if (s->finished.empty()) {
          // nothing to retire and no room: wait for the compute thread to finish an instance
          s->cv.wait(lk, [&] { return s->stop || s->fatal || !s->finished.empty(); });
          continue;
        }
      }
      s->stats.queued = (int64_t)s->queue.size();
    }
    for (Request *r : fin) {
      const int re = r->status == ALW_OK ? retire_one(s, r, r->slot, r->steps_cur) : 0;
      if (re) {
        set_fatal(s, re);
        return;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_done = now_s();
      r->done = 1;
      s->rows.give(r->row_off, r->rows);
      s->slot_req[r->slot] = nullptr;
      s->stats.completed++;
      s->done_cv.notify_all();
      s->cv.notify_all();
    }
    if (adm) {
      const int e = admit_one(s, adm, adm_slot);
      if (e) {
        set_fatal(s, e);
        return;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->ready.push_back(adm);
      s->cv.notify_all();
    }
  }
}

// Compute thread: rounds of RK steps over every active instance.
void worker_main(alw_server *s) {
  cudaSetDevice(s->device);
  std::vector<int> list, new_tiles, tmp;
  std::vector<Request *> active, round;  // active: in admission order
  for (;;) {
    std::vector<Request *> fresh;
    int steps = 1, tile_limit = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || s->fatal || !active.empty() || !s->ready.empty(); });
      if (s->stop || s->fatal) return;
      fresh.swap(s->ready);
      steps = s->steps_per_round;
      tile_limit = s->round_tiles;
    }
    for (Request *r : fresh) active.push_back(r);
    // members of this round, oldest first: the oldest always; the others while the round's
    // tiles stay within the limit, and small instances always.  Large solves then run in
    // arrival order (as one at a time would), with the small ones beside them.
    // under load the limit grows to half of the resident tiles: fuller launches and fewer rounds
    // when many instances wait, arrival order when few do
    if (tile_limit > 0) {
      long long resident = 0;
      for (Request *r : active) resident += s->h_inst[r->slot].ntiles;
      tile_limit = (int)std::max<long long>(tile_limit, resident / 2);
    }
    round.clear();
    long long round_tiles = 0;
    bool any_new = false;
    for (Request *r : active) {
      const int nt = s->h_inst[r->slot].ntiles;
      if (round.empty() || tile_limit <= 0 || round_tiles + nt <= tile_limit || nt <= kSmallTiles) {
        round.push_back(r);
        round_tiles += nt;
        any_new |= !r->primed;
      }
    }
    // round length: long enough to amortise the round trip, short enough that the first
    // member to finish is retired promptly (its remaining steps, at most 16); short while
    // new instances are joining
    if (!any_new) {
      double rem_min = 1e30;
      for (Request *r : round) {
        const DevState &ds = s->h_state[r->slot];
        if (ds.dt > 0.0) rem_min = std::min(rem_min, std::ceil((ds.t_final - ds.t) / ds.dt));
      }
      if (rem_min < 1e29) steps = std::max(steps, std::min(16, (int)rem_min));
    }
    // work lists of the round, one group per Hamiltonian (each launch runs that Hamiltonian's own
    // kernel), each in admission order and laid out over the CTAs in blocks of 4 entries (fewer
    // instance changes per CTA): first the new instances' first-alpha pass, then the steps
    struct Seg {
      int off, n, kind;
    };
    std::vector<Seg> prime_segs, step_segs;
    list.clear();
    auto add_groups = [&](bool only_new, std::vector<Seg> &segs) {
      for (int kind = 0; kind < 16; ++kind) {
        new_tiles.clear();
        for (Request *r : round)
          if (r->ham == kind && (!only_new || !r->primed))
            for (int t = 0; t < s->h_inst[r->slot].ntiles; ++t) new_tiles.push_back(r->slot * 65536 + t);
        if (new_tiles.empty()) continue;
        cta_blocks(new_tiles, stage2d_grid((int)new_tiles.size(), 0, s->grid_cap), 4, tmp);
        segs.push_back({(int)list.size(), (int)tmp.size(), kind});
        list.insert(list.end(), tmp.begin(), tmp.end());
      }
    };
    add_groups(true, prime_segs);
    add_groups(false, step_segs);
    for (Request *r : round) r->primed = true;
    cudaError_t e = cudaMemcpyAsync(s->d_tiles, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    s->stream);
    int le = 0;
    for (const Seg &g : prime_segs) {  // first lagged alpha of the new instances
      if (e != cudaSuccess || le) break;
      Stage2DParams q = server_params(s, 0, LOOP_ADVANCE, g.n);
      q.tiles = s->d_tiles + g.off;
      q.batch_kind1 = g.kind + 1;
      le = launch(s, q);
    }
    for (int k = 0; k < steps && e == cudaSuccess && !le; ++k)
      for (int stage = 1; stage <= 3 && !le; ++stage)
        for (const Seg &g : step_segs) {
          if (le) break;
          Stage2DParams q = server_params(s, stage, LOOP_STEP_TO, g.n);
          q.tiles = s->d_tiles + g.off;
          q.batch_kind1 = g.kind + 1;
          le = launch(s, q);
        }
    if (e == cudaSuccess && !le)
      e = cudaMemcpyAsync(s->h_state, s->d_state, sizeof(DevState) * s->max_slots, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && !le) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess || le) {
      set_fatal(s, e != cudaSuccess ? (int)e : le);
      return;
    }
    // instances that reached t_final (or failed) leave the active set for the copier
    std::vector<Request *> keep, done;
    for (Request *r : active) {
      const DevState &ds = s->h_state[r->slot];
      if (ds.t < ds.t_final && !ds.err) {
        keep.push_back(r);
      } else {
        r->status = ds.err ? ALW_ENONFINITE : ALW_OK;
        r->steps = ds.steps;
        r->steps_cur = ds.cur;
        done.push_back(r);
      }
    }
    active.swap(keep);
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.rounds++;
    if (!done.empty()) {
      for (Request *r : done) s->finished.push_back(r);
      s->cv.notify_all();
    }
  }
}

}  // namespace

extern "C" {

alw_status alw_server_create(const alw_scheme *scheme, size_t hbm_budget_bytes, int32_t max_slots, int32_t max_side,
                             void *cuda_stream, alw_server **out) {
  if (!scheme || !out) return serr(ALW_EINVAL, "NULL argument");
  *out = nullptr;
  if (scheme->precision != ALW_PREC_MIXED && scheme->precision != ALW_PREC_FP32)
    return serr(ALW_EINVAL, "the server runs the float kernels: precision must be FP32 or MIXED");
  if (scheme->alpha_mode != ALW_ALPHA_DEFAULT && scheme->alpha_mode != ALW_ALPHA_GLOBAL_LAGGED &&
      scheme->alpha_mode != ALW_ALPHA_LOCAL_LAGGED && scheme->alpha_mode != ALW_ALPHA_FIXED)
    return serr(ALW_EINVAL, "the server supports the lagged and fixed alpha modes");
  if (max_slots < 1 || max_slots > 32768 || max_side < 8 || max_side > 16384) return serr(ALW_EINVAL, "bad limits");
  if (!(scheme->eps > 0.0) || !(scheme->cfl > 0.0)) return serr(ALW_EINVAL, "eps and cfl must be > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return serr(ALW_ECUDA, "no CUDA device");
  }
  alw_server *s = new (std::nothrow) alw_server();
  if (!s) return serr(ALW_ENOMEM, "host allocation failed");
  cudaGetDevice(&s->device);
  s->scheme = *scheme;
  s->prec = scheme->precision == ALW_PREC_MIXED ? P_MIXED : P_F32;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->max_side = max_side;
  s->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (!s->stream) {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return serr(ALW_ECUDA, "stream creation failed");
    }
    s->own_stream = true;
  }
  auto fail_destroy = [&](alw_status st) {
    alw_server_destroy(s);
    return st;
  };
  s->pitch = ((max_side + kTile2DX - 1) / kTile2DX) * kTile2DX + 2 * GX;
  s->narr = s->prec == P_MIXED ? 6 : 3;
  const int tiles_max = ((max_side + kTile2DX - 1) / kTile2DX) * ((max_side + kTile2DY - 1) / kTile2DY);
  // fixed per-server memory first, the rest of the budget is the arena
  const size_t fixed = sizeof(InstDesc) * max_slots + sizeof(DevState) * max_slots +
                       sizeof(int) * (size_t)max_slots * tiles_max + sizeof(double) * (size_t)max_side * max_side;
  const size_t per_row = (size_t)s->pitch * sizeof(float) * s->narr;
  if (hbm_budget_bytes <= fixed + per_row * rows_of(max_side))
    return fail_destroy(serr(ALW_EBUDGET, "budget below one maximal instance (%zu bytes needed)",
                             fixed + per_row * rows_of(max_side)));
  s->rows_total = (long long)((hbm_budget_bytes - fixed) / per_row);
  if (s->rows_total > (1ll << 31) - 1) s->rows_total = (1ll << 31) - 1;
  s->rows.init(s->rows_total);
  for (int i = 0; i < s->narr; ++i) {
    const size_t bytes = (size_t)s->pitch * sizeof(float) * (size_t)s->rows_total;
    s->arr[i] = dev_alloc(bytes, s->stream);
    if (!s->arr[i]) return fail_destroy(serr(ALW_ENOMEM, "device allocation of %zu bytes failed", bytes));
    s->allocs.emplace_back(s->arr[i], bytes);
    if (cudaMemsetAsync(s->arr[i], 0, bytes, s->stream) != cudaSuccess) return fail_destroy(serr(ALW_ECUDA, "memset"));
    const int r = encode_tile_map(&s->maps[i], s->arr[i], s->pitch, s->rows_total);
    if (r) return fail_destroy(serr(ALW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", r));
  }
  auto grab = [&](size_t bytes) -> void * {
    void *p = dev_alloc(bytes, s->stream);
    if (p) s->allocs.emplace_back(p, bytes);
    return p;
  };
  s->tiles_cap = 2 * max_slots * tiles_max;  // new instances' tiles, then the whole work list
  s->d_inst = (InstDesc *)grab(sizeof(InstDesc) * max_slots);
  s->d_state = (DevState *)grab(sizeof(DevState) * max_slots);
  s->d_tiles = (int *)grab(sizeof(int) * (size_t)s->tiles_cap);
  s->d_stage = (double *)grab(sizeof(double) * (size_t)max_side * max_side);
  if (!s->d_inst || !s->d_state || !s->d_tiles || !s->d_stage) return fail_destroy(serr(ALW_ENOMEM, "device allocation failed"));
  if (cudaHostAlloc((void **)&s->h_state, sizeof(DevState) * max_slots, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void **)&s->h_stage, sizeof(double) * (size_t)max_side * max_side, cudaHostAllocDefault) !=
          cudaSuccess) {
    cudaGetLastError();
    return fail_destroy(serr(ALW_ENOMEM, "pinned host allocation failed"));
  }
  memset(s->h_state, 0, sizeof(DevState) * max_slots);
  if (cudaMemsetAsync(s->d_state, 0, sizeof(DevState) * max_slots, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return fail_destroy(serr(ALW_ECUDA, "initialisation failed"));
  s->h_inst.assign(max_slots, InstDesc{});
  s->slot_req.assign(max_slots, nullptr);
  s->stats.arena_rows = s->rows_total;
  if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail_destroy(serr(ALW_ECUDA, "stream creation failed"));
  {  // default tile limit of a round: four waves of the persistent stage kernel
    const int cap = s->prec == P_MIXED ? stage2d_grid_cap_mixed(scheme->weights) : stage2d_grid_cap_f32(scheme->weights);
    s->grid_cap = std::max(cap, 1);
    s->round_tiles = 4 * s->grid_cap;
  }
  s->worker = std::thread(worker_main, s);
  s->copier = std::thread(copier_main, s);
  *out = s;
  return ALW_OK;
}

alw_status alw_server_set_round_tiles(alw_server *s, int32_t tiles) {
  if (!s || tiles < 0) return serr(ALW_EINVAL, "the tile limit must be >= 0");
  std::lock_guard<std::mutex> lk(s->mu);
  s->round_tiles = tiles;
  return ALW_OK;
}

alw_status alw_server_set_round_steps(alw_server *s, int32_t steps) {
  if (!s || steps < 1 || steps > 64) return serr(ALW_EINVAL, "steps per round must be 1..64");
  std::lock_guard<std::mutex> lk(s->mu);
  s->steps_per_round = steps;
  return ALW_OK;
}

alw_status alw_server_submit(alw_server *s, const alw_grid *grid, const alw_hamiltonian *ham, const double *host_phi0,
                             size_t n, double t_final, uint64_t *req_id) {
  if (!s || !grid || !ham || !host_phi0 || !req_id) return serr(ALW_EINVAL, "NULL argument");
  if (grid->dim != 2 || grid->bc != ALW_BC_PERIODIC || grid->nx < 1 || grid->ny < 1)
    return serr(ALW_EINVAL, "the server takes 2D periodic grids");
  if (grid->nx > s->max_side || grid->ny > s->max_side) return serr(ALW_EBUDGET, "grid larger than max_side");
  if (rows_of(grid->ny) > s->rows_total) return serr(ALW_EBUDGET, "grid larger than the memory budget");
  if (n != (size_t)grid->nx * grid->ny) return serr(ALW_EINVAL, "n = %zu but nx*ny = %zu", n, (size_t)grid->nx * grid->ny);
  if (ham->kind != ALW_H_BURGERS2D && ham->kind != ALW_H_NEGCOS2D && ham->kind != ALW_H_SIN2D &&
      ham->kind != ALW_H_EIKONAL2D)
    return serr(ALW_EINVAL, "the server takes 2D Hamiltonians");
  if (!std::isfinite(t_final) || t_final < 0.0) return serr(ALW_EINVAL, "bad t_final");
  if (!(grid->xhi > grid->xlo) || !(grid->yhi > grid->ylo)) return serr(ALW_EINVAL, "empty extent");
  Request *r = new (std::nothrow) Request();
  if (!r) return serr(ALW_ENOMEM, "host allocation failed");
  r->grid = *grid;
  r->ham = ham->kind;
  r->t_final = t_final;
  r->phi0.assign(host_phi0, host_phi0 + n);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal) {
    delete r;
    return serr((alw_status)s->fatal, "server stopped after an error");
  }
  r->id = s->next_id++;
  r->t_submit = now_s();
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  s->stats.submitted++;
  *req_id = r->id;
  s->cv.notify_one();
  return ALW_OK;
}

alw_status alw_server_poll(alw_server *s, uint64_t req_id, double timeout_s, int32_t *done, double *host_out,
                           size_t n, alw_request_info *info) {
  if (!s || !done) return serr(ALW_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return serr(ALW_ENOTFOUND, "no request %llu", (unsigned long long)req_id);
  Request *r = it->second;
  if (!r->done && timeout_s > 0.0)
    s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done || s->fatal; });
  if (!r->done && s->fatal) return serr((alw_status)s->fatal, "server stopped after an error");
  *done = r->done;
  if (!r->done) return ALW_OK;
  if (info) {
    info->status = r->status;
    info->steps = r->steps;
    info->queue_s = r->t_admit - r->t_submit;
    info->latency_s = r->t_done - r->t_submit;
  }
  if (host_out) {
    if (n != r->result.size()) return serr(ALW_EINVAL, "n = %zu but the result has %zu values", n, r->result.size());
    memcpy(host_out, r->result.data(), n * sizeof(double));
  }
  // a request whose result has been copied out is forgotten
  if (host_out) {
    const int st = r->status;
    s->reqs.erase(it);
    delete r;
    if (st != ALW_OK) return serr((alw_status)st, "request failed");
  }
  return ALW_OK;
}

alw_status alw_server_stats_get(alw_server *s, alw_server_stats *out) {
  if (!s || !out) return serr(ALW_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.free_rows = s->rows.free_rows();
  *out = s->stats;
  return ALW_OK;
}

alw_status alw_server_destroy(alw_server *s) {
  if (!s) return ALW_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->copier.joinable()) s->copier.join();
  cudaStreamSynchronize(s->stream);
  if (s->copy_stream) {
    cudaStreamSynchronize(s->copy_stream);
    cudaStreamDestroy(s->copy_stream);
  }
  for (auto &a : s->allocs) dev_free(a.first, a.second, s->stream);
  cudaStreamSynchronize(s->stream);
  if (s->h_state) cudaFreeHost(s->h_state);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  for (auto &kv : s->reqs) delete kv.second;
  if (s->own_stream) cudaStreamDestroy(s->stream);
  cudaGetLastError();
  delete s;
  return ALW_OK;
}

}  // extern "C"
