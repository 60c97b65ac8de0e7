// api.cu -- the C ABI of include/vplbm.h: validation, workspace carving,
// body placement (SIM polygon of Eq. defFf built on the host in FP64), step
// scheduling with CUDA-graph replay, and read-back of forces and fields.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "vplbm_internal.cuh"

using namespace vplbm;

namespace {

// An NVTX range around a call, for timelines taken with a profiler (the
// calls cost nothing measurable when no profiler is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

constexpr size_t kAlign = 256;
// Runs of steps are replayed from CUDA graphs of up to kGraphMax steps, one
// per length and per starting buffer: always 1, 2, 4, ..., 32 steps (any
// step count is then a sum of at most six launches per 63 steps), and any
// other length a caller prepares (vplbm_prepare) for runs of that length.
constexpr int kGraphMax = 32;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_bytes(int dtype) {
  switch (dtype) {
    case VPLBM_F64: return 8;
    case VPLBM_F32: return 4;
    case VPLBM_F16_OFS:
    case VPLBM_BF16_OFS:
    case VPLBM_F16_SR:
    case VPLBM_BF16_SR: return 2;
  }
  return 0;
}

struct Layout {
  size_t buf[2], prev[2], chi, sim_pts, sim_nodes, hist, body[2], region[2], sums, counts,
      dev_step, ticket, status, acc, rng, total;
};

int effective_max_sim(const vplbm_config &c) { return c.max_sim_points > 0 ? c.max_sim_points : 4096; }
int effective_hist(const vplbm_config &c) { return c.history_len > 0 ? c.history_len : 1024; }
int pitch_of(int nx) { return (int)align_up((size_t)nx, 64); }

// elements between two population planes: the padded rows plus an offset
// that keeps the nine planes from sharing address bits with each other
#ifndef VPLBM_PLANE_PAD
#define VPLBM_PLANE_PAD 0
#endif
int64_t plane_of(const vplbm_config &c) {
  return (int64_t)pitch_of(c.nx) * c.ny + VPLBM_PLANE_PAD;
}

Layout make_layout(const vplbm_config &c) {
  Layout l{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, kAlign);
    return at;
  };
  const size_t plane = (size_t)plane_of(c);
  const size_t fbytes = 9 * plane * elem_bytes(c.dtype);
  l.buf[0] = take(fbytes);
  l.buf[1] = take(fbytes);
  l.prev[0] = take(3 * (size_t)c.ny * sizeof(double));
  l.prev[1] = take(3 * (size_t)c.ny * sizeof(double));
  l.chi = take((size_t)pitch_of(c.nx) * (size_t)c.ny);
  const size_t ms = (size_t)effective_max_sim(c);
  l.sim_pts = take(ms * sizeof(SimPoint));
  l.sim_nodes = take(ms * sizeof(int32_t));
  l.hist = take((size_t)effective_hist(c) * kHistCols * sizeof(double));
  l.body[0] = take(sizeof(BodyState));
  l.body[1] = take(sizeof(BodyState));
  l.region[0] = take(sizeof(ForceRegion));
  l.region[1] = take(sizeof(ForceRegion));
  l.sums = take(6 * sizeof(double));
  l.counts = take(2 * sizeof(long long));
  l.dev_step = take(sizeof(long long));
  l.ticket = take(sizeof(unsigned int));
  l.status = take(sizeof(int32_t));
  l.acc = take(2 * kAccWords * sizeof(unsigned long long));  // by step parity
  l.rng = take(2 * sizeof(unsigned long long));                // rounding counter, by parity
  l.total = off;
  return l;
}

std::string g_err;  // failures of calls without a context (create / workspace_bytes)

std::string fmt(const char *f, ...) {
  char b[512];
  va_list ap;
  va_start(ap, f);
  vsnprintf(b, sizeof b, f, ap);
  va_end(ap);
  return b;
}

const char *check_config(const vplbm_config *c) {
  if (!c) return "config is NULL";
  if (c->nx < 3 || c->ny < 3) return "nx and ny must be >= 3";
  if ((int64_t)c->nx * c->ny > (int64_t)1 << 31) return "lattice too large";
  if (elem_bytes(c->dtype) == 0) return "unknown dtype";
  if (c->collision != VPLBM_BGK && c->collision != VPLBM_TRT) return "unknown collision";
  if (c->forcing != VPLBM_FORCING_PAPER && c->forcing != VPLBM_FORCING_SPLIT) return "unknown forcing";
  if (!(c->tau_plus > 0.5) || !std::isfinite(c->tau_plus)) return "tau_plus must be > 1/2";
  if (c->collision == VPLBM_TRT && !(c->lambda_trt > 0.0)) return "lambda_trt must be > 0";
  if (!(c->eta > 0.0)) return "eta must be > 0";
  if (c->sim_every < 0 || c->max_sim_points < 0 || c->history_len < 0) return "negative count";
  if (c->sim_order != 0 && c->sim_order != 1) return "sim_order must be 0 or 1";
  for (int k = 0; k < 2; ++k)
    if (!std::isfinite(c->u_in[k]) || !std::isfinite(c->body_force[k]) || !std::isfinite(c->u_ref[k]))
      return "non-finite velocity or force";
  if (c->u_ref[0] * c->u_ref[0] + c->u_ref[1] * c->u_ref[1] > 0.09) return "|u_ref| must be below 0.3";
  const int x0 = c->bc[0], x1 = c->bc[1], y0 = c->bc[2], y1 = c->bc[3];
  auto xok = [](int b) {
    return b == VPLBM_PERIODIC || b == VPLBM_INLET_BB || b == VPLBM_OUTLET_CONVECTIVE ||
           b == VPLBM_OUTLET_FREE || b == VPLBM_NOSLIP_BB;
  };
  auto yok = [](int b) { return b == VPLBM_PERIODIC || b == VPLBM_SYMMETRY || b == VPLBM_NOSLIP_BB; };
  if (!xok(x0) || !xok(x1) || !yok(y0) || !yok(y1)) return "side condition not allowed on that side";
  if (x0 == VPLBM_OUTLET_CONVECTIVE || x0 == VPLBM_OUTLET_FREE) return "outlets are x_hi conditions";
  if ((x0 == VPLBM_PERIODIC) != (x1 == VPLBM_PERIODIC)) return "x periodicity must hold on both sides";
  if ((y0 == VPLBM_PERIODIC) != (y1 == VPLBM_PERIODIC)) return "y periodicity must hold on both sides";
  return nullptr;
}

double naca_yt(double t, double xi) {
  return 5.0 * t *
         (0.2969 * sqrt(xi) - 0.1260 * xi - 0.3516 * (xi * xi) + 0.2843 * (xi * xi * xi) -
          0.1015 * (xi * xi * xi * xi));
}

// Closed counter-clockwise polygon on the body surface; one SIM point per
// edge at its midpoint with the outward normal and the edge length.
bool build_polygon(const vplbm_body &b, int n, std::vector<SimPoint> &pts) {
  std::vector<double> vx, vy;
  if (b.kind == VPLBM_BODY_DISK) {
    if (n < 3) return false;
    const double r = 0.5 * b.length;
    for (int k = 0; k < n; ++k) {
      const double th = 2.0 * M_PI * (double)k / (double)n;
      vx.push_back(r * cos(th));
      vy.push_back(r * sin(th));
    }
  } else if (b.kind == VPLBM_BODY_NACA4) {
    if (n < 5 || n % 2 == 0) return false;
    const int m = (n - 1) / 2;
    const double ca = cos(b.angle), sa = sin(b.angle);
    auto put = [&](int k, double sign) {
      const double xi = 0.5 * (1.0 - cos(M_PI * (double)k / (double)m));
      const double zt = sign * naca_yt(b.thickness, xi);
      const double s = (xi - b.pivot_chord_frac) * b.length, z = zt * b.length;
      vx.push_back(s * ca + z * sa);
      vy.push_back(-s * sa + z * ca);
    };
    for (int k = m; k >= 0; --k) put(k, 1.0);  // upper surface, trailing to leading edge
    for (int k = 1; k <= m; ++k) put(k, -1.0); // lower surface, back to the trailing edge
  } else {
    return false;
  }
  const int nv = (int)vx.size();
  if (nv != n) return false;
  pts.resize(n);
  for (int k = 0; k < nv; ++k) {
    const int k2 = (k + 1) % nv;
    const double ex = vx[k2] - vx[k], ey = vy[k2] - vy[k];
    const double len = sqrt(ex * ex + ey * ey);
    SimPoint &p = pts[k];
    p.dx = 0.5 * (vx[k] + vx[k2]);
    p.dy = 0.5 * (vy[k] + vy[k2]);
    p.nx = ey / len;
    p.ny = -ex / len;
    p.s = len;
    // lattice direction closest to the normal, ties to the lowest index
    int best = 1;
    double bv = -1e300;
    for (int a = 1; a < 9; ++a) {
      const double cl = a <= 4 ? 1.0 : sqrt(2.0);
      const double v = (cx_of(a) * p.nx + cy_of(a) * p.ny) / cl;
      if (v > bv) {
        bv = v;
        best = a;
      }
    }
    p.dir = best;
    p.f_dx = (float)p.dx;
    p.f_dy = (float)p.dy;
    p.f_nx = (float)p.nx;
    p.f_ny = (float)p.ny;
    p.f_s = (float)p.s;
    p.n_cand = -1;  // walked every step, unless a fixed body's walk is cached
    for (uint32_t &q : p.cand) q = 0u;
  }
  return true;
}

int default_sim_points(const vplbm_body &b) {
  if (b.n_sim_points > 0) return b.n_sim_points;
  if (b.kind == VPLBM_BODY_DISK) return (int)ceil(2.0 * M_PI * (0.5 * b.length) / 0.5);
  return 849;
}

}  // namespace

struct vplbm_ctx {
  vplbm_config cfg;
  Lattice L;
  Layout lay;
  cudaStream_t stream;
  cudaStream_t capture_stream = nullptr;
  int device;
  char *ws;
  void *buf[2];
  void *prev[2];  // outlet column in the compute type
  uint8_t *chi;
  SimPoint *sim_pts;
  unsigned long long *acc;
  unsigned long long *rng;
  int32_t *sim_nodes;
  double *hist;
  BodyState *body[2];
  ForceRegion *region[2];
  double *sums;
  long long *counts;
  long long *dev_step;
  unsigned int *ticket;
  int32_t *status;
  int cur = 0;        // buffer holding the state
  bool pre = true;    // the state is a pre-collision field (first step reads in place)
  bool pending = false;      // the last queued step's force sums still await finalizing
  bool pending_sim = false;  // ... and that step evaluated SIM
  bool mask_stale = false;   // a moving body's chi lags its body by a step
  bool has_body = false;
  vplbm_body body_cfg{};
  BodyState body_host{};
  ForceRegion region_host{};
  int n_sim = 0;
  int sim_every = 0;  // effective
  long long steps = 0;
  int64_t launches = 0;
  uint64_t generation = 0;  // bumped whenever captured step graphs go stale
  // graphs[p][n]: n steps starting from buffer p, ending with finalized forces
  cudaGraphExec_t graphs[2][kGraphMax + 1] = {};
  cudaGraph_t graph_defs[2][kGraphMax + 1] = {};  // their definitions (batch graphs clone them)
  bool graph_wanted[kGraphMax + 1] = {};  // lengths beyond the powers of two
  bool graphs_ready = false;
  cudaStream_t side = nullptr;      // the special kernel's stream
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int region_slots = 1;             // blocks reserved for force-region tiles
  int bulk_variant = 0;             // launch form of the bulk kernel (kBulkVariants)
  double sim_const[3] = {0.0, 0.0, 0.0};  // -(1/3) sum S n and its moment
  std::string err;
  double s_plus, s_minus, a_plus, a_minus, half_pen;
};

namespace {

}  // namespace

void vplbm::set_global_error(const std::string &msg) { g_err = msg; }

namespace {

vplbm_status fail(vplbm_ctx *c, vplbm_status st, const std::string &msg) {
  if (c)
    c->err = msg;
  else
    g_err = msg;
  return st;
}

vplbm_status cuda_fail(vplbm_ctx *c, cudaError_t e, const char *where) {
  return fail(c, VPLBM_ECUDA, fmt("%s: %s", where, cudaGetErrorString(e)));
}

#define VPLBM_CUDA(ctx, expr)                                  \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #expr); \
  } while (0)

StepArgs step_args(vplbm_ctx *c, int src, bool do_sim) {
  StepArgs a{};
  a.L = c->L;
  a.src = c->buf[src];
  a.dst = c->buf[1 - src];
  a.prev_src = c->prev[src];
  a.prev_dst = c->prev[1 - src];
  a.chi = c->chi;
  a.body_src = c->body[src];
  a.body_dst = c->body[1 - src];
  a.reg_src = c->region[src];
  a.reg_dst = c->region[1 - src];
  a.acc = c->acc + kAccWords * src;
  a.acc_prev = c->acc + kAccWords * (1 - src);
  a.sim_pts = c->sim_pts;
  for (int k = 0; k < 3; ++k) a.sim_const[k] = c->sim_const[k];
  a.sim_nodes = c->sim_nodes;
  a.n_sim = c->n_sim;
  a.sim_order = c->cfg.sim_order;
  a.sim_per_block = c->body_host.moving ? kSimPointsMoving : kSimPointsFixed;
  a.sim_blocks = do_sim ? (c->n_sim + a.sim_per_block - 1) / a.sim_per_block : 0;
  a.hist = c->hist;
  a.hist_len = effective_hist(c->cfg);
  a.sums = c->sums;
  a.counts = c->counts;
  a.dev_step = c->dev_step;
  a.ticket = c->ticket;
  a.status = c->status;
  a.s_plus = c->s_plus;
  a.s_minus = c->s_minus;
  a.a_plus = c->a_plus;
  a.a_minus = c->a_minus;
  a.half_pen = c->half_pen;
  a.tau_plus = c->cfg.tau_plus;
  a.f_s_plus = (float)a.s_plus;
  a.f_s_minus = (float)a.s_minus;
  a.f_a_plus = (float)a.a_plus;
  a.f_a_minus = (float)a.a_minus;
  a.f_half_pen = (float)a.half_pen;
  a.f_sim_s = (float)(1.0 - 0.5 / a.tau_plus);
  a.tile_w = kTileX;
  a.ntiles_x = (c->L.nx + kTileX - 1) / kTileX;
  a.ntiles_y = (c->L.ny + kTileY - 1) / kTileY;
  a.all_tiles = 0;
  a.n_edge = edge_count(c->L.nx, c->L.ny);
  a.edge_blocks = (a.n_edge + kThreads - 1) / kThreads;
  a.region_slots = c->region_slots;
  a.region_capacity = kRegionCapacity;
  a.raster = c->body_host.moving ? 1 : 0;
  a.sr = stochastic_dtype(c->cfg.dtype) ? 1 : 0;
  a.rng_src = c->rng + src;
  a.rng_dst = c->rng + (1 - src);
  return a;
}

bool sim_due(const vplbm_ctx *c, long long step) {
  return c->sim_every > 0 && c->n_sim > 0 && step % c->sim_every == 0;
}

// One time step on stream s.  The first step after a pre-collision state
// updates every tile with the special kernel.  Later steps split the nodes:
// the special kernel (edge nodes, force region, SIM, tail: a few latency-bound
// blocks) runs on the context's high-priority side stream beside the bulk
// kernel (all other nodes, bandwidth-bound) on s; the two write disjoint
// nodes, and s waits for both before the next step.
// Finalizes the force sums of the last queued step if they were deferred: one
// block on s (history row, running sums, step counter).
cudaError_t flush_forces(vplbm_ctx *c, cudaStream_t s) {
  if (!c->pending) return cudaSuccess;
  StepArgs a = step_args(c, c->cur, false);  // acc_prev: the last step's sums
  a.prev_sim = c->pending_sim ? 1 : 0;
  c->pending = false;
  ++c->launches;
  return launch_finalize(storage_dtype(c->cfg.dtype), a, s);
}

// A moving body's steps leave chi one time level behind the body (each step
// rasterises the level it updates): one launch brings it to the current
// level, at the end of every call and every step graph.
cudaError_t refresh_mask(vplbm_ctx *c, cudaStream_t s) {
  if (!c->mask_stale) return cudaSuccess;
  c->mask_stale = false;
  ++c->launches;
  return launch_mask(step_args(c, c->cur, false), s);
}

cudaError_t queue_step(vplbm_ctx *c, cudaStream_t s, int src, bool pre, bool do_sim) {
  if (c->body_host.moving) c->mask_stale = true;
  if (pre) {
    cudaError_t e = flush_forces(c, s);
    StepArgs a = step_args(c, src, do_sim);
    a.all_tiles = 1;
    ++c->launches;
    if (e == cudaSuccess) e = launch_special(storage_dtype(c->cfg.dtype), false, a, s);
    return e;
  }
  StepArgs a = step_args(c, src, do_sim);
  // a fixed body needs its force sums only after the call: the special kernel
  // skips the ticket and tail, and the next step's special kernel (one extra
  // block beside its work) or flush_forces finalizes them.  A moving body's
  // update needs them within the step.
  a.defer = c->body_host.moving ? 0 : 1;
  a.finalize_prev = c->pending ? 1 : 0;
  a.prev_sim = c->pending_sim ? 1 : 0;
  cudaError_t e = cudaEventRecord(c->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  if (e == cudaSuccess) e = launch_special(storage_dtype(c->cfg.dtype), true, a, c->side);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
  if (e == cudaSuccess) e = launch_bulk(storage_dtype(c->cfg.dtype), c->bulk_variant, a, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join, 0);
  c->launches += 2;
  c->pending = a.defer != 0;
  c->pending_sim = do_sim;
  return e;
}

vplbm_status one_step(vplbm_ctx *c, cudaStream_t s) {
  VPLBM_CUDA(c, queue_step(c, s, c->cur, c->pre, sim_due(c, c->steps)));
  c->cur = 1 - c->cur;
  c->pre = false;
  ++c->steps;
  return VPLBM_OK;
}

void drop_graphs(vplbm_ctx *c) {
  for (auto &row : c->graphs)
    for (cudaGraphExec_t &g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  for (auto &row : c->graph_defs)
    for (cudaGraph_t &g : row)
      if (g) {
        cudaGraphDestroy(g);
        g = nullptr;
      }
  c->graphs_ready = false;
  ++c->generation;  // batch graphs made of these go stale
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// the longest captured graph from buffer cur that fits in `left` steps
int graph_length_from(const vplbm_ctx *c, int cur, int left) {
  for (int n = std::min(left, kGraphMax); n > 1; --n)
    if (c->graphs[cur][n]) return n;
  return 1;
}

int graph_length(const vplbm_ctx *c, int left) {
  return graph_length_from(c, c->cur, left);
}

// Captures the step graphs of every wanted length (the powers of two up to
// kGraphMax and the prepared lengths) and both starting buffers that are not
// captured yet (valid when SIM runs every step or never: the step kernels are
// then the same for every step).  Each graph begins with no force sums
// pending and ends with its last step's sums finalized (and a moving body's
// mask refreshed).  They are captured together, at the first run that needs
// one, so that later runs of any length find theirs; each is uploaded on the
// stream s that will launch it.
vplbm_status ensure_graphs(vplbm_ctx *c, cudaStream_t s) {
  if (c->graphs_ready) return VPLBM_OK;
  VPLBM_CUDA(c, flush_forces(c, s));  // the graphs start with nothing pending
  if (!c->capture_stream)
    VPLBM_CUDA(c, cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
  const int64_t launches = c->launches;
  const bool stale = c->mask_stale;
  const bool do_sim = c->sim_every == 1 && c->n_sim > 0;
  for (int n = 1; n <= kGraphMax; ++n) {
    if (!is_pow2(n) && !c->graph_wanted[n]) continue;
    for (int p = 0; p < 2; ++p) {
      if (c->graphs[p][n]) continue;
      cudaGraph_t g = nullptr;
      VPLBM_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      const int cur = c->cur;
      c->cur = (p + n) & 1;  // the level the graph ends at, for the end-of-run work
      for (int q = 0; q < n && e == cudaSuccess; ++q)
        e = queue_step(c, c->capture_stream, (p + q) & 1, false, do_sim);
      if (e == cudaSuccess) e = flush_forces(c, c->capture_stream);
      if (e == cudaSuccess) e = refresh_mask(c, c->capture_stream);
      c->cur = cur;
      c->launches = launches;  // counted when a graph is launched
      c->mask_stale = stale;
      const cudaError_t e2 = cudaStreamEndCapture(c->capture_stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        drop_graphs(c);
        return cuda_fail(c, e, "capture of a step graph");
      }
      if (e2 != cudaSuccess) {
        drop_graphs(c);
        return cuda_fail(c, e2, "cudaStreamEndCapture");
      }
      e = cudaGraphInstantiate(&c->graphs[p][n], g, 0);
      c->graph_defs[p][n] = g;
      if (e != cudaSuccess) {
        c->graphs[p][n] = nullptr;
        drop_graphs(c);
        return cuda_fail(c, e, "cudaGraphInstantiate");
      }
      e = cudaGraphUpload(c->graphs[p][n], s);  // so that its first launch does not pay for it
      if (e != cudaSuccess) {
        drop_graphs(c);
        return cuda_fail(c, e, "cudaGraphUpload");
      }
    }
  }
  c->graphs_ready = true;
  return VPLBM_OK;
}

// Queues nsteps steps of one lattice on stream s: each run from the longest
// step graph that fits (when the lattice is past its first step and SIM runs
// every step or never), single steps otherwise; ends with the forces
// finalized and a moving body's mask refreshed.
vplbm_status run_steps(vplbm_ctx *c, cudaStream_t s, int nsteps) {
  int left = nsteps;
  const bool graphable = c->sim_every <= 1;
  while (left > 0) {
    if (graphable && !c->pre) {
      VPLBM_CUDA(c, flush_forces(c, s));  // a graph starts with nothing pending
      if (vplbm_status st = ensure_graphs(c, s)) return st;
      const int n = graph_length(c, left);
      VPLBM_CUDA(c, cudaGraphLaunch(c->graphs[c->cur][n], s));
      c->launches += 2 * n + 1 + (c->body_host.moving ? 1 : 0);
      c->steps += n;
      c->cur ^= n & 1;
      c->pending = false;
      c->mask_stale = false;  // the graph ends with the mask refreshed
      left -= n;
      continue;
    }
    if (vplbm_status st = one_step(c, s)) return st;
    --left;
  }
  VPLBM_CUDA(c, flush_forces(c, s));  // every call returns with its forces finalized
  VPLBM_CUDA(c, refresh_mask(c, s));  // and with the mask of the current level
  return VPLBM_OK;
}

vplbm_status sync(vplbm_ctx *c) {
  VPLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return VPLBM_OK;
}

vplbm_status read_status(vplbm_ctx *c, int32_t *st) {
  VPLBM_CUDA(c, cudaMemcpyAsync(st, c->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  return sync(c);
}

constexpr int kTuneRounds = 3;

void set_variant(vplbm_ctx *c, int v) {
  if (v == c->bulk_variant) return;
  c->bulk_variant = v;
  drop_graphs(c);
  ++c->generation;  // batches re-capture their graphs
}

// Elapsed milliseconds of the work `queue` puts on stream s, per step.
template <typename F>
vplbm_status timed(cudaStream_t s, int steps, float *ms, F queue, vplbm_ctx *c) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  vplbm_status st = VPLBM_OK;
  if (e == cudaSuccess) st = queue();
  if (e == cudaSuccess && st == VPLBM_OK) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess && st == VPLBM_OK) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess && st == VPLBM_OK) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != VPLBM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(c, e, "timing a launch form");
  *ms /= (float)steps;
  return VPLBM_OK;
}

}  // namespace

extern "C" {

vplbm_status vplbm_workspace_bytes(const vplbm_config *cfg, size_t *bytes) {
  if (const char *m = check_config(cfg)) return fail(nullptr, VPLBM_EINVAL, m);
  if (!bytes) return fail(nullptr, VPLBM_EINVAL, "bytes is NULL");
  *bytes = make_layout(*cfg).total;
  return VPLBM_OK;
}

vplbm_status vplbm_create(const vplbm_config *cfg, void *dev_workspace, size_t bytes,
                          void *cuda_stream, vplbm_ctx **out) {
  if (const char *m = check_config(cfg)) return fail(nullptr, VPLBM_EINVAL, m);
  if (!out) return fail(nullptr, VPLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!dev_workspace || ((uintptr_t)dev_workspace % kAlign) != 0)
    return fail(nullptr, VPLBM_EINVAL, "workspace must be a 256-byte aligned device pointer");
  const Layout lay = make_layout(*cfg);
  if (bytes < lay.total)
    return fail(nullptr, VPLBM_ENOMEM, fmt("workspace of %zu bytes, %zu needed", bytes, lay.total));
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, dev_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(nullptr, VPLBM_EINVAL, "workspace is not device memory");
  }
  vplbm_ctx *c = new vplbm_ctx();
  c->cfg = *cfg;
  c->lay = lay;
  c->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&c->device);
  c->ws = (char *)dev_workspace;
  c->buf[0] = c->ws + lay.buf[0];
  c->buf[1] = c->ws + lay.buf[1];
  c->prev[0] = c->ws + lay.prev[0];
  c->prev[1] = c->ws + lay.prev[1];
  c->chi = (uint8_t *)(c->ws + lay.chi);
  c->sim_pts = (SimPoint *)(c->ws + lay.sim_pts);
  c->acc = (unsigned long long *)(c->ws + lay.acc);
  c->rng = (unsigned long long *)(c->ws + lay.rng);
  c->sim_nodes = (int32_t *)(c->ws + lay.sim_nodes);
  c->hist = (double *)(c->ws + lay.hist);
  c->body[0] = (BodyState *)(c->ws + lay.body[0]);
  c->body[1] = (BodyState *)(c->ws + lay.body[1]);
  c->region[0] = (ForceRegion *)(c->ws + lay.region[0]);
  c->region[1] = (ForceRegion *)(c->ws + lay.region[1]);
  c->sums = (double *)(c->ws + lay.sums);
  c->counts = (long long *)(c->ws + lay.counts);
  c->dev_step = (long long *)(c->ws + lay.dev_step);
  c->ticket = (unsigned int *)(c->ws + lay.ticket);
  c->status = (int32_t *)(c->ws + lay.status);

  Lattice &L = c->L;
  L.nx = cfg->nx;
  L.ny = cfg->ny;
  L.pitch = pitch_of(cfg->nx);
  L.plane = plane_of(*cfg);
  for (int k = 0; k < 4; ++k) L.bc[k] = cfg->bc[k];
  // offsets from E_a = feq_a(1, u_ref) and the side-condition constants on
  // them: E_abar - E_a = -6 w_a c_a.u_ref (the odd part of the equilibrium),
  // plus the moving-wall term 2 w_a rho_w (c_a.u_in) / cs2 (rho_w = 1) at the
  // inlet; a symmetry wall flips c_y
  // FP32 paths carry u_ref in FP32: the offsets are defined from exactly that
  // value so that the kernels and the conversions agree on E to the last bit
  const bool f64 = cfg->dtype == VPLBM_F64;
  L.ur[0] = f64 ? cfg->u_ref[0] : (double)(float)cfg->u_ref[0];
  L.ur[1] = f64 ? cfg->u_ref[1] : (double)(float)cfg->u_ref[1];
  for (int a = 0; a < 9; ++a) {
    const double cr = cx_of(a) * L.ur[0] + cy_of(a) * L.ur[1];
    const double uu = L.ur[0] * L.ur[0] + L.ur[1] * L.ur[1];
    L.E[a] = w_of(a) * (1.0 + 3.0 * cr + 4.5 * cr * cr - 1.5 * uu);
    const double cin = cx_of(a) * (cfg->u_in[0] - L.ur[0]) + cy_of(a) * (cfg->u_in[1] - L.ur[1]);
    L.kin[a] = 6.0 * w_of(a) * cin;
    L.knos[a] = -6.0 * w_of(a) * cr;
    L.ksym[a] = w_of(a) * (-6.0 * cy_of(a) * L.ur[1] - 18.0 * cx_of(a) * cy_of(a) * L.ur[0] * L.ur[1]);
    L.E_f[a] = (float)L.E[a];
    L.kin_f[a] = (float)L.kin[a];
    L.knos_f[a] = (float)L.knos[a];
    L.ksym_f[a] = (float)L.ksym[a];
  }
  L.ur_f[0] = (float)L.ur[0];
  L.ur_f[1] = (float)L.ur[1];
  L.uc = sqrt(cfg->u_in[0] * cfg->u_in[0] + cfg->u_in[1] * cfg->u_in[1]);
  L.bf[0] = cfg->body_force[0];
  L.bf[1] = cfg->body_force[1];
  L.uc_f = (float)L.uc;
  L.bf_f[0] = (float)L.bf[0];
  L.bf_f[1] = (float)L.bf[1];
  L.has_bf = (L.bf[0] != 0.0 || L.bf[1] != 0.0) ? 1 : 0;

  const double tp = cfg->tau_plus;
  const double tm = cfg->collision == VPLBM_BGK ? tp : cfg->lambda_trt / (tp - 0.5) + 0.5;
  c->s_plus = 1.0 / tp;
  c->s_minus = 1.0 / tm;
  c->a_plus = 1.0 - 0.5 / tp;
  c->a_minus = (cfg->collision == VPLBM_TRT && cfg->forcing == VPLBM_FORCING_SPLIT) ? 1.0 - 0.5 / tm
                                                                                  : c->a_plus;
  c->half_pen = 0.5 / cfg->eta;

  const int64_t ntiles = (int64_t)((L.nx + kTileX - 1) / kTileX) * ((L.ny + kTileY - 1) / kTileY);
  if (ntiles + 64 > (int64_t)INT32_MAX) {
    delete c;
    return fail(nullptr, VPLBM_EINVAL, "lattice too large for one launch");
  }

  cudaError_t e = cudaMemsetAsync(c->ws, 0, lay.total, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  // the side stream runs the special kernel (forces, edges, tail) at the
  // highest priority so that its few blocks are dispatched ahead of the bulk
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    vplbm_destroy(c);
    return cuda_fail(nullptr, e, "setting up the workspace and streams");
  }
  *out = c;
  return VPLBM_OK;
}

vplbm_status vplbm_set_stream(vplbm_ctx *c, void *cuda_stream) {
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  c->stream = (cudaStream_t)cuda_stream;
  return VPLBM_OK;
}

vplbm_status vplbm_set_body(vplbm_ctx *c, const vplbm_body *b) {
  Range range_("vplbm_set_body");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!b) return fail(c, VPLBM_EINVAL, "body is NULL");
  const Lattice &L = c->L;
  BodyState bs{};
  bs.kind = b->kind;
  bs.xg = b->x_c;
  bs.yg = b->y_c;
  bs.theta = b->angle;
  bs.ux = b->u[0];
  bs.uy = b->u[1];
  bs.omega = b->omega;
  bs.length = b->length;
  bs.thickness = b->thickness;
  bs.pivot_frac = b->pivot_chord_frac;
  bs.cos_a = cos(b->angle);
  bs.sin_a = sin(b->angle);
  bs.density_ratio = b->density_ratio;
  bs.gx = b->gravity[0];
  bs.gy = b->gravity[1];
  bs.moving = b->moving;
  bs.estimator = b->estimator;
  body_sync_f32(bs);
  std::vector<SimPoint> pts;
  int n_sim = 0;
  if (b->kind != VPLBM_BODY_NONE) {
    if (b->kind != VPLBM_BODY_DISK && b->kind != VPLBM_BODY_NACA4)
      return fail(c, VPLBM_EINVAL, "unknown body kind");
    if (!(b->length > 0.0)) return fail(c, VPLBM_EINVAL, "body length must be > 0");
    if (b->kind == VPLBM_BODY_NACA4) {
      if (!(b->thickness > 0.0 && b->thickness < 0.5)) return fail(c, VPLBM_EINVAL, "bad NACA thickness");
      if (!(b->pivot_chord_frac >= 0.0 && b->pivot_chord_frac <= 1.0))
        return fail(c, VPLBM_EINVAL, "pivot must lie on the chord");
      if (b->moving) return fail(c, VPLBM_EINVAL, "only a disk can move");
    }
    if (b->moving) {
      if (!(b->density_ratio > 0.0)) return fail(c, VPLBM_EINVAL, "density ratio must be > 0");
      if (b->estimator != VPLBM_MEM && b->estimator != VPLBM_SIM)
        return fail(c, VPLBM_EINVAL, "unknown estimator");
    }
    n_sim = default_sim_points(*b);
    if (n_sim > effective_max_sim(c->cfg))
      return fail(c, VPLBM_EINVAL, fmt("%d SIM points exceed the capacity %d", n_sim, effective_max_sim(c->cfg)));
    if (!build_polygon(*b, n_sim, pts)) return fail(c, VPLBM_EINVAL, "bad SIM point count for this body");
    // the body (its polygon, with one node of margin) must lie inside the lattice
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (const SimPoint &p : pts) {
      x0 = std::min(x0, b->x_c + p.dx - 0.5 * p.s);
      x1 = std::max(x1, b->x_c + p.dx + 0.5 * p.s);
      y0 = std::min(y0, b->y_c + p.dy - 0.5 * p.s);
      y1 = std::max(y1, b->y_c + p.dy + 0.5 * p.s);
    }
    if (!(x0 >= 0.0 && y0 >= 0.0 && x1 <= L.nx - 1.0 && y1 <= L.ny - 1.0))
      return fail(c, VPLBM_EINVAL, "body does not fit in the lattice");
  }
  // force region: tiles around the body (its farthest polygon point from the
  // reference point sets the extent); tile (0, 0) alone for an empty lattice
  double extent = 0.0, bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
  for (const SimPoint &p : pts) {
    extent = std::max(extent, sqrt(p.dx * p.dx + p.dy * p.dy) + 0.5 * p.s);
    bx0 = std::min(bx0, b->x_c + p.dx - 0.5 * p.s);
    bx1 = std::max(bx1, b->x_c + p.dx + 0.5 * p.s);
    by0 = std::min(by0, b->y_c + p.dy - 0.5 * p.s);
    by1 = std::max(by1, b->y_c + p.dy + 0.5 * p.s);
  }
  const int tw = kTileX;
  const int ntx = (L.nx + tw - 1) / tw, nty = (L.ny + kTileY - 1) / kTileY;
  ForceRegion reg{};
  if (b->kind != VPLBM_BODY_NONE) {
    reg = b->moving ? make_region(L, b->x_c, b->y_c, 0.5 * b->length, ntx, nty, tw)
                    : make_region_box(L, bx0, bx1, by0, by1, ntx, nty, tw);
    reg.error = 0;
    if (reg.count > kRegionCapacity)
      return fail(c, VPLBM_EINVAL, fmt("body too large: %d force-region tiles (capacity %d)", reg.count, kRegionCapacity));
  } else {
    reg.count = 1;
  }
  // blocks reserved for region tiles: the region's tile count, or for a
  // moving body the most tiles a box of its size can cover anywhere
  int slots = reg.count;
  if (b->kind != VPLBM_BODY_NONE && b->moving) {
    const double span = 2.0 * (0.5 * b->length + kRegionMargin) + 3.0;
    slots = ((int)(span / tw) + 2) * ((int)(span / kTileY) + 2);
    slots = std::min(slots, kRegionCapacity);
  }
  // the constant part of the SIM sum: -(1/3) sum S_i n_i and its moment
  // (zero for a closed polygon up to round-off), in FP64 in point order
  double cfx = 0.0, cfy = 0.0, ctq = 0.0;
  for (const SimPoint &p : pts) {
    const double tx = p.s * (-1.0 / 3.0) * p.nx, ty = p.s * (-1.0 / 3.0) * p.ny;
    cfx += tx;
    cfy += ty;
    ctq += p.dx * ty - p.dy * tx;
  }
  // The step graphs carry, by value, what a body sets beyond its device data:
  // the SIM point count and constant part, the region's block count, whether
  // it moves, the SIM cadence.  A body with the same ones (the same body placed
  // again, as a restarted solve does) keeps them: its geometry and state are
  // read from device memory at every step.
  const int new_slots = std::max(1, slots);
  const int new_every = (b->moving && b->estimator == VPLBM_SIM) ? 1 : c->cfg.sim_every;
  const double new_const[3] = {cfx, cfy, ctq};
  const bool keep_graphs = c->has_body && c->n_sim == n_sim && c->region_slots == new_slots &&
                           c->body_host.moving == bs.moving && c->sim_every == new_every &&
                           std::memcmp(c->sim_const, new_const, sizeof(new_const)) == 0;
  c->sim_const[0] = cfx;
  c->sim_const[1] = cfy;
  c->sim_const[2] = ctq;
  c->body_cfg = *b;
  c->body_host = bs;
  c->region_slots = new_slots;
  c->n_sim = n_sim;
  c->sim_every = new_every;
  if (!keep_graphs) drop_graphs(c);
  cudaStream_t s = c->stream;
  c->region_host = reg;
  for (int k = 0; k < 2; ++k) {
    VPLBM_CUDA(c, cudaMemcpyAsync(c->body[k], &c->body_host, sizeof(BodyState), cudaMemcpyHostToDevice, s));
    VPLBM_CUDA(c, cudaMemcpyAsync(c->region[k], &c->region_host, sizeof(ForceRegion), cudaMemcpyHostToDevice, s));
  }
  if (n_sim > 0)
    VPLBM_CUDA(c, cudaMemcpyAsync(c->sim_pts, pts.data(), n_sim * sizeof(SimPoint), cudaMemcpyHostToDevice, s));
  VPLBM_CUDA(c, cudaMemsetAsync(c->chi, 0, (size_t)L.pitch * L.ny, s));
  if (b->kind != VPLBM_BODY_NONE) {
    // the predicate only where the body can be: its polygon's box with a
    // margin of three nodes (the surface bulges beyond the polygon's edges
    // by far less than a node); interface bits one node wider
    int i0 = std::max(0, (int)floor(bx0) - 3), i1 = std::min(L.nx - 1, (int)ceil(bx1) + 3);
    int j0 = std::max(0, (int)floor(by0) - 3), j1 = std::min(L.ny - 1, (int)ceil(by1) + 3);
    // a box reaching a periodic side: its neighbours across the side too
    if (L.bc[0] == VPLBM_PERIODIC && (i0 == 0 || i1 == L.nx - 1)) i0 = 0, i1 = L.nx - 1;
    if (L.bc[2] == VPLBM_PERIODIC && (j0 == 0 || j1 == L.ny - 1)) j0 = 0, j1 = L.ny - 1;
    VPLBM_CUDA(c, launch_raster(L, c->body[0], c->chi, i0, j0, i1, j1, s));
    VPLBM_CUDA(c, launch_interface(L, c->chi, std::max(0, i0 - 1), std::max(0, j0 - 1),
                                   std::min(L.nx - 1, i1 + 1), std::min(L.ny - 1, j1 + 1), s));
    c->launches += 2;
  }
  VPLBM_CUDA(c, launch_init(storage_dtype(c->cfg.dtype), L, c->body[0], c->chi, c->buf[0], c->cfg.u_in[0], c->cfg.u_in[1], s));
  ++c->launches;
  // a fixed body's SIM points sample the same nodes at every step: walk once
  if (n_sim > 0 && !b->moving && L.nx <= 0xffff && L.ny <= 0xffff) {
    VPLBM_CUDA(c, launch_sim_cache(step_args(c, 0, true), s));
    ++c->launches;
  }
  // histories, sums, counters, status
  VPLBM_CUDA(c, cudaMemsetAsync(c->ws + c->lay.hist, 0, c->lay.body[0] - c->lay.hist, s));
  VPLBM_CUDA(c, cudaMemsetAsync(c->ws + c->lay.sums, 0, c->lay.total - c->lay.sums, s));
  VPLBM_CUDA(c, cudaMemsetAsync(c->prev[0], 0, 3 * (size_t)L.ny * sizeof(double), s));
  VPLBM_CUDA(c, cudaMemsetAsync(c->prev[1], 0, 3 * (size_t)L.ny * sizeof(double), s));
  VPLBM_CUDA(c, cudaGetLastError());
  c->cur = 0;
  c->pre = true;
  c->steps = 0;
  c->pending = false;  // the accumulators were cleared with the other counters
  c->mask_stale = false;
  c->has_body = true;
  return sync(c);
}

vplbm_status vplbm_step(vplbm_ctx *c, int32_t nsteps) {
  Range range_("vplbm_step");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(c, VPLBM_EINVAL, "nsteps must be >= 0");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "no body placed (vplbm_set_body)");
  return run_steps(c, c->stream, nsteps);
}

}  // extern "C"

namespace {

// marks the graph length a run of nsteps steps ends with (beyond the full
// kGraphMax runs) for capture; true when a new length was marked
bool want_length(vplbm_ctx *c, int nsteps) {
  const int r = nsteps > kGraphMax ? nsteps % kGraphMax : nsteps;
  if (r <= 1 || is_pow2(r) || c->graph_wanted[r]) return false;
  c->graph_wanted[r] = true;
  c->graphs_ready = false;  // ensure_graphs captures the missing lengths only
  return true;
}

}  // namespace

extern "C" {

vplbm_status vplbm_prepare(vplbm_ctx *c, int32_t nsteps) {
  Range range_("vplbm_prepare");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(c, VPLBM_EINVAL, "nsteps must be >= 0");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "no body placed (vplbm_set_body)");
  want_length(c, nsteps);
  if (c->sim_every > 1) return VPLBM_OK;  // steps are queued one by one
  if (vplbm_status st = ensure_graphs(c, c->stream)) return st;
  return sync(c);
}

// one history row: MEM (F_x, F_y, T), SIM (same), volume integral (same)
static vplbm_status read_hist_entry(vplbm_ctx *c, long long step, double out[kHistCols]) {
  const int len = effective_hist(c->cfg);
  VPLBM_CUDA(c, cudaMemcpyAsync(out, c->hist + kHistCols * (step % len), kHistCols * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  return sync(c);
}

vplbm_status vplbm_force_mem(vplbm_ctx *c, double F[2], double *T) {
  Range range_("vplbm_force_mem");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!F || !T) return fail(c, VPLBM_EINVAL, "NULL output");
  if (c->steps == 0) return fail(c, VPLBM_ESTATE, "no step taken");
  double e[kHistCols];
  if (vplbm_status st = read_hist_entry(c, c->steps - 1, e)) return st;
  int32_t status = 0;
  if (vplbm_status st = read_status(c, &status)) return st;
  F[0] = e[0];
  F[1] = e[1];
  *T = e[2];
  if (status & kStatusUnstable) return fail(c, VPLBM_EUNSTABLE, "non-finite or non-positive density");
  return VPLBM_OK;
}

vplbm_status vplbm_force_sim(vplbm_ctx *c, double F[2], double *T) {
  Range range_("vplbm_force_sim");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!F || !T) return fail(c, VPLBM_EINVAL, "NULL output");
  if (c->sim_every <= 0 || c->n_sim <= 0 || c->steps == 0) return fail(c, VPLBM_ESTATE, "SIM not evaluated");
  const long long last = (c->steps - 1) / c->sim_every * c->sim_every;
  if (c->steps - 1 - last >= effective_hist(c->cfg)) return fail(c, VPLBM_ESTATE, "SIM entry left the history");
  double e[kHistCols];
  if (vplbm_status st = read_hist_entry(c, last, e)) return st;
  int32_t status = 0;
  if (vplbm_status st = read_status(c, &status)) return st;
  F[0] = e[3];
  F[1] = e[4];
  *T = e[5];
  if (status & kStatusUnstable) return fail(c, VPLBM_EUNSTABLE, "non-finite or non-positive density");
  if (status & kStatusSimMissing) return fail(c, VPLBM_ESTATE, "a SIM point found no fluid node");
  return VPLBM_OK;
}

vplbm_status vplbm_force_angot(vplbm_ctx *c, double F[2], double *T) {
  Range range_("vplbm_force_angot");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!F || !T) return fail(c, VPLBM_EINVAL, "NULL output");
  if (c->steps == 0) return fail(c, VPLBM_ESTATE, "no step taken");
  double e[kHistCols];
  if (vplbm_status st = read_hist_entry(c, c->steps - 1, e)) return st;
  F[0] = e[6];
  F[1] = e[7];
  *T = e[8];
  return VPLBM_OK;
}

vplbm_status vplbm_forces_async(vplbm_ctx *c, double *out) {
  Range range_("vplbm_forces_async");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!out) return fail(c, VPLBM_EINVAL, "NULL output");
  if (c->steps == 0) return fail(c, VPLBM_ESTATE, "no step taken");
  const int len = effective_hist(c->cfg);
  VPLBM_CUDA(c, cudaMemcpyAsync(out, c->hist + kHistCols * ((c->steps - 1) % len), 6 * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  return VPLBM_OK;
}

vplbm_status vplbm_force_history(vplbm_ctx *c, int32_t estimator, int32_t count, double *out) {
  Range range_("vplbm_force_history");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  const int len = effective_hist(c->cfg);
  if (!out || count < 0 || count > len || count > c->steps)
    return fail(c, VPLBM_EINVAL, "bad history request");
  if (estimator != VPLBM_MEM && estimator != VPLBM_SIM && estimator != VPLBM_ANGOT)
    return fail(c, VPLBM_EINVAL, "unknown estimator");
  if (count == 0) return VPLBM_OK;
  // the requested rows only: one copy, or two where they wrap around the ring
  std::vector<double> rows((size_t)count * kHistCols);
  const int first = (int)((c->steps - count) % len);
  const int n1 = std::min(count, len - first);
  VPLBM_CUDA(c, cudaMemcpyAsync(rows.data(), c->hist + kHistCols * (size_t)first, (size_t)n1 * kHistCols * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  if (count > n1)
    VPLBM_CUDA(c, cudaMemcpyAsync(rows.data() + kHistCols * (size_t)n1, c->hist, (size_t)(count - n1) * kHistCols * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
  if (vplbm_status st = sync(c)) return st;
  const int off = estimator == VPLBM_SIM ? 3 : (estimator == VPLBM_ANGOT ? 6 : 0);
  for (int k = 0; k < count; ++k)
    for (int q = 0; q < 3; ++q) out[3 * k + q] = rows[kHistCols * (size_t)k + off + q];
  return VPLBM_OK;
}

vplbm_status vplbm_force_history_async(vplbm_ctx *c, int32_t count, double *out) {
  Range range_("vplbm_force_history_async");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  const int len = effective_hist(c->cfg);
  if (!out || count < 0 || count > len || count > c->steps)
    return fail(c, VPLBM_EINVAL, "bad history request");
  if (count == 0) return VPLBM_OK;
  const int first = (int)((c->steps - count) % len);
  const int n1 = std::min(count, len - first);
  const size_t row = kHistCols * sizeof(double);
  VPLBM_CUDA(c, cudaMemcpyAsync(out, c->hist + kHistCols * (size_t)first, (size_t)n1 * row,
                                cudaMemcpyDeviceToHost, c->stream));
  if (count > n1)
    VPLBM_CUDA(c, cudaMemcpyAsync(out + kHistCols * (size_t)n1, c->hist, (size_t)(count - n1) * row,
                                  cudaMemcpyDeviceToHost, c->stream));
  return VPLBM_OK;
}

vplbm_status vplbm_force_sums(vplbm_ctx *c, double sums[6], int64_t n[2]) {
  Range range_("vplbm_force_sums");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!sums || !n) return fail(c, VPLBM_EINVAL, "NULL output");
  long long cnt[2];
  VPLBM_CUDA(c, cudaMemcpyAsync(sums, c->sums, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  VPLBM_CUDA(c, cudaMemcpyAsync(cnt, c->counts, 2 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  if (vplbm_status st = sync(c)) return st;
  n[0] = cnt[0];
  n[1] = cnt[1];
  return VPLBM_OK;
}

vplbm_status vplbm_reset_sums(vplbm_ctx *c) {
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  VPLBM_CUDA(c, cudaMemsetAsync(c->sums, 0, 6 * sizeof(double), c->stream));
  VPLBM_CUDA(c, cudaMemsetAsync(c->counts, 0, 2 * sizeof(long long), c->stream));
  return VPLBM_OK;
}

vplbm_status vplbm_step_count(vplbm_ctx *c, int64_t *n) {
  if (!c || !n) return fail(c, VPLBM_EINVAL, "NULL argument");
  *n = c->steps;
  return VPLBM_OK;
}

vplbm_status vplbm_get_f_dev(vplbm_ctx *c, double *f_dev) {
  Range range_("vplbm_get_f_dev");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!f_dev) return fail(c, VPLBM_EINVAL, "f_dev is NULL");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "no state yet");
  VPLBM_CUDA(c, launch_get_f(storage_dtype(c->cfg.dtype), !c->pre, c->L, c->buf[c->cur], c->prev[c->cur], f_dev, 0,
                             9, 0, c->L.ny, c->stream));
  ++c->launches;
  return VPLBM_OK;
}

vplbm_status vplbm_get_fields_dev(vplbm_ctx *c, double *rho, double *ux, double *uy) {
  Range range_("vplbm_get_fields_dev");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!rho || !ux || !uy) return fail(c, VPLBM_EINVAL, "NULL output");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "no state yet");
  VPLBM_CUDA(c, launch_get_fields(storage_dtype(c->cfg.dtype), !c->pre, c->L, c->buf[c->cur], c->prev[c->cur], c->chi,
                                  c->body[c->cur], c->half_pen, rho, ux, uy, 0, c->L.ny, c->stream));
  ++c->launches;
  return VPLBM_OK;
}

vplbm_status vplbm_get_mask_dev(vplbm_ctx *c, uint8_t *chi_dev) {
  Range range_("vplbm_get_mask_dev");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!chi_dev) return fail(c, VPLBM_EINVAL, "chi_dev is NULL");
  VPLBM_CUDA(c, launch_get_mask(c->L, c->chi, chi_dev, 0, c->L.ny, c->stream));
  ++c->launches;
  return VPLBM_OK;
}

}  // extern "C"

namespace {

// The host read-backs stage their rows in the population buffer that does
// not hold the state (the next step overwrites it anyway), a few rows at a
// time, so that they need no device memory beyond the workspace.
void *staging(const vplbm_ctx *c, size_t *bytes) {
  *bytes = 9 * (size_t)c->L.plane * elem_bytes(c->cfg.dtype);
  return c->buf[1 - c->cur];
}

int rows_per_chunk(size_t staging_bytes, size_t row_bytes, int ny) {
  const size_t r = staging_bytes / row_bytes;
  return (int)std::min<size_t>(r, (size_t)ny);
}

}  // namespace

extern "C" {

vplbm_status vplbm_get_f(vplbm_ctx *c, double *f) {
  Range range_("vplbm_get_f");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!f) return fail(c, VPLBM_EINVAL, "NULL output");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "no state yet");
  size_t sb = 0;
  double *st = static_cast<double *>(staging(c, &sb));
  const int nx = c->L.nx, ny = c->L.ny;
  const size_t n = (size_t)nx * ny;
  // all nine planes of a chunk of rows at once, or (16-bit storage on very
  // short lattices) one plane at a time
  const int na = rows_per_chunk(sb, 9 * (size_t)nx * sizeof(double), ny) >= 1 ? 9 : 1;
  const int rows = rows_per_chunk(sb, (size_t)na * nx * sizeof(double), ny);
  if (rows < 1) return fail(c, VPLBM_EINVAL, "lattice row too long to stage");
  for (int a0 = 0; a0 < 9; a0 += na)
    for (int j0 = 0; j0 < ny; j0 += rows) {
      const int r = std::min(rows, ny - j0);
      VPLBM_CUDA(c, launch_get_f(storage_dtype(c->cfg.dtype), !c->pre, c->L, c->buf[c->cur], c->prev[c->cur], st, a0,
                                 na, j0, r, c->stream));
      ++c->launches;
      const size_t w = (size_t)r * nx * sizeof(double);
      VPLBM_CUDA(c, cudaMemcpy2DAsync(f + a0 * n + (size_t)j0 * nx, n * sizeof(double), st, w, w, na,
                                      cudaMemcpyDeviceToHost, c->stream));
    }
  return sync(c);
}

vplbm_status vplbm_get_fields(vplbm_ctx *c, double *rho, double *ux, double *uy) {
  Range range_("vplbm_get_fields");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!rho || !ux || !uy) return fail(c, VPLBM_EINVAL, "NULL output");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "no state yet");
  size_t sb = 0;
  double *st = static_cast<double *>(staging(c, &sb));
  const int nx = c->L.nx, ny = c->L.ny;
  const int rows = rows_per_chunk(sb, 3 * (size_t)nx * sizeof(double), ny);
  if (rows < 1) return fail(c, VPLBM_EINVAL, "lattice row too long to stage");
  double *out[3] = {rho, ux, uy};
  for (int j0 = 0; j0 < ny; j0 += rows) {
    const int r = std::min(rows, ny - j0);
    const size_t m = (size_t)r * nx;
    VPLBM_CUDA(c, launch_get_fields(storage_dtype(c->cfg.dtype), !c->pre, c->L, c->buf[c->cur], c->prev[c->cur], c->chi,
                                    c->body[c->cur], c->half_pen, st, st + m, st + 2 * m, j0, r,
                                    c->stream));
    ++c->launches;
    for (int q = 0; q < 3; ++q)
      VPLBM_CUDA(c, cudaMemcpyAsync(out[q] + (size_t)j0 * nx, st + q * m, m * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
  }
  return sync(c);
}

vplbm_status vplbm_get_mask(vplbm_ctx *c, uint8_t *chi) {
  Range range_("vplbm_get_mask");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!chi) return fail(c, VPLBM_EINVAL, "NULL output");
  size_t sb = 0;
  uint8_t *st = static_cast<uint8_t *>(staging(c, &sb));
  const int nx = c->L.nx, ny = c->L.ny;
  const int rows = rows_per_chunk(sb, (size_t)nx, ny);
  for (int j0 = 0; j0 < ny; j0 += rows) {
    const int r = std::min(rows, ny - j0);
    VPLBM_CUDA(c, launch_get_mask(c->L, c->chi, st, j0, r, c->stream));
    ++c->launches;
    VPLBM_CUDA(c, cudaMemcpyAsync(chi + (size_t)j0 * nx, st, (size_t)r * nx, cudaMemcpyDeviceToHost,
                                  c->stream));
  }
  return sync(c);
}

vplbm_status vplbm_set_state(vplbm_ctx *c, const double *f_dev, const double *prev_dev,
                             int32_t post_collision) {
  Range range_("vplbm_set_state");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!f_dev) return fail(c, VPLBM_EINVAL, "f_dev is NULL");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "place a body first");
  if (post_collision && c->cfg.bc[1] == VPLBM_OUTLET_CONVECTIVE && !prev_dev)
    return fail(c, VPLBM_EINVAL, "the convective outlet needs the previous pre-collision field");
  VPLBM_CUDA(c, launch_set_state(storage_dtype(c->cfg.dtype), c->L, f_dev, c->buf[c->cur], c->stream));
  ++c->launches;
  if (post_collision && prev_dev) {
    VPLBM_CUDA(c, launch_set_prev(storage_dtype(c->cfg.dtype), c->L, prev_dev, c->prev[c->cur], c->stream));
    ++c->launches;
  }
  c->pre = post_collision == 0;
  return VPLBM_OK;
}

}  // extern "C"

namespace {

// A snapshot: this header, then the workspace from the outlet columns to its
// end (outlet columns, mask, SIM points and nodes, force history, body and
// force-region states, running sums, counters, fixed-point accumulators),
// then the population buffer that holds the state.  Raw bytes: a restored
// lattice continues bit for bit as the saved one would have.
struct SnapHeader {
  char magic[8];
  int32_t version, header_bytes;
  vplbm_config cfg;
  vplbm_body body_cfg;
  BodyState body_host;
  ForceRegion region_host;
  double sim_const[3];
  int64_t steps;
  int32_t cur, pre, n_sim, sim_every, region_slots, pad;
  uint64_t tail_bytes, pop_bytes;
};
constexpr char kSnapMagic[8] = {'V', 'P', 'L', 'B', 'M', 'S', 'N', 'P'};
constexpr int32_t kSnapVersion = 3;  // 3: SIM points carry their cached walk

size_t snap_header_bytes() { return align_up(sizeof(SnapHeader), 64); }
size_t snap_tail_bytes(const vplbm_ctx *c) { return c->lay.total - c->lay.prev[0]; }
size_t snap_pop_bytes(const vplbm_ctx *c) { return 9 * (size_t)c->L.plane * elem_bytes(c->cfg.dtype); }

bool same_config(const vplbm_config &a, const vplbm_config &b) {
  bool eq = a.nx == b.nx && a.ny == b.ny && a.dtype == b.dtype && a.collision == b.collision &&
            a.forcing == b.forcing && a.sim_every == b.sim_every &&
            effective_max_sim(a) == effective_max_sim(b) && effective_hist(a) == effective_hist(b) &&
            a.sim_order == b.sim_order && a.tau_plus == b.tau_plus && a.lambda_trt == b.lambda_trt &&
            a.eta == b.eta;
  for (int k = 0; k < 4; ++k) eq = eq && a.bc[k] == b.bc[k];
  for (int k = 0; k < 2; ++k)
    eq = eq && a.u_in[k] == b.u_in[k] && a.body_force[k] == b.body_force[k] && a.u_ref[k] == b.u_ref[k];
  return eq;
}

}  // namespace

extern "C" {

vplbm_status vplbm_state_bytes(vplbm_ctx *c, size_t *bytes) {
  if (!c || !bytes) return fail(c, VPLBM_EINVAL, "NULL argument");
  *bytes = snap_header_bytes() + snap_tail_bytes(c) + snap_pop_bytes(c);
  return VPLBM_OK;
}

vplbm_status vplbm_save_state(vplbm_ctx *c, void *host, size_t bytes) {
  Range range_("vplbm_save_state");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!host) return fail(c, VPLBM_EINVAL, "NULL output");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "no state yet");
  const size_t hb = snap_header_bytes(), tb = snap_tail_bytes(c), pb = snap_pop_bytes(c);
  if (bytes < hb + tb + pb) return fail(c, VPLBM_EINVAL, fmt("snapshot needs %zu bytes", hb + tb + pb));
  VPLBM_CUDA(c, flush_forces(c, c->stream));  // the last step's sums into the history first
  VPLBM_CUDA(c, refresh_mask(c, c->stream));
  SnapHeader h{};
  memcpy(h.magic, kSnapMagic, sizeof h.magic);
  h.version = kSnapVersion;
  h.header_bytes = (int32_t)hb;
  h.cfg = c->cfg;
  h.body_cfg = c->body_cfg;
  h.body_host = c->body_host;
  h.region_host = c->region_host;
  for (int k = 0; k < 3; ++k) h.sim_const[k] = c->sim_const[k];
  h.steps = c->steps;
  h.cur = c->cur;
  h.pre = c->pre ? 1 : 0;
  h.n_sim = c->n_sim;
  h.sim_every = c->sim_every;
  h.region_slots = c->region_slots;
  h.tail_bytes = tb;
  h.pop_bytes = pb;
  char *out = static_cast<char *>(host);
  memset(out, 0, hb);
  memcpy(out, &h, sizeof h);
  VPLBM_CUDA(c, cudaMemcpyAsync(out + hb, c->ws + c->lay.prev[0], tb, cudaMemcpyDeviceToHost, c->stream));
  VPLBM_CUDA(c, cudaMemcpyAsync(out + hb + tb, c->buf[c->cur], pb, cudaMemcpyDeviceToHost, c->stream));
  return sync(c);
}

vplbm_status vplbm_load_state(vplbm_ctx *c, const void *host, size_t bytes) {
  Range range_("vplbm_load_state");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!host) return fail(c, VPLBM_EINVAL, "NULL input");
  const size_t hb = snap_header_bytes(), tb = snap_tail_bytes(c), pb = snap_pop_bytes(c);
  if (bytes < hb + tb + pb) return fail(c, VPLBM_EINVAL, "snapshot too short for this lattice");
  SnapHeader h;
  memcpy(&h, host, sizeof h);
  if (memcmp(h.magic, kSnapMagic, sizeof h.magic) != 0 || h.version != kSnapVersion ||
      h.header_bytes != (int32_t)hb)
    return fail(c, VPLBM_EINVAL, "not a snapshot of this library version");
  if (!same_config(h.cfg, c->cfg) || h.tail_bytes != tb || h.pop_bytes != pb)
    return fail(c, VPLBM_EINVAL, "snapshot of a lattice with another configuration");
  if ((h.cur != 0 && h.cur != 1) || h.n_sim < 0 || h.n_sim > effective_max_sim(c->cfg))
    return fail(c, VPLBM_EINVAL, "corrupt snapshot header");
  const char *in = static_cast<const char *>(host);
  VPLBM_CUDA(c, cudaMemcpyAsync(c->ws + c->lay.prev[0], in + hb, tb, cudaMemcpyHostToDevice, c->stream));
  VPLBM_CUDA(c, cudaMemcpyAsync(c->buf[h.cur], in + hb + tb, pb, cudaMemcpyHostToDevice, c->stream));
  if (vplbm_status st = sync(c)) return st;
  c->body_cfg = h.body_cfg;
  c->body_host = h.body_host;
  c->region_host = h.region_host;
  for (int k = 0; k < 3; ++k) c->sim_const[k] = h.sim_const[k];
  c->steps = h.steps;
  c->cur = h.cur;
  c->pre = h.pre != 0;
  c->n_sim = h.n_sim;
  c->sim_every = h.sim_every;
  c->region_slots = h.region_slots;
  c->pending = false;
  c->pending_sim = false;
  c->mask_stale = false;
  c->has_body = true;
  drop_graphs(c);
  ++c->generation;  // batches re-capture their graphs
  return VPLBM_OK;
}

vplbm_status vplbm_get_body(vplbm_ctx *c, double state[6]) {
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!state) return fail(c, VPLBM_EINVAL, "NULL output");
  BodyState b;
  VPLBM_CUDA(c, cudaMemcpyAsync(&b, c->body[c->cur], sizeof b, cudaMemcpyDeviceToHost, c->stream));
  if (vplbm_status st = sync(c)) return st;
  state[0] = b.xg;
  state[1] = b.yg;
  state[2] = b.theta;
  state[3] = b.ux;
  state[4] = b.uy;
  state[5] = b.omega;
  return VPLBM_OK;
}

vplbm_status vplbm_get_sim_nodes(vplbm_ctx *c, int32_t *nodes, int32_t capacity, int32_t *n) {
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (!n || (capacity > 0 && !nodes)) return fail(c, VPLBM_EINVAL, "NULL output");
  *n = c->n_sim;
  if (capacity < c->n_sim) return fail(c, VPLBM_EINVAL, "capacity below the SIM point count");
  if (c->n_sim > 0) {
    VPLBM_CUDA(c, cudaMemcpyAsync(nodes, c->sim_nodes, c->n_sim * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
  }
  return VPLBM_OK;
}

vplbm_status vplbm_check(vplbm_ctx *c) {
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  int32_t status = 0;
  if (vplbm_status st = read_status(c, &status)) return st;
  if (status & kStatusUnstable) return fail(c, VPLBM_EUNSTABLE, "non-finite or non-positive density");
  return VPLBM_OK;
}

vplbm_status vplbm_launch_count(vplbm_ctx *c, int64_t *n) {
  if (!c || !n) return fail(c, VPLBM_EINVAL, "NULL argument");
  *n = c->launches;
  return VPLBM_OK;
}

vplbm_status vplbm_autotune(vplbm_ctx *c, int32_t trials, int32_t *variant) {
  Range range_("vplbm_autotune");
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (trials < 1 || trials > 10000) return fail(c, VPLBM_EINVAL, "trials must be in 1 .. 10000");
  if (!c->has_body) return fail(c, VPLBM_ESTATE, "place a body first");
  // the forms in turn, kTuneRounds times: per form kGraphMax untimed steps
  // (the step graphs are captured there), then `trials` timed steps;
  // each form's fastest round counts
  float t[kBulkVariants];
  for (int r = 0; r < kTuneRounds; ++r)
    for (int v = 0; v < kBulkVariants; ++v) {
      set_variant(c, v);
      if (vplbm_status st = vplbm_step(c, kGraphMax)) return st;
      float ms = 0.f;
      if (vplbm_status st = timed(c->stream, trials, &ms, [&] { return vplbm_step(c, trials); }, c))
        return st;
      t[v] = r == 0 ? ms : std::min(t[v], ms);
    }
  int best = 0;
  for (int v = 1; v < kBulkVariants; ++v)
    if (t[v] < t[best]) best = v;
  set_variant(c, best);
  if (variant) *variant = best;
  return VPLBM_OK;
}

vplbm_status vplbm_set_bulk_variant(vplbm_ctx *c, int32_t variant) {
  if (!c) return fail(nullptr, VPLBM_EINVAL, "ctx is NULL");
  if (variant < 0 || variant >= kBulkVariants) return fail(c, VPLBM_EINVAL, "no such variant");
  set_variant(c, variant);
  return VPLBM_OK;
}

vplbm_status vplbm_bulk_variant(vplbm_ctx *c, int32_t *variant) {
  if (!c || !variant) return fail(c, VPLBM_EINVAL, "NULL argument");
  *variant = c->bulk_variant;
  return VPLBM_OK;
}

void vplbm_destroy(vplbm_ctx *c) {
  if (!c) return;
  drop_graphs(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

const char *vplbm_last_error(const vplbm_ctx *c) { return c ? c->err.c_str() : g_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------

// One launch for a whole call of n steps: every lattice's run of step graphs
// (the graphs run_steps would launch) as a chain of child graphs, the chains
// side by side in one graph.  Valid while each lattice starts from the buffer
// and the step graphs it was built from.
struct BatchGraph {
  int n = 0;
  std::vector<int> cur;
  std::vector<uint64_t> gen;
  cudaGraphExec_t exec = nullptr;
};

struct vplbm_batch {
  std::vector<vplbm_ctx *> ctxs;
  std::vector<BatchGraph> graphs;   // for prepared step counts
  cudaStream_t stream = nullptr;
  std::vector<cudaEvent_t> ev_in;   // each lattice's stream -> the batch stream
  cudaEvent_t ev_out = nullptr;     // the batch stream -> each lattice's stream
  std::vector<cudaStream_t> chain;  // one stream per lattice: the lattices' steps run side by side
  std::vector<cudaEvent_t> ev_chain;  // end of each chain -> the batch stream
  cudaEvent_t ev_fork = nullptr;      // start of a call on the batch stream
};

namespace {

vplbm_status batch_fail(vplbm_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

vplbm_status batch_cuda(cudaError_t e, const char *where) {
  return batch_fail(VPLBM_ECUDA, fmt("%s: %s", where, cudaGetErrorString(e)));
}

// a failure of a per-lattice call, reported through the global text
vplbm_status batch_ctx_fail(vplbm_status st, int k, const vplbm_ctx *c) {
  return batch_fail(st, fmt("lattice %d: %s", k, c->err.c_str()));
}

// The lattices share no data, so each runs its steps on a stream of its own
// (its chain), forked from s and joined back into s: the steps of different
// lattices overlap, and one lattice's latency-bound special kernel runs while
// other lattices' bulk kernels use the memory bandwidth.
cudaError_t batch_fork(vplbm_batch *b, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->ev_fork, s);
  for (size_t q = 0; q < b->chain.size() && e == cudaSuccess; ++q)
    e = cudaStreamWaitEvent(b->chain[q], b->ev_fork, 0);
  return e;
}

cudaError_t batch_join(vplbm_batch *b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (size_t q = 0; q < b->chain.size() && e == cudaSuccess; ++q) {
    e = cudaEventRecord(b->ev_chain[q], b->chain[q]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_chain[q], 0);
  }
  return e;
}

// Every lattice replays step graphs (no per-step launches) from where it is.
bool batch_graphable(const vplbm_batch *b) {
  for (const vplbm_ctx *c : b->ctxs)
    if (c->sim_every > 1 || c->pre || !c->graphs_ready) return false;
  return true;
}

// The step graphs of a call of n steps of lattice c from buffer cur, in the
// order vplbm_batch_step's rounds of at most kGraphMax steps launch them.
template <typename F>
void for_pieces(const vplbm_ctx *c, int cur, int n, F piece) {
  for (int left = n; left > 0; left -= std::min(left, kGraphMax))
    for (int r = std::min(left, kGraphMax); r > 0;) {
      const int len = graph_length_from(c, cur, r);
      piece(cur, len);
      cur ^= len & 1;
      r -= len;
    }
}

const BatchGraph *find_batch_graph(const vplbm_batch *b, int n) {
  for (const BatchGraph &bg : b->graphs) {
    if (bg.n != n) continue;
    bool ok = true;
    for (size_t k = 0; k < b->ctxs.size() && ok; ++k)
      ok = bg.cur[k] == b->ctxs[k]->cur && bg.gen[k] == b->ctxs[k]->generation;
    if (ok) return &bg;
  }
  return nullptr;
}

constexpr size_t kBatchGraphsKept = 8;

// Builds (and uploads on s) the batch graph of n steps from the buffers cur.
vplbm_status build_batch_graph(vplbm_batch *b, int n, const std::vector<int> &cur, cudaStream_t s) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  for (size_t k = 0; k < b->ctxs.size() && e == cudaSuccess; ++k) {
    const vplbm_ctx *c = b->ctxs[k];
    cudaGraphNode_t prev = nullptr;
    for_pieces(c, cur[k], n, [&](int p, int len) {
      if (e != cudaSuccess) return;
      if (!c->graph_defs[p][len]) {
        e = cudaErrorInvalidValue;
        return;
      }
      cudaGraphNode_t node = nullptr;
      e = cudaGraphAddChildGraphNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0,
                                     c->graph_defs[p][len]);
      prev = node;
    });
  }
  BatchGraph bg;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&bg.exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e == cudaSuccess) e = cudaGraphUpload(bg.exec, s);
  if (e != cudaSuccess) {
    if (bg.exec) cudaGraphExecDestroy(bg.exec);
    return batch_cuda(e, "building a batch graph");
  }
  bg.n = n;
  bg.cur = cur;
  for (const vplbm_ctx *c : b->ctxs) bg.gen.push_back(c->generation);
  if (b->graphs.size() >= kBatchGraphsKept) {
    cudaGraphExecDestroy(b->graphs.front().exec);
    b->graphs.erase(b->graphs.begin());
  }
  b->graphs.push_back(std::move(bg));
  return VPLBM_OK;
}

}  // namespace

extern "C" {

vplbm_status vplbm_batch_create(vplbm_ctx *const *ctxs, int32_t n, void *cuda_stream,
                                vplbm_batch **out) {
  if (!out) return batch_fail(VPLBM_EINVAL, "vplbm_batch_create: out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1) return batch_fail(VPLBM_EINVAL, "vplbm_batch_create: no lattices");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess)
    return batch_fail(VPLBM_ECUDA, "vplbm_batch_create: no current device");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return batch_fail(VPLBM_EINVAL, fmt("vplbm_batch_create: lattice %d is NULL", k));
    for (int q = 0; q < k; ++q)
      if (ctxs[q] == ctxs[k])
        return batch_fail(VPLBM_EINVAL, fmt("vplbm_batch_create: lattice %d repeats lattice %d", k, q));
    if (ctxs[k]->device != dev)
      return batch_fail(VPLBM_EINVAL, fmt("vplbm_batch_create: lattice %d is on device %d, not the current %d",
                                          k, ctxs[k]->device, dev));
  }
  vplbm_batch *b = new vplbm_batch;
  b->ctxs.assign(ctxs, ctxs + n);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->ev_in.assign(n, nullptr);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&b->ev_in[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  b->chain.assign(n, nullptr);
  b->ev_chain.assign(n, nullptr);
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->chain[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_chain[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    vplbm_batch_destroy(b);
    return batch_cuda(e, "vplbm_batch_create: cudaEventCreateWithFlags");
  }
  *out = b;
  return VPLBM_OK;
}

vplbm_status vplbm_batch_autotune(vplbm_batch *b, int32_t trials, int32_t *variants) {
  Range range_("vplbm_batch_autotune");
  if (!b) return batch_fail(VPLBM_EINVAL, "vplbm_batch_autotune: batch is NULL");
  if (trials < 1 || trials > 10000)
    return batch_fail(VPLBM_EINVAL, "vplbm_batch_autotune: trials must be in 1 .. 10000");
  const int n = (int)b->ctxs.size();
  for (int k = 0; k < n; ++k)
    if (!b->ctxs[k]->has_body)
      return batch_fail(VPLBM_ESTATE, fmt("vplbm_batch_autotune: lattice %d has no body placed", k));
  // classes: lattices of one size and storage form share a launch form
  std::vector<int> cls(n, -1);
  int ncls = 0;
  for (int k = 0; k < n; ++k) {
    const vplbm_config &a = b->ctxs[k]->cfg;
    for (int q = 0; q < k && cls[k] < 0; ++q) {
      const vplbm_config &o = b->ctxs[q]->cfg;
      if (o.nx == a.nx && o.ny == a.ny && o.dtype == a.dtype) cls[k] = cls[q];
    }
    if (cls[k] < 0) cls[k] = ncls++;
  }
  // coordinate descent: each pass visits the classes in turn and times every
  // form of one class on the whole batch's steps, the other classes held at
  // their current forms (so the overlap with them is part of the timing);
  // the class keeps its form of the fastest time seen so far
  std::vector<float> t((size_t)ncls * kBulkVariants, 0.f);
  for (int r = 0; r < kTuneRounds; ++r)
    for (int g = 0; g < ncls; ++g) {
      for (int v = 0; v < kBulkVariants; ++v) {
        for (int k = 0; k < n; ++k)
          if (cls[k] == g) set_variant(b->ctxs[k], v);
        if (vplbm_status st = vplbm_batch_step(b, kGraphMax)) return st;
        float ms = 0.f;
        if (vplbm_status st = timed(b->stream, trials, &ms,
                                    [&] { return vplbm_batch_step(b, trials); }, nullptr))
          return st;
        float &tv = t[(size_t)g * kBulkVariants + v];
        tv = r == 0 ? ms : std::min(tv, ms);
      }
      int best = 0;
      for (int v = 1; v < kBulkVariants; ++v)
        if (t[(size_t)g * kBulkVariants + v] < t[(size_t)g * kBulkVariants + best]) best = v;
      for (int k = 0; k < n; ++k)
        if (cls[k] == g) set_variant(b->ctxs[k], best);
    }
  if (variants)
    for (int k = 0; k < n; ++k) variants[k] = b->ctxs[k]->bulk_variant;
  return VPLBM_OK;
}

vplbm_status vplbm_batch_prepare(vplbm_batch *b, int32_t nsteps) {
  Range range_("vplbm_batch_prepare");
  if (!b) return batch_fail(VPLBM_EINVAL, "vplbm_batch_prepare: batch is NULL");
  if (nsteps < 0) return batch_fail(VPLBM_EINVAL, "vplbm_batch_prepare: nsteps must be >= 0");
  for (size_t k = 0; k < b->ctxs.size(); ++k) {
    vplbm_ctx *c = b->ctxs[k];
    if (!c->has_body)
      return batch_fail(VPLBM_ESTATE, fmt("vplbm_batch_prepare: lattice %zu has no body placed", k));
    // the runs of a batch call are at most kGraphMax steps per lattice
    want_length(c, nsteps);
    if (c->sim_every > 1) continue;
    if (vplbm_status st = ensure_graphs(c, b->chain[k])) return batch_ctx_fail(st, (int)k, c);
  }
  for (cudaStream_t st : b->chain)
    if (const cudaError_t e = cudaStreamSynchronize(st); e != cudaSuccess)
      return batch_cuda(e, "vplbm_batch_prepare: cudaStreamSynchronize");
  // a call of nsteps steps as one graph launch, from the current buffers and
  // from the other ones (where the lattices stand after an odd step count)
  if (nsteps > 0 && batch_graphable(b)) {
    std::vector<int> cur;
    for (const vplbm_ctx *c : b->ctxs) cur.push_back(c->cur);
    for (int flip = 0; flip < 2; ++flip) {
      std::vector<int> from(cur);
      for (int &p : from) p ^= flip;
      bool have = false;
      for (const BatchGraph &bg : b->graphs)
        if (bg.n == nsteps && bg.cur == from) {
          have = true;
          for (size_t k = 0; k < b->ctxs.size() && have; ++k) have = bg.gen[k] == b->ctxs[k]->generation;
        }
      if (!have)
        if (vplbm_status st = build_batch_graph(b, nsteps, from, b->stream)) return st;
    }
    if (const cudaError_t e = cudaStreamSynchronize(b->stream); e != cudaSuccess)
      return batch_cuda(e, "vplbm_batch_prepare: cudaStreamSynchronize");
  }
  return VPLBM_OK;
}

vplbm_status vplbm_batch_step(vplbm_batch *b, int32_t nsteps) {
  Range range_("vplbm_batch_step");
  if (!b) return batch_fail(VPLBM_EINVAL, "vplbm_batch_step: batch is NULL");
  if (nsteps < 0) return batch_fail(VPLBM_EINVAL, "vplbm_batch_step: nsteps must be >= 0");
  const int n = (int)b->ctxs.size();
  for (int k = 0; k < n; ++k)
    if (!b->ctxs[k]->has_body)
      return batch_fail(VPLBM_ESTATE, fmt("vplbm_batch_step: lattice %d has no body placed", k));
  if (nsteps == 0) return VPLBM_OK;
  cudaStream_t s = b->stream;
  // the batch's work follows what each lattice's own stream holds
  for (int k = 0; k < n; ++k) {
    vplbm_ctx *c = b->ctxs[k];
    if (c->stream == s) continue;
    cudaError_t e = cudaEventRecord(b->ev_in[k], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_in[k], 0);
    if (e != cudaSuccess) return batch_cuda(e, "vplbm_batch_step: ordering after a lattice stream");
  }
  // a prepared step count: the whole call is one launch of the batch graph
  if (batch_graphable(b))
    if (const BatchGraph *bg = find_batch_graph(b, nsteps)) {
      for (int k = 0; k < n; ++k)  // a graph starts with nothing pending
        if (const cudaError_t e = flush_forces(b->ctxs[k], s); e != cudaSuccess)
          return batch_cuda(e, "vplbm_batch_step: finalizing pending forces");
      if (const cudaError_t e = cudaGraphLaunch(bg->exec, s); e != cudaSuccess)
        return batch_cuda(e, "vplbm_batch_step: cudaGraphLaunch");
      for (int k = 0; k < n; ++k) {
        vplbm_ctx *c = b->ctxs[k];
        for_pieces(c, c->cur, nsteps, [&](int, int len) {
          c->launches += 2 * len + 1 + (c->body_host.moving ? 1 : 0);
        });
        c->steps += nsteps;
        c->cur ^= nsteps & 1;
        c->pending = false;
        c->mask_stale = false;
      }
      cudaError_t e = cudaEventRecord(b->ev_out, s);
      for (int k = 0; k < n && e == cudaSuccess; ++k)
        if (b->ctxs[k]->stream != s) e = cudaStreamWaitEvent(b->ctxs[k]->stream, b->ev_out, 0);
      if (e != cudaSuccess) return batch_cuda(e, "vplbm_batch_step: ordering of the lattice streams");
      return VPLBM_OK;
    }
  // each lattice runs its own steps (its step graphs where they apply) on its
  // chain, forked from s and joined back; the chains meet only at the end of
  // the call, so no lattice waits for another between runs of steps.  The
  // calls are issued in rounds of at most 32 steps per lattice, so that the
  // lattices' work is interleaved on the host too.
  if (const cudaError_t e = batch_fork(b, s); e != cudaSuccess)
    return batch_cuda(e, "vplbm_batch_step: forking the lattice chains");
  for (int left = nsteps; left > 0; left -= std::min(left, kGraphMax)) {
    const int run = std::min(left, kGraphMax);
    for (int k = 0; k < n; ++k)
      if (vplbm_status st = run_steps(b->ctxs[k], b->chain[k], run)) return batch_ctx_fail(st, k, b->ctxs[k]);
  }
  if (const cudaError_t e = batch_join(b, s); e != cudaSuccess)
    return batch_cuda(e, "vplbm_batch_step: joining the lattice chains");
  // and each lattice's own stream follows the batch's work
  cudaError_t e = cudaEventRecord(b->ev_out, s);
  for (int k = 0; k < n && e == cudaSuccess; ++k)
    if (b->ctxs[k]->stream != s) e = cudaStreamWaitEvent(b->ctxs[k]->stream, b->ev_out, 0);
  if (e != cudaSuccess) return batch_cuda(e, "vplbm_batch_step: ordering of the lattice streams");
  return VPLBM_OK;
}

void vplbm_batch_destroy(vplbm_batch *b) {
  if (!b) return;
  for (BatchGraph &bg : b->graphs)
    if (bg.exec) cudaGraphExecDestroy(bg.exec);
  for (cudaEvent_t ev : b->ev_in)
    if (ev) cudaEventDestroy(ev);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (cudaStream_t st : b->chain)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->ev_chain)
    if (ev) cudaEventDestroy(ev);
  delete b;
}

}  // extern "C"
