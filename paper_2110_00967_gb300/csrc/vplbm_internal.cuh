// vplbm_internal.cuh -- device-side building blocks of the sm_103a VP-LBM
// library: D2Q9 constants, storage conversions, the pull-form streaming
// gather with side conditions, the body mask predicate and the parameter
// blocks passed to the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "vplbm.h"

namespace vplbm {

// ---------------------------------------------------------------------------
// D2Q9 lattice (numbering of Fig. d2q9): a = 0 rest, 1 E, 2 N, 3 W, 4 S,
// 5 NE, 6 NW, 7 SW, 8 SE.  Written as constexpr functions so that unrolled
// loops fold them into immediates.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int cx_of(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int cy_of(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int opp_of(int a) {
  return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4 + 1) : ((a - 5 + 2) % 4 + 5));
}
// direction with c_y negated (specular reflection on a y wall)
__host__ __device__ __forceinline__ constexpr int flipy_of(int a) {
  return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}
__host__ __device__ __forceinline__ constexpr double w_of(int a) {
  return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// A lattice tile is one block: kTileX x kTileY nodes, one node per thread
// (warps along x).
constexpr int kTileX = 128;
constexpr int kTileY = 2;
constexpr int kThreads = kTileX * kTileY;
constexpr int kRegionCapacity = 16384;  // force-region tiles
// SIM points per block of the special kernel: a fixed body's points read
// their cached nodes (memory latency only); a moving body's walk evaluates the
// body's FP64 predicate, and GB300's FP64 rate per SM is low, so its points
// are spread over more blocks (more SMs)
constexpr int kSimPointsFixed = kThreads;
constexpr int kSimPointsMoving = 32;

// mask byte bits
constexpr uint8_t kSolid = 1;      // chi = 1
constexpr uint8_t kInterface = 2;  // some lattice neighbour has the other phase

// latched device status bits
constexpr int kStatusUnstable = 1;
constexpr int kStatusSimMissing = 2;

// ---------------------------------------------------------------------------
// storage conversions: populations are stored as offsets h = f - w
// ---------------------------------------------------------------------------
template <typename S>
struct Store;
template <>
struct Store<double> {
  using T = double;
  static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
  static __device__ __forceinline__ double ld_own(const double *p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
  static __device__ __forceinline__ double from_double(double v) { return v; }
};
template <>
struct Store<float> {
  using T = float;
  static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ float ld_own(const float *p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
  static __device__ __forceinline__ float from_double(double v) { return __double2float_rn(v); }
};
template <>
struct Store<__half> {
  using T = float;
  static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ float ld_own(const __half *p) { return __half2float(__ldcg(p)); }
  static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ __half from_double(double v) { return __double2half(v); }
};
template <>
struct Store<__nv_bfloat16> {
  using T = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ float ld_own(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldcg(p));
  }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ __nv_bfloat16 from_double(double v) {
    return __double2bfloat16(v);
  }
};

// ---------------------------------------------------------------------------
// body state kept on the device (FP64)
// ---------------------------------------------------------------------------
struct BodyState {
  double xg, yg, theta;  // reference point and rotation angle
  double ux, uy, omega;  // rigid velocity
  double length;         // disk diameter / chord
  double thickness;      // NACA t
  double pivot_frac;
  double cos_a, sin_a;   // of the airfoil angle (taken on the host)
  double density_ratio;
  double gx, gy;         // gravity on a moving body
  int32_t kind;
  int32_t moving;
  int32_t estimator;
  int32_t pad;
  float f_ux, f_uy, f_omega, f_xg, f_yg, f_pad;  // FP32 copies for FP32 paths
};

// keeps the FP32 copies in step with the FP64 state
__host__ __device__ inline void body_sync_f32(BodyState &b) {
  b.f_ux = (float)b.ux;
  b.f_uy = (float)b.uy;
  b.f_omega = (float)b.omega;
  b.f_xg = (float)b.xg;
  b.f_yg = (float)b.yg;
}

// rigid velocity u_s = U + Omega x (x - x_G) at node (i, j), in the compute type
template <typename T>
__device__ __forceinline__ void solid_velocity(const BodyState &b, int i, int j, T &usx, T &usy);
template <>
__device__ __forceinline__ void solid_velocity<double>(const BodyState &b, int i, int j,
                                                       double &usx, double &usy) {
  usx = b.ux - b.omega * ((double)j - b.yg);
  usy = b.uy + b.omega * ((double)i - b.xg);
}
template <>
__device__ __forceinline__ void solid_velocity<float>(const BodyState &b, int i, int j,
                                                      float &usx, float &usy) {
  usx = b.f_ux - b.f_omega * ((float)j - b.f_yg);
  usy = b.f_uy + b.f_omega * ((float)i - b.f_xg);
}

struct SimPoint {
  double dx, dy;  // offset of the integration point from the reference point
  double nx, ny;  // outward unit normal
  double s;       // edge length S_i
  int32_t dir;    // lattice direction closest to the normal
  float f_dx, f_dy, f_nx, f_ny, f_s;  // FP32 copies for FP32 paths
  // For a fixed body, the walk's result, found once when the body is placed:
  // the sampled fluid nodes (i in the low 16 bits, j in the high 16), in the
  // order the walk takes them (one, or two or four for a point half-way
  // between nodes).  n_cand: their count; 0 when no fluid node was found;
  // -1 when not cached (a moving body, whose nodes are walked every step).
  int32_t n_cand;
  uint32_t cand[4];
};

// body reference point and rigid velocity in the compute type
template <typename T>
struct BodyRef;
template <>
struct BodyRef<double> {
  double xg, yg, ux, uy, om;
  __device__ __forceinline__ explicit BodyRef(const BodyState &b)
      : xg(b.xg), yg(b.yg), ux(b.ux), uy(b.uy), om(b.omega) {}
};
template <>
struct BodyRef<float> {
  float xg, yg, ux, uy, om;
  __device__ __forceinline__ explicit BodyRef(const BodyState &b)
      : xg(b.f_xg), yg(b.f_yg), ux(b.f_ux), uy(b.f_uy), om(b.f_omega) {}
};

// ---------------------------------------------------------------------------
// Force sums are exact 64-bit fixed-point integers: each term, computed in the
// compute type, is rounded once to a multiple of 2^-kF (forces) or 2^-kT
// (torques) and the integers are added, which is exact and independent of
// the order, so warps can add with integer atomics and the result is
// reproducible bit for bit.  (FP64 arithmetic runs at about 1/58 of the FP32
// rate on this part, so the sums avoid it; the totals are converted to FP64.)
// ---------------------------------------------------------------------------
template <typename T>
struct Fix;
template <>
struct Fix<double> {
  // two words: round(v 2^30) and the exact remainder at 2^-82 (|sum| < 2^33)
  static constexpr int kWords = 2;
  static __device__ __forceinline__ void split(double v, long long (&w)[2]) {
    const long long hi = __double2ll_rn(v * 1073741824.0);              // 2^30
    const double rem = v - (double)hi * 9.313225746154785e-10;          // exact
    w[0] = hi;
    w[1] = __double2ll_rn(rem * 4835703278458516698824704.0);           // 2^82
  }
  static __host__ __device__ double value(long long w0, long long w1) {
    return (double)w0 * 9.313225746154785e-10 + (double)w1 * 2.0679515313825692e-25;
  }
};
template <>
struct Fix<float> {
  // one word at 2^-40 (|sum| < 2^23); the terms carry FP32 precision anyway
  static constexpr int kWords = 1;
  // round(t) for an FP32 value t with |t| < 2^62, without FP64: split at 2^31
  static __device__ __forceinline__ long long round_ll(float t) {
    const int hi = __float2int_rz(t * 4.656612873077392578125e-10f);  // trunc(t / 2^31)
    const float rem = t - (float)hi * 2147483648.0f;                  // exact
    return ((long long)hi << 31) + (long long)__float2int_rn(rem);
  }
  static __device__ __forceinline__ void split(float v, long long (&w)[1]) {
    w[0] = round_ll(v * 1099511627776.0f);  // 2^40
  }
  static __host__ __device__ double value(long long w0, long long) {
    return (double)w0 * 9.094947017729282e-13;  // 2^-40
  }
};
// accumulator words: (MEM Fx, Fy, T, SIM Fx, Fy, T) x two words
// fixed-point sum slots: MEM F_x, F_y, T; SIM F_x, F_y, T; volume integral F_x, F_y, T
constexpr int kAccSlots = 9;
constexpr int kHistCols = 9;  // one history row per step: the same nine values
constexpr int kAccWords = 2 * kAccSlots;

// ---------------------------------------------------------------------------
// lattice geometry and side conditions, shared by every kernel
// ---------------------------------------------------------------------------
// Populations are stored as offsets h_a = f_a - E_a from the equilibrium at
// rest density and a reference velocity, E_a = feq_a(1, u_ref): with
// u_ref = 0 these are the offsets from the lattice weights; with u_ref the
// free-stream velocity the stored values are small wherever the flow is
// undisturbed, which keeps rounding small in the reduced-precision forms.
// Every formula below works on these offsets and on small differences
// (rho - 1, u - u_ref) only.
struct Lattice {
  int32_t nx, ny, pitch;
  int32_t bc[4];
  int64_t plane;     // ny * pitch (+ padding)
  double E[9];       // feq_a(1, u_ref)
  double ur[2];      // u_ref
  // side-condition constants on the offsets: a population that returns by
  // bounce-back from an inlet wall gets kin, from a no-slip wall knos, and one
  // reflected on a symmetry wall gets ksym
  double kin[9], knos[9], ksym[9];
  double uc;         // convective outlet velocity |u_in|
  double bf[2];      // uniform body force density
  float E_f[9], ur_f[2], kin_f[9], knos_f[9], ksym_f[9];  // FP32 copies
  float uc_f;
  float bf_f[2];
  int32_t has_bf;    // body force nonzero: every node carries a forcing term
};

// lattice constants in the compute type
template <typename T>
struct LatC;
template <>
struct LatC<double> {
  static __device__ __forceinline__ double kin(const Lattice &L, int a) { return L.kin[a]; }
  static __device__ __forceinline__ double knos(const Lattice &L, int a) { return L.knos[a]; }
  static __device__ __forceinline__ double ksym(const Lattice &L, int a) { return L.ksym[a]; }
  static __device__ __forceinline__ double E(const Lattice &L, int a) { return L.E[a]; }
  static __device__ __forceinline__ double ur(const Lattice &L, int k) { return L.ur[k]; }
  static __device__ __forceinline__ double uc(const Lattice &L) { return L.uc; }
  static __device__ __forceinline__ double bf(const Lattice &L, int k) { return L.bf[k]; }
};
template <>
struct LatC<float> {
  static __device__ __forceinline__ float kin(const Lattice &L, int a) { return L.kin_f[a]; }
  static __device__ __forceinline__ float knos(const Lattice &L, int a) { return L.knos_f[a]; }
  static __device__ __forceinline__ float ksym(const Lattice &L, int a) { return L.ksym_f[a]; }
  static __device__ __forceinline__ float E(const Lattice &L, int a) { return L.E_f[a]; }
  static __device__ __forceinline__ float ur(const Lattice &L, int k) { return L.ur_f[k]; }
  static __device__ __forceinline__ float uc(const Lattice &L) { return L.uc_f; }
  static __device__ __forceinline__ float bf(const Lattice &L, int k) { return L.bf_f[k]; }
};
template <typename T>
__device__ __forceinline__ T lat_bf(const Lattice &L, int k) { return LatC<T>::bf(L, k); }

// Pull-form streaming: the pre-collision population a at node (i, j) of the
// time level whose post-collision field is `post` (previous level) and whose
// outlet column of pre-collision values at the previous level is `prev`
// ([3][ny] for a = 3, 6, 7).  Mirrors Eq. eqBd with the side conditions:
// periodic sides wrap; otherwise the side beyond which the source node lies
// decides, the x side first.
template <typename S>
__device__ __forceinline__ typename Store<S>::T pop_at(const S *post, const Lattice &L, int a,
                                                        int i, int j) {
  return Store<S>::ld(post + (int64_t)a * L.plane + (int64_t)j * L.pitch + i);
}

template <typename S>
__device__ __forceinline__ typename Store<S>::T gather_core(const S *post, const Lattice &L, int a,
                                                             int i, int j) {
  using T = typename Store<S>::T;
  int si = i - cx_of(a), sj = j - cy_of(a);
  if (si < 0 && L.bc[0] == VPLBM_PERIODIC) si += L.nx;
  if (si >= L.nx && L.bc[1] == VPLBM_PERIODIC) si -= L.nx;
  if (sj < 0 && L.bc[2] == VPLBM_PERIODIC) sj += L.ny;
  if (sj >= L.ny && L.bc[3] == VPLBM_PERIODIC) sj -= L.ny;
  const bool xin = si >= 0 && si < L.nx;
  const bool yin = sj >= 0 && sj < L.ny;
  if (xin && yin) return pop_at(post, L, a, si, sj);
  if (!xin) {
    const int kind = L.bc[si < 0 ? 0 : 1];
    if (kind == VPLBM_INLET_BB) return pop_at(post, L, opp_of(a), i, j) + LatC<T>::kin(L, a);
    return pop_at(post, L, opp_of(a), i, j) + LatC<T>::knos(L, a);  // no-slip bounce-back
  }
  const int kind = L.bc[sj < 0 ? 2 : 3];
  if (kind == VPLBM_SYMMETRY) return pop_at(post, L, flipy_of(a), si, j) + LatC<T>::ksym(L, a);
  return pop_at(post, L, opp_of(a), i, j) + LatC<T>::knos(L, a);  // no-slip bounce-back
}

__device__ __forceinline__ int outlet_slot(int a) { return a == 3 ? 0 : (a == 6 ? 1 : 2); }

// The outlet column is kept in the compute type T (FP64 for the FP64 form,
// FP32 otherwise), [3][ny] for a = 3, 6, 7.
template <typename S>
__device__ __forceinline__ typename Store<S>::T gather(const S *post,
                                                        const typename Store<S>::T *prev,
                                                        const Lattice &L, int a, int i, int j) {
  using T = typename Store<S>::T;
  if (cx_of(a) < 0 && i == L.nx - 1 && L.bc[1] == VPLBM_OUTLET_CONVECTIVE) {
    // convective outlet: f^{n+1}(N-1) = (f^n(N-1) + U_c f^{n+1}(N-2)) / (1 + U_c)
    const T inner = gather_core(post, L, a, i - 1, j);
    const T old = prev[outlet_slot(a) * L.ny + j];
    const T uc = LatC<T>::uc(L);
    return (old + uc * inner) / ((T)1 + uc);
  }
  if (cx_of(a) < 0 && i == L.nx - 1 && L.bc[1] == VPLBM_OUTLET_FREE)
    return gather_core(post, L, a, i - 1, j);  // free outlet: zero normal gradient
  return gather_core(post, L, a, i, j);
}

// Pre-collision population of the current level: gathered from the previous
// post-collision field, or read in place when the state is pre-collision.
template <typename S, bool kGather>
__device__ __forceinline__ typename Store<S>::T pre_pop(const S *buf,
                                                         const typename Store<S>::T *prev,
                                                         const Lattice &L, int a, int i, int j) {
  if (kGather) return gather(buf, prev, L, a, i, j);
  return pop_at(buf, L, a, i, j);
}

// ---------------------------------------------------------------------------
// mask predicate (Eq. fcar), evaluated in FP64 with correctly rounded
// operations in a fixed order so that it is reproducible bit for bit
// ---------------------------------------------------------------------------
__device__ __forceinline__ double naca_half_thickness_dev(double t, double xi) {
  const double x2 = __dmul_rn(xi, xi);
  const double x3 = __dmul_rn(x2, xi);
  const double x4 = __dmul_rn(x3, xi);
  double p = __dmul_rn(0.2969, sqrt(xi));
  p = __dsub_rn(p, __dmul_rn(0.1260, xi));
  p = __dsub_rn(p, __dmul_rn(0.3516, x2));
  p = __dadd_rn(p, __dmul_rn(0.2843, x3));
  p = __dsub_rn(p, __dmul_rn(0.1015, x4));
  return __dmul_rn(__dmul_rn(5.0, t), p);
}

__device__ __forceinline__ bool body_contains(const BodyState &b, int i, int j) {
  const double dx = __dsub_rn((double)i, b.xg);
  const double dy = __dsub_rn((double)j, b.yg);
  if (b.kind == VPLBM_BODY_DISK) {
    const double r = __dmul_rn(0.5, b.length);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= __dmul_rn(r, r);
  }
  if (b.kind == VPLBM_BODY_NACA4) {
    const double s = __dsub_rn(__dmul_rn(dx, b.cos_a), __dmul_rn(dy, b.sin_a));
    const double xi = __dadd_rn(__ddiv_rn(s, b.length), b.pivot_frac);
    const double zn = __dadd_rn(__dmul_rn(dx, b.sin_a), __dmul_rn(dy, b.cos_a));
    const double zeta = __ddiv_rn(zn, b.length);
    if (!(xi >= 0.0 && xi <= 1.0)) return false;
    return fabs(zeta) <= naca_half_thickness_dev(b.thickness, xi);
  }
  return false;
}

// neighbour of (i, j) along a inside the lattice (periodic sides wrap);
// false when it lies beyond a non-periodic side
__device__ __forceinline__ bool neighbour(const Lattice &L, int a, int i, int j, int &ni, int &nj) {
  ni = i + cx_of(a);
  nj = j + cy_of(a);
  if (ni < 0 || ni >= L.nx) {
    if (L.bc[0] != VPLBM_PERIODIC) return false;
    ni = ni < 0 ? ni + L.nx : ni - L.nx;
  }
  if (nj < 0 || nj >= L.ny) {
    if (L.bc[2] != VPLBM_PERIODIC) return false;
    nj = nj < 0 ? nj + L.ny : nj - L.ny;
  }
  return true;
}

// ---------------------------------------------------------------------------
// the force region: the tiles that can hold MEM links (the body's box with a
// margin); only their blocks and the SIM blocks take part in the reduction
// ---------------------------------------------------------------------------
struct ForceRegion {
  int32_t ti0, ti1, tj0, tj1;  // inclusive tile ranges
  int32_t count;               // number of region tiles (>= 1)
  int32_t error;               // nonzero: the body left the lattice
};

// nodes of margin around a body for its force region; a moving body travels
// less than one node per step, so its mask update stays inside the region
constexpr int kRegionMargin = 4;

// ---------------------------------------------------------------------------
// parameters of the fused step kernel
// ---------------------------------------------------------------------------
struct StepArgs {
  Lattice L;
  const void *src;      // populations: post-collision of level n-1 (gather)
                        // or pre-collision of level n (first step)
  void *dst;            // post-collision populations of level n
  const void *prev_src;  // outlet column (compute type), pre-collision, level n-1
  void *prev_dst;        // outlet column, pre-collision, level n
  uint8_t *chi;
  const BodyState *body_src;   // body at level n
  BodyState *body_dst;         // body at level n + 1 (written by the tail)
  const ForceRegion *reg_src;
  ForceRegion *reg_dst;
  unsigned long long *acc;       // [6][2] fixed-point sums of this step
  unsigned long long *acc_prev;  // the previous step's sums (finalized by this launch)
  int32_t defer;                 // 1: no ticket and tail; a later launch finalizes the sums
  int32_t finalize_prev;         // 1: an extra last block finalizes acc_prev first
  int32_t prev_sim;              // 1: the step being finalized evaluated SIM
  const SimPoint *sim_pts;
  int32_t *sim_nodes;    // [n_sim]
  int32_t n_sim;
  int32_t sim_order;     // 0: stress copied from the sampled node; 1: extrapolated linearly
  int32_t sim_blocks;    // leading blocks that evaluate SIM (0: SIM not due)
  int32_t sim_per_block; // SIM points per block (a multiple of 32)
  double *hist;          // [hist_len][6]
  int32_t hist_len;
  int32_t pad0;
  double *sums;          // [6]
  long long *counts;     // [2]
  long long *dev_step;   // steps completed
  unsigned int *ticket;
  int32_t *status;
  // collision constants, FP64 and FP32 copies (FP32 paths must not convert
  // from FP64 per node: GB300 runs FP64 at a small fraction of FP32)
  double s_plus, s_minus;  // 1/tau+, 1/tau-
  double a_plus, a_minus;  // forcing prefactors
  double half_pen;         // dt/(2 eta)
  double tau_plus;
  double sim_const[3];     // -(1/3) sum S n and its moment: the SIM constant part
  float f_s_plus, f_s_minus, f_a_plus, f_a_minus, f_half_pen, f_sim_s;
  int32_t ntiles_x, ntiles_y;
  int32_t region_capacity;  // most force-region tiles a step may hold
  int32_t tile_w;           // nodes along x of one tile
  int32_t all_tiles;        // 1: the special kernel updates every tile (first step)
  int32_t n_edge;           // nodes on the lattice edges
  int32_t edge_blocks;      // special-kernel blocks for the edge nodes
  int32_t region_slots;     // special-kernel blocks reserved for force-region tiles
  int32_t raster;           // 1 (a moving body): the force-region tiles rasterise chi
                            // from body_src themselves, and SIM tests nodes with the
                            // predicate instead of reading chi
  int32_t sr;               // 1: 16-bit stores round stochastically
  const unsigned long long *rng_src;  // the rounding counter of this step's level
  unsigned long long *rng_dst;        // ... and of the next (written by the special kernel)
};

// storage type of a dtype's populations, for the kernels' dispatch: the
// stochastically rounded forms store FP16 / BF16 like the nearest-rounded ones
__host__ __device__ inline int storage_dtype(int dtype) {
  return dtype == VPLBM_F16_SR ? VPLBM_F16_OFS : (dtype == VPLBM_BF16_SR ? VPLBM_BF16_OFS : dtype);
}
__host__ __device__ inline bool stochastic_dtype(int dtype) {
  return dtype == VPLBM_F16_SR || dtype == VPLBM_BF16_SR;
}

// ---------------------------------------------------------------------------
// stochastic rounding to 16 bits
// ---------------------------------------------------------------------------
// 32-bit hash of a 32-bit input: the "PCG hash" of Jarzynski and Olano, Hash
// Functions for GPU Rendering, JCGT 9(3), 2020 (one step of a PCG generator
// with an RXS-M-XS output permutation).
__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
  const uint32_t state = v * 747796405u + 2891336453u;
  const uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

// Stochastic rounding by the conversion instruction of sm_100 and later
// (cvt.rs): a pair of FP32 values to a packed pair of 16-bit values, each
// rounded to one of its two neighbours in the format, away from zero with
// probability (distance from the one toward zero) / (their spacing).  The
// instruction adds random bits just below the kept ones and truncates; the
// lower element takes bits 0..12 (FP16) or 0..15 (BF16) of rbits, the upper
// element bits 16..28 or 16..31.  With all of the value's dropped bits covered
// by the random ones (13 for FP16 in its normal range, 16 for BF16) the
// rounding is exactly unbiased.
template <typename S>
struct Stochastic;
template <>
struct Stochastic<__half> {
  static __device__ __forceinline__ uint32_t pair(float lo, float hi, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
  }
};
template <>
struct Stochastic<__nv_bfloat16> {
  static __device__ __forceinline__ uint32_t pair(float lo, float hi, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
  }
};


// the nodes on the lattice edges, enumerated: first row, last row, then the
// first and the last column between them
__host__ __device__ inline int edge_count(int nx, int ny) { return 2 * nx + 2 * (ny - 2); }
__host__ __device__ inline void edge_node(int e, int nx, int ny, int &i, int &j) {
  if (e < nx) {
    i = e;
    j = 0;
    return;
  }
  e -= nx;
  if (e < nx) {
    i = e;
    j = ny - 1;
    return;
  }
  e -= nx;
  if (e < ny - 2) {
    i = 0;
    j = 1 + e;
    return;
  }
  i = nx - 1;
  j = 1 + (e - (ny - 2));
}

// collision constants in the compute type
template <typename T>
struct Consts;
template <>
struct Consts<double> {
  double s_plus, s_minus, a_plus, a_minus, half_pen, sim_s, urx, ury;
  __device__ __forceinline__ explicit Consts(const StepArgs &p)
      : s_plus(p.s_plus), s_minus(p.s_minus), a_plus(p.a_plus), a_minus(p.a_minus),
        half_pen(p.half_pen), sim_s(1.0 - 0.5 / p.tau_plus), urx(p.L.ur[0]), ury(p.L.ur[1]) {}
};
template <>
struct Consts<float> {
  float s_plus, s_minus, a_plus, a_minus, half_pen, sim_s, urx, ury;
  __device__ __forceinline__ explicit Consts(const StepArgs &p)
      : s_plus(p.f_s_plus), s_minus(p.f_s_minus), a_plus(p.f_a_plus), a_minus(p.f_a_minus),
        half_pen(p.f_half_pen), sim_s(p.f_sim_s), urx(p.L.ur_f[0]), ury(p.L.ur_f[1]) {}
};

// tile range of the force region of a body whose bounding box is
// [x0, x1] x [y0, y1], widened by kRegionMargin nodes
__host__ __device__ inline ForceRegion make_region_box(const Lattice &L, double x0, double x1,
                                                       double y0, double y1, int ntiles_x,
                                                       int ntiles_y, int tile_w) {
  ForceRegion g{};
  const double m = kRegionMargin;
  int i0 = (int)floor(x0 - m), i1 = (int)ceil(x1 + m);
  int j0 = (int)floor(y0 - m), j1 = (int)ceil(y1 + m);
  g.error = (i0 < -kRegionMargin || j0 < -kRegionMargin || i1 > L.nx - 1 + kRegionMargin ||
             j1 > L.ny - 1 + kRegionMargin || !(x0 == x0) || !(y0 == y0) || !(x1 == x1) ||
             !(y1 == y1))
                ? 1
                : 0;
  i0 = i0 < 0 ? 0 : (i0 > L.nx - 1 ? L.nx - 1 : i0);
  i1 = i1 < 0 ? 0 : (i1 > L.nx - 1 ? L.nx - 1 : i1);
  j0 = j0 < 0 ? 0 : (j0 > L.ny - 1 ? L.ny - 1 : j0);
  j1 = j1 < 0 ? 0 : (j1 > L.ny - 1 ? L.ny - 1 : j1);
  g.ti0 = i0 / tile_w;
  g.ti1 = i1 / tile_w;
  g.tj0 = j0 / kTileY;
  g.tj1 = j1 / kTileY;
  if (g.ti1 > ntiles_x - 1) g.ti1 = ntiles_x - 1;
  if (g.tj1 > ntiles_y - 1) g.tj1 = ntiles_y - 1;
  g.count = (g.ti1 - g.ti0 + 1) * (g.tj1 - g.tj0 + 1);
  return g;
}

// the same for a disk of radius r centred at (xg, yg)
__host__ __device__ inline ForceRegion make_region(const Lattice &L, double xg, double yg,
                                                   double r, int ntiles_x, int ntiles_y,
                                                   int tile_w) {
  return make_region_box(L, xg - r, xg + r, yg - r, yg + r, ntiles_x, ntiles_y, tile_w);
}

// failure text of calls without a context (api.cu), read by vplbm_last_error(NULL)
void set_global_error(const std::string &msg);

// launches (step.cu)
// the special kernel: SIM blocks, edge nodes, force-region tiles and the
// FP64 tail (or every tile, with all_tiles set)
cudaError_t launch_special(int dtype, bool gather, const StepArgs &a, cudaStream_t s);
// one block that finalizes a deferred step's force sums (acc_prev): history
// row, running sums, step counter
cudaError_t launch_finalize(int dtype, const StepArgs &a, cudaStream_t s);
// chi of a moving body at the current time level on the force-region tiles
// (reg_src, body_src): the mask the read-backs see after a call
cudaError_t launch_mask(const StepArgs &a, cudaStream_t s);
// the walks of a fixed body's SIM points, stored in the points (sim_pts,
// n_sim, chi, body_src of a)
cudaError_t launch_sim_cache(const StepArgs &a, cudaStream_t s);
// the bulk kernel: the nodes off the edges, outside the force-region tiles
// the bulk kernel in one of kBulkVariants launch forms (same results, bit
// for bit): FP32 and FP64 blocks of 1, 2 or 4 tiles; 16-bit storage with
// eight nodes per thread at 96 or 126 registers, or four nodes per thread
constexpr int kBulkVariants = 3;
cudaError_t launch_bulk(int dtype, int variant, const StepArgs &a, cudaStream_t s);

// auxiliary kernels (aux.cu)
cudaError_t launch_raster(const Lattice &L, const BodyState *body, uint8_t *chi, int i0, int j0,
                          int i1, int j1, cudaStream_t s);
cudaError_t launch_interface(const Lattice &L, uint8_t *chi, int i0, int j0, int i1, int j1,
                             cudaStream_t s);
cudaError_t launch_init(int dtype, const Lattice &L, const BodyState *body, const uint8_t *chi,
                        void *buf, double u0x, double u0y, cudaStream_t s);
// read-backs of the rows j0 .. j0 + rows - 1, written compactly ([rows][nx]
// per output plane); get_f writes the planes a0 .. a0 + na - 1
cudaError_t launch_get_f(int dtype, bool gather, const Lattice &L, const void *buf,
                         const void *prev, double *out, int a0, int na, int j0, int rows,
                         cudaStream_t s);
cudaError_t launch_get_fields(int dtype, bool gather, const Lattice &L, const void *buf,
                              const void *prev, const uint8_t *chi, const BodyState *body,
                              double half_pen, double *rho, double *ux, double *uy, int j0,
                              int rows, cudaStream_t s);
cudaError_t launch_set_state(int dtype, const Lattice &L, const double *f, void *buf,
                             cudaStream_t s);
cudaError_t launch_set_prev(int dtype, const Lattice &L, const double *f, void *prev,
                            cudaStream_t s);
cudaError_t launch_get_mask(const Lattice &L, const uint8_t *chi, uint8_t *out, int j0, int rows,
                            cudaStream_t s);

}  // namespace vplbm
