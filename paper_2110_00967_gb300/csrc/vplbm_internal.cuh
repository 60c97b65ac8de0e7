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

constexpr int kTileX = 128;  // threads along x per block (4 warps per row)
constexpr int kTileY = 2;    // rows per block
constexpr int kThreads = kTileX * kTileY;
constexpr int kMaxBlocks = 8192;  // capacity of the MEM partial array

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
  static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
  static __device__ __forceinline__ double from_double(double v) { return v; }
};
template <>
struct Store<float> {
  using T = float;
  static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
  static __device__ __forceinline__ float from_double(double v) { return __double2float_rn(v); }
};
template <>
struct Store<__half> {
  using T = float;
  static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ __half from_double(double v) { return __double2half(v); }
};
template <>
struct Store<__nv_bfloat16> {
  using T = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
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
};

struct SimPoint {
  double dx, dy;  // offset of the integration point from the reference point
  double nx, ny;  // outward unit normal
  double s;       // edge length S_i
  int32_t dir;    // lattice direction closest to the normal
  int32_t pad;
};

// ---------------------------------------------------------------------------
// lattice geometry and side conditions, shared by every kernel
// ---------------------------------------------------------------------------
struct Lattice {
  int32_t nx, ny, pitch;
  int32_t bc[4];
  int64_t plane;     // ny * pitch
  double kin[9];     // inlet bounce-back terms 2 w_a (c_a.u_in)/cs2
  double uc;         // convective outlet velocity |u_in|
  double bf[2];      // uniform body force density
};

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
    if (kind == VPLBM_INLET_BB) return pop_at(post, L, opp_of(a), i, j) + (T)L.kin[a];
    return pop_at(post, L, opp_of(a), i, j);  // no-slip bounce-back
  }
  const int kind = L.bc[sj < 0 ? 2 : 3];
  if (kind == VPLBM_SYMMETRY) return pop_at(post, L, flipy_of(a), si, j);
  return pop_at(post, L, opp_of(a), i, j);  // no-slip bounce-back
}

__device__ __forceinline__ int outlet_slot(int a) { return a == 3 ? 0 : (a == 6 ? 1 : 2); }

template <typename S>
__device__ __forceinline__ typename Store<S>::T gather(const S *post, const double *prev,
                                                        const Lattice &L, int a, int i, int j) {
  using T = typename Store<S>::T;
  if (cx_of(a) < 0 && i == L.nx - 1 && L.bc[1] == VPLBM_OUTLET_CONVECTIVE) {
    // convective outlet: f^{n+1}(N-1) = (f^n(N-1) + U_c f^{n+1}(N-2)) / (1 + U_c)
    const T inner = gather_core(post, L, a, i - 1, j);
    const T old = (T)prev[outlet_slot(a) * L.ny + j];
    return (old + (T)L.uc * inner) / ((T)1 + (T)L.uc);
  }
  return gather_core(post, L, a, i, j);
}

// Pre-collision population of the current level: gathered from the previous
// post-collision field, or read in place when the state is pre-collision.
template <typename S, bool kGather>
__device__ __forceinline__ typename Store<S>::T pre_pop(const S *buf, const double *prev,
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
// parameters of the fused step kernel
// ---------------------------------------------------------------------------
struct StepArgs {
  Lattice L;
  const void *src;      // populations: post-collision of level n-1 (gather)
                        // or pre-collision of level n (first step)
  void *dst;            // post-collision populations of level n
  const double *prev_src;  // outlet column, pre-collision, level n-1
  double *prev_dst;        // outlet column, pre-collision, level n
  uint8_t *chi;
  BodyState *body;
  double *mem_partials;  // [gridDim.x][3]
  const SimPoint *sim_pts;
  double *sim_contrib;   // [n_sim][3]
  int32_t *sim_nodes;    // [n_sim]
  int32_t n_sim;
  int32_t do_sim;
  double *hist;          // [hist_len][6]
  int32_t hist_len;
  int32_t pad0;
  double *sums;          // [6]
  long long *counts;     // [2]
  long long *dev_step;   // steps completed
  unsigned int *ticket;
  int32_t *status;
  // collision constants
  double s_plus, s_minus;  // 1/tau+, 1/tau-
  double a_plus, a_minus;  // forcing prefactors
  double half_pen;         // dt/(2 eta)
  double tau_plus;
  int32_t ntiles_x, ntiles;
};

// launches (step.cu)
cudaError_t launch_step(int dtype, bool gather, const StepArgs &a, int grid, cudaStream_t s);
int step_blocks_per_sm(int dtype, bool gather);

// auxiliary kernels (aux.cu)
cudaError_t launch_raster(const Lattice &L, const BodyState *body, uint8_t *chi, int i0, int j0,
                          int i1, int j1, cudaStream_t s);
cudaError_t launch_interface(const Lattice &L, uint8_t *chi, int i0, int j0, int i1, int j1,
                             cudaStream_t s);
cudaError_t launch_init(int dtype, const Lattice &L, const BodyState *body, const uint8_t *chi,
                        void *buf, double u0x, double u0y, cudaStream_t s);
cudaError_t launch_get_f(int dtype, bool gather, const Lattice &L, const void *buf,
                         const double *prev, double *out, cudaStream_t s);
cudaError_t launch_get_fields(int dtype, bool gather, const Lattice &L, const void *buf,
                              const double *prev, const uint8_t *chi, const BodyState *body,
                              double half_pen, double *rho, double *ux, double *uy,
                              cudaStream_t s);
cudaError_t launch_set_state(int dtype, const Lattice &L, const double *f, void *buf,
                             cudaStream_t s);
cudaError_t launch_set_prev(const Lattice &L, const double *f, double *prev, cudaStream_t s);
cudaError_t launch_get_mask(const Lattice &L, const uint8_t *chi, uint8_t *out, cudaStream_t s);

}  // namespace vplbm
