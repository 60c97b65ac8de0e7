// step.cu -- the VP-LBM time step for sm_103a.
//
// One time step is two launches that write disjoint nodes:
//   * the special kernel: the SIM points (stress of Sec. 2.3.2 at the
//     sampled fluid node from its pre-collision populations, S_i sigma n_i
//     and its moment, Eq. defFf), the nodes on the lattice edges (side
//     conditions of Sec. 3.1/3.2), and the tiles of the force region around
//     the body (penalized nodes and the MEM link terms of Eq. MMEL /
//     Eq. fluidtorque).  Its SIM and region blocks add their force terms into
//     exact fixed-point sums.  For a moving body the region tiles rasterise
//     the mask of the body's current position themselves (each tile with a
//     one-node halo), the blocks take a ticket and the last of them records
//     the step's forces and applies the FP64 rigid-body update (Eqs. dep1,
//     theta2); for a fixed body one extra block of the next step's launch
//     records them.
//   * the bulk kernel: every other node -- pull streaming (Eq. eqBd) and the
//     BGK/TRT collision (Eq. TRT) of fluid nodes whose sources all lie inside
//     the lattice; no mask, no side conditions, no forces.  It comes in
//     several launch forms with identical results (bulk_kernel for FP32/FP64,
//     bulk16_kernel and bulk16x4_kernel for 16-bit storage).
// For the first step after a pre-collision state the special kernel updates
// every tile.
#include "vplbm_internal.cuh"

namespace vplbm {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// exact force sums
// ---------------------------------------------------------------------------
template <typename T>
struct FixAcc {
  long long f[3][Fix<T>::kWords];
  __device__ __forceinline__ FixAcc() {
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int k = 0; k < Fix<T>::kWords; ++k) f[q][k] = 0;
  }
  __device__ __forceinline__ void add(int q, T v) {
    long long w[Fix<T>::kWords];
    Fix<T>::split(v, w);
#pragma unroll
    for (int k = 0; k < Fix<T>::kWords; ++k) f[q][k] += w[k];
  }
};

// adds the warp's fixed-point words into acc[slot][word] for the three
// quantities starting at slot base
template <typename T>
__device__ __forceinline__ void warp_add(const FixAcc<T> &a, unsigned long long *acc, int base) {
  constexpr int W = Fix<T>::kWords;
  long long v[3][W];
  long long any = 0;
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int k = 0; k < W; ++k) {
      v[q][k] = a.f[q][k];
      any |= v[q][k];
    }
  if (!__any_sync(kFull, any != 0)) return;
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int k = 0; k < W; ++k)
      for (int o = 16; o > 0; o >>= 1) v[q][k] += __shfl_xor_sync(kFull, v[q][k], o);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int k = 0; k < W; ++k)
        if (v[q][k]) atomicAdd(acc + 2 * (base + q) + k, (unsigned long long)v[q][k]);
  }
}

// ---------------------------------------------------------------------------
// SIM (Sec. 2.3.2)
// ---------------------------------------------------------------------------

// The part of the stress beyond -(1/3) I at a fluid node,
// sigma + (1/3) I = -(rho - 1)/3 I - (1 - 1/(2 tau+)) sum c c (f - feq),
// from its pre-collision offsets, in the compute type (all terms are small;
// f - feq = h - heq, with heq the equilibrium's offset as in collide()).
template <typename S, bool kGather>
__device__ __forceinline__ void node_stress(const S *buf, const typename Store<S>::T *prev,
                                            const Lattice &L, const Consts<typename Store<S>::T> &c,
                                            int i, int j, typename Store<S>::T sig[3]) {
  using T = typename Store<S>::T;
  T h[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) h[a] = pre_pop<S, kGather>(buf, prev, L, a, i, j);
  T drho = 0, jx = 0, jy = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    drho += h[a];
    jx += (T)cx_of(a) * h[a];
    jy += (T)cy_of(a) * h[a];
  }
  const T rho = (T)1 + drho;
  const T inv = (T)1 / rho;
  const T dux = (jx + (T)0.5 * lat_bf<T>(L, 0) - drho * c.urx) * inv;
  const T duy = (jy + (T)0.5 * lat_bf<T>(L, 1) - drho * c.ury) * inv;
  const T ux = c.urx + dux, uy = c.ury + duy, uu = ux * ux + uy * uy;
  const T dsu = dux * (ux + c.urx) + duy * (uy + c.ury);
  T pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const T cu = (T)cx_of(a) * ux + (T)cy_of(a) * uy;
    const T cdu = (T)cx_of(a) * dux + (T)cy_of(a) * duy;
    const T csu = cu + ((T)cx_of(a) * c.urx + (T)cy_of(a) * c.ury);
    const T heq = (T)w_of(a) * (drho * ((T)1 + (T)3 * cu + (T)4.5 * cu * cu - (T)1.5 * uu) +
                                (T)3 * cdu + (T)4.5 * cdu * csu - (T)1.5 * dsu);
    const T d = h[a] - heq;
    pxx += (T)(cx_of(a) * cx_of(a)) * d;
    pxy += (T)(cx_of(a) * cy_of(a)) * d;
    pyy += (T)(cy_of(a) * cy_of(a)) * d;
  }
  sig[0] = -drho / (T)3 - c.sim_s * pxx;
  sig[1] = -c.sim_s * pxy;
  sig[2] = -drho / (T)3 - c.sim_s * pyy;
}

// mask byte of node (i, j) (inside the lattice) as SIM and MEM see it: chi,
// or for a moving body the predicate of Eq. fcar on the current body, since
// the force-region tiles rewrite chi during the step
__device__ __forceinline__ uint8_t solid_at(const StepArgs &p, int i, int j) {
  if (p.raster) return body_contains(*p.body_src, i, j) ? kSolid : (uint8_t)0;
  return p.chi[(int64_t)j * p.L.pitch + i];
}

// first fluid node of q_k = (qi, qj) + k c_a, k = 0..3, inside the lattice
// (the four mask bytes are loaded together)
__device__ __forceinline__ bool sim_walk(const StepArgs &p, int a, int qi, int qj, int &oi,
                                         int &oj) {
  const Lattice &L = p.L;
  uint8_t m[4];
  bool in[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int ii = qi + k * cx_of(a), jj = qj + k * cy_of(a);
    in[k] = ii >= 0 && ii < L.nx && jj >= 0 && jj < L.ny;
    m[k] = in[k] ? solid_at(p, ii, jj) : (uint8_t)kSolid;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!in[k]) return false;
    if (!(m[k] & kSolid)) {
      oi = qi + k * cx_of(a);
      oj = qj + k * cy_of(a);
      return true;
    }
  }
  return false;
}

template <typename T>
__device__ __forceinline__ void sim_geom(const SimPoint &sp, T &dx, T &dy, T &nx, T &ny, T &s);
template <>
__device__ __forceinline__ void sim_geom<double>(const SimPoint &sp, double &dx, double &dy,
                                                 double &nx, double &ny, double &s) {
  dx = sp.dx; dy = sp.dy; nx = sp.nx; ny = sp.ny; s = sp.s;
}
template <>
__device__ __forceinline__ void sim_geom<float>(const SimPoint &sp, float &dx, float &dy,
                                                float &nx, float &ny, float &s) {
  dx = sp.f_dx; dy = sp.f_dy; nx = sp.f_nx; ny = sp.f_ny; s = sp.f_s;
}

// The sampled nodes of SIM point sp for the reference point (bxg, byg): the
// nearest node (both nodes when the point lies exactly half-way: the
// coordinates are compared in FP64), each walked along the direction closest
// to the normal to the first fluid node.  Returns their count (1, 2 or 4; 0
// when a walk finds no fluid node), the nodes packed i | j << 16 in the order
// the stress sum takes them.
__device__ __forceinline__ int sim_candidates(const StepArgs &p, const SimPoint &sp, double bxg,
                                              double byg, uint32_t (&cand)[4]) {
  const double x = bxg + sp.dx, y = byg + sp.dy;
  const double rx = floor(x + 0.5), ry = floor(y + 0.5);
  const int ncx = (rx == x + 0.5) ? 2 : 1, ncy = (ry == y + 0.5) ? 2 : 1;
  int n = 0;
  for (int u = 0; u < ncy; ++u)
    for (int v = 0; v < ncx; ++v) {
      int qi, qj;
      if (!sim_walk(p, sp.dir, (int)rx - v, (int)ry - u, qi, qj)) return 0;
      cand[n++] = (uint32_t)qi | ((uint32_t)qj << 16);
    }
  return n;
}

// The walks of a fixed body's SIM points, once when the body is placed (the
// mask never changes afterwards): one thread per point.
__global__ void sim_cache_kernel(const StepArgs p) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.n_sim) return;
  SimPoint *sp = const_cast<SimPoint *>(p.sim_pts) + q;
  uint32_t cand[4] = {0u, 0u, 0u, 0u};
  const int n = sim_candidates(p, *sp, p.body_src->xg, p.body_src->yg, cand);
#pragma unroll
  for (int k = 0; k < 4; ++k) sp->cand[k] = cand[k];
  sp->n_cand = n;
}

// One SIM integration point: its sampled nodes (walked now, or for a fixed
// body found when it was placed), the stress averaged over them, then
// S (sigma + I/3) n and its moment; the -(1/3) S n part sums to a constant of
// the polygon added in the tail.
template <typename S, bool kGather>
__device__ __noinline__ FixAcc<typename Store<S>::T> sim_point(const StepArgs &p, const S *buf, double bxg, double byg,
                                         int q, bool &missing) {
  using T = typename Store<S>::T;
  const SimPoint sp = p.sim_pts[q];
  uint32_t cand[4] = {sp.cand[0], sp.cand[1], sp.cand[2], sp.cand[3]};
  const int n = sp.n_cand >= 0 ? sp.n_cand : sim_candidates(p, sp, bxg, byg, cand);
  const T *prev = static_cast<const T *>(p.prev_src);
  T sig[3] = {0, 0, 0};
  int first = -1;
  const bool ok = n > 0;
  for (int k = 0; k < n; ++k) {
    const int qi = (int)(cand[k] & 0xffffu), qj = (int)(cand[k] >> 16);
    if (first < 0) first = qj * p.L.nx + qi;
    T s3[3];
    node_stress<S, kGather>(buf, prev, p.L, Consts<T>(p), qi, qj, s3);
    if (p.sim_order == 1) {
      // first order: extrapolated to the point along the direction from
      // the next node, where that node is fluid and inside the lattice
      const int ni = qi + cx_of(sp.dir), nj = qj + cy_of(sp.dir);
      if (ni >= 0 && ni < p.L.nx && nj >= 0 && nj < p.L.ny && !(solid_at(p, ni, nj) & kSolid)) {
        T s3n[3];
        node_stress<S, kGather>(buf, prev, p.L, Consts<T>(p), ni, nj, s3n);
        const double x = bxg + sp.dx, y = byg + sp.dy;
        const int c2 = cx_of(sp.dir) * cx_of(sp.dir) + cy_of(sp.dir) * cy_of(sp.dir);
        const T t = (T)(((x - qi) * cx_of(sp.dir) + (y - qj) * cy_of(sp.dir)) / (double)c2);
        s3[0] += t * (s3n[0] - s3[0]);
        s3[1] += t * (s3n[1] - s3[1]);
        s3[2] += t * (s3n[2] - s3[2]);
      }
    }
    sig[0] += s3[0];
    sig[1] += s3[1];
    sig[2] += s3[2];
  }
  p.sim_nodes[q] = ok ? first : -1;
  missing = !ok;
  FixAcc<T> r;
  if (!ok) return r;
  // mean over 1, 2 or 4 candidates: an exact power-of-two scaling
  const T inv = (n == 1) ? (T)1 : ((n == 2) ? (T)0.5 : (T)0.25);
  T dx, dy, nx, ny, sl;
  sim_geom<T>(sp, dx, dy, nx, ny, sl);
  const T sxx = sig[0] * inv, sxy = sig[1] * inv, syy = sig[2] * inv;
  const T tx = sl * (sxx * nx + sxy * ny);
  const T ty = sl * (sxy * nx + syy * ny);
  r.add(0, tx);
  r.add(1, ty);
  r.add(2, dx * ty - dy * tx);
  return r;
}

// ---------------------------------------------------------------------------
// the mask of a moving body, rasterised tile by tile (Eq. fcar)
// ---------------------------------------------------------------------------
// Solid bits of one tile and a one-node halo around it: the predicate of
// Eq. fcar on the body at the step's time level, evaluated by the tile's own
// block, so that no single block re-rasterises the body between steps.
struct TileMask {
  uint8_t s[kTileY + 2][kTileX + 2];
};

__device__ __forceinline__ void tile_solid(const StepArgs &p, int ti, int tj, TileMask &tm) {
  const Lattice &L = p.L;
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  for (int q = tid; q < (kTileY + 2) * (kTileX + 2); q += kThreads) {
    const int hx = q % (kTileX + 2), hy = q / (kTileX + 2);
    int gi = ti * kTileX + hx - 1, gj = tj * kTileY + hy - 1;
    // halo nodes across a periodic side are the nodes there; beyond another
    // side they are never a neighbour (neighbour() gives false)
    if (L.bc[0] == VPLBM_PERIODIC) gi = gi < 0 ? gi + L.nx : (gi >= L.nx ? gi - L.nx : gi);
    if (L.bc[2] == VPLBM_PERIODIC) gj = gj < 0 ? gj + L.ny : (gj >= L.ny ? gj - L.ny : gj);
    const bool in = gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny;
    tm.s[hy][hx] = (in && body_contains(*p.body_src, gi, gj)) ? kSolid : (uint8_t)0;
  }
}

// mask byte (solid bit and interface bit) of the tile node (tx, ty) at (i, j)
__device__ __forceinline__ uint8_t tile_mask_byte(const Lattice &L, const TileMask &tm, int i,
                                                  int j, int tx, int ty) {
  const uint8_t self = tm.s[ty + 1][tx + 1];
  bool iface = false;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    int ni, nj;
    if (neighbour(L, a, i, j, ni, nj) && tm.s[ty + 1 + cy_of(a)][tx + 1 + cx_of(a)] != self)
      iface = true;
  }
  return (uint8_t)(self | (iface ? kInterface : 0));
}

// ---------------------------------------------------------------------------
// MEM (Sec. 2.3.1)
// ---------------------------------------------------------------------------

// The link terms of one interface node (Eq. MMEL): for each lattice
// neighbour of the other phase, the fluid end adds (c_a - u_Gamma) f~_a and
// the solid end subtracts its own (c_a - u_Gamma) f~_a, with x_Gamma the link
// midpoint and u_Gamma the rigid velocity there; torques about the reference
// point (Eq. fluidtorque).  f~ = h~ + E is split so that the E parts, which
// cancel in pairs around a fixed body, are rounded exactly.  The neighbours'
// phases come from chi, or from the tile's mask when it rasterises its own.
template <typename T>
__device__ __forceinline__ void mem_terms(const StepArgs &p, const T (&o)[9], int i, int j,
                                          uint8_t m, const TileMask *tm, FixAcc<T> &acc) {
  const Lattice &L = p.L;
  const BodyRef<T> b(*p.body_src);
  const bool solid = m & kSolid;
  const T sg = solid ? (T)-1 : (T)1;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    int ni, nj;
    if (!neighbour(L, a, i, j, ni, nj)) continue;
    const bool nsolid = tm ? (tm->s[threadIdx.y + 1 + cy_of(a)][threadIdx.x + 1 + cx_of(a)] & kSolid)
                           : (p.chi[(int64_t)nj * L.pitch + ni] & kSolid);
    if (nsolid == solid) continue;
    const T rx = ((T)i - b.xg) + (T)(0.5 * cx_of(a));
    const T ry = ((T)j - b.yg) + (T)(0.5 * cy_of(a));
    const T vx = (T)cx_of(a) - (b.ux - b.om * ry);
    const T vy = (T)cy_of(a) - (b.uy + b.om * rx);
    const T ah = sg * o[a], aw = sg * LatC<T>::E(L, a);
    const T lxh = vx * ah, lyh = vy * ah, lxw = vx * aw, lyw = vy * aw;
    acc.add(0, lxh);
    acc.add(0, lxw);
    acc.add(1, lyh);
    acc.add(1, lyw);
    acc.add(2, rx * lyh - ry * lxh);
    acc.add(2, rx * lyw - ry * lxw);
  }
}

// ---------------------------------------------------------------------------
// rigid body and the tail
// ---------------------------------------------------------------------------

// Rigid-body update (Eqs. dep1 and theta2, explicit trapezoid in time) for a
// disk of density ratio rho_s/rho in a fluid of density 1.
__device__ void rigid_update(BodyState &b, const double F[3]) {
  const double r = 0.5 * b.length;
  const double m = b.density_ratio * 3.14159265358979323846 * r * r;
  const double inertia = 0.5 * m * r * r;
  const double buoy = 1.0 - 1.0 / b.density_ratio;
  const double ax = F[0] / m + buoy * b.gx;
  const double ay = F[1] / m + buoy * b.gy;
  const double u0x = b.ux, u0y = b.uy, w0 = b.omega;
  b.ux = u0x + ax;
  b.uy = u0y + ay;
  b.omega = w0 + F[2] / inertia;
  b.xg += 0.5 * (u0x + b.ux);
  b.yg += 0.5 * (u0y + b.uy);
  b.theta += 0.5 * (w0 + b.omega);
  body_sync_f32(b);
}

// Force bookkeeping of a step whose tail was deferred (a fixed body): its
// fixed-point sums (acc) become the step's history row and are added to the
// running sums; the step counter advances and acc is cleared for reuse two
// steps later.  Runs in one block beside the next step's work, or alone at
// the end of a call.  Loads are spread over threads and issued together.
template <typename T>
__device__ void finalize(const StepArgs &p, unsigned long long *acc) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  __shared__ double tot[kAccSlots];
  __shared__ long long step_s;
  const bool do_sim = p.prev_sim != 0;
  if (tid < kAccSlots) {
    const long long w0 = (long long)__ldcg(acc + 2 * tid);
    const long long w1 = (long long)__ldcg(acc + 2 * tid + 1);
    double v = Fix<T>::value(w0, w1);
    if (tid >= 3 && tid < 6) v += p.sim_const[tid - 3];
    tot[tid] = v;
  } else if (tid == 64) {
    step_s = __ldcg(p.dev_step);
  }
  __syncthreads();
  if (tid < kHistCols) {
    // MEM (0-2) and the volume integral (6-8) every step, SIM (3-5) when due
    const bool have = tid < 3 || tid >= 6 || do_sim;
    p.hist[kHistCols * (step_s % p.hist_len) + tid] =
        have ? tot[tid] : __longlong_as_double(0x7ff8000000000000LL);
    if (have && tid < 6) p.sums[tid] += tot[tid];
  } else if (tid == 16) {
    p.counts[0] += 1;
  } else if (tid == 17 && do_sim) {
    p.counts[1] += 1;
  } else if (tid == 32) {
    *p.dev_step = step_s + 1;
  }
  if (tid < kAccWords) acc[tid] = 0ull;  // every read of acc above precedes the barrier
}

// The last participating block: the step's forces from the fixed-point sums
// (plus the polygon's constant SIM part), histories, running sums, body.
// Its loads are spread over threads and issued together, and each thread then
// stores its own words: the tail costs a few memory round trips, not one per
// word.
template <typename T>
__device__ void tail(const StepArgs &p, const ForceRegion &reg) {
  constexpr int kBodyWords = (int)(sizeof(BodyState) / sizeof(unsigned long long));
  static_assert(sizeof(BodyState) % sizeof(unsigned long long) == 0, "BodyState in 8-byte words");
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  __shared__ double tot[kAccSlots];
  __shared__ BodyState old_b, new_b;
  __shared__ long long step_s;
  const bool do_sim = p.sim_blocks > 0;
  if (tid < kAccSlots) {
    // the sums were added by other SMs: read them through L2
    const long long w0 = (long long)__ldcg(p.acc + 2 * tid);
    const long long w1 = (long long)__ldcg(p.acc + 2 * tid + 1);
    double v = Fix<T>::value(w0, w1);
    if (tid >= 3 && tid < 6) v += p.sim_const[tid - 3];
    tot[tid] = v;
  } else if (tid >= 32 && tid < 32 + kBodyWords) {
    reinterpret_cast<unsigned long long *>(&old_b)[tid - 32] =
        __ldcg(reinterpret_cast<const unsigned long long *>(p.body_src) + (tid - 32));
  } else if (tid == 64) {
    step_s = __ldcg(p.dev_step);
  }
  __syncthreads();
  if (tid < kHistCols) {
    // MEM (0-2) and the volume integral (6-8) every step, SIM (3-5) when due
    const bool have = tid < 3 || tid >= 6 || do_sim;
    p.hist[kHistCols * (step_s % p.hist_len) + tid] =
        have ? tot[tid] : __longlong_as_double(0x7ff8000000000000LL);
    if (have && tid < 6) p.sums[tid] += tot[tid];
  } else if (tid == 16) {
    p.counts[0] += 1;
  } else if (tid == 17 && do_sim) {
    p.counts[1] += 1;
  } else if (tid == 32) {
    new_b = old_b;
    ForceRegion nreg = reg;
    if (old_b.moving) {
      const bool sim = old_b.estimator == VPLBM_SIM;
      const double F[3] = {sim ? tot[3] : tot[0], sim ? tot[4] : tot[1], sim ? tot[5] : tot[2]};
      rigid_update(new_b, F);
      nreg = make_region(p.L, new_b.xg, new_b.yg, 0.5 * new_b.length, p.ntiles_x, p.ntiles_y,
                         p.tile_w);
      if (nreg.error || nreg.count > p.region_slots || nreg.count > p.region_capacity ||
          fabs(new_b.xg - old_b.xg) >= 1.0 || fabs(new_b.yg - old_b.yg) >= 1.0) {
        // the body left the lattice or moved a node in one step: keep it
        // where it was and flag the run as unstable
        atomicOr(p.status, kStatusUnstable);
        new_b = old_b;
        nreg = reg;
      }
    }
    *p.reg_dst = nreg;
    *p.dev_step = step_s + 1;
  }
  __syncthreads();
  if (tid >= 32 && tid < 32 + kBodyWords)
    reinterpret_cast<unsigned long long *>(p.body_dst)[tid - 32] =
        reinterpret_cast<const unsigned long long *>(&new_b)[tid - 32];
  __syncthreads();
  if (tid < kAccWords) p.acc[tid] = 0ull;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    *p.ticket = 0u;
  }
}

// ---------------------------------------------------------------------------
// node update
// ---------------------------------------------------------------------------

// Coefficients 3 w_a of the odd (momentum-carrying) part of the equilibrium
// and of the forcing term, for the axis directions (k1 = 3 w_1 = 1/3) and the
// diagonals (k2 = 3 w_5 = 1/12).  In the compute type they are chosen with
// 2 k1 + 4 k2 = 1 exactly, so that the odd equilibrium carries exactly the
// node's momentum: with the rounded weights 1/9 and 1/36 of FP32 (both
// 7.45e-9 too large) every collision would add 7.45e-9 s- of the momentum
// offset, a bias that compounds step after step.
template <typename T>
struct OddW;
template <>
struct OddW<double> {
  static constexpr double k1 = 1.0 / 3.0;
  static constexpr double k2 = (1.0 - 2.0 * (1.0 / 3.0)) / 4.0;  // exact: 2 k1 + 4 k2 = 1
};
template <>
struct OddW<float> {
  static constexpr float k1 = 0x1.555556p-2f;  // 1/3 rounded
  static constexpr float k2 = 0x1.555554p-4f;  // (1 - 2 k1) / 4, exactly
};
template <typename T>
__device__ __forceinline__ constexpr T odd_w(int a) {
  return a <= 4 ? OddW<T>::k1 : OddW<T>::k2;
}

// BGK/TRT collision with the forcing term (Eq. TRT) of one node, into o.
// The equilibrium enters through its offset heq = feq(rho, u) - E, written
// with the small quantities drho = rho - 1 and du = u - u_ref only:
// heq_a = w_a [drho (1 + Q_a(u)) + Q_a(u) - Q_a(u_ref)],
// Q_a(u) = 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2, split into its even and odd parts
// for TRT.  kForce = false drops the forcing term (G = 0: a fluid node
// without body force).  The rest population takes what the moving
// populations' even parts give up, o_0 = h_0 - sum_{a>0} (even change of a):
// equal to the relaxation of h_0 towards heq_0 (plus F_0) in exact
// arithmetic, and conserving mass exactly up to the rounding of that sum,
// where rounded weights would make the collision a mass source proportional
// to rho - 1.
template <typename T, bool kForce>
__device__ __forceinline__ void collide(const T (&h)[9], T drho, T dux, T duy, T gx, T gy,
                                        const Consts<T> &c, T (&o)[9]) {
  const T ux = c.urx + dux, uy = c.ury + duy;
  const T uu = ux * ux + uy * uy;
  const T dsu = dux * (ux + c.urx) + duy * (uy + c.ury);  // |u|^2 - |u_ref|^2
  const T ug = kForce ? ux * gx + uy * gy : (T)0;
  T even = 0;  // sum over the pairs of the even change of one population
#pragma unroll
  for (int a = 1; a <= 6; ++a) {
    if (a == 3 || a == 4) continue;
    const int b = opp_of(a);
    const T w = (T)w_of(a);
    const T k = odd_w<T>(a);
    const T cu = (T)cx_of(a) * ux + (T)cy_of(a) * uy;
    const T cdu = (T)cx_of(a) * dux + (T)cy_of(a) * duy;
    const T csu = cu + ((T)cx_of(a) * c.urx + (T)cy_of(a) * c.ury);
    const T heqp = w * (drho * ((T)1 + (T)4.5 * cu * cu - (T)1.5 * uu) + (T)4.5 * cdu * csu -
                        (T)1.5 * dsu);
    const T heqm = k * (drho * cu + cdu);
    const T hp = (T)0.5 * (h[a] + h[b]);
    const T hm = (T)0.5 * (h[a] - h[b]);
    T dp = -c.s_plus * (hp - heqp);
    T dm = -c.s_minus * (hm - heqm);
    if (kForce) {
      const T cg = (T)cx_of(a) * gx + (T)cy_of(a) * gy;
      dp += c.a_plus * (w * ((T)9 * cu * cg - (T)3 * ug));
      dm += c.a_minus * (k * cg);
    }
    even += dp;
    o[a] = h[a] + dp + dm;
    o[b] = h[b] + dp - dm;
  }
  o[0] = h[0] - (T)2 * even;
}

// ---------------------------------------------------------------------------
// FP32 arithmetic of the 16-bit forms' fluid-node update in the packed f32x2
// instructions of sm_100 and later (one instruction for two nodes).  The
// special kernel updates its 16-bit fluid nodes with the same instructions,
// the node in both lanes: the compiler fuses some packed multiplies with a
// following add (even when the PTX names a rounding mode), so only the same
// instruction sequence gives a node the same bits in either kernel.
// ---------------------------------------------------------------------------
struct F2 {
  float2 v;
};
__device__ __forceinline__ unsigned long long f2_bits(F2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.v.x), "f"(a.v.y));
  return r;
}
__device__ __forceinline__ F2 bits_f2(unsigned long long r) {
  F2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.v.x), "=f"(a.v.y) : "l"(r));
  return a;
}
template <typename V>
__device__ __forceinline__ V vsplat(float c);
template <>
__device__ __forceinline__ F2 vsplat<F2>(float c) { return F2{make_float2(c, c)}; }
__device__ __forceinline__ F2 vpair(float x, float y) { return F2{make_float2(x, y)}; }
__device__ __forceinline__ F2 vsame(float x) { return F2{make_float2(x, x)}; }
__device__ __forceinline__ F2 vadd(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 vmul(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 vsub(F2 a, F2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
__device__ __forceinline__ F2 vrcp(F2 a) { return vpair(__frcp_rn(a.v.x), __frcp_rn(a.v.y)); }
__device__ __forceinline__ float vlo(F2 a) { return a.v.x; }
__device__ __forceinline__ float vhi(F2 a) { return a.v.y; }
__device__ __forceinline__ bool rho_bad(float r) { return !(r > 0.f) || !isfinite(r); }

// The collision of collide() in the packed FP32 arithmetic above, with the
// relaxation rate and weights folded into the even part's coefficients: for
// each pair
// (a, opp(a))
//   s+ heq+ = s+ w K + 4.5 s+ w X,  X = drho (c.u)^2 + (c.du)(c.u + c.u_ref),
//   K = drho (1 - 1.5 |u|^2) - 1.5 (|u|^2 - |u_ref|^2),
// the same terms as heq_a = w_a [drho (1 + Q_a(u)) + Q_a(u) - Q_a(u_ref)].  The
// odd part keeps collide()'s form -s- (h- - k (drho c.u + c.du)) with the
// coefficients k of odd_w (its momentum is then exact: a folded s- k would
// round differently from s-), and the rest population takes the even
// changes' remainder as in collide().
template <typename V, typename T, bool kForce>
__device__ __forceinline__ void collide2(const V (&h)[9], V drho, V dux, V duy, V gx, V gy,
                                         const Consts<T> &c, V (&o)[9]) {
  const V urx = vsplat<V>(c.urx), ury = vsplat<V>(c.ury);
  const V ux = vadd(urx, dux), uy = vadd(ury, duy);
  const V uu = vfma(ux, ux, vmul(uy, uy));
  const V dsu = vfma(dux, vadd(ux, urx), vmul(duy, vadd(uy, ury)));
  const V m15 = vsplat<V>((T)-1.5);
  const V K = vfma(m15, dsu, vmul(drho, vfma(m15, uu, vsplat<V>((T)1))));
  V ug{};
  if (kForce) ug = vfma(ux, gx, vmul(uy, gy));
  const V nsph = vsplat<V>((T)-0.5 * c.s_plus), nsm = vsplat<V>(-c.s_minus), half = vsplat<V>((T)0.5);
  V even = vsplat<V>((T)0);
#pragma unroll
  for (int a = 1; a <= 6; ++a) {
    if (a == 3 || a == 4) continue;
    const int b = opp_of(a);
    const T w = (T)w_of(a);
    const V k = vsplat<V>(odd_w<T>(a));
    // c.u, c.du for the four directions 1 (1,0), 2 (0,1), 5 (1,1), 6 (-1,1)
    V cu, cdu;
    if (a == 1) {
      cu = ux;
      cdu = dux;
    } else if (a == 2) {
      cu = uy;
      cdu = duy;
    } else if (a == 5) {
      cu = vadd(ux, uy);
      cdu = vadd(dux, duy);
    } else {
      cu = vsub(uy, ux);
      cdu = vsub(duy, dux);
    }
    const V csu = vadd(cu, vsplat<V>((T)cx_of(a) * c.urx + (T)cy_of(a) * c.ury));
    const V dc = vmul(drho, cu);
    const V X = vfma(dc, cu, vmul(cdu, csu));
    const V P = vfma(vsplat<V>((T)4.5 * c.s_plus * w), X, vmul(vsplat<V>(c.s_plus * w), K));
    V dp = vfma(nsph, vadd(h[a], h[b]), P);
    // -s- (h- - heq-), h- = (h_a - h_b) / 2, heq- = k (drho c.u + c.du)
    V dm = vmul(nsm, vsub(vmul(half, vsub(h[a], h[b])), vmul(k, vadd(dc, cdu))));
    if (kForce) {
      V cg;
      if (a == 1)
        cg = gx;
      else if (a == 2)
        cg = gy;
      else if (a == 5)
        cg = vadd(gx, gy);
      else
        cg = vsub(gy, gx);
      dp = vfma(vsplat<V>(c.a_plus * w * (T)9), vmul(cu, cg), vfma(vsplat<V>(c.a_plus * w * (T)-3), ug, dp));
      dm = vfma(vsplat<V>(c.a_minus), vmul(k, cg), dm);
    }
    even = vadd(even, dp);
    o[a] = vadd(vadd(h[a], dp), dm);
    o[b] = vsub(vadd(h[b], dp), dm);
  }
  o[0] = vfma(vsplat<V>((T)-2), even, h[0]);
}

// The update of fluid nodes (no penalization) in FP32: moments, velocity and
// the collision, from the pre-collision offsets h of a node pair (or of one
// node in both lanes); kForce adds the uniform body force.  Returns rho.
template <typename V, bool kForce>
__device__ __forceinline__ V fluid_update(const Lattice &L, const Consts<float> &cst,
                                          const V (&h)[9], V (&o)[9]) {
  const V drho = vadd(vadd(vadd(h[0], h[1]), vadd(h[2], h[3])),
                      vadd(vadd(vadd(h[4], h[5]), vadd(h[6], h[7])), h[8]));
  V djx = vadd(vadd(vsub(h[1], h[3]), vsub(h[5], h[6])), vsub(h[8], h[7]));
  V djy = vadd(vadd(vsub(h[2], h[4]), vsub(h[5], h[7])), vsub(h[6], h[8]));
  const V rho = vadd(vsplat<V>(1.0f), drho);
  const V inv = vrcp(rho);
  if (kForce) {
    const V gx = vsplat<V>(lat_bf<float>(L, 0)), gy = vsplat<V>(lat_bf<float>(L, 1));
    djx = vfma(vsplat<V>(0.5f), gx, djx);
    djy = vfma(vsplat<V>(0.5f), gy, djy);
    collide2<V, float, true>(h, drho, vmul(vfma(drho, vsplat<V>(-cst.urx), djx), inv),
                             vmul(vfma(drho, vsplat<V>(-cst.ury), djy), inv), gx, gy, cst, o);
  } else {
    collide2<V, float, false>(h, drho, vmul(vfma(drho, vsplat<V>(-cst.urx), djx), inv),
                              vmul(vfma(drho, vsplat<V>(-cst.ury), djy), inv), V{}, V{}, cst, o);
  }
  return rho;
}

// Moments, penalized velocity and force density of one node (Eqs. updatestep
// .. updatestepm: G = -rho (chi/eta)(u - u_s) in the rearranged form
// -(chi/eta)(j - rho u_s)/(1 + chi dt/(2 eta)), plus the body force), then
// the collision.  Returns true for a non-finite or non-positive density.
template <typename T, bool kPacked>
__device__ __forceinline__ bool update_node(const T (&h)[9], uint8_t m, int i, int j,
                                            const Lattice &L, const BodyState *body,
                                            const Consts<T> &cst, T (&o)[9], T &pen_x,
                                            T &pen_y) {
  pen_x = pen_y = (T)0;  // the penalization part of G (solid nodes only)
  if constexpr (kPacked) {
    // FP32 compute (FP32 and 16-bit storage): the packed arithmetic of
    // fluid_update, which the bulk kernels of these forms use, with the node
    // in both lanes, so that a fluid node gets the same bits in either kernel
    F2 hv[9], ov[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) hv[a] = vsame(h[a]);
    F2 rho;
    if (!(m & kSolid)) {
      rho = L.has_bf ? fluid_update<F2, true>(L, cst, hv, ov) : fluid_update<F2, false>(L, cst, hv, ov);
    } else {
      const F2 drho = vadd(vadd(vadd(hv[0], hv[1]), vadd(hv[2], hv[3])),
                           vadd(vadd(vadd(hv[4], hv[5]), vadd(hv[6], hv[7])), hv[8]));
      F2 djx = vadd(vadd(vsub(hv[1], hv[3]), vsub(hv[5], hv[6])), vsub(hv[8], hv[7]));
      F2 djy = vadd(vadd(vsub(hv[2], hv[4]), vsub(hv[5], hv[7])), vsub(hv[6], hv[8]));
      rho = vadd(vsame(1.0f), drho);
      const float bfx = lat_bf<float>(L, 0), bfy = lat_bf<float>(L, 1);
      djx = vfma(vsame(0.5f), vsame(bfx), djx);
      djy = vfma(vsame(0.5f), vsame(bfy), djy);
      float usx, usy;
      solid_velocity<float>(*body, i, j, usx, usy);
      const float k = cst.half_pen, r = vlo(rho), dr = vlo(drho);
      const float den = r + k * r;
      // the momentum defect j - rho u_s, and u - u_ref written as
      // (u_s - u_ref) + (j - rho u_s)/(rho (1 + k)) (see below)
      const float defx = vlo(djx) - dr * usx + (cst.urx - usx);
      const float defy = vlo(djy) - dr * usy + (cst.ury - usy);
      const float dux = (usx - cst.urx) + defx / den, duy = (usy - cst.ury) + defy / den;
      const float pen = 2.0f * k;
      pen_x = -pen * defx / (1.0f + k);
      pen_y = -pen * defy / (1.0f + k);
      collide2<F2, float, true>(hv, drho, vsame(dux), vsame(duy), vsame(bfx + pen_x),
                                vsame(bfy + pen_y), cst, ov);
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) o[a] = vlo(ov[a]);
    return rho_bad(vlo(rho));
  } else {
  const T drho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
  const T rho = (T)1 + drho;
  // j - u_ref (the offsets' first moment; sum_a c_a E_a = u_ref)
  T djx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
  T djy = (h[2] - h[4]) + (h[5] - h[7]) + (h[6] - h[8]);
  if ((m & kSolid) || L.has_bf) {
    const T bfx = lat_bf<T>(L, 0), bfy = lat_bf<T>(L, 1);
    djx += (T)0.5 * bfx;
    djy += (T)0.5 * bfy;
    T dux, duy, gx = bfx, gy = bfy;
    if (m & kSolid) {
      T usx, usy;
      solid_velocity<T>(*body, i, j, usx, usy);
      const T k = cst.half_pen;
      const T den = rho + k * rho;
      // the momentum defect j - rho u_s, from the offsets' first moment
      const T defx = djx - drho * usx + (cst.urx - usx);
      const T defy = djy - drho * usy + (cst.ury - usy);
      // u - u_ref = (j + k rho u_s)/(rho (1 + k)) - u_ref, written as
      // (u_s - u_ref) + (j - rho u_s)/(rho (1 + k)): the large part is exact
      // and the small one keeps its relative precision (k rho u_s alone
      // would carry an FP32 rounding of 1e-3 into the division by k rho)
      dux = (usx - cst.urx) + defx / den;
      duy = (usy - cst.ury) + defy / den;
      // G = -(chi/eta)(j - rho u_s)/(1 + k)
      const T pen = (T)2 * k;
      pen_x = -pen * defx / ((T)1 + k);
      pen_y = -pen * defy / ((T)1 + k);
      gx += pen_x;
      gy += pen_y;
    } else {
      const T inv = (T)1 / rho;
      dux = (djx - drho * cst.urx) * inv;
      duy = (djy - drho * cst.ury) * inv;
    }
    collide<T, true>(h, drho, dux, duy, gx, gy, cst, o);
  } else {
    const T inv = (T)1 / rho;
    collide<T, false>(h, drho, (djx - drho * cst.urx) * inv, (djy - drho * cst.ury) * inv, (T)0,
                      (T)0, cst, o);
  }
  return !(rho > (T)0) || !isfinite(rho);
  }
}

// ---------------------------------------------------------------------------
// stochastic rounding of the stored populations (the _SR storage forms)
// ---------------------------------------------------------------------------
// hash of the level being written: the rounding counter, which the special
// kernel advances by one per step
__device__ __forceinline__ uint32_t sr_level(const StepArgs &p) {
  const unsigned long long n = __ldg(p.rng_src);
  return pcg_hash((uint32_t)n ^ (uint32_t)(n >> 32));
}

// The random bits of a node pair (the nodes 2q and 2q + 1 of the linear index
// j * pitch + i; a row starts at an even index, the pitch being a multiple of
// 64) for the eighteen values it stores: four hashes, and nine words made of
// distinct exclusive-ors of them, one word per population.  The low half of
// population a's word serves the even node, the high half the odd one (the
// lanes of the conversion).  Distinct subsets of independent uniform words
// are pairwise independent, so any two roundings of the pair are
// uncorrelated.  Every kernel that stores a node draws the same bits.
struct SrBits {
  uint32_t h[4];
  __device__ __forceinline__ SrBits(uint32_t level, uint32_t pair) {
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = pcg_hash(level + pair * 4u + (uint32_t)q);
  }
  __device__ __forceinline__ uint32_t word(int a) const {
    switch (a) {
      case 0: return h[0];
      case 1: return h[1];
      case 2: return h[2];
      case 3: return h[3];
      case 4: return h[0] ^ h[1];
      case 5: return h[2] ^ h[3];
      case 6: return h[0] ^ h[2];
      case 7: return h[1] ^ h[3];
      default: return h[0] ^ h[3];
    }
  }
};

// stores population value v of node `node`, rounded to the storage type (to
// nearest, or stochastically with the bits of the node's pair)
template <typename S, bool kSR>
__device__ __forceinline__ void store_pop(S *ptr, typename Store<S>::T v, const SrBits *r, int a,
                                          uint32_t node) {
  if constexpr (sizeof(S) == 2 && kSR) {
    const uint32_t w = r->word(a);
    *reinterpret_cast<unsigned short *>(ptr) =
        (unsigned short)(Stochastic<S>::pair(v, v, (node & 1u) ? w >> 16 : w) & 0xffffu);
  } else {
    Store<S>::st(ptr, v);
  }
}

// pre-collision populations of an edge node, with the side conditions
template <typename S, bool kGather>
__device__ __forceinline__ void edge_pops(const S *src, const typename Store<S>::T *prev,
                                          const Lattice &L, int i, int j,
                                          typename Store<S>::T (&h)[9]) {
#pragma unroll
  for (int a = 0; a < 9; ++a) h[a] = pre_pop<S, kGather>(src, prev, L, a, i, j);
}

// One node of the special kernel: pull (with the side conditions where
// needed), keep the outlet column, update, store, and the MEM link terms of
// an interface node of the force region.
template <typename S, bool kGather>
__device__ __forceinline__ bool special_node(const StepArgs &p, int i, int j, bool in_reg,
                                             const TileMask *tm, FixAcc<typename Store<S>::T> &acc,
                                             FixAcc<typename Store<S>::T> &vol) {
  using T = typename Store<S>::T;
  const Lattice &L = p.L;
  const S *__restrict__ src = static_cast<const S *>(p.src);
  S *dst = static_cast<S *>(p.dst);
  const T *prev = static_cast<const T *>(p.prev_src);
  const int64_t node = (int64_t)j * L.pitch + i;
  T h[9];
  if (kGather && i > 0 && i < L.nx - 1 && j > 0 && j < L.ny - 1) {
#pragma unroll
    for (int a = 0; a < 9; ++a)
      h[a] = Store<S>::ld(src + (int64_t)a * L.plane + node - cy_of(a) * L.pitch - cx_of(a));
  } else {
    edge_pops<S, kGather>(src, prev, L, i, j, h);
  }
  if (i == L.nx - 1 && L.bc[1] == VPLBM_OUTLET_CONVECTIVE) {
    // the outlet column's pre-collision values, for the next step
    T *pd = static_cast<T *>(p.prev_dst);
    pd[0 * L.ny + j] = h[3];
    pd[1 * L.ny + j] = h[6];
    pd[2 * L.ny + j] = h[7];
  }
  uint8_t m;
  if (tm) {
    // a moving body's tile: its mask byte from the tile's predicate, kept in
    // chi for the read-backs
    m = tile_mask_byte(L, *tm, i, j, threadIdx.x, threadIdx.y);
    p.chi[node] = m;
  } else {
    m = p.chi[node];
  }
  T o[9], pen_x, pen_y;
  const bool bad = update_node<T, sizeof(T) == 4>(h, m, i, j, L, p.body_src, Consts<T>(p), o, pen_x,
                                                  pen_y);
  if (sizeof(S) == 2 && p.sr) {
    const SrBits r(sr_level(p), (uint32_t)node >> 1);
#pragma unroll
    for (int a = 0; a < 9; ++a)
      store_pop<S, true>(dst + (int64_t)a * L.plane + node, o[a], &r, a, (uint32_t)node);
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a)
      store_pop<S, false>(dst + (int64_t)a * L.plane + node, o[a], nullptr, a, (uint32_t)node);
  }
  if (in_reg && (m & kInterface)) mem_terms<T>(p, o, i, j, m, tm, acc);
  if (in_reg && (m & kSolid)) {
    // volume integral (Eq. Angotforce, reading R19): the penalization force
    // on the fluid, reversed, and its moment about the reference point
    const BodyRef<T> b(*p.body_src);
    const T fx = -pen_x, fy = -pen_y;
    vol.add(0, fx);
    vol.add(1, fy);
    vol.add(2, ((T)i - b.xg) * fy - ((T)j - b.yg) * fx);
  }
  return bad;
}

// ---------------------------------------------------------------------------
// special kernel: SIM blocks, then blocks of edge nodes, then the
// force-region tiles (or, for the first step, every tile)
// ---------------------------------------------------------------------------
// The special kernels of lattices stepped side by side share the SMs with the
// bulk kernels, whose bytes in flight need the register file: for a fixed
// body with FP32 compute the special kernel is capped at 64 registers (four
// blocks per SM), at the price of a few spilled values.  A moving body's
// special kernel is on the step's critical path (its force feeds the next
// step), so it keeps all the registers it wants (kMinBlocks 1).
template <typename S>
constexpr int kSpecialMinBlocks = sizeof(S) <= 4 ? 4 : 1;

template <typename S, bool kGather, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) special_kernel(const StepArgs p) {
  using T = typename Store<S>::T;
  __shared__ int is_last;
  __shared__ TileMask tmask;
  const Lattice &L = p.L;
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  const ForceRegion reg = *p.reg_src;
  const int b = blockIdx.x;
  if (p.sr && b == 0 && tid == 0) *p.rng_dst = *p.rng_src + 1ull;  // the next level's counter
  if (p.finalize_prev && b == (int)gridDim.x - 1) {
    // the previous step's force sums, beside this step's work
    finalize<T>(p, p.acc_prev);
    return;
  }

  if (b < p.sim_blocks) {
    // ---- SIM points of this level ----
    const int q = b * p.sim_per_block + tid;
    FixAcc<T> acc;
    bool missing = false;
    if (tid < p.sim_per_block && q < p.n_sim) {
      const BodyState *body = p.body_src;
      acc = sim_point<S, kGather>(p, static_cast<const S *>(p.src), body->xg, body->yg, q,
                                  missing);
    }
    if (__any_sync(kFull, missing) && (tid & 31) == 0) atomicOr(p.status, kStatusSimMissing);
    warp_add(acc, p.acc, 3);
  } else if (!p.all_tiles && b < p.sim_blocks + p.edge_blocks) {
    // ---- one edge node per thread (nodes of force-region tiles excluded) ----
    const int e = (b - p.sim_blocks) * kThreads + tid;
    bool bad = false;
    if (e < p.n_edge) {
      int i, j;
      edge_node(e, L.nx, L.ny, i, j);
      const int ti = i / kTileX, tj = j / kTileY;
      const bool in_reg = ti >= reg.ti0 && ti <= reg.ti1 && tj >= reg.tj0 && tj <= reg.tj1;
      if (!in_reg) {
        FixAcc<T> unused, unused_vol;
        bad = special_node<S, kGather>(p, i, j, false, nullptr, unused, unused_vol);
      }
    }
    if (__any_sync(kFull, bad) && (tid & 31) == 0) atomicOr(p.status, kStatusUnstable);
    return;
  } else {
    // ---- a whole tile: every tile (first step) or a force-region tile ----
    int ti, tj;
    const int r = b - p.sim_blocks;
    if (p.all_tiles) {
      ti = r % p.ntiles_x;
      tj = r / p.ntiles_x;
    } else {
      const int k = r - p.edge_blocks;
      if (k >= reg.count) return;  // spare slot (moving bodies)
      const int rw = reg.ti1 - reg.ti0 + 1;
      ti = reg.ti0 + k % rw;
      tj = reg.tj0 + k / rw;
    }
    const bool in_reg = ti >= reg.ti0 && ti <= reg.ti1 && tj >= reg.tj0 && tj <= reg.tj1;
    const int i = ti * kTileX + threadIdx.x;
    const int j = tj * kTileY + threadIdx.y;
    // a moving body: the region tiles rasterise its mask at this level
    const bool raster = p.raster && in_reg;  // uniform over the block
    if (raster) {
      tile_solid(p, ti, tj, tmask);
      __syncthreads();
    }
    bool bad = false;
    FixAcc<T> acc, vol;
    if (i < L.nx && j < L.ny)
      bad = special_node<S, kGather>(p, i, j, in_reg, raster ? &tmask : nullptr, acc, vol);
    if (__any_sync(kFull, bad) && (tid & 31) == 0) atomicOr(p.status, kStatusUnstable);
    if (!in_reg) return;  // uniform over the block
    warp_add(acc, p.acc, 0);
    warp_add(vol, p.acc, 6);
  }

  if (p.defer) return;  // a later launch finalizes this step's sums

  // ---- ticket among the SIM blocks and the force-region tiles ----
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned int expected = (unsigned int)(p.sim_blocks + reg.count);
    const unsigned int prev = atomicAdd(p.ticket, 1u);
    is_last = (prev == expected - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  tail<T>(p, reg);
}

// ---------------------------------------------------------------------------
// bulk kernel: every node off the lattice edges and outside the force-region
// tiles -- fluid nodes whose pull sources all lie inside the lattice.
// ---------------------------------------------------------------------------
template <typename S, bool kForce, int kTiles>
__global__ void __launch_bounds__(kThreads * kTiles) bulk_kernel(const StepArgs p) {
  using T = typename Store<S>::T;
  const Lattice &L = p.L;
  const int ti = blockIdx.x;
  const int i = ti * kTileX + threadIdx.x;
  const int j = blockIdx.y * (kTileY * kTiles) + threadIdx.y;  // a block is kTiles tiles high
  const int tj = j / kTileY;
  if (i < 1 || i > L.nx - 2 || j < 1 || j > L.ny - 2) return;  // edge nodes: special kernel
  const S *__restrict__ src = static_cast<const S *>(p.src);
  S *__restrict__ dst = static_cast<S *>(p.dst);
  const int64_t node = (int64_t)j * L.pitch + i;
  // the populations are requested before the force-region bounds are known,
  // so that their latency is not added to that of the bounds
  T h[9];
#pragma unroll
  for (int a = 0; a < 9; ++a)
    h[a] = Store<S>::ld(src + (int64_t)a * L.plane + node - cy_of(a) * L.pitch - cx_of(a));
  {
    const ForceRegion reg = *p.reg_src;
    if (ti >= reg.ti0 && ti <= reg.ti1 && tj >= reg.tj0 && tj <= reg.tj1) return;  // special kernel
  }
  const Consts<T> cst(p);
  const T drho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
  const T rho = (T)1 + drho;
  T djx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
  T djy = (h[2] - h[4]) + (h[5] - h[7]) + (h[6] - h[8]);
  T o[9];
  const T inv = (T)1 / rho;
  if (kForce) {
    const T bfx = lat_bf<T>(L, 0), bfy = lat_bf<T>(L, 1);
    djx += (T)0.5 * bfx;
    djy += (T)0.5 * bfy;
    collide<T, true>(h, drho, (djx - drho * cst.urx) * inv, (djy - drho * cst.ury) * inv, bfx,
                     bfy, cst, o);
  } else {
    collide<T, false>(h, drho, (djx - drho * cst.urx) * inv, (djy - drho * cst.ury) * inv, (T)0,
                      (T)0, cst, o);
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) Store<S>::st(dst + (int64_t)a * L.plane + node, o[a]);
  if (!(rho > (T)0) || !isfinite(rho)) atomicOr(p.status, kStatusUnstable);
}

// ---------------------------------------------------------------------------
// bulk kernel for FP32 storage: two adjacent nodes per thread, one 64-bit
// load and one 64-bit store per plane, the +-x neighbour from the next lane by
// a shuffle, and the collision of both nodes in packed f32x2 arithmetic (the
// special kernel updates its fluid nodes with the same arithmetic, one node
// in both lanes).  A tile row of 128 nodes is two warps; a block is kTiles
// tiles high.
// ---------------------------------------------------------------------------
template <bool kForce, int kTiles>
__global__ void __launch_bounds__(kThreads / 2 * kTiles) bulk32x2_kernel(const StepArgs p) {
  const Lattice &L = p.L;
  const int ti = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const int i = ti * kTileX + 2 * threadIdx.x;  // the thread's nodes i, i + 1
  const int j = blockIdx.y * (kTileY * kTiles) + threadIdx.y;
  const int tj = j / kTileY;
  // every lane loads from inside its row (clamped), so that the shuffles see
  // all lanes; results of clamped lanes are never stored.  Rows start on
  // 256-byte boundaries (the pitch is a multiple of 64 values).
  const int ic = i < L.pitch - 2 ? i : L.pitch - 2;
  const float *__restrict__ src = static_cast<const float *>(p.src);
  F2 h[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int r = j - cy_of(a);
    r = r < 0 ? 0 : (r > L.ny - 1 ? L.ny - 1 : r);
    const float *row = src + (int64_t)a * L.plane + (int64_t)r * L.pitch;
    const float2 v = __ldg(reinterpret_cast<const float2 *>(row + ic));
    if (cx_of(a) == 0) {
      h[a] = vpair(v.x, v.y);
    } else if (cx_of(a) > 0) {  // sources i - 1 (the left lane's second value), i
      float left = __shfl_up_sync(0xffffffffu, v.y, 1);
      if (lane == 0) left = ic >= 1 ? __ldg(row + ic - 1) : 0.f;
      h[a] = vpair(left, v.x);
    } else {  // sources i + 1, i + 2 (the right lane's first value)
      float right = __shfl_down_sync(0xffffffffu, v.x, 1);
      if (lane == 31) right = ic + 2 < L.pitch ? __ldg(row + ic + 2) : 0.f;
      h[a] = vpair(v.y, right);
    }
  }
  {
    const ForceRegion reg = *p.reg_src;
    if (ti >= reg.ti0 && ti <= reg.ti1 && tj >= reg.tj0 && tj <= reg.tj1) return;  // special kernel
  }
  if (j < 1 || j > L.ny - 2) return;  // edge rows: special kernel
  const bool ok0 = i >= 1 && i <= L.nx - 2, ok1 = i + 1 <= L.nx - 2;
  if (!ok0 && !ok1) return;
  F2 o[9];
  const F2 rho = fluid_update<F2, kForce>(L, Consts<float>(p), h, o);
  float *dst = static_cast<float *>(p.dst) + (int64_t)j * L.pitch + i;
  if (ok0 && ok1) {
#pragma unroll
    for (int a = 0; a < 9; ++a)
      *reinterpret_cast<float2 *>(dst + (int64_t)a * L.plane) = make_float2(vlo(o[a]), vhi(o[a]));
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (ok0) dst[(int64_t)a * L.plane] = vlo(o[a]);
      if (ok1) dst[(int64_t)a * L.plane + 1] = vhi(o[a]);
    }
  }
  if ((ok0 && rho_bad(vlo(rho))) || (ok1 && rho_bad(vhi(rho)))) atomicOr(p.status, kStatusUnstable);
}

// ---------------------------------------------------------------------------
// bulk kernel for 16-bit storage: eight nodes per thread.  HBM stays busy
// only with enough bytes in flight per SM, and a thread holds what it loads
// in registers until it is used; with 2-byte values the registers, not the
// threads, cap what is in flight.  So each thread takes the nodes i .. i+7
// (i a multiple of 8) of a tile row, a half-warp per row and one warp per
// 128 x 2 tile: one aligned 128-bit load per plane brings eight values, kept
// packed (four 32-bit words per plane, 36 registers for 8 nodes: 144 bytes
// in flight per thread).  For c_x = +1 (sources i-1 .. i+6) and c_x = -1
// (sources i+1 .. i+8) the value beyond the thread's eight comes from the
// next lane of the half-warp by a shuffle (one extra 2-byte load at the
// row's edge) and a funnel shift realigns the words.  The nodes are collided
// two at a time in packed f32x2 (collide2) and leave in one 128-bit store per
// plane.  96 registers, 20 one-warp blocks per SM: about 90 KB in flight per
// SM.
// ---------------------------------------------------------------------------
template <typename S>
struct Pair16;
template <>
struct Pair16<__half> {
  static __device__ __forceinline__ float lo(uint32_t w) {
    return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
  }
  static __device__ __forceinline__ float hi(uint32_t w) {
    return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
  }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};
template <>
struct Pair16<__nv_bfloat16> {
  static __device__ __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
  static __device__ __forceinline__ float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};

// (lo half of b, hi half of a) -> the pair starting one value later
__device__ __forceinline__ uint32_t shift16(uint32_t a, uint32_t b) {
  return __funnelshift_r(a, b, 16);
}

// the update of the node pair whose pre-collision values are the packed
// words w[a], nodes `node` and `node + 1`; returns the packed post-collision
// words (rounded to nearest, or stochastically with the level's bits) and rho
template <typename S, bool kForce, bool kSR>
__device__ __forceinline__ F2 collide_pair16(const StepArgs &p, const uint32_t (&w)[9],
                                             uint32_t (&out)[9], uint32_t level, uint32_t node) {
  using P = Pair16<S>;
  F2 h[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) h[a] = vpair(P::lo(w[a]), P::hi(w[a]));
  F2 o[9];
  const F2 rho = fluid_update<F2, kForce>(p.L, Consts<float>(p), h, o);
  if constexpr (kSR) {
    const SrBits r(level, node >> 1);
#pragma unroll
    for (int a = 0; a < 9; ++a) out[a] = Stochastic<S>::pair(vlo(o[a]), vhi(o[a]), r.word(a));
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) out[a] = P::pack(vlo(o[a]), vhi(o[a]));
  }
  return rho;
}

template <typename S, bool kForce, bool kSR, int kMinBlocks>
__global__ void __launch_bounds__(32, kMinBlocks) bulk16_kernel(const StepArgs p) {
  const int ti = blockIdx.x, tj = blockIdx.y;
  const Lattice &L = p.L;
  const int lane = threadIdx.x & 15;               // lane within the tile row
  const int i = ti * kTileX + 8 * lane;            // the thread's nodes i .. i + 7
  const int j = tj * kTileY + (threadIdx.x >> 4);  // half-warp per tile row
  // every lane loads from inside its row (clamped), so that the shuffles see
  // all lanes; results of clamped lanes are never stored.  Rows and planes
  // start on 16-byte boundaries (the pitch is a multiple of 64 values).
  const int ic = i < L.pitch - 8 ? i : L.pitch - 8;
  const S *__restrict__ src = static_cast<const S *>(p.src);
  uint32_t w[4][9];  // sources of the node pairs (i, i+1) .. (i+6, i+7), packed
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int r = j - cy_of(a);
    r = r < 0 ? 0 : (r > L.ny - 1 ? L.ny - 1 : r);
    const S *row = src + (int64_t)a * L.plane + (int64_t)r * L.pitch;
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(row + ic));
    if (cx_of(a) == 0) {
      w[0][a] = v.x;
      w[1][a] = v.y;
      w[2][a] = v.z;
      w[3][a] = v.w;
    } else if (cx_of(a) > 0) {  // sources i-1 (the left lane's last value) .. i+6
      uint32_t left = __shfl_up_sync(0xffffffffu, v.w, 1, 16);
      if (lane == 0)
        left = ic >= 1 ? ((uint32_t)__ldg(reinterpret_cast<const unsigned short *>(row + ic - 1)) << 16)
                       : 0u;
      w[0][a] = shift16(left, v.x);
      w[1][a] = shift16(v.x, v.y);
      w[2][a] = shift16(v.y, v.z);
      w[3][a] = shift16(v.z, v.w);
    } else {  // sources i+1 .. i+8 (the right lane's first value)
      uint32_t right = __shfl_down_sync(0xffffffffu, v.x, 1, 16);
      if (lane == 15)
        right = ic + 8 < L.pitch ? (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(row + ic + 8))
                                 : 0u;
      w[0][a] = shift16(v.x, v.y);
      w[1][a] = shift16(v.y, v.z);
      w[2][a] = shift16(v.z, v.w);
      w[3][a] = shift16(v.w, right);
    }
  }
  {
    const ForceRegion reg = *p.reg_src;
    if (ti >= reg.ti0 && ti <= reg.ti1 && tj >= reg.tj0 && tj <= reg.tj1) return;  // special kernel
  }
  if (j < 1 || j > L.ny - 2) return;  // edge rows: special kernel
  const int n_ok_lo = i >= 1 ? 0 : 1;                    // first node to store
  const int n_ok_hi = L.nx - 2 - i < 7 ? L.nx - 2 - i : 7;  // last node to store
  if (n_ok_hi < n_ok_lo) return;
  uint32_t out[4][9];
  bool bad = false;
  const uint32_t level = kSR ? sr_level(p) : 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const F2 r = collide_pair16<S, kForce, kSR>(p, w[k], out[k], level,
                                           (uint32_t)((int64_t)j * L.pitch + i + 2 * k));
    bad |= (2 * k >= n_ok_lo && 2 * k <= n_ok_hi && rho_bad(vlo(r))) ||
           (2 * k + 1 >= n_ok_lo && 2 * k + 1 <= n_ok_hi && rho_bad(vhi(r)));
  }
  S *dst = static_cast<S *>(p.dst) + (int64_t)j * L.pitch + i;
  if (n_ok_lo == 0 && n_ok_hi == 7) {
#pragma unroll
    for (int a = 0; a < 9; ++a)
      *reinterpret_cast<uint4 *>(dst + (int64_t)a * L.plane) =
          make_uint4(out[0][a], out[1][a], out[2][a], out[3][a]);
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      unsigned short *d = reinterpret_cast<unsigned short *>(dst + (int64_t)a * L.plane);
#pragma unroll
      for (int n = 0; n < 8; ++n)
        if (n >= n_ok_lo && n <= n_ok_hi)
          d[n] = (unsigned short)(n & 1 ? out[n >> 1][a] >> 16 : out[n >> 1][a] & 0xffffu);
    }
  }
  if (bad) atomicOr(p.status, kStatusUnstable);
}

// The same update with four nodes per thread (one 64-bit load per plane, one
// warp per tile row, 80 registers): a variant for the tuner.
template <typename S, bool kForce, bool kSR>
__global__ void __launch_bounds__(32 * kTileY, 12) bulk16x4_kernel(const StepArgs p) {
  const int ti = blockIdx.x, tj = blockIdx.y;
  const Lattice &L = p.L;
  const int lane = threadIdx.x;
  const int i = ti * kTileX + 4 * lane;  // the thread's nodes i .. i + 3
  const int j = tj * kTileY + threadIdx.y;
  // every lane loads from inside its row (clamped), so that the shuffles see
  // all 32 lanes; results of clamped lanes are never stored.  Rows and planes
  // start on 8-byte boundaries (the pitch is a multiple of 64 values).
  const int ic = i < L.pitch - 4 ? i : L.pitch - 4;
  const S *__restrict__ src = static_cast<const S *>(p.src);
  uint32_t wa[9], wb[9];  // sources of nodes (i, i+1) and (i+2, i+3), packed
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int r = j - cy_of(a);
    r = r < 0 ? 0 : (r > L.ny - 1 ? L.ny - 1 : r);
    const S *row = src + (int64_t)a * L.plane + (int64_t)r * L.pitch;
    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(row + ic));
    if (cx_of(a) == 0) {
      wa[a] = w.x;
      wb[a] = w.y;
    } else if (cx_of(a) > 0) {  // sources i-1 (the left lane's last value) .. i+2
      uint32_t left = __shfl_up_sync(0xffffffffu, w.y, 1);
      if (lane == 0)
        left = ic >= 1 ? ((uint32_t)__ldg(reinterpret_cast<const unsigned short *>(row + ic - 1)) << 16)
                       : 0u;
      wa[a] = shift16(left, w.x);
      wb[a] = shift16(w.x, w.y);
    } else {  // sources i+1 .. i+4 (the right lane's first value)
      uint32_t right = __shfl_down_sync(0xffffffffu, w.x, 1);
      if (lane == 31)
        right = ic + 4 < L.pitch ? (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(row + ic + 4))
                                 : 0u;
      wa[a] = shift16(w.x, w.y);
      wb[a] = shift16(w.y, right);
    }
  }
  {
    const ForceRegion reg = *p.reg_src;
    if (ti >= reg.ti0 && ti <= reg.ti1 && tj >= reg.tj0 && tj <= reg.tj1) return;  // special kernel
  }
  if (j < 1 || j > L.ny - 2) return;  // edge rows: special kernel
  bool ok[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) ok[k] = i + k >= 1 && i + k <= L.nx - 2;
  if (!ok[0] && !ok[1] && !ok[2] && !ok[3]) return;
  S *dst = static_cast<S *>(p.dst) + (int64_t)j * L.pitch + i;
  // the two pairs one after the other, each stored as soon as it is done
  bool bad = false;
  const uint32_t level = kSR ? sr_level(p) : 0u;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t o[9];
    const F2 r = collide_pair16<S, kForce, kSR>(p, half ? wb : wa, o, level,
                                           (uint32_t)((int64_t)j * L.pitch + i + 2 * half));
    const bool ok0 = ok[2 * half], ok1 = ok[2 * half + 1];
    S *d2 = dst + 2 * half;
    if (ok0 && ok1) {
#pragma unroll
      for (int a = 0; a < 9; ++a) *reinterpret_cast<uint32_t *>(d2 + (int64_t)a * L.plane) = o[a];
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        unsigned short *d = reinterpret_cast<unsigned short *>(d2 + (int64_t)a * L.plane);
        if (ok0) d[0] = (unsigned short)(o[a] & 0xffffu);
        if (ok1) d[1] = (unsigned short)(o[a] >> 16);
      }
    }
    bad |= (ok0 && rho_bad(vlo(r))) || (ok1 && rho_bad(vhi(r)));
  }
  if (bad) atomicOr(p.status, kStatusUnstable);
}

template <typename S, bool kGather>
cudaError_t special_t(const StepArgs &a, cudaStream_t s) {
  const int tiles = a.all_tiles ? a.ntiles_x * a.ntiles_y : a.edge_blocks + a.region_slots;
  const int blocks = a.sim_blocks + tiles + (a.finalize_prev ? 1 : 0);
  if (a.raster || kSpecialMinBlocks<S> == 1)
    special_kernel<S, kGather, 1><<<blocks, dim3(kTileX, kTileY), 0, s>>>(a);
  else
    special_kernel<S, kGather, kSpecialMinBlocks<S>><<<blocks, dim3(kTileX, kTileY), 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(kThreads) finalize_kernel(const StepArgs p) {
  finalize<T>(p, p.acc_prev);
}

// chi of a moving body on the force-region tiles, tile by tile as the special
// kernel rasterises it
__global__ void __launch_bounds__(kThreads) mask_kernel(const StepArgs p) {
  __shared__ TileMask tm;
  const ForceRegion reg = *p.reg_src;
  const int k = blockIdx.x;
  if (k >= reg.count) return;
  const int rw = reg.ti1 - reg.ti0 + 1;
  const int ti = reg.ti0 + k % rw, tj = reg.tj0 + k / rw;
  tile_solid(p, ti, tj, tm);
  __syncthreads();
  const int i = ti * kTileX + threadIdx.x, j = tj * kTileY + threadIdx.y;
  if (i < p.L.nx && j < p.L.ny)
    p.chi[(int64_t)j * p.L.pitch + i] = tile_mask_byte(p.L, tm, i, j, threadIdx.x, threadIdx.y);
}

template <typename S, bool kForce, bool kSR>
cudaError_t bulk16_v(int variant, const StepArgs &a, cudaStream_t s) {
  static_assert(kTileX == 8 * 16 && kTileY == 2, "bulk16_kernel maps a tile onto one warp");
  const dim3 grid(a.ntiles_x, a.ntiles_y);
  switch (variant) {
    case 0: bulk16_kernel<S, kForce, kSR, 20><<<grid, dim3(32), 0, s>>>(a); break;  // 8 nodes, 96 regs
    case 1: bulk16_kernel<S, kForce, kSR, 16><<<grid, dim3(32), 0, s>>>(a); break;  // 8 nodes, 126 regs
    case 2: bulk16x4_kernel<S, kForce, kSR><<<grid, dim3(32, kTileY), 0, s>>>(a); break;  // 4 nodes
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename S, bool kForce>
cudaError_t bulk_v(int variant, const StepArgs &a, cudaStream_t s) {
  if constexpr (sizeof(S) == 2) {
    return a.sr ? bulk16_v<S, kForce, true>(variant, a, s) : bulk16_v<S, kForce, false>(variant, a, s);
  } else if constexpr (sizeof(S) == 4) {
    const int k = variant == 0 ? 1 : (variant == 1 ? 2 : 4);  // tiles per block
    if (variant < 0 || variant > 2) return cudaErrorInvalidValue;
    const dim3 grid(a.ntiles_x, (a.ntiles_y + k - 1) / k), block(kTileX / 2, kTileY * k);
    if (k == 1) bulk32x2_kernel<kForce, 1><<<grid, block, 0, s>>>(a);
    else if (k == 2) bulk32x2_kernel<kForce, 2><<<grid, block, 0, s>>>(a);
    else bulk32x2_kernel<kForce, 4><<<grid, block, 0, s>>>(a);
  } else {
    const int k = variant == 0 ? 1 : (variant == 1 ? 2 : 4);  // tiles per block
    if (variant < 0 || variant > 2) return cudaErrorInvalidValue;
    const dim3 grid(a.ntiles_x, (a.ntiles_y + k - 1) / k), block(kTileX, kTileY * k);
    if (k == 1) bulk_kernel<S, kForce, 1><<<grid, block, 0, s>>>(a);
    else if (k == 2) bulk_kernel<S, kForce, 2><<<grid, block, 0, s>>>(a);
    else bulk_kernel<S, kForce, 4><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename S>
cudaError_t bulk_t(int variant, const StepArgs &a, cudaStream_t s) {
  return a.L.has_bf ? bulk_v<S, true>(variant, a, s) : bulk_v<S, false>(variant, a, s);
}

}  // namespace

cudaError_t launch_special(int dtype, bool gather, const StepArgs &a, cudaStream_t s) {
  switch (dtype) {
    case VPLBM_F64: return gather ? special_t<double, true>(a, s) : special_t<double, false>(a, s);
    case VPLBM_F32: return gather ? special_t<float, true>(a, s) : special_t<float, false>(a, s);
    case VPLBM_F16_OFS: return gather ? special_t<__half, true>(a, s) : special_t<__half, false>(a, s);
    case VPLBM_BF16_OFS:
      return gather ? special_t<__nv_bfloat16, true>(a, s) : special_t<__nv_bfloat16, false>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_finalize(int dtype, const StepArgs &a, cudaStream_t s) {
  if (dtype == VPLBM_F64)
    finalize_kernel<double><<<1, dim3(kTileX, kTileY), 0, s>>>(a);
  else
    finalize_kernel<float><<<1, dim3(kTileX, kTileY), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mask(const StepArgs &a, cudaStream_t s) {
  mask_kernel<<<a.region_slots, dim3(kTileX, kTileY), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sim_cache(const StepArgs &a, cudaStream_t s) {
  if (a.n_sim <= 0) return cudaSuccess;
  sim_cache_kernel<<<(a.n_sim + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bulk(int dtype, int variant, const StepArgs &a, cudaStream_t s) {
  switch (dtype) {
    case VPLBM_F64: return bulk_t<double>(variant, a, s);
    case VPLBM_F32: return bulk_t<float>(variant, a, s);
    case VPLBM_F16_OFS: return bulk_t<__half>(variant, a, s);
    case VPLBM_BF16_OFS: return bulk_t<__nv_bfloat16>(variant, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace vplbm
