// step.cu -- the fused VP-LBM time step for sm_103a.
//
// One launch advances the lattice by one time step and produces that step's
// forces.  Blocks are of three kinds:
//   * SIM blocks (the first few, when SIM is due): one integration point per
//     thread -- the stress of Sec. 2.3.2 at the sampled fluid node from its
//     pre-collision populations, then S_i sigma n_i and its moment (Eq. defFf),
//     stored per point;
//   * lattice tiles (128 x 2 nodes, one node per thread): pull-stream the
//     pre-collision populations (Eq. eqBd with the side conditions of Sec. 3.1
//     and 3.2), moments and penalized velocity (Eqs. updatestep ..
//     updatestepm), force density G, equilibrium and BGK/TRT collision with
//     the forcing term (Eq. TRT), store;
//   * tiles of the force region (around the body) additionally sum the MEM
//     link terms of their interface nodes (Eq. MMEL, Eq. fluidtorque) in FP64
//     into one partial per tile.
// The SIM blocks and the force-region tiles take a ticket when done; the last
// of them sums the partials and the SIM entries in a fixed order in FP64,
// records the step's forces and, for a moving body, applies the FP64
// rigid-body update (Eqs. dep1, theta2) and re-rasterises the mask.  Every
// other block only streams and collides: no barrier, no atomic, no FP64.
#include "vplbm_internal.cuh"

// resident blocks per SM the register allocation is sized for (80 registers)
#ifndef VPLBM_STEP_MIN_BLOCKS
#define VPLBM_STEP_MIN_BLOCKS 3
#endif

namespace vplbm {

namespace {

__device__ __forceinline__ double block_sum(double v, double *red) {
  // fixed-order block reduction: warp butterfly, then warp 0 over warp sums
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int nwarps = (blockDim.x * blockDim.y) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < nwarps ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// Deviatoric-plus-density part of the stress of Sec. 2.3.2 at a fluid node,
// sigma + (1/3) I = -(rho - 1)/3 I - (1 - 1/(2 tau+)) sum c c (f - feq),
// from the pre-collision offsets, in the compute type (all terms are small).
template <typename S, bool kGather>
__device__ void node_stress(const S *buf, const typename Store<S>::T *prev, const Lattice &L,
                            double tau_plus, int i, int j, typename Store<S>::T sig[3]) {
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
  jx += (T)0.5 * lat_bf<T>(L, 0);
  jy += (T)0.5 * lat_bf<T>(L, 1);
  const T ux = jx / rho, uy = jy / rho, uu = ux * ux + uy * uy;
  T pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const T cu = (T)cx_of(a) * ux + (T)cy_of(a) * uy;
    const T heq = (T)w_of(a) * (drho + rho * ((T)3 * cu + (T)4.5 * cu * cu - (T)1.5 * uu));
    const T d = h[a] - heq;
    pxx += (T)(cx_of(a) * cx_of(a)) * d;
    pxy += (T)(cx_of(a) * cy_of(a)) * d;
    pyy += (T)(cy_of(a) * cy_of(a)) * d;
  }
  const T s = (T)(1.0 - 0.5 / tau_plus);
  sig[0] = -drho / (T)3 - s * pxx;
  sig[1] = -s * pxy;
  sig[2] = -drho / (T)3 - s * pyy;
}

// pre-collision populations of an edge node, with the side conditions (kept
// out of line: only edge nodes take this path)
template <typename S, bool kGather>
__device__ __noinline__ void edge_pops(const S *src, const typename Store<S>::T *prev,
                                       const Lattice &L, int i, int j,
                                       typename Store<S>::T *h) {
#pragma unroll
  for (int a = 0; a < 9; ++a) h[a] = pre_pop<S, kGather>(src, prev, L, a, i, j);
}

// MEM link terms of one interface node (Eq. MMEL, Eq. fluidtorque), FP64,
// from its post-collision populations just stored (kept out of line: only
// interface nodes of the force region take this path)
template <typename S>
__device__ __noinline__ void mem_terms(const StepArgs &p, const S *dst, int i, int j,
                                       uint8_t m, double acc[3]) {
  const Lattice &L = p.L;
  const BodyState &b = *p.body_src;
  const int64_t node = (int64_t)j * L.pitch + i;
  const bool solid = m & kSolid;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    int ni, nj;
    if (!neighbour(L, a, i, j, ni, nj)) continue;
    const bool nsolid = p.chi[(int64_t)nj * L.pitch + ni] & kSolid;
    if (nsolid == solid) continue;
    // link midpoint x_Gamma and the wall velocity u_Gamma there
    const double xgam = (double)i + 0.5 * cx_of(a), ygam = (double)j + 0.5 * cy_of(a);
    const double ugx = b.ux - b.omega * (ygam - b.yg);
    const double ugy = b.uy + b.omega * (xgam - b.xg);
    // the node's own store of this launch: read back through L2, not the
    // read-only path
    const double fa = (double)Store<S>::ld_own(dst + (int64_t)a * L.plane + node) + w_of(a);
    const double sg = solid ? -1.0 : 1.0;
    const double lx = sg * (cx_of(a) - ugx) * fa;
    const double ly = sg * (cy_of(a) - ugy) * fa;
    acc[0] += lx;
    acc[1] += ly;
    acc[2] += (xgam - b.xg) * ly - (ygam - b.yg) * lx;
  }
}

__device__ __forceinline__ bool sim_walk(const Lattice &L, const uint8_t *chi, int a, int qi,
                                         int qj, int &oi, int &oj) {
#pragma unroll 1
  for (int k = 0; k <= 3; ++k) {
    const int ii = qi + k * cx_of(a), jj = qj + k * cy_of(a);
    if (ii < 0 || ii >= L.nx || jj < 0 || jj >= L.ny) return false;
    if (!(chi[(int64_t)jj * L.pitch + ii] & kSolid)) {
      oi = ii;
      oj = jj;
      return true;
    }
  }
  return false;
}

// One SIM integration point: the nearest node (both nodes when the point lies
// exactly half-way), the walk along the direction closest to the normal to the
// first fluid node, sigma averaged over the candidates, then S sigma n and its
// moment about the reference point in FP64.
template <typename S, bool kGather>
__device__ __noinline__ void sim_point(const StepArgs &p, const S *buf, const BodyState &b,
                                       int q) {
  using T = typename Store<S>::T;
  const SimPoint sp = p.sim_pts[q];
  const double x = b.xg + sp.dx, y = b.yg + sp.dy;
  const double rx = floor(x + 0.5), ry = floor(y + 0.5);
  const int ncx = (rx == x + 0.5) ? 2 : 1, ncy = (ry == y + 0.5) ? 2 : 1;
  const T *prev = static_cast<const T *>(p.prev_src);
  T sig[3] = {0, 0, 0};
  int first = -1;
  bool ok = true;
  for (int u = 0; u < ncy && ok; ++u)
    for (int v = 0; v < ncx && ok; ++v) {
      int qi, qj;
      if (!sim_walk(p.L, p.chi, sp.dir, (int)rx - v, (int)ry - u, qi, qj)) {
        ok = false;
        break;
      }
      if (first < 0) first = qj * p.L.nx + qi;
      T s3[3];
      node_stress<S, kGather>(buf, prev, p.L, p.tau_plus, qi, qj, s3);
      sig[0] += s3[0];
      sig[1] += s3[1];
      sig[2] += s3[2];
    }
  double *out = p.sim_contrib + 3 * (int64_t)q;
  if (!ok) {
    p.sim_nodes[q] = -1;
    out[0] = out[1] = out[2] = 0.0;
    return;
  }
  const double cnt = (double)(ncx * ncy);
  // sigma = -(1/3) I + (the small part); the constant part in FP64
  const double sxx = (double)sig[0] / cnt - 1.0 / 3.0;
  const double sxy = (double)sig[1] / cnt;
  const double syy = (double)sig[2] / cnt - 1.0 / 3.0;
  const double tx = sp.s * (sxx * sp.nx + sxy * sp.ny);
  const double ty = sp.s * (sxy * sp.nx + syy * sp.ny);
  p.sim_nodes[q] = first;
  out[0] = tx;
  out[1] = ty;
  out[2] = sp.dx * ty - sp.dy * tx;
}

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

// Re-rasterise the disk mask inside the box covering the old and the new
// position, then refresh the interface bits one node wider.
__device__ void tail_reraster(const StepArgs &p, const BodyState &old_b, const BodyState &new_b) {
  const Lattice &L = p.L;
  const double r = 0.5 * new_b.length;
  const int i0 = max(0, (int)floor(fmin(old_b.xg, new_b.xg) - r) - 2);
  const int i1 = min(L.nx - 1, (int)ceil(fmax(old_b.xg, new_b.xg) + r) + 2);
  const int j0 = max(0, (int)floor(fmin(old_b.yg, new_b.yg) - r) - 2);
  const int j1 = min(L.ny - 1, (int)ceil(fmax(old_b.yg, new_b.yg) + r) + 2);
  const int w = i1 - i0 + 1, h = j1 - j0 + 1;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int k = tid; k < w * h; k += nt) {
    const int i = i0 + k % w, j = j0 + k / w;
    p.chi[(int64_t)j * L.pitch + i] = body_contains(new_b, i, j) ? kSolid : 0;
  }
  __syncthreads();
  const int a0 = max(0, i0 - 1), a1 = min(L.nx - 1, i1 + 1);
  const int b0 = max(0, j0 - 1), b1 = min(L.ny - 1, j1 + 1);
  const int w2 = a1 - a0 + 1, h2 = b1 - b0 + 1;
  for (int k = tid; k < w2 * h2; k += nt) {
    const int i = a0 + k % w2, j = b0 + k / w2;
    const uint8_t self = p.chi[(int64_t)j * L.pitch + i] & kSolid;
    bool iface = false;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      int ni, nj;
      if (neighbour(L, a, i, j, ni, nj) && ((p.chi[(int64_t)nj * L.pitch + ni] & kSolid) != self))
        iface = true;
    }
    // only bit 1 changes here, the solid bits other threads read stay put
    p.chi[(int64_t)j * L.pitch + i] = (uint8_t)(self | (iface ? kInterface : 0));
  }
}

// The last participating block: FP64 sums in a fixed order, histories, body.
__device__ void tail(const StepArgs &p, const ForceRegion &reg, double *red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  __shared__ double tot[6];
  __shared__ BodyState old_b, new_b;
  // partials and SIM entries were written by other SMs: read them through L2
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  for (int k = tid; k < reg.count; k += nt) {
    m0 += __ldcg(p.mem_partials + 3 * k + 0);
    m1 += __ldcg(p.mem_partials + 3 * k + 1);
    m2 += __ldcg(p.mem_partials + 3 * k + 2);
  }
  const bool do_sim = p.sim_blocks > 0;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  int missing = 0;
  if (do_sim) {
    for (int q = tid; q < p.n_sim; q += nt) {
      s0 += __ldcg(p.sim_contrib + 3 * q + 0);
      s1 += __ldcg(p.sim_contrib + 3 * q + 1);
      s2 += __ldcg(p.sim_contrib + 3 * q + 2);
      missing |= __ldcg(p.sim_nodes + q) < 0;
    }
  }
  missing = __syncthreads_or(missing);
  const double v[6] = {m0, m1, m2, s0, s1, s2};
  for (int k = 0; k < 6; ++k) {
    const double r = block_sum(v[k], red);
    if (tid == 0) tot[k] = r;
  }
  __syncthreads();
  const long long step = *p.dev_step;
  if (tid == 0) {
    double *h = p.hist + 6 * (step % p.hist_len);
    for (int k = 0; k < 3; ++k) h[k] = tot[k];
    for (int k = 3; k < 6; ++k) h[k] = do_sim ? tot[k] : __longlong_as_double(0x7ff8000000000000LL);
    for (int k = 0; k < 3; ++k) p.sums[k] += tot[k];
    p.counts[0] += 1;
    if (do_sim) {
      for (int k = 3; k < 6; ++k) p.sums[k] += tot[k];
      p.counts[1] += 1;
      if (missing) atomicOr(p.status, kStatusSimMissing);
    }
    old_b = *p.body_src;
    new_b = old_b;
    ForceRegion nreg = reg;
    if (old_b.moving) {
      const bool sim = old_b.estimator == VPLBM_SIM;
      const double F[3] = {sim ? tot[3] : tot[0], sim ? tot[4] : tot[1], sim ? tot[5] : tot[2]};
      rigid_update(new_b, F);
      nreg = make_region(p.L, new_b.xg, new_b.yg, 0.5 * new_b.length, p.ntiles_x, p.ntiles_y);
      if (nreg.error || nreg.count > p.region_capacity ||
          fabs(new_b.xg - old_b.xg) >= 1.0 || fabs(new_b.yg - old_b.yg) >= 1.0) {
        // the body left the lattice or moved a node in one step: keep it
        // where it was and flag the run as unstable
        atomicOr(p.status, kStatusUnstable);
        new_b = old_b;
        nreg = reg;
      }
    }
    *p.body_dst = new_b;
    *p.reg_dst = nreg;
  }
  __syncthreads();
  if (old_b.moving && (new_b.xg != old_b.xg || new_b.yg != old_b.yg)) tail_reraster(p, old_b, new_b);
  __syncthreads();
  if (tid == 0) {
    *p.dev_step = step + 1;
    __threadfence();
    *p.ticket = 0u;
  }
}

template <typename S, bool kGather>
__global__ void __launch_bounds__(kThreads, VPLBM_STEP_MIN_BLOCKS) step_kernel(const StepArgs p) {
  using T = typename Store<S>::T;
  __shared__ double red[32];
  __shared__ int is_last;
  const Lattice &L = p.L;
  const S *__restrict__ src = static_cast<const S *>(p.src);
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  const ForceRegion reg = *p.reg_src;

  if ((int)blockIdx.x < p.sim_blocks) {
    // ---- SIM points of this level ----
    const BodyState b = *p.body_src;
    const int q = blockIdx.x * kThreads + tid;
    if (q < p.n_sim) sim_point<S, kGather>(p, src, b, q);
  } else {
    const int t = blockIdx.x - p.sim_blocks;
    const int ti = t % p.ntiles_x, tj = t / p.ntiles_x;
    const bool in_reg = ti >= reg.ti0 && ti <= reg.ti1 && tj >= reg.tj0 && tj <= reg.tj1;
    const int i = ti * kTileX + threadIdx.x;
    const int j = tj * kTileY + threadIdx.y;
    const bool valid = i < L.nx && j < L.ny;
    bool bad = false;
    double macc[3] = {0.0, 0.0, 0.0};
    if (valid) {
      S *dst = static_cast<S *>(p.dst);
      const T *prev = static_cast<const T *>(p.prev_src);
      const int64_t node = (int64_t)j * L.pitch + i;

      // ---- streaming (pull) ----
      T h[9];
      if (kGather && i > 0 && i < L.nx - 1 && j > 0 && j < L.ny - 1) {
#pragma unroll
        for (int a = 0; a < 9; ++a)
          h[a] = Store<S>::ld(src + (int64_t)a * L.plane + node - cy_of(a) * L.pitch - cx_of(a));
      } else {
        edge_pops<S, kGather>(src, prev, L, i, j, h);
      }
      if (i == L.nx - 1 && L.bc[1] == VPLBM_OUTLET_CONVECTIVE) {
        T *pd = static_cast<T *>(p.prev_dst);
        pd[0 * L.ny + j] = h[3];
        pd[1 * L.ny + j] = h[6];
        pd[2 * L.ny + j] = h[7];
      }

      // ---- moments and penalized velocity ----
      const T drho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
      const T rho = (T)1 + drho;
      const T bfx = lat_bf<T>(L, 0), bfy = lat_bf<T>(L, 1);
      T jx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
      T jy = (h[2] - h[4]) + (h[5] - h[7]) + (h[6] - h[8]);
      jx += (T)0.5 * bfx;
      jy += (T)0.5 * bfy;
      const uint8_t m = p.chi[node];
      T ux, uy, gx = bfx, gy = bfy;
      if (m & kSolid) {
        T usx, usy;
        solid_velocity<T>(*p.body_src, i, j, usx, usy);
        const T k = (T)p.half_pen;
        const T den = rho + k * rho;
        ux = (jx + k * rho * usx) / den;
        uy = (jy + k * rho * usy) / den;
        const T pen = (T)2 * k;
        gx -= pen * (jx - rho * usx) / ((T)1 + k);
        gy -= pen * (jy - rho * usy) / ((T)1 + k);
      } else {
        const T inv = (T)1 / rho;
        ux = jx * inv;
        uy = jy * inv;
      }
      bad = !(rho > (T)0) || !isfinite(rho);

      // ---- collision (BGK / TRT with the forcing term) ----
      const T s_plus = (T)p.s_plus, s_minus = (T)p.s_minus;
      const T a_plus = (T)p.a_plus, a_minus = (T)p.a_minus;
      const T uu = ux * ux + uy * uy;
      const T ug = ux * gx + uy * gy;
      T ht[9];
      {
        const T w0 = (T)w_of(0);
        const T heq0 = w0 * (drho - (T)1.5 * rho * uu);
        const T f0 = w0 * ((T)-3 * ug);
        ht[0] = h[0] - s_plus * (h[0] - heq0) + a_plus * f0;
      }
#pragma unroll
      for (int a = 1; a <= 6; ++a) {
        if (a == 3 || a == 4) continue;
        const int o = opp_of(a);
        const T w = (T)w_of(a);
        const T cu = (T)cx_of(a) * ux + (T)cy_of(a) * uy;
        const T cg = (T)cx_of(a) * gx + (T)cy_of(a) * gy;
        const T heqp = w * (drho + rho * ((T)4.5 * cu * cu - (T)1.5 * uu));
        const T heqm = w * (T)3 * rho * cu;
        const T fp = w * ((T)9 * cu * cg - (T)3 * ug);
        const T fm = w * (T)3 * cg;
        const T hp = (T)0.5 * (h[a] + h[o]);
        const T hm = (T)0.5 * (h[a] - h[o]);
        const T dp = a_plus * fp - s_plus * (hp - heqp);
        const T dm = a_minus * fm - s_minus * (hm - heqm);
        ht[a] = h[a] + dp + dm;
        ht[o] = h[o] + dp - dm;
      }
#pragma unroll
      for (int a = 0; a < 9; ++a) Store<S>::st(dst + (int64_t)a * L.plane + node, ht[a]);

      // ---- MEM link terms of this node ----
      if (in_reg && (m & kInterface)) mem_terms<S>(p, dst, i, j, m, macc);
    }
    // instability flag, one atomic per warp that saw it
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(p.status, kStatusUnstable);
    if (!in_reg) return;  // uniform over the block
    const double r0 = block_sum(macc[0], red);
    const double r1 = block_sum(macc[1], red);
    const double r2 = block_sum(macc[2], red);
    if (tid == 0) {
      const int k = (tj - reg.tj0) * (reg.ti1 - reg.ti0 + 1) + (ti - reg.ti0);
      p.mem_partials[3 * k + 0] = r0;
      p.mem_partials[3 * k + 1] = r1;
      p.mem_partials[3 * k + 2] = r2;
    }
  }

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
  tail(p, reg, red);
}

template <typename S, bool kGather>
cudaError_t launch_t(const StepArgs &a, cudaStream_t s) {
  const int grid = a.sim_blocks + a.ntiles_x * a.ntiles_y;
  step_kernel<S, kGather><<<grid, dim3(kTileX, kTileY), 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(int dtype, bool gather, const StepArgs &a, cudaStream_t s) {
  switch (dtype) {
    case VPLBM_F64: return gather ? launch_t<double, true>(a, s) : launch_t<double, false>(a, s);
    case VPLBM_F32: return gather ? launch_t<float, true>(a, s) : launch_t<float, false>(a, s);
    case VPLBM_F16_OFS: return gather ? launch_t<__half, true>(a, s) : launch_t<__half, false>(a, s);
    case VPLBM_BF16_OFS:
      return gather ? launch_t<__nv_bfloat16, true>(a, s) : launch_t<__nv_bfloat16, false>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace vplbm
