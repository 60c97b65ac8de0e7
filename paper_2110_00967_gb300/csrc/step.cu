// step.cu -- the fused VP-LBM time step for sm_103a.
//
// One launch advances the lattice by one time step and produces that step's
// forces:
//   * every node: pull-stream the pre-collision populations (Eq. eqBd with the
//     side conditions of Sec. 3.1/3.2), moments and penalized velocity
//     (Eqs. updatestep .. updatestepm), force density G, equilibrium and the
//     BGK/TRT collision with the forcing term (Eq. TRT), store;
//   * interface nodes: their MEM link terms (Eq. MMEL, Eq. fluidtorque) in
//     FP64, reduced per block;
//   * SIM points (when due): stress of Sec. 2.3.2 at the sampled fluid node,
//     S_i sigma n_i and its moment (Eq. defFf) in FP64, one entry per point;
//   * the last block to finish: fixed-order FP64 sums of the MEM partials and
//     the SIM entries, force history and running sums, and for a moving body
//     the FP64 rigid-body update (Eqs. dep1, theta2) and the re-rasterised mask.
//
// The grid is persistent (a fixed number of blocks per SM, each looping over
// 128x2 tiles), so the MEM partial count and the reduction order depend only
// on the lattice and the device.
#include "vplbm_internal.cuh"

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

// Stress of Sec. 2.3.2 at node (i, j) from its pre-collision populations
// (a fluid node: no penalization), FP64.
template <typename S, bool kGather>
__device__ void node_stress(const S *buf, const double *prev, const Lattice &L, double tau_plus,
                            int i, int j, double sig[3]) {
  double f[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) f[a] = (double)pre_pop<S, kGather>(buf, prev, L, a, i, j) + w_of(a);
  double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    rho += f[a];
    jx += cx_of(a) * f[a];
    jy += cy_of(a) * f[a];
  }
  jx += 0.5 * L.bf[0];
  jy += 0.5 * L.bf[1];
  const double ux = jx / rho, uy = jy / rho, uu = ux * ux + uy * uy;
  double pxx = 0.0, pxy = 0.0, pyy = 0.0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const double cu = cx_of(a) * ux + cy_of(a) * uy;
    const double feq = w_of(a) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    const double d = f[a] - feq;
    pxx += cx_of(a) * cx_of(a) * d;
    pxy += cx_of(a) * cy_of(a) * d;
    pyy += cy_of(a) * cy_of(a) * d;
  }
  const double s = 1.0 - 0.5 / tau_plus;
  sig[0] = -rho / 3.0 - s * pxx;
  sig[1] = -s * pxy;
  sig[2] = -rho / 3.0 - s * pyy;
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

// One SIM integration point: nearest node(s), walk along the direction
// closest to the normal to the first fluid node, sigma (mean over tied
// candidates), then S sigma n and its moment about the reference point.
template <typename S, bool kGather>
__device__ void sim_point(const StepArgs &p, const S *buf, double bxg, double byg, int q) {
  const SimPoint sp = p.sim_pts[q];
  const double x = bxg + sp.dx, y = byg + sp.dy;
  const double rx = floor(x + 0.5), ry = floor(y + 0.5);
  const int ncx = (rx == x + 0.5) ? 2 : 1, ncy = (ry == y + 0.5) ? 2 : 1;
  double sig[3] = {0.0, 0.0, 0.0};
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
      double s3[3];
      node_stress<S, kGather>(buf, p.prev_src, p.L, p.tau_plus, qi, qj, s3);
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
  sig[0] /= cnt;
  sig[1] /= cnt;
  sig[2] /= cnt;
  const double tx = sp.s * (sig[0] * sp.nx + sig[1] * sp.ny);
  const double ty = sp.s * (sig[1] * sp.nx + sig[2] * sp.ny);
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
}

// Re-rasterise the disk mask inside the box covering the old and the new
// position (one margin node), then refresh the interface bits one node wider.
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
    uint8_t *m = p.chi + (int64_t)j * L.pitch + i;
    *m = body_contains(new_b, i, j) ? kSolid : 0;
  }
  __syncthreads();
  const int a0 = max(0, i0 - 1), a1 = min(L.nx - 1, i1 + 1);
  const int b0 = max(0, j0 - 1), b1 = min(L.ny - 1, j1 + 1);
  const int w2 = a1 - a0 + 1, h2 = b1 - b0 + 1;
  // compute the new interface bits first, then write them, so every thread
  // reads consistent solid bits
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
    // the solid bit is untouched by this pass; only bit 1 changes
    uint8_t *m = p.chi + (int64_t)j * L.pitch + i;
    *m = (uint8_t)(self | (iface ? kInterface : 0));
  }
}

// The last block: FP64 sums in a fixed order, histories, rigid body.
__device__ void tail(const StepArgs &p, double *red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  __shared__ double tot[6];
  __shared__ BodyState old_b, new_b;
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  // partials and SIM entries were written by other SMs: read through L2
  for (int b = tid; b < (int)gridDim.x; b += nt) {
    m0 += __ldcg(p.mem_partials + 3 * b + 0);
    m1 += __ldcg(p.mem_partials + 3 * b + 1);
    m2 += __ldcg(p.mem_partials + 3 * b + 2);
  }
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  int missing = 0;
  if (p.do_sim) {
    for (int q = tid; q < p.n_sim; q += nt) {
      s0 += __ldcg(p.sim_contrib + 3 * q + 0);
      s1 += __ldcg(p.sim_contrib + 3 * q + 1);
      s2 += __ldcg(p.sim_contrib + 3 * q + 2);
      missing |= __ldcg(p.sim_nodes + q) < 0;
    }
  }
  missing = __syncthreads_or(missing);
  double v[6] = {m0, m1, m2, s0, s1, s2};
  for (int k = 0; k < 6; ++k) {
    const double r = block_sum(v[k], red);
    if (tid == 0) tot[k] = r;
  }
  __syncthreads();
  const long long step = *p.dev_step;
  if (tid == 0) {
    double *h = p.hist + 6 * (step % p.hist_len);
    for (int k = 0; k < 3; ++k) h[k] = tot[k];
    if (p.do_sim) {
      for (int k = 3; k < 6; ++k) h[k] = tot[k];
    } else {
      // keep the previous SIM entry visible as "not evaluated" (NaN)
      for (int k = 3; k < 6; ++k) h[k] = __longlong_as_double(0x7ff8000000000000LL);
    }
    for (int k = 0; k < 3; ++k) p.sums[k] += tot[k];
    p.counts[0] += 1;
    if (p.do_sim) {
      for (int k = 3; k < 6; ++k) p.sums[k] += tot[k];
      p.counts[1] += 1;
      if (missing) atomicOr(p.status, kStatusSimMissing);
    }
    old_b = *p.body;
    new_b = old_b;
    if (old_b.moving) {
      const double F[3] = {old_b.estimator == VPLBM_SIM ? tot[3] : tot[0],
                           old_b.estimator == VPLBM_SIM ? tot[4] : tot[1],
                           old_b.estimator == VPLBM_SIM ? tot[5] : tot[2]};
      rigid_update(new_b, F);
      *p.body = new_b;
    }
  }
  __syncthreads();
  if (old_b.moving) tail_reraster(p, old_b, new_b);
  __syncthreads();
  if (tid == 0) {
    *p.dev_step = step + 1;
    __threadfence();
    *p.ticket = 0u;
  }
}

template <typename S, bool kGather>
__global__ void __launch_bounds__(kThreads) step_kernel(const StepArgs p) {
  using T = typename Store<S>::T;
  __shared__ double red[32];
  __shared__ bool is_last;
  const Lattice &L = p.L;
  const S *__restrict__ src = static_cast<const S *>(p.src);
  S *__restrict__ dst = static_cast<S *>(p.dst);

  const BodyState b = *p.body;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;

  // SIM points spread over the blocks (pre-collision field of this level)
  if (p.do_sim) {
    for (int q = blockIdx.x * kThreads + tid; q < p.n_sim; q += gridDim.x * kThreads)
      sim_point<S, kGather>(p, src, b.xg, b.yg, q);
  }

  const T s_plus = (T)p.s_plus, s_minus = (T)p.s_minus;
  const T a_plus = (T)p.a_plus, a_minus = (T)p.a_minus;
  const T half_pen = (T)p.half_pen;
  const T bfx = (T)L.bf[0], bfy = (T)L.bf[1];
  bool bad = false;
  double mfx = 0.0, mfy = 0.0, mtq = 0.0;

  for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
    const int i = (t % p.ntiles_x) * kTileX + threadIdx.x;
    const int j = (t / p.ntiles_x) * kTileY + threadIdx.y;
    if (i >= L.nx || j >= L.ny) continue;
    const int64_t node = (int64_t)j * L.pitch + i;

    // ---- streaming (pull) ----
    T h[9];
    if (kGather && i > 0 && i < L.nx - 1 && j > 0 && j < L.ny - 1) {
#pragma unroll
      for (int a = 0; a < 9; ++a)
        h[a] = Store<S>::ld(src + (int64_t)a * L.plane + node - cy_of(a) * L.pitch - cx_of(a));
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) h[a] = pre_pop<S, kGather>(src, p.prev_src, L, a, i, j);
    }
    if (i == L.nx - 1 && L.bc[1] == VPLBM_OUTLET_CONVECTIVE) {
      p.prev_dst[0 * L.ny + j] = (double)h[3];
      p.prev_dst[1 * L.ny + j] = (double)h[6];
      p.prev_dst[2 * L.ny + j] = (double)h[7];
    }

    // ---- moments and penalized velocity ----
    const T drho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
    const T rho = (T)1 + drho;
    T jx = (h[1] - h[3]) + (h[5] - h[6]) + (h[8] - h[7]);
    T jy = (h[2] - h[4]) + (h[5] - h[7]) + (h[6] - h[8]);
    jx += (T)0.5 * bfx;
    jy += (T)0.5 * bfy;
    const uint8_t m = p.chi[node];
    T ux, uy, gx = bfx, gy = bfy;
    if (m & kSolid) {
      const T usx = (T)(b.ux - b.omega * ((double)j - b.yg));
      const T usy = (T)(b.uy + b.omega * ((double)i - b.xg));
      const T k = half_pen;
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
    bad |= !(rho > (T)0) || !isfinite(rho);

    // ---- collision (BGK / TRT with the forcing term) ----
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

    // ---- MEM link terms of this node (Eq. MMEL), FP64 ----
    if (m & kInterface) {
      const bool solid = m & kSolid;
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        int ni, nj;
        if (!neighbour(L, a, i, j, ni, nj)) continue;
        const bool nsolid = p.chi[(int64_t)nj * L.pitch + ni] & kSolid;
        if (nsolid == solid) continue;
        // link midpoint and the wall velocity there
        const double xgam = (double)i + 0.5 * cx_of(a), ygam = (double)j + 0.5 * cy_of(a);
        const double ugx = b.ux - b.omega * (ygam - b.yg);
        const double ugy = b.uy + b.omega * (xgam - b.xg);
        const double fa = (double)ht[a] + w_of(a);
        const double sg = solid ? -1.0 : 1.0;
        const double lx = sg * (cx_of(a) - ugx) * fa;
        const double ly = sg * (cy_of(a) - ugy) * fa;
        mfx += lx;
        mfy += ly;
        mtq += (xgam - b.xg) * ly - (ygam - b.yg) * lx;
      }
    }
  }

  // ---- block partials of MEM, instability flag ----
  if (__syncthreads_or(bad) && tid == 0) atomicOr(p.status, kStatusUnstable);
  const double r0 = block_sum(mfx, red);
  const double r1 = block_sum(mfy, red);
  const double r2 = block_sum(mtq, red);
  if (tid == 0) {
    p.mem_partials[3 * blockIdx.x + 0] = r0;
    p.mem_partials[3 * blockIdx.x + 1] = r1;
    p.mem_partials[3 * blockIdx.x + 2] = r2;
    __threadfence();
    const unsigned int prev = atomicAdd(p.ticket, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  tail(p, red);
}

template <typename S, bool kGather>
cudaError_t launch_t(const StepArgs &a, int grid, cudaStream_t s) {
  step_kernel<S, kGather><<<grid, dim3(kTileX, kTileY), 0, s>>>(a);
  return cudaGetLastError();
}

template <typename S, bool kGather>
int occ_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<S, kGather>, kThreads, 0) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace

cudaError_t launch_step(int dtype, bool gather, const StepArgs &a, int grid, cudaStream_t s) {
  switch (dtype) {
    case VPLBM_F64: return gather ? launch_t<double, true>(a, grid, s) : launch_t<double, false>(a, grid, s);
    case VPLBM_F32: return gather ? launch_t<float, true>(a, grid, s) : launch_t<float, false>(a, grid, s);
    case VPLBM_F16_OFS: return gather ? launch_t<__half, true>(a, grid, s) : launch_t<__half, false>(a, grid, s);
    case VPLBM_BF16_OFS:
      return gather ? launch_t<__nv_bfloat16, true>(a, grid, s) : launch_t<__nv_bfloat16, false>(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

int step_blocks_per_sm(int dtype, bool gather) {
  switch (dtype) {
    case VPLBM_F64: return gather ? occ_t<double, true>() : occ_t<double, false>();
    case VPLBM_F32: return gather ? occ_t<float, true>() : occ_t<float, false>();
    case VPLBM_F16_OFS: return gather ? occ_t<__half, true>() : occ_t<__half, false>();
    case VPLBM_BF16_OFS: return gather ? occ_t<__nv_bfloat16, true>() : occ_t<__nv_bfloat16, false>();
  }
  return 1;
}

}  // namespace vplbm
