// static_sim.cu -- the SIM force of a caller-supplied state without any
// device allocation: the scratch the evaluation needs (the integration
// points, one force term per point, a flag) lives in a fixed array in this
// file.  For callers that must not allocate device memory themselves (see
// vplbm_sim_force_static in include/vplbm.h).
#include <string>

#include "vplbm_internal.cuh"

// most integration points one call takes (the scratch holds 8 doubles per
// point: 4096 points are 256 KiB, held by every GPU that loads the library)
#ifndef VPLBM_STATIC_SIM_MAX_POINTS
#define VPLBM_STATIC_SIM_MAX_POINTS 4096
#endif

namespace {

using vplbm::cx_of;
using vplbm::cy_of;
using vplbm::w_of;

constexpr int kMaxPts = VPLBM_STATIC_SIM_MAX_POINTS;
constexpr int kDoubles = 8;  // per point: dx, dy, nx, ny, S, then Fx, Fy, T

// scratch layout: [0] missing-point count (as a double), [1..3] result,
// [4..7] unused, then kMaxPts rows of kDoubles
constexpr int kHeader = 8;
static __device__ __align__(256) double g_scratch[kHeader + kMaxPts * kDoubles];

// SIM term of one point from FP64 pre-collision populations (the same
// definition as the library's step: nearest node or both nodes of an exact
// tie, walk along the lattice direction closest to the normal to the first
// fluid node, stress of Sec. 2.3.2 averaged over the candidates)
__global__ void sim_terms_kernel(double *scratch, const double *f, const uint8_t *chi, int nx,
                                 int ny, int n, double xg, double yg, double tau_plus, double bfx,
                                 double bfy) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double *row = scratch + kHeader + (size_t)q * kDoubles;
  const double dx = row[0], dy = row[1], nxv = row[2], nyv = row[3], sl = row[4];
  // lattice direction closest to the normal, ties to the lowest index
  int dir = 1;
  double best = -1e300;
  for (int a = 1; a < 9; ++a) {
    const double cl = a <= 4 ? 1.0 : sqrt(2.0);
    const double v = (cx_of(a) * nxv + cy_of(a) * nyv) / cl;
    if (v > best) {
      best = v;
      dir = a;
    }
  }
  const double x = xg + dx, y = yg + dy;
  const double rx = floor(x + 0.5), ry = floor(y + 0.5);
  const int ncx = (rx == x + 0.5) ? 2 : 1, ncy = (ry == y + 0.5) ? 2 : 1;
  const int64_t plane = (int64_t)nx * ny;
  double s[3] = {0.0, 0.0, 0.0};
  bool ok = true;
  for (int u = 0; u < ncy && ok; ++u)
    for (int v = 0; v < ncx && ok; ++v) {
      int qi = (int)rx - v, qj = (int)ry - u;
      bool found = false;
      for (int k = 0; k <= 3 && !found; ++k) {
        const int ii = qi + k * cx_of(dir), jj = qj + k * cy_of(dir);
        if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) break;
        if (!chi[(int64_t)jj * nx + ii]) {
          qi = ii;
          qj = jj;
          found = true;
        }
      }
      if (!found) {
        ok = false;
        break;
      }
      double fl[9], rho = 0.0, jx = 0.5 * bfx, jy = 0.5 * bfy;
      for (int a = 0; a < 9; ++a) {
        fl[a] = f[a * plane + (int64_t)qj * nx + qi];
        rho += fl[a];
        jx += cx_of(a) * fl[a];
        jy += cy_of(a) * fl[a];
      }
      const double ux = jx / rho, uy = jy / rho, uu = ux * ux + uy * uy;
      double pxx = 0.0, pxy = 0.0, pyy = 0.0;
      for (int a = 0; a < 9; ++a) {
        const double cu = cx_of(a) * ux + cy_of(a) * uy;
        const double d = fl[a] - w_of(a) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        pxx += cx_of(a) * cx_of(a) * d;
        pxy += cx_of(a) * cy_of(a) * d;
        pyy += cy_of(a) * cy_of(a) * d;
      }
      const double sf = 1.0 - 0.5 / tau_plus;
      s[0] += -rho / 3.0 - sf * pxx;
      s[1] += -sf * pxy;
      s[2] += -rho / 3.0 - sf * pyy;
    }
  if (!ok) {
    row[5] = row[6] = row[7] = 0.0;
    atomicAdd(scratch, 1.0);
    return;
  }
  const double inv = 1.0 / (double)(ncx * ncy);
  const double sxx = s[0] * inv, sxy = s[1] * inv, syy = s[2] * inv;
  const double tx = sl * (sxx * nxv + sxy * nyv);
  const double ty = sl * (sxy * nxv + syy * nyv);
  row[5] = tx;
  row[6] = ty;
  row[7] = dx * ty - dy * tx;
}

// the sum over the points in point order (one thread: the order is fixed)
__global__ void sim_sum_kernel(double *scratch, int n) {
  double fx = 0.0, fy = 0.0, tq = 0.0;
  for (int q = 0; q < n; ++q) {
    const double *row = scratch + kHeader + (size_t)q * kDoubles;
    fx += row[5];
    fy += row[6];
    tq += row[7];
  }
  scratch[1] = fx;
  scratch[2] = fy;
  scratch[3] = tq;
}

vplbm_status static_fail(vplbm_status st, const std::string &msg) {
  vplbm::set_global_error(msg);  // read back with vplbm_last_error(NULL)
  return st;
}

}  // namespace

extern "C" vplbm_status vplbm_sim_force_static(const vplbm_config *cfg, const double *f_dev,
                                               const uint8_t *chi_dev, int32_t n_pts,
                                               const double *pts, const double ref[2],
                                               double out[3], void *cuda_stream) {
  if (!cfg || !f_dev || !chi_dev || !pts || !ref || !out)
    return static_fail(VPLBM_EINVAL, "vplbm_sim_force_static: NULL argument");
  if (cfg->nx < 3 || cfg->ny < 3 || !(cfg->tau_plus > 0.5))
    return static_fail(VPLBM_EINVAL, "vplbm_sim_force_static: bad lattice size or tau_plus");
  if (cfg->sim_order != 0)
    return static_fail(VPLBM_EINVAL, "vplbm_sim_force_static: only the stress copied from the "
                                     "sampled node (sim_order 0) is evaluated here");
  if (n_pts < 1 || n_pts > kMaxPts)
    return static_fail(VPLBM_EINVAL, "vplbm_sim_force_static: " + std::to_string(n_pts) +
                                         " points; this entry point holds at most " +
                                         std::to_string(kMaxPts));
  // the device address of the scratch array on the current device (its name
  // in host code is not a device address).  Taken on every call, with the
  // device current: cudaGetSymbolAddress allocates nothing, and a context
  // torn down and re-created between calls (a device reset by the embedding
  // application) gets the array's new address.  On the first call on a
  // device it also loads this library's device code there.
  double *scratch = nullptr;
  {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr)
      return static_fail(VPLBM_ECUDA, std::string("vplbm_sim_force_static: cudaGetSymbolAddress: ") +
                                          cudaGetErrorString(e));
    scratch = static_cast<double *>(ptr);
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the points into the scratch rows (columns 0..4), the header cleared
  cudaError_t e = cudaMemsetAsync(scratch, 0, kHeader * sizeof(double), s);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(scratch + kHeader, kDoubles * sizeof(double), pts, 5 * sizeof(double),
                          5 * sizeof(double), (size_t)n_pts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    sim_terms_kernel<<<(n_pts + 127) / 128, 128, 0, s>>>(
        scratch, f_dev, chi_dev, cfg->nx, cfg->ny, n_pts, ref[0], ref[1], cfg->tau_plus,
        cfg->body_force[0], cfg->body_force[1]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    sim_sum_kernel<<<1, 1, 0, s>>>(scratch, n_pts);
    e = cudaGetLastError();
  }
  double head[4];
  if (e == cudaSuccess) e = cudaMemcpyAsync(head, scratch, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return static_fail(VPLBM_ECUDA, std::string("vplbm_sim_force_static: ") + cudaGetErrorString(e));
  out[0] = head[1];
  out[1] = head[2];
  out[2] = head[3];
  if (head[0] != 0.0)
    return static_fail(VPLBM_ESTATE, "vplbm_sim_force_static: a point found no fluid node");
  return VPLBM_OK;
}
