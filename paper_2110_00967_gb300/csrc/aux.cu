// aux.cu -- mask rasterisation (Eq. fcar), interface flags, initial state and
// the conversions between the stored offsets and FP64 fields.
#include "vplbm_internal.cuh"

namespace vplbm {

namespace {

constexpr int kAuxThreads = 256;

inline int blocks_for(int64_t n) { return (int)((n + kAuxThreads - 1) / kAuxThreads); }

// chi on the box [i0, i1] x [j0, j1] (Eq. fcar: 1 inside or on the body)
__global__ void raster_kernel(Lattice L, const BodyState *body, uint8_t *chi, int i0, int j0,
                              int w, int h) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= w * h) return;
  const int i = i0 + k % w, j = j0 + k / w;
  const BodyState b = *body;
  chi[(int64_t)j * L.pitch + i] = body_contains(b, i, j) ? kSolid : 0;
}

// interface bit: some lattice neighbour (inside the lattice) has the other phase
__global__ void interface_kernel(Lattice L, uint8_t *chi, int i0, int j0, int w, int h) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= w * h) return;
  const int i = i0 + k % w, j = j0 + k / w;
  const uint8_t self = chi[(int64_t)j * L.pitch + i] & kSolid;
  bool iface = false;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    int ni, nj;
    if (neighbour(L, a, i, j, ni, nj) && ((chi[(int64_t)nj * L.pitch + ni] & kSolid) != self))
      iface = true;
  }
  chi[(int64_t)j * L.pitch + i] = (uint8_t)(self | (iface ? kInterface : 0));
}

// f = feq(1, u0) with u0 = u_in on fluid nodes and the rigid velocity on
// solid nodes; stored as offsets f - E
template <typename S>
__global__ void init_kernel(Lattice L, const BodyState *body, const uint8_t *chi, S *buf,
                            double u0x, double u0y) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)L.nx * L.ny) return;
  const int i = (int)(k % L.nx), j = (int)(k / L.nx);
  const int64_t node = (int64_t)j * L.pitch + i;
  double ux = u0x, uy = u0y;
  if (chi[node] & kSolid) {
    const BodyState b = *body;
    ux = b.ux - b.omega * ((double)j - b.yg);
    uy = b.uy + b.omega * ((double)i - b.xg);
  }
  // feq(1, u0) - E = w (Q(u0) - Q(u_ref)) with Q(u) = 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2,
  // written with du = u0 - u_ref
  const double dux = ux - L.ur[0], duy = uy - L.ur[1];
  const double dsu = dux * (ux + L.ur[0]) + duy * (uy + L.ur[1]);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const double cdu = cx_of(a) * dux + cy_of(a) * duy;
    const double csu = cx_of(a) * (ux + L.ur[0]) + cy_of(a) * (uy + L.ur[1]);
    const double h = w_of(a) * (3.0 * cdu + 4.5 * cdu * csu - 1.5 * dsu);
    buf[(int64_t)a * L.plane + node] = Store<S>::from_double(h);
  }
}

// Read-back kernels cover the rows j0 .. j0 + rows - 1 and write them
// compactly, [rows][nx] per output plane, so that the host read-backs can
// stage a few rows at a time.

// planes a0 .. a0 + na - 1 of the pre-collision populations f = h + E
template <typename S, bool kGather>
__global__ void get_f_kernel(Lattice L, const S *buf, const typename Store<S>::T *prev,
                             double *out, int a0, int na, int j0, int rows) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)L.nx * rows;
  if (k >= n) return;
  const int i = (int)(k % L.nx), j = j0 + (int)(k / L.nx);
#pragma unroll
  for (int a = 0; a < 9; ++a)
    if (a >= a0 && a < a0 + na)
      out[(a - a0) * n + k] = (double)pre_pop<S, kGather>(buf, prev, L, a, i, j) + L.E[a];
}

// macroscopic fields of Eqs. updatestep and updatestepm, FP64
template <typename S, bool kGather>
__global__ void get_fields_kernel(Lattice L, const S *buf, const typename Store<S>::T *prev,
                                  const uint8_t *chi, const BodyState *body, double half_pen,
                                  double *rho_o, double *ux_o, double *uy_o, int j0, int rows) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)L.nx * rows;
  if (k >= n) return;
  const int i = (int)(k % L.nx), j = j0 + (int)(k / L.nx);
  double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const double f = (double)pre_pop<S, kGather>(buf, prev, L, a, i, j) + L.E[a];
    rho += f;
    jx += cx_of(a) * f;
    jy += cy_of(a) * f;
  }
  jx += 0.5 * L.bf[0];
  jy += 0.5 * L.bf[1];
  double ux = jx / rho, uy = jy / rho;
  if (chi[(int64_t)j * L.pitch + i] & kSolid) {
    const BodyState b = *body;
    const double usx = b.ux - b.omega * ((double)j - b.yg);
    const double usy = b.uy + b.omega * ((double)i - b.xg);
    ux = (jx + half_pen * rho * usx) / (rho + half_pen * rho);
    uy = (jy + half_pen * rho * usy) / (rho + half_pen * rho);
  }
  rho_o[k] = rho;
  ux_o[k] = ux;
  uy_o[k] = uy;
}

template <typename S>
__global__ void set_state_kernel(Lattice L, const double *f, S *buf) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)L.nx * L.ny;
  if (k >= n) return;
  const int i = (int)(k % L.nx), j = (int)(k / L.nx);
  const int64_t node = (int64_t)j * L.pitch + i;
#pragma unroll
  for (int a = 0; a < 9; ++a)
    buf[(int64_t)a * L.plane + node] = Store<S>::from_double(f[a * n + k] - L.E[a]);
}

// outlet column (a = 3, 6, 7 at i = nx - 1) of a pre-collision FP64 field,
// kept as offsets in the compute type
template <typename T>
__global__ void set_prev_kernel(Lattice L, const double *f, T *prev) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.ny) return;
  const int64_t n = (int64_t)L.nx * L.ny;
  const int64_t k = (int64_t)j * L.nx + (L.nx - 1);
  prev[0 * L.ny + j] = (T)(f[3 * n + k] - L.E[3]);
  prev[1 * L.ny + j] = (T)(f[6 * n + k] - L.E[6]);
  prev[2 * L.ny + j] = (T)(f[7 * n + k] - L.E[7]);
}

__global__ void get_mask_kernel(Lattice L, const uint8_t *chi, uint8_t *out, int j0, int rows) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)L.nx * rows) return;
  const int i = (int)(k % L.nx), j = j0 + (int)(k / L.nx);
  out[k] = chi[(int64_t)j * L.pitch + i] & kSolid;
}

template <typename S>
cudaError_t get_f_t(bool gather, const Lattice &L, const void *buf, const void *prev_v,
                    double *out, int a0, int na, int j0, int rows, cudaStream_t s) {
  using T = typename Store<S>::T;
  const T *prev = static_cast<const T *>(prev_v);
  const int g = blocks_for((int64_t)L.nx * rows);
  if (gather)
    get_f_kernel<S, true><<<g, kAuxThreads, 0, s>>>(L, (const S *)buf, prev, out, a0, na, j0, rows);
  else
    get_f_kernel<S, false><<<g, kAuxThreads, 0, s>>>(L, (const S *)buf, prev, out, a0, na, j0, rows);
  return cudaGetLastError();
}

template <typename S>
cudaError_t get_fields_t(bool gather, const Lattice &L, const void *buf, const void *prev_v,
                         const uint8_t *chi, const BodyState *body, double half_pen, double *rho,
                         double *ux, double *uy, int j0, int rows, cudaStream_t s) {
  using T = typename Store<S>::T;
  const T *prev = static_cast<const T *>(prev_v);
  const int g = blocks_for((int64_t)L.nx * rows);
  if (gather)
    get_fields_kernel<S, true><<<g, kAuxThreads, 0, s>>>(L, (const S *)buf, prev, chi, body,
                                                         half_pen, rho, ux, uy, j0, rows);
  else
    get_fields_kernel<S, false><<<g, kAuxThreads, 0, s>>>(L, (const S *)buf, prev, chi, body,
                                                          half_pen, rho, ux, uy, j0, rows);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster(const Lattice &L, const BodyState *body, uint8_t *chi, int i0, int j0,
                          int i1, int j1, cudaStream_t s) {
  const int w = i1 - i0 + 1, h = j1 - j0 + 1;
  if (w <= 0 || h <= 0) return cudaSuccess;
  raster_kernel<<<blocks_for((int64_t)w * h), kAuxThreads, 0, s>>>(L, body, chi, i0, j0, w, h);
  return cudaGetLastError();
}

cudaError_t launch_interface(const Lattice &L, uint8_t *chi, int i0, int j0, int i1, int j1,
                             cudaStream_t s) {
  const int w = i1 - i0 + 1, h = j1 - j0 + 1;
  if (w <= 0 || h <= 0) return cudaSuccess;
  interface_kernel<<<blocks_for((int64_t)w * h), kAuxThreads, 0, s>>>(L, chi, i0, j0, w, h);
  return cudaGetLastError();
}

cudaError_t launch_init(int dtype, const Lattice &L, const BodyState *body, const uint8_t *chi,
                        void *buf, double u0x, double u0y, cudaStream_t s) {
  const int g = blocks_for((int64_t)L.nx * L.ny);
  switch (dtype) {
    case VPLBM_F64: init_kernel<double><<<g, kAuxThreads, 0, s>>>(L, body, chi, (double *)buf, u0x, u0y); break;
    case VPLBM_F32: init_kernel<float><<<g, kAuxThreads, 0, s>>>(L, body, chi, (float *)buf, u0x, u0y); break;
    case VPLBM_F16_OFS: init_kernel<__half><<<g, kAuxThreads, 0, s>>>(L, body, chi, (__half *)buf, u0x, u0y); break;
    case VPLBM_BF16_OFS:
      init_kernel<__nv_bfloat16><<<g, kAuxThreads, 0, s>>>(L, body, chi, (__nv_bfloat16 *)buf, u0x, u0y);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_get_f(int dtype, bool gather, const Lattice &L, const void *buf,
                         const void *prev, double *out, int a0, int na, int j0, int rows,
                         cudaStream_t s) {
  if (rows <= 0 || na <= 0) return cudaSuccess;
  switch (dtype) {
    case VPLBM_F64: return get_f_t<double>(gather, L, buf, prev, out, a0, na, j0, rows, s);
    case VPLBM_F32: return get_f_t<float>(gather, L, buf, prev, out, a0, na, j0, rows, s);
    case VPLBM_F16_OFS: return get_f_t<__half>(gather, L, buf, prev, out, a0, na, j0, rows, s);
    case VPLBM_BF16_OFS: return get_f_t<__nv_bfloat16>(gather, L, buf, prev, out, a0, na, j0, rows, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_get_fields(int dtype, bool gather, const Lattice &L, const void *buf,
                              const void *prev, const uint8_t *chi, const BodyState *body,
                              double half_pen, double *rho, double *ux, double *uy, int j0,
                              int rows, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  switch (dtype) {
    case VPLBM_F64:
      return get_fields_t<double>(gather, L, buf, prev, chi, body, half_pen, rho, ux, uy, j0, rows, s);
    case VPLBM_F32:
      return get_fields_t<float>(gather, L, buf, prev, chi, body, half_pen, rho, ux, uy, j0, rows, s);
    case VPLBM_F16_OFS:
      return get_fields_t<__half>(gather, L, buf, prev, chi, body, half_pen, rho, ux, uy, j0, rows, s);
    case VPLBM_BF16_OFS:
      return get_fields_t<__nv_bfloat16>(gather, L, buf, prev, chi, body, half_pen, rho, ux, uy, j0,
                                         rows, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_set_state(int dtype, const Lattice &L, const double *f, void *buf,
                             cudaStream_t s) {
  const int g = blocks_for((int64_t)L.nx * L.ny);
  switch (dtype) {
    case VPLBM_F64: set_state_kernel<double><<<g, kAuxThreads, 0, s>>>(L, f, (double *)buf); break;
    case VPLBM_F32: set_state_kernel<float><<<g, kAuxThreads, 0, s>>>(L, f, (float *)buf); break;
    case VPLBM_F16_OFS: set_state_kernel<__half><<<g, kAuxThreads, 0, s>>>(L, f, (__half *)buf); break;
    case VPLBM_BF16_OFS:
      set_state_kernel<__nv_bfloat16><<<g, kAuxThreads, 0, s>>>(L, f, (__nv_bfloat16 *)buf);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_set_prev(int dtype, const Lattice &L, const double *f, void *prev,
                            cudaStream_t s) {
  if (dtype == VPLBM_F64)
    set_prev_kernel<double><<<blocks_for(L.ny), kAuxThreads, 0, s>>>(L, f, (double *)prev);
  else
    set_prev_kernel<float><<<blocks_for(L.ny), kAuxThreads, 0, s>>>(L, f, (float *)prev);
  return cudaGetLastError();
}

cudaError_t launch_get_mask(const Lattice &L, const uint8_t *chi, uint8_t *out, int j0, int rows,
                            cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  get_mask_kernel<<<blocks_for((int64_t)L.nx * rows), kAuxThreads, 0, s>>>(L, chi, out, j0, rows);
  return cudaGetLastError();
}

}  // namespace vplbm
