// cc_tab.cu -- tabulated collapse and the GPU-native interpolation routines.
//
// Sec. 3: in the "Tabulated" option collapse times are precomputed on a grid
// of delta = sum l_i, x = l1 - l2, y = l2 - l3 and interpolated with a cubic
// spline along delta and bilinear interpolation in x and y. Sec. 4.2: because
// the table changes at every smoothing radius, its splines are built on the
// device (one tridiagonal solve per (x, y) node here, one thread each) instead
// of on the host. Sec. 4.3 validates the two routines on toys (y = x^2 on 512
// random knots; a 64 x 64 grid with a 128-knot spline per node): cc_spline_eval
// and cc_table_query expose them for exactly that use.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cc_device.cuh"

namespace cc {
namespace {

// Natural cubic spline through (xs[k], ys[k]), k < n, as per-interval
// coefficients; work holds 2 n doubles. Continuity of the first derivative
// gives h_{k-1} s_{k-1} + 2 (h_{k-1} + h_k) s_k + h_k s_{k+1} = 6 (m_k - m_{k-1})
// for the second derivatives s (s_0 = s_{n-1} = 0), solved by elimination.
__device__ void natural_spline_device(int n, const double* __restrict__ xs, const double* __restrict__ ys,
                                      int ystride, Coef4* __restrict__ out, double* __restrict__ work) {
  double* diag = work;      // n
  double* rhs = work + n;   // n, then the second derivatives in place
  for (int i = 1; i + 1 < n; ++i) {
    const double hl = xs[i] - xs[i - 1], hr = xs[i + 1] - xs[i];
    diag[i] = 2.0 * (hl + hr);
    rhs[i] = 6.0 * ((ys[(i + 1) * ystride] - ys[i * ystride]) / hr - (ys[i * ystride] - ys[(i - 1) * ystride]) / hl);
  }
  for (int i = 2; i + 1 < n; ++i) {
    const double f = (xs[i] - xs[i - 1]) / diag[i - 1];
    diag[i] -= f * (xs[i] - xs[i - 1]);
    rhs[i] -= f * rhs[i - 1];
  }
  rhs[0] = 0.0;
  rhs[n - 1] = 0.0;
  if (n > 2) rhs[n - 2] = rhs[n - 2] / diag[n - 2];
  for (int i = n - 3; i >= 1; --i) rhs[i] = (rhs[i] - (xs[i + 1] - xs[i]) * rhs[i + 1]) / diag[i];
  for (int k = 0; k + 1 < n; ++k) {
    const double h = xs[k + 1] - xs[k];
    const double y0 = ys[k * ystride], y1 = ys[(k + 1) * ystride];
    Coef4 c;
    c.c0 = y0;
    c.c1 = (y1 - y0) / h - h * (2.0 * rhs[k] + rhs[k + 1]) / 6.0;
    c.c2 = 0.5 * rhs[k];
    c.c3 = (rhs[k + 1] - rhs[k]) / (6.0 * h);
    out[k] = c;
  }
}

__global__ void tab_spline_build_kernel(const double* __restrict__ vals, const double* __restrict__ dg, int nd,
                                        int nsys, Coef4* __restrict__ coef, double* __restrict__ work) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  natural_spline_device(nd, dg, vals + static_cast<size_t>(s) * nd, 1, coef + static_cast<size_t>(s) * (nd - 1),
                        work + static_cast<size_t>(s) * 2 * nd);
}

// Largest real root of u^3 + b u^2 + c u + d in FP64: closed form (Cardano or
// trigonometric) and two Newton steps with the exact derivative.
__device__ double cubic_largest_root_fp64(double b, double c, double d) {
  const double b3 = b * (1.0 / 3.0);
  const double pp = c - b * b3;
  const double qq = b3 * (2.0 * b3 * b3 - c) + d;
  const double disc = 0.25 * qq * qq + pp * pp * pp * (1.0 / 27.0);
  double t;
  if (disc > 0.0) {
    const double A = cbrt(0.5 * fabs(qq) + sqrt(disc));
    const double C = (qq > 0.0) ? -A : A;
    t = (C != 0.0) ? C - pp / (3.0 * C) : 0.0;
  } else {
    const double m = sqrt(-pp * (1.0 / 3.0));
    double arg = (m > 0.0) ? (-0.5 * qq) / (m * m * m) : 0.0;
    arg = fmin(1.0, fmax(-1.0, arg));
    t = 2.0 * m * cos(acos(arg) * (1.0 / 3.0));
  }
  double u = t - b3;
  for (int it = 0; it < 2; ++it) {
    const double P = fma(fma(u + b, u, c), u, d);
    const double dP = fma(fma(3.0, u, 2.0 * b), u, c);
    u = (dP != 0.0) ? u - P / dP : u;
  }
  return u;
}

// u = 1/D_c at every node: eigenvalues from (delta, x, y), the R-LPT cubic in u.
__global__ void tab_nodes_kernel(const double* __restrict__ dg, const double* __restrict__ xg,
                                 const double* __restrict__ yg, int nd, int nx, int ny, double* __restrict__ out) {
  const int64_t total = static_cast<int64_t>(nd) * nx * ny;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(i % nd);
    const int64_t s = i / nd;
    const int iy = static_cast<int>(s % ny), ix = static_cast<int>(s / ny);
    const double delta = dg[k], x = xg[ix], y = yg[iy];
    const double l2 = (delta - x + y) / 3.0, l1 = l2 + x, l3 = l2 - y;
    const double c2 = -3.0 / 7.0 * l2 * l3;
    const double c3 = l1 * l2 * l3 / 9.0 - 5.0 / 21.0 * l1 * (l2 * l2 + l3 * l3);
    out[i] = cubic_largest_root_fp64(-l1, c2, c3);
  }
}

__global__ void tab_query_kernel(TabDev td, const double* __restrict__ d, const double* __restrict__ x,
                                 const double* __restrict__ y, int64_t m, double* __restrict__ out) {
  extern __shared__ double s_ax[];
  const int nwords = static_cast<int>((td.axes_bytes() + 7) / 8);
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) s_ax[i] = td.axes[i];
  __syncthreads();
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = tab_interp(td, s_ax, td.coef, d[i], fmax(x[i], 0.0), fmax(y[i], 0.0));
}

// y(q) for m queries: FP32 binary search on the FP32 knots (C2 spline: the
// neighbouring interval gives the same value to rounding), FP64 Horner.
__global__ void spline_eval_kernel(const double* __restrict__ xk, const float* __restrict__ xkf,
                                   const Coef4* __restrict__ coef, int n, int steps, const double* __restrict__ q,
                                   int64_t m, double* __restrict__ out) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double t = q[i];
    const float tf = static_cast<float>(t);
    int k = 0;
    for (int step = steps; step > 0; step >>= 1) {
      const int j = k + step;
      k = (j <= n - 2 && __ldg(xkf + j) <= tf) ? j : k;
    }
    const Coef4 c = coef[k];
    out[i] = horner(c, t - __ldg(xk + k));
  }
}

int pow2_steps(int n) {  // largest power of two <= n - 2 (0 when n <= 2)
  int s = 0;
  if (n - 2 >= 1) {
    s = 1;
    while (s * 2 <= n - 2) s *= 2;
  }
  return s;
}

int grow(void** p, size_t* cap, size_t bytes, const char* what) {
  if (bytes <= *cap) return CC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (int rc = check_cuda(cudaMalloc(p, bytes), what)) return rc;
  *cap = bytes;
  return CC_OK;
}

int check_axes(const double* dg, int nd, const double* xg, int nx, const double* yg, int ny) {
  if (!dg || !xg || !yg) return set_error(CC_EINVAL, "table axes must be non-NULL");
  if (nd < 4 || nd > kTabMaxD || nx < 2 || nx > kTabMaxXY || ny < 2 || ny > kTabMaxXY)
    return set_error(CC_EINVAL, "table sizes: 4 <= nd <= 256, 2 <= nx, ny <= 256");
  for (int i = 0; i + 1 < nd; ++i)
    if (!(dg[i + 1] > dg[i])) return set_error(CC_EINVAL, "delta axis must be strictly increasing");
  for (int i = 0; i + 1 < nx; ++i)
    if (!(xg[i + 1] > xg[i])) return set_error(CC_EINVAL, "x axis must be strictly increasing");
  for (int i = 0; i + 1 < ny; ++i)
    if (!(yg[i + 1] > yg[i])) return set_error(CC_EINVAL, "y axis must be strictly increasing");
  if (!(xg[0] >= 0.0) || !(yg[0] >= 0.0)) return set_error(CC_EINVAL, "x and y axes must start at >= 0");
  return CC_OK;
}

}  // namespace

int launch_tab_checked(cc_ctx* ctx, const LaunchArgs& a) {
  if (!ctx->tab_valid) return set_error(CC_EINVAL, "CC_MODE_TABULATED needs a table: call cc_set_table first");
  return launch_tab(a, ctx->tab, ctx->tabdev);
}

}  // namespace cc

using namespace cc;

extern "C" {

int cc_set_table(cc_ctx* ctx, const double* dgrid, int32_t nd, const double* xgrid, int32_t nx,
                 const double* ygrid, int32_t ny, const double* values, void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (int rc = check_axes(dgrid, nd, xgrid, nx, ygrid, ny)) return rc;
  if (!values) return set_error(CC_EINVAL, "values is NULL");
  const size_t nv = static_cast<size_t>(nx) * ny * nd;
  for (size_t i = 0; i < nv; ++i)
    if (!std::isfinite(values[i])) return set_error(CC_EINVAL, "table values must be finite");
  if (int rc = select_device(ctx)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TabDev td{};
  td.nd = nd;
  td.nx = nx;
  td.ny = ny;
  const size_t ab = td.axes_bytes();
  const size_t nsys = static_cast<size_t>(nx) * ny;
  if (int rc = grow(&ctx->d_tab_axes, &ctx->tab_axes_cap, ab, "cudaMalloc(table axes)")) return rc;
  if (int rc = grow(reinterpret_cast<void**>(&ctx->d_tab_coef), &ctx->tab_coef_cap, sizeof(Coef4) * nsys * (nd - 1),
                    "cudaMalloc(table coefficients)"))
    return rc;
  if (int rc = grow(reinterpret_cast<void**>(&ctx->d_tab_work), &ctx->tab_work_cap, sizeof(double) * nsys * nd * 3,
                    "cudaMalloc(table scratch)"))
    return rc;
  std::vector<double> img((ab + 7) / 8, 0.0);
  double* p = img.data();
  std::memcpy(p, dgrid, sizeof(double) * nd);
  std::memcpy(p + nd, xgrid, sizeof(double) * nx);
  std::memcpy(p + nd + nx, ygrid, sizeof(double) * ny);
  for (int i = 0; i + 1 < nx; ++i) p[nd + nx + ny + i] = 1.0 / (xgrid[i + 1] - xgrid[i]);
  for (int i = 0; i + 1 < ny; ++i) p[nd + nx + ny + (nx - 1) + i] = 1.0 / (ygrid[i + 1] - ygrid[i]);
  // cell offsets: the bilinear weight (x - x_i) / h_i as one FMA, x (1/h_i) + (-x_i / h_i)
  for (int i = 0; i + 1 < nx; ++i) p[nd + nx + ny + (nx - 1) + (ny - 1) + i] = -(xgrid[i] * p[nd + nx + ny + i]);
  for (int i = 0; i + 1 < ny; ++i)
    p[nd + nx + ny + 2 * (nx - 1) + (ny - 1) + i] = -(ygrid[i] * p[nd + nx + ny + (nx - 1) + i]);
  float* pf = reinterpret_cast<float*>(p + nd + nx + ny + 2 * (nx - 1) + 2 * (ny - 1));
  for (int k = 0; k < nd; ++k) pf[k] = static_cast<float>(dgrid[k]);
  ctx->tab_valid = false;
  // pageable sources: each call returns once its data is staged
  if (int rc = check_cuda(cudaMemcpyAsync(ctx->d_tab_axes, img.data(), ab, cudaMemcpyHostToDevice, st), "H2D table axes"))
    return rc;
  double* d_vals = ctx->d_tab_work;
  if (int rc = check_cuda(cudaMemcpyAsync(d_vals, values, sizeof(double) * nv, cudaMemcpyHostToDevice, st), "H2D table values"))
    return rc;
  const int threads = 128;
  const int blocks = static_cast<int>((nsys + threads - 1) / threads);
  tab_spline_build_kernel<<<blocks, threads, 0, st>>>(d_vals, static_cast<const double*>(ctx->d_tab_axes), nd,
                                                      static_cast<int>(nsys), ctx->d_tab_coef, d_vals + nv);
  if (int rc = check_cuda(cudaGetLastError(), "tab_spline_build_kernel launch")) return rc;
  td.axes = static_cast<const double*>(ctx->d_tab_axes);
  td.coef = ctx->d_tab_coef;
  td.d_steps = pow2_steps(nd);
  td.x_steps = pow2_steps(nx);
  td.y_steps = pow2_steps(ny);
  td.d_lo = dgrid[0];
  td.d_hi = dgrid[nd - 1];
  // integer keys that order like the values: the hull test on delta takes
  // no FP64 compare
  td.d_lo_key = order_key(td.d_lo);
  td.d_hi_key = order_key(td.d_hi);
  td.x_lo = xgrid[0];
  td.x_hi = xgrid[nx - 1];
  td.y_lo = ygrid[0];
  td.y_hi = ygrid[ny - 1];
  ctx->tabdev = td;
  ctx->tab_valid = true;
  return CC_OK;
}

int cc_table_nodes_rlpt(cc_ctx* ctx, const double* dgrid, int32_t nd, const double* xgrid, int32_t nx,
                        const double* ygrid, int32_t ny, double* values, void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (int rc = check_axes(dgrid, nd, xgrid, nx, ygrid, ny)) return rc;
  if (!values) return set_error(CC_EINVAL, "values is NULL");
  if (int rc = select_device(ctx)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nv = static_cast<size_t>(nx) * ny * nd;
  double* buf = nullptr;
  if (int rc = check_cuda(cudaMalloc(reinterpret_cast<void**>(&buf), sizeof(double) * (nv + nd + nx + ny)), "cudaMalloc(nodes)"))
    return rc;
  int rc = check_cuda(cudaMemcpyAsync(buf + nv, dgrid, sizeof(double) * nd, cudaMemcpyHostToDevice, st), "H2D");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(buf + nv + nd, xgrid, sizeof(double) * nx, cudaMemcpyHostToDevice, st), "H2D");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(buf + nv + nd + nx, ygrid, sizeof(double) * ny, cudaMemcpyHostToDevice, st), "H2D");
  if (!rc) {
    const int blocks = static_cast<int>(std::min<size_t>((nv + 255) / 256, 4096));
    tab_nodes_kernel<<<blocks, 256, 0, st>>>(buf + nv, buf + nv + nd, buf + nv + nd + nx, nd, nx, ny, buf);
    rc = check_cuda(cudaGetLastError(), "tab_nodes_kernel launch");
  }
  if (!rc) rc = check_cuda(cudaMemcpyAsync(values, buf, sizeof(double) * nv, cudaMemcpyDeviceToHost, st), "D2H nodes");
  if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  cudaFree(buf);
  return rc;
}

int cc_table_query(cc_ctx* ctx, const double* d, const double* x, const double* y, int64_t m, double* out,
                   void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (!ctx->tab_valid) return set_error(CC_EINVAL, "no table: call cc_set_table first");
  if (m < 0) return set_error(CC_EINVAL, "m must be >= 0");
  if (m > 0 && (!d || !x || !y || !out)) return set_error(CC_EINVAL, "NULL query or output array");
  if (m == 0) return CC_OK;
  if (int rc = select_device(ctx)) return rc;
  const TabDev& td = ctx->tabdev;
  const size_t smem = ((td.axes_bytes() + 15) / 16) * 16;
  const int64_t need = (m + 255) / 256;
  const int grid = static_cast<int>(std::min<int64_t>(need, static_cast<int64_t>(ctx->num_sms) * 8));
  tab_query_kernel<<<grid, 256, smem, static_cast<cudaStream_t>(stream)>>>(td, d, x, y, m, out);
  return check_cuda(cudaGetLastError(), "tab_query_kernel launch");
}

int cc_spline_eval(cc_ctx* ctx, const double* xk, const double* yk, int32_t n, const double* q, int64_t m,
                   double* out, void* stream) {
  if (!ctx) return set_error(CC_EINVAL, "ctx is NULL");
  if (!xk || !yk || n < 2 || n > kMaxKnots) return set_error(CC_EINVAL, "need 2 <= n <= 4096 host knots");
  for (int i = 0; i + 1 < n; ++i)
    if (!(xk[i + 1] > xk[i])) return set_error(CC_EINVAL, "knots must be strictly increasing");
  if (m < 0 || (m > 0 && (!q || !out))) return set_error(CC_EINVAL, "bad query arrays");
  if (int rc = select_device(ctx)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // One spline is a serial O(n) tridiagonal solve: a single device thread
  // took ~1.5 ms for 512 knots (dependent FP64 divisions), the host takes a
  // few microseconds. Built on the host in FP64, uploaded as one image:
  // coef (n-1) | xk (n) | xkf (n, FP32 copies for the interval search).
  std::vector<double> img(4 * static_cast<size_t>(n - 1) + n + (n + 1) / 2);
  std::vector<double> work(6 * static_cast<size_t>(n));
  if (int rc = natural_spline_into(n, xk, yk, img.data(), work.data())) return set_error(rc, "spline build failed");
  double* hx = img.data() + 4 * (n - 1);
  std::memcpy(hx, xk, sizeof(double) * n);
  float* hxf = reinterpret_cast<float*>(hx + n);
  for (int k = 0; k < n; ++k) hxf[k] = static_cast<float>(xk[k]);
  const size_t bytes = sizeof(double) * img.size();
  if (int rc = grow(&ctx->d_spl, &ctx->spl_cap, bytes, "cudaMalloc(spline image)")) return rc;
  // pageable source: the call returns once the image is staged
  if (int rc = check_cuda(cudaMemcpyAsync(ctx->d_spl, img.data(), bytes, cudaMemcpyHostToDevice, st), "H2D spline"))
    return rc;
  const Coef4* coef = static_cast<const Coef4*>(ctx->d_spl);
  const double* dx = reinterpret_cast<const double*>(coef + (n - 1));
  const float* xkf = reinterpret_cast<const float*>(dx + n);
  if (m == 0) return CC_OK;
  const int64_t need = (m + 255) / 256;
  const int grid = static_cast<int>(std::min<int64_t>(need, static_cast<int64_t>(ctx->num_sms) * 8));
  spline_eval_kernel<<<grid, 256, 0, st>>>(dx, xkf, coef, n, pow2_steps(n), q, m, out);
  return check_cuda(cudaGetLastError(), "spline_eval_kernel launch");
}

}  // extern "C"
