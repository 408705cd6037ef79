// Residual check that allocates nothing (hz_residual_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they want to check a
// solution: real-time or serving loops that forbid device allocation (it can
// synchronise the device and fragment a memory pool), and frameworks that hand
// out all device memory themselves.  For them this entry point computes the same
// per-RHS relative residual ||M f - A u||_2 / ||M f||_2 as hz_residual, but keeps
// its scratch (per-CTA partial sums and the per-RHS results) in the fixed device
// array below instead of the plan's workspace, and writes no residual field.
//
// The array lives as long as the library is loaded, on every GPU that loads
// it, and is shared by all calls and plans: calls that overlap on the GPU
// (different streams or host threads at the same time) race on it and must be
// serialised by the caller.  It keeps the last call's contents; every slot a
// call reads is written earlier in the same call, so nothing needs clearing.
// The first call on a device looks the array's address up with
// cudaGetSymbolAddress while that device is current (make that first call
// before any stream capture).  The plan's kernels and stream belong to the
// device the plan was created on, so the call requires that device to be the
// current one.
#include <cmath>
#include <mutex>

#include "hz_internal.h"

namespace hz {

// Accessors of plan internals (defined in hz_api.cu).
StencilArgs plan_stencil_args(hz_plan_t p, int nrhs);
cudaStream_t plan_stream(hz_plan_t p);
int plan_device(hz_plan_t p);

namespace {

constexpr int kMaxRhs = 64;            // largest nrhs accepted
constexpr int kParts = 256;            // partial sums per RHS (one per CTA)
constexpr int kScratchDoubles = kMaxRhs * kParts * 2 + kMaxRhs * 2;   // 32,896 doubles = 263 KB

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int NT = 256;
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 c, double2 y, double2 acc) {
  return make_double2(fma(c.x, y.x, fma(-c.y, y.y, acc.x)), fma(c.x, y.y, fma(c.y, y.x, acc.y)));
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < NT / 32; ++q) s += sh[q];
  return s;
}

// Same 7-point residual as the refinement stencil, without storing rho:
// partial[r][part][0] = sum |M (f - M^{-1} A u)|^2, partial[r][part][1] = sum |M f|^2.
__global__ void __launch_bounds__(NT) resid_norms_kernel(const StencilArgs a, const double2* __restrict__ f,
                                                         const double2* __restrict__ u,
                                                         double* __restrict__ partial) {
  __shared__ double sh[NT / 32];
  const int r = blockIdx.y;
  const long long nxy = (long long)a.nx * a.ny;
  const long long n = nxy * a.nz;
  const double2* __restrict__ ur = u + r * n;
  const double2* __restrict__ fr = f + r * n;
  double nr2 = 0.0, nf2 = 0.0;
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT) {
    const int i = (int)(t % a.nx);
    const long long q = t / a.nx;
    const int j = (int)(q % a.ny);
    const int k = (int)(q / a.ny);
    const double2 uc = ur[t];
    const double2* kx = a.kxs + 3 * i;
    const double2* ky = a.kys + 3 * j;
    const double2* tz = a.tzs + 3 * k;
    const double s = a.sig ? a.sig[k] : 1.0;
    double2 h = cmul(make_double2(kx[1].x + ky[1].x, kx[1].y + ky[1].y), uc);
    if (i > 0) h = cfma(kx[0], ur[t - 1], h);
    if (i < a.nx - 1) h = cfma(kx[2], ur[t + 1], h);
    if (j > 0) h = cfma(ky[0], ur[t - a.nx], h);
    if (j < a.ny - 1) h = cfma(ky[2], ur[t + a.nx], h);
    double2 au = cmul(tz[1], uc);
    au.x = fma(s, h.x, au.x);
    au.y = fma(s, h.y, au.y);
    if (k > 0) au = cfma(tz[0], ur[t - nxy], au);
    if (k < a.nz - 1) au = cfma(tz[2], ur[t + nxy], au);
    const double2 fv = fr[t];
    const double rx = fv.x - au.x, ry = fv.y - au.y;
    const double2 mx = a.mx[i], my = a.my[j], mz = a.mz[k];
    const double w2 = (mx.x * mx.x + mx.y * mx.y) * (my.x * my.x + my.y * my.y) * (mz.x * mz.x + mz.y * mz.y);
    nr2 = fma(w2, rx * rx + ry * ry, nr2);
    nf2 = fma(w2, fv.x * fv.x + fv.y * fv.y, nf2);
  }
  const double s1 = block_sum(nr2, sh);
  const double s2 = block_sum(nf2, sh);
  if (threadIdx.x == 0) {
    partial[((long long)r * gridDim.x + blockIdx.x) * 2 + 0] = s1;
    partial[((long long)r * gridDim.x + blockIdx.x) * 2 + 1] = s2;
  }
}

// rel[r] = sqrt(sum_parts nr2 / sum_parts nf2), in fixed order.
__global__ void resid_finish_kernel(const double* __restrict__ partial, int nparts, double* __restrict__ rel) {
  const int r = blockIdx.x;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int p = 0; p < nparts; ++p) {
      a += partial[((long long)r * nparts + p) * 2 + 0];
      b += partial[((long long)r * nparts + p) * 2 + 1];
    }
    rel[r] = b > 0.0 ? sqrt(a / b) : sqrt(a);
  }
}

// Device address of g_scratch on device dev, which must be the current device (looked up
// once per device).
cudaError_t scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaError_t e = cudaSuccess;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace hz

extern "C" hz_status hz_residual_noalloc(hz_plan_t plan, const hz_c128* f_dev, const hz_c128* u_dev, int nrhs,
                                         double* rel_host) {
  using namespace hz;
  if (!plan || !f_dev || !u_dev || !rel_host || nrhs < 1) return HZ_ERR_ARG;
  if (nrhs > kMaxRhs) return HZ_ERR_ARG;          // beyond the fixed scratch array
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HZ_ERR_CUDA;
  if (dev != plan_device(plan)) return HZ_ERR_ARG;   // the plan's stream and tables live on its device
  double* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return HZ_ERR_CUDA;
  const StencilArgs a = plan_stencil_args(plan, nrhs);
  cudaStream_t st = plan_stream(plan);
  const long long n = (long long)a.nx * a.ny * a.nz;
  long long parts = (n + NT * 8 - 1) / (NT * 8);
  if (parts > kParts) parts = kParts;
  if (parts < 1) parts = 1;
  double* partial = scratch;
  double* rel = scratch + (size_t)kMaxRhs * kParts * 2;
  resid_norms_kernel<<<dim3((unsigned)parts, nrhs), NT, 0, st>>>(a, reinterpret_cast<const double2*>(f_dev),
                                                                 reinterpret_cast<const double2*>(u_dev), partial);
  count_launch();
  resid_finish_kernel<<<nrhs, 32, 0, st>>>(partial, (int)parts, rel);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return HZ_ERR_CUDA;
  double out[kMaxRhs];
  if (cudaMemcpyAsync(out, rel, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return HZ_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HZ_ERR_CUDA;
  for (int r = 0; r < nrhs; ++r) {
    if (!std::isfinite(out[r])) return HZ_ERR_NONFINITE;
    rel_host[r] = out[r];
  }
  return HZ_OK;
}
