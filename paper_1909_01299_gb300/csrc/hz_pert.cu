// Vector kernels of the restarted GMRES that solves a locally perturbed layered medium
// with the layered solve as its operator (Sec. 1: the fast layered solver as a
// preconditioner for media with embedded inhomogeneities).
//
// Vectors are the solver's volumes: nrhs right-hand sides of n complex values each,
// [r][n]; a Krylov basis is a run of such volumes, [i][r][n].  Everything is FP64 and
// bound by HBM: each kernel streams its vectors once (grid-stride, coalesced), the
// multi-vector dot products and updates take up to kMaxVec basis vectors per pass so that
// the vector they are applied to is read once per pass, and the dot products reduce in a
// fixed order (per-CTA partial sums, then one ordered sum per output).
#include "hz_convert.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int NT = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

unsigned grid_for(long long n) {
  const long long g = (n + NT - 1) / NT;
  return (unsigned)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}
// per-RHS kernels: grid (x, R), blockIdx.y = RHS, grid-stride over its n values
dim3 grid_rhs(long long n, int R) {
  const long long g = (n + NT - 1) / NT;
  return dim3((unsigned)(g < 1024 ? (g > 0 ? g : 1) : 1024), (unsigned)R);
}

// out[r][n] = d[n] * v[r][n]
__global__ void pert_mul_kernel(const double2* __restrict__ d, const double2* __restrict__ v,
                                double2* __restrict__ out, long long n) {
  const long long off = (long long)blockIdx.y * n;
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT)
    out[off + t] = cmul(d[t], v[off + t]);
}

// out = a - b + c (b or c may be NULL)
__global__ void lin3_kernel(const double2* __restrict__ a, const double2* __restrict__ b,
                            const double2* __restrict__ c, double2* __restrict__ out, long long total) {
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < total; t += (long long)gridDim.x * NT) {
    double2 x = a[t];
    if (b) {
      const double2 y = b[t];
      x.x -= y.x;
      x.y -= y.y;
    }
    if (c) {
      const double2 z = c[t];
      x.x += z.x;
      x.y += z.y;
    }
    out[t] = x;
  }
}

// out[r][n] = s[r] * w[r][n]
__global__ void scale_kernel(const double2* __restrict__ s, const double2* __restrict__ w,
                             double2* __restrict__ out, long long n) {
  const long long off = (long long)blockIdx.y * n;
  const double2 sr = s[blockIdx.y];
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT)
    out[off + t] = cmul(sr, w[off + t]);
}

// partial[(blockIdx.y * gridDim.x + blockIdx.x) * CNT + i] = sum over this CTA's slice of
// conj(V_i[r][.]) w[r][.], r = blockIdx.y, V_i = V + i * vstride.  CNT is a compile-time
// count: with a run-time count the predicated-off FP64 arithmetic of the unrolled loop
// still issues, and FP64 is the bound here (4 FMA per complex element and vector).
template <int CNT>
__global__ void __launch_bounds__(NT) multi_dot_kernel(const double2* __restrict__ V, long long vstride,
                                                       const double2* __restrict__ w, long long n,
                                                       double2* __restrict__ partial) {
  __shared__ double2 sh[NT / 32][CNT];
  const int r = blockIdx.y;
  const long long off = (long long)r * n;
  double2 acc[CNT];
#pragma unroll
  for (int i = 0; i < CNT; ++i) acc[i] = make_double2(0.0, 0.0);
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT) {
    const double2 x = w[off + t];
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const double2 v = V[i * vstride + off + t];
      acc[i].x = fma(v.x, x.x, fma(v.y, x.y, acc[i].x));       // conj(v) * x
      acc[i].y = fma(v.x, x.y, fma(-v.y, x.x, acc[i].y));
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    double2 a = acc[i];
    for (int o = 16; o > 0; o >>= 1) {
      a.x += __shfl_down_sync(0xffffffffu, a.x, o);
      a.y += __shfl_down_sync(0xffffffffu, a.y, o);
    }
    if (lane == 0) sh[wid][i] = a;
  }
  __syncthreads();
  if (threadIdx.x < CNT) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < NT / 32; ++q) {
      s.x += sh[q][threadIdx.x].x;
      s.y += sh[q][threadIdx.x].y;
    }
    partial[((long long)blockIdx.y * gridDim.x + blockIdx.x) * CNT + threadIdx.x] = s;
  }
}

// out[r * cnt + i] = sum_p partial[(r * parts + p) * cnt + i]: one warp per output, lane l
// sums p = l, l + 32, ..., then a shuffle tree (fixed order)
__global__ void dot_finish_kernel(const double2* __restrict__ partial, int parts, int cnt,
                                  double2* __restrict__ out) {
  const int t = blockIdx.x;                                 // = r * cnt + i
  const int r = t / cnt, i = t - r * cnt;
  const int lane = threadIdx.x;
  double2 s = make_double2(0.0, 0.0);
  for (int p = lane; p < parts; p += 32) {
    const double2 v = partial[((long long)r * parts + p) * cnt + i];
    s.x += v.x;
    s.y += v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_down_sync(0xffffffffu, s.x, o);
    s.y += __shfl_down_sync(0xffffffffu, s.y, o);
  }
  if (lane == 0) out[t] = s;
}

// w[r][n] -= sum_{i < CNT} c[r * CNT + i] V_i[r][n]  (compile-time CNT, as multi_dot)
template <int CNT>
__global__ void __launch_bounds__(NT) multi_axpy_kernel(const double2* __restrict__ V, long long vstride,
                                                        const double2* __restrict__ c, double2* __restrict__ w,
                                                        long long n) {
  const int r = blockIdx.y;
  const long long off = (long long)r * n;
  double2 cr[CNT];
#pragma unroll
  for (int i = 0; i < CNT; ++i) cr[i] = c[r * CNT + i];
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT) {
    double2 x = w[off + t];
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const double2 v = V[i * vstride + off + t];
      x.x = fma(-cr[i].x, v.x, fma(cr[i].y, v.y, x.x));
      x.y = fma(-cr[i].x, v.y, fma(-cr[i].y, v.x, x.y));
    }
    w[off + t] = x;
  }
}

// ---- FP32 Krylov basis (mixed plans): the basis is stored and combined in FP32, the
// vector it is applied to stays FP64 (converted with integer operations, no FP64 work) ----

// out[r][n] = d[n] * v[r][n], v FP32
__global__ void pert_mul32_kernel(const double2* __restrict__ d, const float2* __restrict__ v,
                                  double2* __restrict__ out, long long n) {
  const long long off = (long long)blockIdx.y * n;
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT)
    out[off + t] = cmul(d[t], to_c128(v[off + t]));
}

// out32[r][n] = s[r] * w[r][n] rounded to FP32
__global__ void scale32_kernel(const double2* __restrict__ s, const double2* __restrict__ w,
                               float2* __restrict__ out, long long n) {
  const long long off = (long long)blockIdx.y * n;
  const float2 sr = to_c64t(s[blockIdx.y]);
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT) {
    const float2 x = to_c64t(w[off + t]);
    out[off + t] = make_float2(fmaf(sr.x, x.x, -sr.y * x.y), fmaf(sr.x, x.y, sr.y * x.x));
  }
}

template <int CNT>
__global__ void __launch_bounds__(NT) multi_dot32_kernel(const float2* __restrict__ V, long long vstride,
                                                         const double2* __restrict__ w, long long n,
                                                         double2* __restrict__ partial) {
  __shared__ double2 sh[NT / 32][CNT];
  const int r = blockIdx.y;
  const long long off = (long long)r * n;
  float2 acc[CNT];
#pragma unroll
  for (int i = 0; i < CNT; ++i) acc[i] = make_float2(0.f, 0.f);
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT) {
    const float2 x = to_c64t(w[off + t]);
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const float2 v = V[i * vstride + off + t];
      acc[i].x = fmaf(v.x, x.x, fmaf(v.y, x.y, acc[i].x));       // conj(v) * x
      acc[i].y = fmaf(v.x, x.y, fmaf(-v.y, x.x, acc[i].y));
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    double2 a = to_c128(acc[i]);                           // the reduction across threads in FP64
    for (int o = 16; o > 0; o >>= 1) {
      a.x += __shfl_down_sync(0xffffffffu, a.x, o);
      a.y += __shfl_down_sync(0xffffffffu, a.y, o);
    }
    if (lane == 0) sh[wid][i] = a;
  }
  __syncthreads();
  if (threadIdx.x < CNT) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < NT / 32; ++q) {
      s.x += sh[q][threadIdx.x].x;
      s.y += sh[q][threadIdx.x].y;
    }
    partial[((long long)blockIdx.y * gridDim.x + blockIdx.x) * CNT + threadIdx.x] = s;
  }
}

// w[r][n] -= sum_{i < CNT} c[r * CNT + i] V_i[r][n]: the sum in FP32, the update in FP64
template <int CNT>
__global__ void __launch_bounds__(NT) multi_axpy32_kernel(const float2* __restrict__ V, long long vstride,
                                                          const double2* __restrict__ c, double2* __restrict__ w,
                                                          long long n) {
  const int r = blockIdx.y;
  const long long off = (long long)r * n;
  float2 cr[CNT];
#pragma unroll
  for (int i = 0; i < CNT; ++i) cr[i] = to_c64t(c[r * CNT + i]);
  for (long long t = blockIdx.x * (long long)NT + threadIdx.x; t < n; t += (long long)gridDim.x * NT) {
    float2 sum = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < CNT; ++i) {
      const float2 v = V[i * vstride + off + t];
      sum.x = fmaf(cr[i].x, v.x, fmaf(-cr[i].y, v.y, sum.x));
      sum.y = fmaf(cr[i].x, v.y, fmaf(cr[i].y, v.x, sum.y));
    }
    const double2 sd = to_c128(sum);
    double2 x = w[off + t];
    x.x -= sd.x;
    x.y -= sd.y;
    w[off + t] = x;
  }
}

// s[r] = 1 / sqrt(Re d[r]) (0 where that is not positive): the scale that normalises a
// vector from its <w, w>
__global__ void inv_norm_kernel(const double2* __restrict__ d, double2* __restrict__ s, int R) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) s[r] = make_double2(d[r].x > 0.0 ? 1.0 / sqrt(d[r].x) : 0.0, 0.0);
}

}  // namespace

void vec_inv_norm(const double2* d, double2* s, int R, cudaStream_t st) {
  inv_norm_kernel<<<(R + 127) / 128, 128, 0, st>>>(d, s, R);
  count_launch();
}

void pert_mul(const double2* d, const double2* v, double2* out, long long n, int R, cudaStream_t st) {
  pert_mul_kernel<<<grid_rhs(n, R), NT, 0, st>>>(d, v, out, n);
  count_launch();
}

void vec_lin3(const double2* a, const double2* b, const double2* c, double2* out, long long total,
              cudaStream_t st) {
  lin3_kernel<<<grid_for(total), NT, 0, st>>>(a, b, c, out, total);
  count_launch();
}

void vec_scale(const double2* s, const double2* w, double2* out, long long n, int R, cudaStream_t st) {
  scale_kernel<<<grid_rhs(n, R), NT, 0, st>>>(s, w, out, n);
  count_launch();
}

int multi_dot_parts(long long n) {
  const long long g = (n + NT - 1) / NT;
  return (int)(g < 512 ? (g > 0 ? g : 1) : 512);
}

void pert_mul(const double2* d, const float2* v, double2* out, long long n, int R, cudaStream_t st) {
  pert_mul32_kernel<<<grid_rhs(n, R), NT, 0, st>>>(d, v, out, n);
  count_launch();
}

void vec_scale(const double2* s, const double2* w, float2* out, long long n, int R, cudaStream_t st) {
  scale32_kernel<<<grid_rhs(n, R), NT, 0, st>>>(s, w, out, n);
  count_launch();
}

template <int CNT>
void multi_dot_t(const double2* V, long long vstride, const double2* w, long long n, int R, double2* partial,
                 double2* out, cudaStream_t st) {
  const int parts = multi_dot_parts(n);
  multi_dot_kernel<CNT><<<dim3(parts, R), NT, 0, st>>>(V, vstride, w, n, partial);
  dot_finish_kernel<<<R * CNT, 32, 0, st>>>(partial, parts, CNT, out);
  count_launch(2);
}
template <int CNT>
void multi_axpy_t(const double2* V, long long vstride, const double2* c, double2* w, long long n, int R,
                  cudaStream_t st) {
  multi_axpy_kernel<CNT><<<grid_rhs(n, R), NT, 0, st>>>(V, vstride, c, w, n);
  count_launch();
}

// run-time count -> the compile-time instantiation
template <template <int> class Op, int C = 1>
struct CountDispatch {
  template <typename... A>
  static void run(int cnt, A... a) {
    if (cnt == C) Op<C>::go(a...);
    else CountDispatch<Op, C + 1>::run(cnt, a...);
  }
};
template <template <int> class Op>
struct CountDispatch<Op, kMaxVec + 1> {
  template <typename... A>
  static void run(int, A...) {}
};
template <int CNT>
void multi_dot32_t(const float2* V, long long vstride, const double2* w, long long n, int R, double2* partial,
                   double2* out, cudaStream_t st) {
  const int parts = multi_dot_parts(n);
  multi_dot32_kernel<CNT><<<dim3(parts, R), NT, 0, st>>>(V, vstride, w, n, partial);
  dot_finish_kernel<<<R * CNT, 32, 0, st>>>(partial, parts, CNT, out);
  count_launch(2);
}
template <int CNT>
void multi_axpy32_t(const float2* V, long long vstride, const double2* c, double2* w, long long n, int R,
                    cudaStream_t st) {
  multi_axpy32_kernel<CNT><<<grid_rhs(n, R), NT, 0, st>>>(V, vstride, c, w, n);
  count_launch();
}
template <int C>
struct Dot32Op {
  static void go(const float2* V, long long vs, const double2* w, long long n, int R, double2* p, double2* o,
                 cudaStream_t st) {
    multi_dot32_t<C>(V, vs, w, n, R, p, o, st);
  }
};
template <int C>
struct Axpy32Op {
  static void go(const float2* V, long long vs, const double2* c, double2* w, long long n, int R,
                 cudaStream_t st) {
    multi_axpy32_t<C>(V, vs, c, w, n, R, st);
  }
};

template <int C>
struct DotOp {
  static void go(const double2* V, long long vs, const double2* w, long long n, int R, double2* p, double2* o,
                 cudaStream_t st) {
    multi_dot_t<C>(V, vs, w, n, R, p, o, st);
  }
};
template <int C>
struct AxpyOp {
  static void go(const double2* V, long long vs, const double2* c, double2* w, long long n, int R,
                 cudaStream_t st) {
    multi_axpy_t<C>(V, vs, c, w, n, R, st);
  }
};

void multi_dot(const double2* V, long long vstride, int cnt, const double2* w, long long n, int R,
               double2* partial, double2* out, cudaStream_t st) {
  if (cnt < 1 || cnt > kMaxVec) return;
  CountDispatch<DotOp>::run(cnt, V, vstride, w, n, R, partial, out, st);
}

void multi_axpy(const double2* V, long long vstride, int cnt, const double2* c, double2* w, long long n, int R,
                cudaStream_t st) {
  if (cnt < 1 || cnt > kMaxVec) return;
  CountDispatch<AxpyOp>::run(cnt, V, vstride, c, w, n, R, st);
}

void multi_dot(const float2* V, long long vstride, int cnt, const double2* w, long long n, int R,
               double2* partial, double2* out, cudaStream_t st) {
  if (cnt < 1 || cnt > kMaxVec) return;
  CountDispatch<Dot32Op>::run(cnt, V, vstride, w, n, R, partial, out, st);
}

void multi_axpy(const float2* V, long long vstride, int cnt, const double2* c, double2* w, long long n, int R,
                cudaStream_t st) {
  if (cnt < 1 || cnt > kMaxVec) return;
  CountDispatch<Axpy32Op>::run(cnt, V, vstride, c, w, n, R, st);
}

}  // namespace hz
