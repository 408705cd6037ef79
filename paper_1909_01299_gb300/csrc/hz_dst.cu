// Fast sine transforms of uniform blocks on the FP64 path (steps 1 and 7 of Sec. 2).
//
// A block whose steps are all equal to h has the discrete sine eigenvectors, so its
// forward table (M W) and inverse table (W) are both a scaled DST-I,
//     X_m = S sum_{j=1}^{n} x_j sin(pi j m / N),   N = n + 1,
// which the paper's cost estimate for a uniform survey core (Sec. 2) computes with an FFT
// instead of a dense product.  Here each row of a block is transformed through one complex
// FFT of length N, valid for complex data because the transform has real coefficients:
//   pre:   y_0 = 0,  y_j = p_j x_j + q_j x_{N-j}  (j = 1..N-1),
//          p_j = (S/2)(sin(pi j / N) + 1/2),  q_j = (S/2)(sin(pi j / N) - 1/2);
//   FFT:   Y_k = sum_j y_j exp(-2 pi i j k / N);
//   post:  X_1 = Y_0,  X_{2k} = i (Y_k - Y_{N-k}),  X_{2k+1} = X_{2k-1} + Y_k + Y_{N-k}.
// (The symmetric part of y picks out sin(pi j / N) (x_j + x_{N-j}), whose cosine sums give
// X_{2k+1} - X_{2k-1}; the antisymmetric part gives the sine sums X_{2k}.)  With FP64 as
// scarce as it is on this GPU (2 DFMA per SM per clock), the count that matters is FP64
// instructions per transformed value: about 4 (pre) + 20-27 (FFT, N = 80 or 81) + 3 (post)
// against n for the folded dense product.
//
// The FFT is the iterative mixed-radix decimation in frequency: the pre step writes y_j in
// natural order (consecutive lanes on consecutive positions, free of bank conflicts), stage s
// (radix r, sub-transforms of length L = N / (r_1 .. r_{s-1})) applies an r-point DFT and
// multiplies output q by exp(-2 pi i j1 q / L), and Y_k ends at the digit-reversed position
// pos[k].  The post step runs in place: X_{2k} replaces Y_k and X_{2k+1} replaces Y_{N-k}
// (X_1 = Y_0 stays at 0), and the store gathers the columns from those positions.
//
// Kernel layout: one CTA takes 32 rows of one block; the rows are staged in shared memory
// (odd row stride in 16-byte units, so that threads on different rows hit distinct banks);
// the load, the pre step and the store are shared by all threads with consecutive columns
// (coalesced); four lanes of a warp then run the FFT stages and the post step of each row
// (the post step's running sum as a four-lane scan).  About 43 KB of shared memory per CTA
// keeps five CTAs (20 warps) on an SM, enough to keep the FP64 pipe busy while other CTAs
// load or store.
#include <algorithm>
#include <cmath>

#include "hz_convert.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

// Complex helpers over V = double2 (FP64 path) or float2 (mixed path), scalar type S.
template <typename V> struct Scalar;
template <> struct Scalar<double2> { using T = double; };
template <> struct Scalar<float2> { using T = float; };
template <typename V>
__host__ __device__ __forceinline__ V mk(typename Scalar<V>::T x, typename Scalar<V>::T y) {
  V r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
// a * w (4 operations)
template <typename V> __host__ __device__ __forceinline__ V cmulw(V a, V w) {
  return mk<V>(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}

// r-point DFTs (exp(-2 pi i q q' / r)) of a[0..r-1], in place.
template <typename V> __host__ __device__ __forceinline__ void dft2(V* a) {
  const V t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <typename V> __host__ __device__ __forceinline__ void dft3(V* a) {
  using S = typename Scalar<V>::T;
  const S c = (S)0.86602540378443864676;            // sin(2 pi / 3)
  const S h = (S)-0.5;
  const V s = cadd(a[1], a[2]);
  const V d = csub(a[1], a[2]);
  const V m = mk<V>(fma(h, s.x, a[0].x), fma(h, s.y, a[0].y));
  a[0] = cadd(a[0], s);
  // X1 = m - i c d, X2 = m + i c d
  a[1] = mk<V>(fma(c, d.y, m.x), fma(-c, d.x, m.y));
  a[2] = mk<V>(fma(-c, d.y, m.x), fma(c, d.x, m.y));
}

template <typename V> __host__ __device__ __forceinline__ void dft4(V* a) {
  const V t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  const V t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = mk<V>(t1.x + t3.y, t1.y - t3.x);              // t1 - i t3
  a[3] = mk<V>(t1.x - t3.y, t1.y + t3.x);              // t1 + i t3
}

template <typename V> __host__ __device__ __forceinline__ void dft5(V* a) {
  using S = typename Scalar<V>::T;
  const S c1 = (S)0.30901699437494742410, c2 = (S)-0.80901699437494742410;  // cos(2 pi / 5), cos(4 pi / 5)
  const S s1 = (S)0.95105651629515357212, s2 = (S)0.58778525229247312917;   // sin(2 pi / 5), sin(4 pi / 5)
  const V a1 = cadd(a[1], a[4]), a2 = cadd(a[2], a[3]);
  const V b1 = csub(a[1], a[4]), b2 = csub(a[2], a[3]);
  const V x0 = a[0];
  const V m1 = mk<V>(fma(c2, a2.x, fma(c1, a1.x, x0.x)), fma(c2, a2.y, fma(c1, a1.y, x0.y)));
  const V m2 = mk<V>(fma(c1, a2.x, fma(c2, a1.x, x0.x)), fma(c1, a2.y, fma(c2, a1.y, x0.y)));
  const V n1 = mk<V>(fma(s2, b2.x, s1 * b1.x), fma(s2, b2.y, s1 * b1.y));
  const V n2 = mk<V>(fma(-s1, b2.x, s2 * b1.x), fma(-s1, b2.y, s2 * b1.y));
  a[0] = cadd(cadd(x0, a1), a2);
  a[1] = mk<V>(m1.x + n1.y, m1.y - n1.x);              // m1 - i n1
  a[4] = mk<V>(m1.x - n1.y, m1.y + n1.x);              // m1 + i n1
  a[2] = mk<V>(m2.x + n2.y, m2.y - n2.x);              // m2 - i n2
  a[3] = mk<V>(m2.x - n2.y, m2.y + n2.x);              // m2 + i n2
}

// y_j and y_{N-j} from x_j and x_{N-j} (equal when 2 j = N).
template <typename V, typename S>
__host__ __device__ __forceinline__ void pre_pair(V xj, V xm, S p, S q, V* yj, V* ym) {
  *yj = mk<V>(fma(p, xj.x, q * xm.x), fma(p, xj.y, q * xm.y));
  *ym = mk<V>(fma(p, xm.x, q * xj.x), fma(p, xm.y, q * xj.y));
}

constexpr int kTM = 32;      // rows per CTA
constexpr int kTPR = 4;      // threads per row in the FFT and post phases (lanes 4r..4r+3 of a warp)
constexpr int kNT = kTM * kTPR;

// Odd row stride (16-byte units) for rows of N values: threads of a warp on different rows
// then address distinct shared-memory banks.
__host__ __device__ __forceinline__ int row_stride(int N) { return N | 1; }


// Mode m of column c in the symmetric-modes-first order of a uniform block (and back).
int sym_mode(int c, int n) {
  const int ns = (n + 1) / 2;
  return c < ns ? 2 * c + 1 : 2 * (c - ns) + 2;
}
int sym_col(int m, int n) {
  const int ns = (n + 1) / 2;
  return (m % 2 == 1) ? (m - 1) / 2 : ns + m / 2 - 1;
}

// One radix-R decimation-in-frequency stage of a row shared by its kTPR threads (sub =
// 0..kTPR-1), butterflies sub, sub + kTPR, ...: sub-transforms of length L, M = L / R; element q
// of butterfly (b, j1) is x[b L + j1 + q M]; after the R-point DFT output q is multiplied by
// exp(-2 pi i j1 q / L) (tw[j1][q-1]; none for j1 = 0).  The caller synchronises the row's lanes
// after the stage; the host reference calls it for every sub in turn.
template <int R, typename V>
__host__ __device__ __forceinline__ void fft_stage_par(V* x, int N, int L, const V* tw, int sub) {
  const int M = L / R;
  const int nb = N / R;
  // FP32: lane sub takes the contiguous butterflies [t0, t1) (neighbouring lanes a chunk apart,
  // spread over the shared-memory banks, indices stepped without division); FP64 (bound by
  // the FP64 pipe, where this measured slower): butterflies sub, sub + kTPR, ...
  constexpr bool CONTIG = sizeof(V) == 8;
  const int chunk = CONTIG ? (nb + kTPR - 1) / kTPR : 1;
  const int t0 = sub * chunk, t1 = CONTIG ? (t0 + chunk < nb ? t0 + chunk : nb) : nb;
  const int step = CONTIG ? 1 : kTPR;
  int blk = t0 / M, j1 = t0 - (t0 / M) * M;
  for (int t = t0; t < t1; t += step) {
    if (!CONTIG) {
      blk = t / M;
      j1 = t - blk * M;
    }
    V a[R];
    V* p = x + blk * L + j1;
#pragma unroll
    for (int q = 0; q < R; ++q) a[q] = p[q * M];
    if (R == 2) dft2(a);
    else if (R == 3) dft3(a);
    else if (R == 4) dft4(a);
    else dft5(a);
    if (tw && j1 > 0) {                              // no table: a prime-factor stage
#pragma unroll
      for (int q = 1; q < R; ++q) a[q] = cmulw(a[q], tw[j1 * (R - 1) + q - 1]);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) p[q * M] = a[q];
    if (CONTIG && ++j1 == M) {
      j1 = 0;
      ++blk;
    }
  }
}

template <typename V>
__host__ __device__ __forceinline__ void fft_stage_any(V* x, int N, int L, int r, const V* tw, int sub) {
  switch (r) {
    case 2: fft_stage_par<2>(x, N, L, tw, sub); break;
    case 3: fft_stage_par<3>(x, N, L, tw, sub); break;
    case 4: fft_stage_par<4>(x, N, L, tw, sub); break;
    default: fft_stage_par<5>(x, N, L, tw, sub); break;
  }
}

// The post step, shared by the kTPR threads of a row: each takes a contiguous range of pairs
// k; part A writes X_{2k} = i (Y_k - Y_{N-k}) in place of Y_k and the pair sum in place of
// Y_{N-k} and returns the range's total; part B adds the running sum (Y_0 + the totals of the
// lower ranges, excl) in place.  pos[k]: where the FFT left Y_k (digit-reversed order).
__host__ __device__ __forceinline__ void post_range(int N, int sub, int* k0, int* k1) {
  const int K = (N - 1) / 2;
  const int chunk = (K + kTPR - 1) / kTPR;
  *k0 = 1 + sub * chunk;
  *k1 = K < *k0 + chunk - 1 ? K : *k0 + chunk - 1;
}
template <typename V>
__host__ __device__ __forceinline__ V post_part_a(V* x, const int* pos, int N, int sub) {
  int k0, k1;
  post_range(N, sub, &k0, &k1);
  V part = mk<V>(0, 0);
  for (int k = k0; k <= k1; ++k) {
    const int pk = pos[k], pm = pos[N - k];
    const V yk = x[pk], ym = x[pm];
    const V sk = cadd(yk, ym);
    part = cadd(part, sk);
    x[pk] = mk<V>(ym.y - yk.y, yk.x - ym.x);
    x[pm] = sk;
  }
  return part;
}
template <typename V>
__host__ __device__ __forceinline__ void post_part_b(V* x, const int* pos, int N, int sub, V excl) {
  int k0, k1;
  post_range(N, sub, &k0, &k1);
  V acc = cadd(x[0], excl);                        // Y_0 sits at position 0
  for (int k = k0; k <= k1; ++k) {
    const int pm = pos[N - k];
    acc = cadd(acc, x[pm]);
    x[pm] = acc;
  }
}

template <typename V>
__device__ __forceinline__ void fft_row_par(V* x, const DstBlock& b, const V* tw, int sub) {
  const int N = b.n + 1;
  int L = N, off = 0;
  for (int s = 0; s < b.nst; ++s) {
    const int r = b.rad[s];
    const bool twiddled = !(b.pfa && s == 0);
    fft_stage_any(x, N, L, r, twiddled ? tw + off : static_cast<const V*>(nullptr), sub);
    __syncwarp();
    if (twiddled) off += (L / r) * (r - 1);
    L /= r;
  }
}

template <typename V>
__device__ __forceinline__ void post_row_par(V* x, const int* pos, int N, int sub) {
  const V part = post_part_a(x, pos, N, sub);
  V excl = mk<V>(0, 0);                              // sum of the lower lanes' parts
  V incl = part;
#pragma unroll
  for (int o = 1; o < kTPR; o <<= 1) {
    const auto ox = __shfl_up_sync(0xffffffffu, incl.x, o, kTPR);
    const auto oy = __shfl_up_sync(0xffffffffu, incl.y, o, kTPR);
    if (sub >= o) {
      incl.x += ox;
      incl.y += oy;
      excl.x += ox;
      excl.y += oy;
    }
  }
  __syncwarp();
  post_part_b(x, pos, N, sub, excl);
}

// Rows per CTA: 32 rows of complex128 or 64 of complex64 fill the same 43 KB.
template <typename V> constexpr int rows_per_cta() { return sizeof(V) == 16 ? 32 : 64; }

// V: arithmetic (double2: FP64 path; float2: mixed path, FP32 arithmetic); TI / TO: input and
// output elements (complex128 or complex64; FP64 <-> FP32 by the integer conversions, which
// keep the FP64 pipe free).  An accumulating store adds to a complex128 output in FP64.
template <typename V, typename TI, typename TO>
__global__ void __launch_bounds__(rows_per_cta<V>() * kTPR)
dst_kernel(const TI* __restrict__ in, TO* __restrict__ out, const DstBlock* __restrict__ blocks,
           const int* __restrict__ idx, const typename Scalar<V>::T* __restrict__ coef, const V* __restrict__ twg,
           int nblk, long long nrows, int rows_per_plane, int ncols, int trans, int store, int conj_out,
           const signed char* __restrict__ rowskip, int stride) {
  constexpr int TM = rows_per_cta<V>(), NT = TM * kTPR;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  __shared__ int s_ok[TM];
  __shared__ long long s_base[TM];          // first output element of the row (trans: the plane slot)
  const int blk = (int)(blockIdx.x % (unsigned)nblk);
  const long long row0 = (long long)(blockIdx.x / (unsigned)nblk) * TM;
  const DstBlock b = blocks[blk];
  const int n = b.n, N = n + 1;
  V* tw = sm + TM * stride;
  for (int t = threadIdx.x; t < b.ntw; t += NT) tw[t] = twg[b.tw_off + t];
  if (threadIdx.x < TM) {
    const long long row = row0 + threadIdx.x;
    int ok = row < nrows;
    long long base = 0;
    if (ok) {
      const long long plane = row / rows_per_plane;
      const int rip = (int)(row - plane * rows_per_plane);
      if (rowskip && rowskip[rip]) ok = 0;
      base = trans ? plane * (long long)ncols * rows_per_plane + rip : row * (long long)ncols;
    }
    s_ok[threadIdx.x] = ok;
    s_base[threadIdx.x] = base;
    sm[threadIdx.x * stride] = mk<V>(0, 0);                 // y_0
  }
  __syncthreads();
  const int* __restrict__ pos = idx + b.ioff;
  const int* __restrict__ gin = pos + N;
  const int* __restrict__ src = gin + N;
  const int* __restrict__ pin = src + n;
  const typename Scalar<V>::T* __restrict__ pq = coef + b.coff;
  // phase 1: load the row pairs (x_j, x_{N-j}) and write y_j, y_{N-j} in natural order (rows
  // that are skipped or past the end transform zeros and are not stored).  FP32: one warp per
  // row at a time, lanes on consecutive j; FP64: all (row, j) pairs spread over the threads.
  const int np = N / 2;
  auto pre_one = [&](int r, int j, bool ok) {
    const TI* rp = in + (row0 + r) * (long long)ncols + b.start;
    V xj = mk<V>(0, 0), xm = xj;
    if (ok) {
      if constexpr (sizeof(V) == 16) {
        xj = to_c128(rp[gin[j]]);
        xm = to_c128(rp[gin[N - j]]);
      } else {
        xj = to_c64t(rp[gin[j]]);
        xm = to_c64t(rp[gin[N - j]]);
      }
    }
    V yj, ym;
    pre_pair(xj, xm, pq[2 * j], pq[2 * j + 1], &yj, &ym);
    V* x = sm + r * stride;
    x[pin[j]] = yj;
    if (N - j != j) x[pin[N - j]] = ym;
  };
  if constexpr (sizeof(V) == 8) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < TM; r += NT / 32) {
      const bool ok = s_ok[r] != 0;
      for (int j = 1 + lane; j <= np; j += 32) pre_one(r, j, ok);
    }
  } else {
#pragma unroll 4
    for (int e = threadIdx.x; e < TM * np; e += NT) {
      const int r = e / np, j = 1 + (e - r * np);
      pre_one(r, j, s_ok[r] != 0);
    }
  }
  __syncthreads();
  // phase 2: FFT and post step, kTPR lanes per row
  {
    V* x = sm + (threadIdx.x / kTPR) * stride;
    const int sub = threadIdx.x % kTPR;
    fft_row_par(x, b, tw, sub);
    post_row_par(x, pos, N, sub);
  }
  __syncthreads();
  // phase 3: store.  Transposed: a warp's lanes take consecutive rows of one column (contiguous
  // in the output, conflict-free in shared memory).  Row-contiguous: lanes take G consecutive
  // columns (64 bytes) of 32 / G rows, so that each row's segment is one or two sectors and the
  // gathers from the scattered positions spread over rows.
  constexpr int G = 64 / (int)sizeof(V);
  const int ncg = (n + G - 1) / G;
  for (int e = threadIdx.x; e < TM * (trans ? n : ncg * G); e += NT) {
    int r, c;
    if (trans) {
      c = e / TM;
      r = e - c * TM;
    } else {
      const int cl = e % G, rest = e / G;
      r = rest % TM;
      c = (rest / TM) * G + cl;
      if (c >= n) continue;
    }
    if (!s_ok[r]) continue;
    V v = sm[r * stride + src[c]];
    if (conj_out) v.y = -v.y;
    TO* p = out + s_base[r] + (long long)(b.start + c) * (trans ? rows_per_plane : 1);
    if constexpr (sizeof(TO) == 16) {
      double2 w = to_c128(v);
      if (store == XS_ACCUM) {
        const double2 o = *p;
        w.x += o.x;
        w.y += o.y;
      }
      *p = w;
    } else {
      *p = to_c64t(v);
    }
  }
}

template <typename V>
size_t dst_smem(int nmax) { return sizeof(V) * ((size_t)rows_per_cta<V>() * row_stride(nmax) + nmax); }

template <typename V, typename TI, typename TO>
void dst_launch(const DstSet& ds, const V* tw, const typename Scalar<V>::T* coef, const TI* in, TO* out,
                int rows_per_plane, long long nplanes, int ncols, int trans, int store, int conj_out,
                const signed char* rowskip, cudaStream_t st) {
  const long long nrows = nplanes * (long long)rows_per_plane;
  if (nrows <= 0 || ds.nblk == 0) return;
  constexpr int TM = rows_per_cta<V>();
  const long long ctas = ((nrows + TM - 1) / TM) * ds.nblk;
  dst_kernel<V, TI, TO><<<(unsigned)ctas, TM * kTPR, dst_smem<V>(ds.nmax), st>>>(
      in, out, ds.d_blk, ds.d_idx, coef, tw, ds.nblk, nrows, rows_per_plane, ncols, trans, store, conj_out,
      rowskip, row_stride(ds.nmax));
  count_launch();
}

template <typename V, typename TI, typename TO>
void set_attr(int nmax) {
  cudaFuncSetAttribute(dst_kernel<V, TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dst_smem<V>(nmax));
}

}  // namespace

void dst_prepare(int nmax) {
  set_attr<double2, double2, double2>(nmax);
  set_attr<float2, double2, float2>(nmax);
  set_attr<float2, float2, float2>(nmax);
  set_attr<float2, float2, double2>(nmax);
}

void dst_f64(const DstSet& ds, const double2* in, double2* out, int rows_per_plane, long long nplanes, int ncols,
             int trans, int store, int conj_out, const signed char* rowskip, cudaStream_t st) {
  dst_launch<double2>(ds, ds.d_tw, ds.d_coef, in, out, rows_per_plane, nplanes, ncols, trans, store, conj_out,
                      rowskip, st);
}

bool dst_f32(const DstSet& ds, const void* in, int in32, void* out, int out32, int rows_per_plane, long long nplanes,
             int ncols, int trans, int store, const signed char* rowskip, cudaStream_t st) {
  if (!ds.d_tw32 || (out32 && store != XS_STORE)) return false;
  if (in32 && out32)
    dst_launch<float2>(ds, ds.d_tw32, ds.d_coef32, static_cast<const float2*>(in), static_cast<float2*>(out),
                       rows_per_plane, nplanes, ncols, trans, store, 0, rowskip, st);
  else if (in32)
    dst_launch<float2>(ds, ds.d_tw32, ds.d_coef32, static_cast<const float2*>(in), static_cast<double2*>(out),
                       rows_per_plane, nplanes, ncols, trans, store, 0, rowskip, st);
  else if (out32)
    dst_launch<float2>(ds, ds.d_tw32, ds.d_coef32, static_cast<const double2*>(in), static_cast<float2*>(out),
                       rows_per_plane, nplanes, ncols, trans, store, 0, rowskip, st);
  else
    return false;
  return true;
}

bool dst_supported(int n) {
  int N = n + 1;
  if (n < 2 || N > kDstMaxN) return false;
  for (int r : {2, 3, 5})
    while (N % r == 0) N /= r;
  return N == 1;
}

bool dst_plan_block(int n, int start, int dir, double S, std::vector<DstBlock>& blk, std::vector<int>& idx,
                    std::vector<double>& coef, std::vector<double2>& tw) {
  const int N = n + 1;
  if (n < 2 || N > kDstMaxN || (dir != 1 && dir != 2)) return false;
  DstBlock b{};
  b.start = start;
  b.n = n;
  // prime-factor split N = m N1 (m = 3 or 5, N1 = 2^a >= 4): the radix-m stage first, without
  // twiddles, then the radix-4/2 stages of the length-N1 transforms
  int N1 = N, pm = 1;
  while (N1 % 2 == 0) N1 /= 2;
  if ((N1 == 3 || N1 == 5) && N / N1 >= 4) {
    pm = N1;
    N1 = N / pm;
    b.pfa = 1;
    b.rad[b.nst++] = pm;
  } else {
    N1 = N;
  }
  int m = N1;
  for (int r : {4, 3, 5, 2}) {
    while (m % r == 0) {
      if (b.nst == kDstMaxStages) return false;
      b.rad[b.nst++] = r;
      m /= r;
    }
  }
  if (m != 1) return false;
  const double pi = 3.14159265358979323846;
  // stage twiddles exp(-2 pi i j1 q / L), j1 = 0..L/r-1, q = 1..r-1 (argument reduced exactly),
  // sub-transform length L = N, N / r_1, ... (a prime-factor first stage has none)
  b.tw_off = (long long)tw.size();
  int L = N;
  for (int s = 0; s < b.nst; ++s) {
    const int r = b.rad[s], M = L / r;
    if (!(b.pfa && s == 0))
      for (int j1 = 0; j1 < M; ++j1)
        for (int q = 1; q < r; ++q) {
          const int e = (j1 * q) % L;
          const double th = -2.0 * pi * e / L;
          tw.push_back(make_double2(std::cos(th), std::sin(th)));
        }
    L = M;
  }
  b.ntw = (int)(tw.size() - b.tw_off);
  // pos[N]: where the FFT leaves Y_k: the digits of k (radix r_1 first, weighted N / r_1, ...)
  // of the mixed-radix transform, or with the prime-factor split N1 (k mod m) + the digits of
  // k mod N1 within the length-N1 transform; gin[N]: column of input index j (1..n); src[n]:
  // position holding output column c; pin[N]: position of y_j (the identity without the split)
  b.ioff = (long long)idx.size();
  std::vector<int> pos(N), pin(N);
  const int s0 = b.pfa ? 1 : 0;
  for (int k = 0; k < N; ++k) {
    int kk = b.pfa ? k % N1 : k, p = 0, Ls = N1;
    for (int s = s0; s < b.nst; ++s) {
      Ls /= b.rad[s];
      p += (kk % b.rad[s]) * Ls;
      kk /= b.rad[s];
    }
    pos[k] = b.pfa ? N1 * (k % pm) + p : p;
  }
  for (int j = 0; j < N; ++j) pin[j] = j;
  if (b.pfa)
    for (int n1 = 0; n1 < N1; ++n1)
      for (int n2 = 0; n2 < pm; ++n2) pin[(pm * n1 + N1 * n2) % N] = n1 + N1 * n2;
  for (int k = 0; k < N; ++k) idx.push_back(pos[k]);
  for (int j = 0; j < N; ++j) idx.push_back(j == 0 ? 0 : (dir == 1 ? j - 1 : sym_col(j, n)));
  for (int c = 0; c < n; ++c) {
    const int m = dir == 1 ? sym_mode(c, n) : c + 1;
    idx.push_back(pos[m == 1 ? 0 : (m % 2 == 0 ? m / 2 : N - (m - 1) / 2)]);
  }
  for (int j = 0; j < N; ++j) idx.push_back(pin[j]);
  b.coff = (long long)coef.size();
  for (int j = 0; j <= N / 2; ++j) {
    const double sj = std::sin(pi * j / N);
    coef.push_back(0.5 * S * (sj + 0.5));
    coef.push_back(0.5 * S * (sj - 0.5));
  }
  blk.push_back(b);
  return true;
}

bool dst_apply_host(int n, int dir, double S, const double2* in, double2* out) {
  std::vector<DstBlock> blk;
  std::vector<int> idx;
  std::vector<double> coef;
  std::vector<double2> tw;
  if (!dst_plan_block(n, 0, dir, S, blk, idx, coef, tw)) return false;
  const DstBlock& b = blk[0];
  const int N = n + 1;
  const int* pos = idx.data() + b.ioff;
  const int* gin = pos + N;
  const int* src = gin + N;
  const int* pin = src + n;
  std::vector<double2> x(N);
  x[0] = make_double2(0.0, 0.0);
  for (int j = 1; 2 * j <= N; ++j) {
    double2 yj, ym;
    pre_pair(in[gin[j]], in[gin[N - j]], coef[b.coff + 2 * j], coef[b.coff + 2 * j + 1], &yj, &ym);
    x[pin[j]] = yj;
    if (N - j != j) x[pin[N - j]] = ym;
  }
  // the kernel's per-lane code, the lanes of a row taken in turn
  int L = N, off = 0;
  for (int st = 0; st < b.nst; ++st) {
    const bool twiddled = !(b.pfa && st == 0);
    for (int sub = 0; sub < kTPR; ++sub)
      fft_stage_any(x.data(), N, L, b.rad[st], twiddled ? tw.data() + b.tw_off + off : nullptr, sub);
    if (twiddled) off += (L / b.rad[st]) * (b.rad[st] - 1);
    L /= b.rad[st];
  }
  double2 part[kTPR];
  for (int sub = 0; sub < kTPR; ++sub) part[sub] = post_part_a(x.data(), pos, N, sub);
  double2 excl = make_double2(0.0, 0.0);
  for (int sub = 0; sub < kTPR; ++sub) {
    post_part_b(x.data(), pos, N, sub, excl);
    excl = cadd(excl, part[sub]);
  }
  for (int c = 0; c < n; ++c) out[c] = x[src[c]];
  return true;
}

}  // namespace hz
