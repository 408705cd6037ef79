// Block-diagonal row transforms on CUDA cores (steps 1, 3, 5, 6, 7 of Sec. 2).
//
// Every x/y eigen-transform of the method is a product of a row of the data
// (contiguous complex values along the contracted axis) with the block's
// eigenvector matrix: forward W^T M (Eq. (fdmtrprjfr)), inverse W, or the
// global W of Eq. (fdmtrprjfrerr).  A launch processes all rows of all
// planes; one CTA computes a 32 x 32 output tile of one block, staging a
// 32 x 16 data tile and a 16 x 32 table tile in shared memory.
//
// FP64 variant: complex tables use the 3M product (Gauss): for data a = ar + i ai
// and table entry c + i d the table stores (c, d - c, c + d) and
//   Re = sum c (ar + ai) - sum (c + d) ai,   Im = sum c (ar + ai) + sum (d - c) ar,
// three DFMA per complex multiply-add instead of four.  Real tables (blocks whose
// steps are all real) take two DFMA.  FP32 variant (mixed path): the same tiling in
// FFMA with the four-product form on an FP32 copy of the tables.
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int TM = 32, TN = 32, TK = 16, NT = 256;

template <typename Acc, bool REAL>
struct Tile {
  Acc a[(REAL || sizeof(Acc) == 4) ? 2 : 3][TK][TM];
  Acc b[REAL ? 1 : (sizeof(Acc) == 8 ? 3 : 2)][TK][TN];
};

template <typename Acc, bool REAL>
__device__ __forceinline__ void run_tile(const double2* __restrict__ in, double2* __restrict__ out,
                                         const Acc* __restrict__ tab, const XBlock& b, const XTile& t,
                                         int rows_per_plane, int ncols, long long plane, int row0,
                                         int trans, int store, int conj_out,
                                         const signed char* __restrict__ rowskip, char* smem_raw) {
  constexpr bool F64 = sizeof(Acc) == 8;
  constexpr int NB = REAL ? 1 : (F64 ? 3 : 2);
  Tile<Acc, REAL>& sm = *reinterpret_cast<Tile<Acc, REAL>*>(smem_raw);
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int n = b.size;
  const long long plane_base = plane * (long long)rows_per_plane;

  // accumulators: [row r][col c][component]; complex FP64 3M: P1, P2, P3; FP32: re, im
  Acc acc[2][2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[r][c][q] = Acc(0);

  const int la_row = tid >> 3, la_k = (tid & 7) * 2;       // A tile loader
  const int lb_k = tid >> 4, lb_c = (tid & 15) * 2;        // B tile loader
  for (int k0 = 0; k0 < n; k0 += TK) {
    {
      const int row = row0 + la_row;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int kk = la_k + e;
        double2 v = make_double2(0.0, 0.0);
        if (row < rows_per_plane && k0 + kk < n)
          v = in[(plane_base + row) * (long long)ncols + b.start + k0 + kk];
        sm.a[0][kk][la_row] = Acc(v.x);
        sm.a[1][kk][la_row] = Acc(v.y);
        if (!REAL && F64) sm.a[(REAL || !F64) ? 1 : 2][kk][la_row] = Acc(v.x + v.y);
      }
    }
    {
      const int a = k0 + lb_k;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int cc = lb_c + e;
        const bool ok = a < n && cc < t.cw;
#pragma unroll
        for (int p = 0; p < NB; ++p)
          sm.b[p][lb_k][cc] = ok ? tab[(long long)p * n * n + (long long)a * n + t.c0 + cc] : Acc(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      Acc ar[2], ai[2], as[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        ar[r] = sm.a[0][kk][ty + 16 * r];
        ai[r] = sm.a[1][kk][ty + 16 * r];
        if (!REAL && F64) as[r] = sm.a[(REAL || !F64) ? 1 : 2][kk][ty + 16 * r];
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const Acc b0 = sm.b[0][kk][tx + 16 * c];
        if (REAL) {
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            acc[r][c][0] = fma(ar[r], b0, acc[r][c][0]);
            acc[r][c][1] = fma(ai[r], b0, acc[r][c][1]);
          }
        } else if (F64) {
          const Acc b1 = sm.b[NB > 1 ? 1 : 0][kk][tx + 16 * c];
          const Acc b2 = sm.b[NB > 2 ? 2 : 0][kk][tx + 16 * c];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            acc[r][c][0] = fma(b0, as[r], acc[r][c][0]);    // c (ar + ai)
            acc[r][c][1] = fma(b1, ar[r], acc[r][c][1]);    // (d - c) ar
            acc[r][c][2] = fma(b2, ai[r], acc[r][c][2]);    // (c + d) ai
          }
        } else {
          const Acc bi = sm.b[NB > 1 ? 1 : 0][kk][tx + 16 * c];
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            acc[r][c][0] = fma(ar[r], b0, acc[r][c][0]);
            acc[r][c][0] = fma(-ai[r], bi, acc[r][c][0]);
            acc[r][c][1] = fma(ar[r], bi, acc[r][c][1]);
            acc[r][c][1] = fma(ai[r], b0, acc[r][c][1]);
          }
        }
      }
    }
    __syncthreads();
  }

  double2 res[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      double re, im;
      if (REAL || !F64) {
        re = double(acc[r][c][0]);
        im = double(acc[r][c][1]);
      } else {
        re = double(acc[r][c][0]) - double(acc[r][c][2]);
        im = double(acc[r][c][0]) + double(acc[r][c][1]);
      }
      res[r][c] = make_double2(re, conj_out ? -im : im);
    }

  if (!trans) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int row = row0 + ty + 16 * r;
      if (row >= rows_per_plane || (rowskip && rowskip[row])) continue;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = tx + 16 * c;
        if (col >= t.cw) continue;
        double2* p = out + (plane_base + row) * (long long)ncols + b.start + t.c0 + col;
        if (store == XS_ACCUM) {
          double2 o = *p;
          o.x += res[r][c].x;
          o.y += res[r][c].y;
          *p = o;
        } else {
          *p = res[r][c];
        }
      }
    }
  } else {
    // stage the tile and write it transposed: out[plane][col][row], rows contiguous
    double2 (*os)[TM + 1] = reinterpret_cast<double2 (*)[TM + 1]>(smem_raw);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) os[tx + 16 * c][ty + 16 * r] = res[r][c];
    __syncthreads();
    const long long out_plane = plane * (long long)ncols * rows_per_plane;
    const int wr = tid & 31;
#pragma unroll
    for (int pass = 0; pass < TN / 8; ++pass) {
      const int col = (tid >> 5) + 8 * pass;
      const int row = row0 + wr;
      if (col < t.cw && row < rows_per_plane && !(rowskip && rowskip[row])) {
        double2* p = out + out_plane + (long long)(b.start + t.c0 + col) * rows_per_plane + row;
        if (store == XS_ACCUM) {
          double2 o = *p;
          o.x += os[col][wr].x;
          o.y += os[col][wr].y;
          *p = o;
        } else {
          *p = os[col][wr];
        }
      }
    }
  }
}

template <typename Acc>
__global__ void __launch_bounds__(NT)
xform_kernel(const double2* __restrict__ in, double2* __restrict__ out, const Acc* __restrict__ tab,
             const XBlock* __restrict__ blocks, const XTile* __restrict__ tiles, int rows_per_plane,
             int ncols, long long plane0, int trans, int store, int conj_out,
             const signed char* __restrict__ rowskip) {
  constexpr int SA = sizeof(Tile<Acc, false>) > sizeof(double2) * TN * (TM + 1)
                         ? sizeof(Tile<Acc, false>) : sizeof(double2) * TN * (TM + 1);
  __shared__ __align__(16) char smem[SA];
  const XTile t = tiles[blockIdx.z];
  const XBlock b = blocks[t.blk];
  const long long plane = plane0 + blockIdx.y;
  const int row0 = blockIdx.x * TM;
  const Acc* tb = tab + (sizeof(Acc) == 8 ? b.toff : b.toff32);
  if (b.real)
    run_tile<Acc, true>(in, out, tb, b, t, rows_per_plane, ncols, plane, row0, trans, store, conj_out,
                        rowskip, smem);
  else
    run_tile<Acc, false>(in, out, tb, b, t, rows_per_plane, ncols, plane, row0, trans, store, conj_out,
                         rowskip, smem);
}

template <typename Acc>
void launch(const XformSet& xs, const Acc* tab, const double2* in, double2* out, int rows_per_plane,
            long long nplanes, int trans, int store, int conj_out, const signed char* rowskip,
            cudaStream_t st) {
  if (nplanes <= 0 || rows_per_plane <= 0 || xs.ntiles == 0) return;
  const int gx = (rows_per_plane + TM - 1) / TM;
  for (long long p0 = 0; p0 < nplanes; p0 += 65535) {
    const int gy = (int)((nplanes - p0) < 65535 ? (nplanes - p0) : 65535);
    dim3 grid(gx, gy, xs.ntiles);
    xform_kernel<Acc><<<grid, NT, 0, st>>>(in, out, tab, xs.d_blocks, xs.d_tiles, rows_per_plane,
                                          xs.ncols, p0, trans, store, conj_out, rowskip);
    count_launch();
  }
}

}  // namespace

void xform_f64(const XformSet& xs, const double2* in, double2* out, int rows_per_plane,
               long long nplanes, int trans, int store, int conj_out, const signed char* rowskip,
               cudaStream_t st) {
  launch<double>(xs, xs.d_tab, in, out, rows_per_plane, nplanes, trans, store, conj_out, rowskip, st);
}

void xform_f32(const XformSet& xs, const double2* in, double2* out, int rows_per_plane,
               long long nplanes, int trans, int store, int conj_out, const signed char* rowskip,
               cudaStream_t st) {
  launch<float>(xs, xs.d_tab32, in, out, rows_per_plane, nplanes, trans, store, conj_out, rowskip, st);
}

}  // namespace hz
