// Block-diagonal row transforms on CUDA cores (steps 1, 3, 5, 6, 7 of Sec. 2).
//
// Every x/y eigen-transform of the method is a product of a row of the data
// (contiguous complex values along the contracted axis) with the block's
// eigenvector matrix: forward W^T M (Eq. (fdmtrprjfr)), inverse W, or the
// global W of Eq. (fdmtrprjfrerr).  A launch treats the rows of all planes as
// one list; one CTA computes a 64 x 16 output tile of one block (64 rows,
// 16 eigen-columns; 16 x 16 for short launches), staging the data tile and a
// 16 x 16 table tile in shared memory per 16-deep slice of the contraction.  Sixteen-column tiles
// keep the padding waste small for the block widths of layered grids
// (79, 80, 95, 96, 32, ...), where it would otherwise cost idle FMAs.
//
// FP64 variant: complex tables use the 3M product (Gauss): for data a = ar + i ai
// and table entry c + i d the table stores (c, d - c, c + d) and
//   Re = sum c (ar + ai) - sum (c + d) ai,   Im = sum c (ar + ai) + sum (d - c) ar,
// three DFMA per complex multiply-add instead of four.  Real tables (blocks whose
// steps are all real) take two DFMA; uniform blocks (sine eigenvectors) fold or unfold
// the data around the block centre and contract over half the block (run_tile_sym).
// FP32 variant (mixed path): the same tiling in FFMA with the four-product form on an
// FP32 copy of the tables.
#include "hz_convert.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int TN = 16, TK = 16, NT = 256;

// data in and results out: FP32 through the integer conversions (no FP64-pipe work)
template <typename Acc> __device__ __forceinline__ Acc to_acc(double v);
template <> __device__ __forceinline__ double to_acc<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_acc<float>(double v) { return f64_to_f32(v); }
__device__ __forceinline__ double from_acc(double v) { return v; }
__device__ __forceinline__ double from_acc(float v) { return f32_to_f64(v); }
static_assert(TN == 16, "host tiling (kTileN) assumes 16-column tiles");

template <typename Acc, bool REAL, int TM>
struct Tile {
  Acc a[(REAL || sizeof(Acc) == 4) ? 2 : 3][TK][TM];
  Acc b[REAL ? 1 : (sizeof(Acc) == 8 ? 3 : 2)][TK][TN];
};

// TM = 64 rows per CTA (4 per thread) for the bulk transforms; TM = 16 (1 per thread)
// for the short interface-row launches, which would otherwise leave SMs idle.
template <typename Acc, bool REAL, int TM>
__device__ __forceinline__ void run_tile(const double2* __restrict__ in, double2* __restrict__ out,
                                         const Acc* __restrict__ tab, const XBlock& b, const XTile& t,
                                         long long nrows, int rows_per_plane, int ncols, long long row0,
                                         int trans, int store, int conj_out,
                                         const signed char* __restrict__ rowskip, char* smem_raw) {
  constexpr bool F64 = sizeof(Acc) == 8;
  constexpr int NB = REAL ? 1 : (F64 ? 3 : 2);
  constexpr int RPT = TM / 16;                             // rows per thread
  constexpr int EPT = TM * TK / NT;                        // A elements loaded per thread
  Tile<Acc, REAL, TM>& sm = *reinterpret_cast<Tile<Acc, REAL, TM>*>(smem_raw);
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int n = b.size;

  // accumulators: [row r][component]; complex FP64 3M: P1, P2, P3; otherwise re, im
  Acc acc[RPT][3];
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) acc[r][q] = Acc(0);

  const int la_row = tid / (TK / EPT), la_k = (tid % (TK / EPT)) * EPT;   // A loader: EPT consecutive k
  const int lb_k = tid >> 4, lb_c = tid & 15;              // B tile loader
  const long long arow = row0 + la_row;
  const bool arow_ok = arow < nrows;
  const double2* __restrict__ ain = in + arow * (long long)ncols + b.start;
  for (int k0 = 0; k0 < n; k0 += TK) {
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int kk = la_k + e;
      double2 v = make_double2(0.0, 0.0);
      if (arow_ok && k0 + kk < n) v = ain[k0 + kk];
      sm.a[0][kk][la_row] = to_acc<Acc>(v.x);
      sm.a[1][kk][la_row] = to_acc<Acc>(v.y);
      if (!REAL && F64) sm.a[(REAL || !F64) ? 1 : 2][kk][la_row] = Acc(v.x + v.y);
    }
    {
      const int a = k0 + lb_k;
      const bool ok = a < n && lb_c < t.cw;
#pragma unroll
      for (int p = 0; p < NB; ++p)
        sm.b[p][lb_k][lb_c] = ok ? tab[(long long)p * n * n + (long long)a * n + t.c0 + lb_c] : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const Acc b0 = sm.b[0][kk][tx];
      if (REAL) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          acc[r][0] = fma(sm.a[0][kk][ty + 16 * r], b0, acc[r][0]);
          acc[r][1] = fma(sm.a[1][kk][ty + 16 * r], b0, acc[r][1]);
        }
      } else if (F64) {
        const Acc b1 = sm.b[NB > 1 ? 1 : 0][kk][tx];
        const Acc b2 = sm.b[NB > 2 ? 2 : 0][kk][tx];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          acc[r][0] = fma(b0, sm.a[(REAL || !F64) ? 1 : 2][kk][ty + 16 * r], acc[r][0]);   // c (ar + ai)
          acc[r][1] = fma(b1, sm.a[0][kk][ty + 16 * r], acc[r][1]);                        // (d - c) ar
          acc[r][2] = fma(b2, sm.a[1][kk][ty + 16 * r], acc[r][2]);                        // (c + d) ai
        }
      } else {
        const Acc bi = sm.b[NB > 1 ? 1 : 0][kk][tx];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const Acc ar = sm.a[0][kk][ty + 16 * r], ai = sm.a[1][kk][ty + 16 * r];
          acc[r][0] = fma(ar, b0, acc[r][0]);
          acc[r][0] = fma(-ai, bi, acc[r][0]);
          acc[r][1] = fma(ar, bi, acc[r][1]);
          acc[r][1] = fma(ai, b0, acc[r][1]);
        }
      }
    }
    __syncthreads();
  }

  double2 res[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    double re, im;
    if (REAL || !F64) {
      re = from_acc(acc[r][0]);
      im = from_acc(acc[r][1]);
    } else {
      re = double(acc[r][0]) - double(acc[r][2]);
      im = double(acc[r][0]) + double(acc[r][1]);
    }
    res[r] = make_double2(re, conj_out ? -im : im);
  }

  if (!trans) {
    if (tx >= t.cw) return;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const long long row = row0 + ty + 16 * r;
      if (row >= nrows) continue;
      if (rowskip && rowskip[row % rows_per_plane]) continue;
      double2* p = out + row * (long long)ncols + b.start + t.c0 + tx;
      if (store == XS_ACCUM) {
        double2 o = *p;
        o.x += res[r].x;
        o.y += res[r].y;
        *p = o;
      } else {
        *p = res[r];
      }
    }
  } else {
    // stage the tile and write it transposed: out[plane][col][row], rows contiguous
    double2 (*os)[TM + 1] = reinterpret_cast<double2 (*)[TM + 1]>(smem_raw);
#pragma unroll
    for (int r = 0; r < RPT; ++r) os[tx][ty + 16 * r] = res[r];
    __syncthreads();
    const int wr = tid & (TM - 1);
    const long long row = row0 + wr;
    if (row >= nrows) return;
    const long long plane = row / rows_per_plane;
    const int rip = (int)(row - plane * rows_per_plane);
    if (rowskip && rowskip[rip]) return;
    double2* base = out + plane * (long long)ncols * rows_per_plane + rip;
#pragma unroll
    for (int pass = 0; pass < TN / (NT / TM); ++pass) {
      const int col = (tid / TM) + (NT / TM) * pass;
      if (col < t.cw) {
        double2* p = base + (long long)(b.start + t.c0 + col) * rows_per_plane;
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

// Mirror-symmetric real blocks (uniform steps): the eigenvectors are the discrete sines,
// mode m (1-based) symmetric under i -> n-1-i for odd m and antisymmetric for even m, and
// the plan stores the ns = (n + 1) / 2 symmetric modes first.  Forward (sym = 1): column c
// needs only the folded data x_a + x_{n-1-a} (c < ns) or x_a - x_{n-1-a} (c >= ns) over
// the first ns nodes, so the contraction is half as long.  Inverse (sym = 2): the tile
// covers the first ns nodes a; S_a sums the symmetric modes, D_a the antisymmetric ones,
// and the two outputs are x_a = S_a + D_a and x_{n-1-a} = S_a - D_a.  Either way a block
// costs about n^2 / 2 multiply-adds per row instead of n^2.
template <typename Acc, int TM>
struct SymTile {
  Acc a[2][2][TK][TM];       // [folded sum | difference][re | im][k][row] (inverse: plane 0 only)
  Acc b[TK][TN];
};

template <typename Acc, int TM>
__device__ __forceinline__ void run_tile_sym(const double2* __restrict__ in, double2* __restrict__ out,
                                             const Acc* __restrict__ tab, const XBlock& b, const XTile& t,
                                             long long nrows, int rows_per_plane, int ncols, long long row0,
                                             int trans, int store, int conj_out,
                                             const signed char* __restrict__ rowskip, char* smem_raw) {
  constexpr int RPT = TM / 16;
  constexpr int EPT = TM * TK / NT;
  SymTile<Acc, TM>& sm = *reinterpret_cast<SymTile<Acc, TM>*>(smem_raw);
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int n = b.size, ns = b.ns;
  const bool fwd = b.sym == 1;
  const int cls = (fwd && t.c0 + tx >= ns) ? 1 : 0;        // forward: which folded plane column tx uses

  Acc sacc[RPT][2], dacc[RPT][2];
#pragma unroll
  for (int r = 0; r < RPT; ++r) sacc[r][0] = sacc[r][1] = dacc[r][0] = dacc[r][1] = Acc(0);

  const int la_row = tid / (TK / EPT), la_k = (tid % (TK / EPT)) * EPT;
  const int lb_k = tid >> 4, lb_c = tid & 15;
  const long long arow = row0 + la_row;
  const bool arow_ok = arow < nrows;
  const double2* __restrict__ ain = in + arow * (long long)ncols + b.start;
  const int klen = fwd ? ns : n;                           // contraction length
  for (int k0 = 0; k0 < klen; k0 += TK) {
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int kk = la_k + e;
      const int a = k0 + kk;
      double2 v = make_double2(0.0, 0.0), w = make_double2(0.0, 0.0);
      if (arow_ok && a < klen) {
        v = ain[a];
        if (fwd && n - 1 - a != a) w = ain[n - 1 - a];
      }
      const Acc vx = to_acc<Acc>(v.x), vy = to_acc<Acc>(v.y);
      if (fwd) {
        const Acc wx = to_acc<Acc>(w.x), wy = to_acc<Acc>(w.y);
        sm.a[0][0][kk][la_row] = vx + wx;
        sm.a[0][1][kk][la_row] = vy + wy;
        sm.a[1][0][kk][la_row] = vx - wx;
        sm.a[1][1][kk][la_row] = vy - wy;
      } else {
        sm.a[0][0][kk][la_row] = vx;
        sm.a[0][1][kk][la_row] = vy;
      }
    }
    {
      const int a = k0 + lb_k;
      sm.b[lb_k][lb_c] = (a < klen && lb_c < t.cw) ? tab[(long long)a * n + t.c0 + lb_c] : Acc(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const Acc bv = sm.b[kk][tx];
      if (fwd || k0 + kk < ns) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          sacc[r][0] = fma(sm.a[cls][0][kk][ty + 16 * r], bv, sacc[r][0]);
          sacc[r][1] = fma(sm.a[cls][1][kk][ty + 16 * r], bv, sacc[r][1]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          dacc[r][0] = fma(sm.a[0][0][kk][ty + 16 * r], bv, dacc[r][0]);
          dacc[r][1] = fma(sm.a[0][1][kk][ty + 16 * r], bv, dacc[r][1]);
        }
      }
    }
    __syncthreads();
  }

  // result columns: forward -> mode c0 + tx; inverse -> node c0 + tx (S + D) and its mirror (S - D)
  double2 rp[RPT], rm[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const double sr = from_acc(sacc[r][0]), si = from_acc(sacc[r][1]);
    const double dr = from_acc(dacc[r][0]), di = from_acc(dacc[r][1]);
    rp[r] = make_double2(sr + dr, conj_out ? -(si + di) : si + di);
    rm[r] = make_double2(sr - dr, conj_out ? -(si - di) : si - di);
  }
  const int col = t.c0 + tx;                               // within the block
  const int mir = n - 1 - col;
  const bool has_mir = !fwd && mir != col;

  if (!trans) {
    if (tx >= t.cw) return;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const long long row = row0 + ty + 16 * r;
      if (row >= nrows) continue;
      if (rowskip && rowskip[row % rows_per_plane]) continue;
      double2* p = out + row * (long long)ncols + b.start;
      if (store == XS_ACCUM) {
        double2 o = p[col];
        o.x += rp[r].x;
        o.y += rp[r].y;
        p[col] = o;
        if (has_mir) {
          double2 q = p[mir];
          q.x += rm[r].x;
          q.y += rm[r].y;
          p[mir] = q;
        }
      } else {
        p[col] = rp[r];
        if (has_mir) p[mir] = rm[r];
      }
    }
  } else {
    // stage [node tile | mirrored tile] and write it transposed: out[plane][col][row]
    double2 (*os)[TM + 1] = reinterpret_cast<double2 (*)[TM + 1]>(smem_raw);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      os[tx][ty + 16 * r] = rp[r];
      os[TN + tx][ty + 16 * r] = rm[r];
    }
    __syncthreads();
    const int wr = tid & (TM - 1);
    const long long row = row0 + wr;
    if (row >= nrows) return;
    const long long plane = row / rows_per_plane;
    const int rip = (int)(row - plane * rows_per_plane);
    if (rowskip && rowskip[rip]) return;
    double2* base = out + plane * (long long)ncols * rows_per_plane + rip;
    const int ncol_st = fwd ? TN : 2 * TN;
    for (int cc = tid / TM; cc < ncol_st; cc += NT / TM) {
      const int ct = cc & (TN - 1);
      if (ct >= t.cw) continue;
      int c = t.c0 + ct;
      if (cc >= TN) {
        if (n - 1 - c == c) continue;                      // the middle node has no mirror
        c = n - 1 - c;
      }
      double2* p = base + (long long)(b.start + c) * rows_per_plane;
      if (store == XS_ACCUM) {
        double2 o = *p;
        o.x += os[cc][wr].x;
        o.y += os[cc][wr].y;
        *p = o;
      } else {
        *p = os[cc][wr];
      }
    }
  }
}

template <typename Acc, int TM>
__global__ void __launch_bounds__(NT)
xform_kernel(const double2* __restrict__ in, double2* __restrict__ out, const Acc* __restrict__ tab,
             const XBlock* __restrict__ blocks, const XTile* __restrict__ tiles, int ntiles, long long nrows,
             int rows_per_plane, int ncols, int trans, int store, int conj_out,
             const signed char* __restrict__ rowskip) {
  constexpr int S1 = sizeof(Tile<Acc, false, TM>), S2 = sizeof(SymTile<Acc, TM>);
  constexpr int S3 = sizeof(double2) * 2 * TN * (TM + 1);      // transposed-store staging
  constexpr int SA = S1 > S2 ? (S1 > S3 ? S1 : S3) : (S2 > S3 ? S2 : S3);
  __shared__ __align__(16) char smem[SA];
  // column tiles of one row tile are consecutive CTAs, so the row tile is read from
  // DRAM once and re-read from L2 by the other column tiles
  const long long cta = blockIdx.x;
  const XTile t = tiles[cta % ntiles];
  const XBlock b = blocks[t.blk];
  const long long row0 = (cta / ntiles) * TM;
  const Acc* tb = tab + (sizeof(Acc) == 8 ? b.toff : b.toff32);
  if (b.sym)
    run_tile_sym<Acc, TM>(in, out, tb, b, t, nrows, rows_per_plane, ncols, row0, trans, store, conj_out, rowskip,
                          smem);
  else if (b.real)
    run_tile<Acc, true, TM>(in, out, tb, b, t, nrows, rows_per_plane, ncols, row0, trans, store, conj_out,
                            rowskip, smem);
  else
    run_tile<Acc, false, TM>(in, out, tb, b, t, nrows, rows_per_plane, ncols, row0, trans, store, conj_out,
                             rowskip, smem);
}

// Launch the dense kernel over the tiles [tiles, tiles + ntiles).
template <typename Acc>
void launch(const XformSet& xs, const XTile* tiles, int ntiles, const Acc* tab, const double2* in, double2* out,
            int rows_per_plane, long long nplanes, int trans, int store, int conj_out,
            const signed char* rowskip, cudaStream_t st, int tile_rows) {
  const long long nrows = nplanes * (long long)rows_per_plane;
  if (nrows <= 0 || ntiles == 0) return;
  const bool big = tile_rows == 64 || (tile_rows != 16 && ((nrows + 63) / 64) * ntiles >= 2 * 152);
  if (big) {
    const long long ctas = ((nrows + 63) / 64) * ntiles;
    xform_kernel<Acc, 64><<<(unsigned)ctas, NT, 0, st>>>(in, out, tab, xs.d_blocks, tiles, ntiles, nrows,
                                                          rows_per_plane, xs.ncols, trans, store, conj_out,
                                                          rowskip);
  } else {
    const long long ctas = ((nrows + 15) / 16) * ntiles;
    xform_kernel<Acc, 16><<<(unsigned)ctas, NT, 0, st>>>(in, out, tab, xs.d_blocks, tiles, ntiles, nrows,
                                                          rows_per_plane, xs.ncols, trans, store, conj_out,
                                                          rowskip);
  }
  count_launch();
}

}  // namespace

void xform_f64(const XformSet& xs, const double2* in, double2* out, int rows_per_plane,
               long long nplanes, int trans, int store, int conj_out, const signed char* rowskip,
               cudaStream_t st, bool fast_sine, int tile_rows) {
  if (fast_sine && xs.dst.nblk > 0) {
    // the two launches write disjoint columns of the output
    launch<double>(xs, xs.d_tiles64, xs.ntiles64, xs.d_tab, in, out, rows_per_plane, nplanes, trans, store,
                   conj_out, rowskip, st, tile_rows);
    dst_f64(xs.dst, in, out, rows_per_plane, nplanes, xs.ncols, trans, store, conj_out, rowskip, st);
    return;
  }
  launch<double>(xs, xs.d_tiles, xs.ntiles, xs.d_tab, in, out, rows_per_plane, nplanes, trans, store, conj_out,
                 rowskip, st, tile_rows);
}

void xform_f32(const XformSet& xs, const double2* in, double2* out, int rows_per_plane,
               long long nplanes, int trans, int store, int conj_out, const signed char* rowskip,
               cudaStream_t st, int tile_rows) {
  launch<float>(xs, xs.d_tiles, xs.ntiles, xs.d_tab32, in, out, rows_per_plane, nplanes, trans, store, conj_out,
                rowskip, st, tile_rows);
}

}  // namespace hz
