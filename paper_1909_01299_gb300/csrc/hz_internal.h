// Internal declarations of the hz library: host plan, device tables, kernel launchers.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hz.h"

namespace hz {

using cd = std::complex<double>;

// Every kernel launcher calls this once per launch (launch accounting for reports).
void count_launch(int n = 1);
long long launch_count();

// Complex-symmetric generalised tridiagonal eigenpairs K W = M W Lambda, W^T M W = I.
// kd: n diagonal, ko: n-1 off-diagonal, m: n diagonal of M.  W is row-major n x n
// (W[i*n + l] = component at node i of mode l).  Returns false on failure.
bool tridiag_eig(int n, const cd* kd, const cd* ko, const cd* m, std::vector<cd>& lam,
                 std::vector<cd>& W, double* eig_residual);
// Closed-form pairs of a uniform real block (every step equal to h): the discrete sine
// transform.  kd, ko, m are the block's pencil, used only for the residual check.
bool sine_eig(int n, double h, const cd* kd, const cd* ko, const cd* m, std::vector<cd>& lam,
              std::vector<cd>& W, double* eig_residual);
// max(||K W - M W Lambda||_F / (||K||_F ||W||_F), max |W^T M W - I|) of a computed pencil.
double eig_check(int n, const cd* kd, const cd* ko, const cd* m, const std::vector<cd>& lam,
                 const std::vector<cd>& W);

// ---------------------------------------------------------------------------
// Row transforms: out_row[s + c] = sum_a in_row[s + a] * B_b[a][c] for every block b
// covering columns [s, s + n) of a row of length ncols (block-diagonal B).
// ---------------------------------------------------------------------------
struct XBlock {
  int start;            // first column of the block in the row
  int size;             // block width n
  int real;             // 1: table is real (one n*n plane); 0: complex
  int sym;              // mirror-symmetric real block (uniform steps, sine eigenvectors with the
                        //   ns = (n + 1) / 2 symmetric modes first): 1 = forward table (rows =
                        //   nodes, folded), 2 = inverse table (rows = modes, outputs unfolded)
  int ns;               // number of symmetric modes when sym != 0
  int pad;
  long long toff;       // offset (doubles) of the FP64 table; complex entries c + i d are
                        //    stored for the 3M product as three planes [c | d - c | c + d]
  long long toff32;     // offset (floats) of the FP32 table; complex: two planes [c | d]
};
struct XTile {
  int blk;              // block index
  int c0;               // first output column within the block
  int cw;               // number of output columns of the tile (<= tile width)
  int pad;
};

// Fast sine transform of a uniform block (FP64 path).  The block's table is
// S sin(pi j m / N), N = n + 1 (forward: rows = nodes j, columns = modes m in the
// symmetric-modes-first order; inverse: the transpose), i.e. a scaled DST-I.  It is
// computed from one complex FFT of length N per row: y_j = p_j x_j + q_j x_{N-j}
// (p_j, q_j = (S / 2) (sin(pi j / N) +- 1/2)), Y = FFT(y) by mixed-radix stages
// (radices 2, 3, 4, 5; decimation in frequency, output in digit-reversed order), then
// X_{2k} = i (Y_k - Y_{N-k}) and X_{2k+1} = X_{2k-1} + Y_k + Y_{N-k}, X_1 = Y_0.
// For N = m 2^a (m = 3 or 5, a >= 2) the FFT is split by the prime-factor map (Good and
// Thomas): y_j is placed at n1 + 2^a n2 for j = (m n1 + 2^a n2) mod N, the radix-m stage
// needs no twiddles, and Y_k lands at 2^a (k mod m) + (digit-reversed k mod 2^a).
constexpr int kDstMaxStages = 8;
constexpr int kDstMaxN = 128;     // largest N = n + 1 handled by the fast transform
struct DstBlock {
  int start;                      // first column of the block in the row
  int n;                          // block width; N = n + 1 = product of the radices
  int nst;                        // radix stages
  int rad[kDstMaxStages];         // radices in stage order
  int ntw;                        // twiddles of all stages (complex entries)
  int pfa;                        // 1: N = m 2^a (m = 3 or 5, a >= 2) split by the prime-factor
                                  //   (Good-Thomas) map: the radix-m first stage has no twiddles
  long long tw_off;               // offset (complex) of the stage twiddles (from the first
                                  //   twiddled stage)
  long long ioff;                 // offset (ints) of pos[N], gin[N], src[n], pin[N]
  long long coff;                 // offset (doubles) of (p_j, q_j), j = 0..N/2
};
struct DstSet {
  int nblk = 0;
  int nmax = 0;                   // largest N of the set
  DstBlock* d_blk = nullptr;
  int* d_idx = nullptr;
  double* d_coef = nullptr;
  double2* d_tw = nullptr;
  float* d_coef32 = nullptr;      // FP32 copies (mixed path)
  float2* d_tw32 = nullptr;
};
// Whether a uniform block of width n takes the fast transform (n >= 2, n + 1 <= kDstMaxN with no
// prime factor above 5).
bool dst_supported(int n);
// Host: the fast-transform descriptor of a block of width n whose table is S sin(pi j m / N);
// dir = 1: forward (natural nodes in, symmetric-modes-first out), 2: inverse (the reverse).
// Appends to the index, coefficient and twiddle arrays; false if N has a prime factor > 5,
// N > kDstMaxN or n < 2.
bool dst_plan_block(int n, int start, int dir, double S, std::vector<DstBlock>& blk, std::vector<int>& idx,
                    std::vector<double>& coef, std::vector<double2>& tw);
// Host reference of the same computation (the code the kernel runs per row), for tests:
// out = table^T applied to one row in (n values each).
bool dst_apply_host(int n, int dir, double S, const double2* in, double2* out);
// Set the kernel's shared-memory limit for blocks up to N = nmax (current device, before any capture).
void dst_prepare(int nmax);
// Mixed path: the same transform in FP32 arithmetic; in32 / out32: complex64 input / output,
// at least one of them (an accumulating store needs a complex128 output).  false: nothing launched.
bool dst_f32(const DstSet& ds, const void* in, int in32, void* out, int out32, int rows_per_plane, long long nplanes,
             int ncols, int trans, int store, const signed char* rowskip, cudaStream_t st);
void dst_f64(const DstSet& ds, const double2* in, double2* out, int rows_per_plane, long long nplanes, int ncols,
             int trans, int store, int conj_out, const signed char* rowskip, cudaStream_t st);

// A device-resident block-diagonal transform (one per axis and use).
struct XformSet {
  int ncols = 0;                  // row length (axis length)
  int nblocks = 0;
  int ntiles = 0;
  XBlock* d_blocks = nullptr;
  XTile* d_tiles = nullptr;
  double* d_tab = nullptr;        // FP64 tables (3M layout for complex blocks)
  float* d_tab32 = nullptr;       // FP32 copy of the same tables for the mixed path
  std::vector<XBlock> h_blocks;
  // FP64 fast sine transforms of the uniform blocks whose N = n + 1 factors into 2, 3, 5:
  // with fast_sine the dense kernel runs only the tiles64 (the other blocks)
  DstSet dst;
  int ntiles64 = 0;
  XTile* d_tiles64 = nullptr;
};

enum XformStore { XS_STORE = 0, XS_ACCUM = 1 };

// Tensor-core (tcgen05 kind::tf32, 3xTF32) version of the bulk transforms.  Per block the
// complex table B (n x n) is stored as the real interleaved matrix B' (2n x 2n) transposed
// to K-major, padded to npad (multiple of 16) rows and kpad (multiple of 16) columns, as
// TF32 hi (npad x kpad floats at toff) followed by TF32 lo (same size).  A block whose table
// is real also has the real table itself, K-major (npad_r x kpad_r at toff_r, hi then lo), for
// the real-table kernel, which transforms the real and imaginary parts of the data as two
// rows of one real GEMM (K = N = n instead of 2n).
struct TCBlock {
  int start;            // first complex column of the block
  int size;             // complex width n
  int npad, kpad;
  long long toff;       // float offset of the hi table (interleaved complex form)
  int npad_r, kpad_r;   // real form (real tables only; npad_r = 0 otherwise)
  long long toff_r;
};
struct TCTile {
  int blk;
  int n0;               // first output column (interleaved: real column, multiple of 16; real
                        //   kernel: complex column, multiple of 16)
  int nt;               // output columns (multiple of 16; <= 160 interleaved, <= 128 real)
  int pad;
};
// A list of output tiles with one 128-byte TMA tensor map per tile (its table rows).
struct TCList {
  int ntiles = 0;
  int nt_max = 16;
  TCTile* d_tiles = nullptr;
  unsigned char* d_tmaps = nullptr;
};
struct TCSet {
  int ncols = 0;
  TCBlock* d_blocks = nullptr;
  float* d_tab = nullptr;
  // Tile lists per variant v = fast + 2 real: fast leaves the uniform blocks with a fast sine
  // transform to dst_f32; real sends the blocks with real tables to the real-table kernel.
  // cl[v]: tiles of the interleaved complex kernel, rl[v]: tiles of the real-table kernel.
  TCList cl[4], rl[4];
};
// Encode the TMA tensor maps of the tiles (tables already on the device at d_tab) into
// 128-byte records; real: the tiles index the real tables.  false if the driver offers no
// encoder or rejects a map.
bool tc_encode_tmaps(const float* d_tab, const std::vector<TCBlock>& blocks, const std::vector<TCTile>& tiles,
                     std::vector<unsigned char>& bytes, bool real = false);
size_t xform_tc_smem(int nt_max, bool in32);
// Set the tensor-core kernels' shared-memory limits on the current device (before any capture).
void xform_tc_prepare();
// Host: append the TF32 hi/lo K-major tables of one block (complex table B, n x n row-major,
// B[a][c]) and its output tiles; with real_tiles (B real) also the real form and its tiles.
void tc_pack_block(const cd* B, int n, int start, std::vector<float>& tab, TCBlock& blk,
                   std::vector<TCTile>& tiles, int blk_index, std::vector<TCTile>* real_tiles = nullptr);
// err: device status word (set to HZ_ERR_TIMEOUT if a bounded wait gives up).
// in32 / out32: the input / output are complex64 (float2) instead of complex128 (double2).
// Returns false (nothing launched) for XS_ACCUM with a complex64 output.
// products: 3 (3xTF32) or 1 (plain TF32).  skip_fast: leave out the blocks with a fast sine
// transform; real_tables: blocks with real tables through the real-table kernel.
bool xform_tc(const TCSet& ts, const void* in, int in32, void* out, int out32, int rows_per_plane,
              long long nplanes, int trans, int store, const signed char* rowskip, int* err,
              cudaStream_t st, int products = 3, bool skip_fast = false, bool real_tables = false);

// FP64 transform (DFMA): rows_per_plane rows of length ncols per plane, nplanes planes.
// trans = 1 writes out[plane][col][row] (plane of ncols x rows_per_plane); else out
// has the input's layout.  store: XS_STORE or XS_ACCUM (out += result).  conj_out
// conjugates the result before it is stored.
// rowskip (may be NULL) flags rows (index within the plane) that are neither computed nor
// written: the interface rows, which belong to no block.
// fast_sine: uniform blocks with a fast-transform descriptor use dst_f64.  tile_rows: data rows
// per CTA of the dense kernel, 16 or 64 (0: 64 when the launch has at least two CTAs per SM).
void xform_f64(const XformSet& xs, const double2* in, double2* out, int rows_per_plane,
               long long nplanes, int trans, int store, int conj_out, const signed char* rowskip,
               cudaStream_t st, bool fast_sine = false, int tile_rows = 0);
// Same contraction with FP32 arithmetic on FP64 data (SIMT FFMA), for the mixed path.
void xform_f32(const XformSet& xs, const double2* in, double2* out, int rows_per_plane,
               long long nplanes, int trans, int store, int conj_out, const signed char* rowskip,
               cudaStream_t st, int tile_rows = 0);

// ---------------------------------------------------------------------------
// z solves per mode (Eq. (fdmtrprjfr), Eq. (fdmtrprjfrerr))
// ---------------------------------------------------------------------------
struct ZFactors {
  double2* P = nullptr;           // [k][i][j]: scaled inverse pivot
  double2* Q = nullptr;           // [k][i][j]: back-substitution multiplier c_{k+1} / d_k
  double2* cm = nullptr;          // [k]: forward multiplier c_k (/ mz_k when folded)
};

// Right-hand side formed inside the sweep (mixed path, complex64 storage), in FP32 with the
// arithmetic of global_rhs / boundary_rhs (so that the separate kernel and its complex64 volume
// round trip are not needed): kind 1, the step-5 global right-hand side
//   sum_p wx32[p][i] aX32[r][k][p][j] + sum_q wy32[q][j] bY32[r][k][q][i];
// kind 2, rhs32 plus the step-6 boundary term
//   sigma_k (cxl32[i] aX32[r][k][gxl[i]][j] + cxr32[i] aX32[..gxr[i]..] + cyl32[j] bY32[r][k][gyl[j]][i]
//            + cyr32[j] bY32[..gyr[j]..]).
constexpr int kGenMaxIface = 4;         // kind 1: interfaces per axis held in registers
struct ZRhsGen {
  int kind = 0;                          // 0: read rhs32
  int nIx = 0, nIy = 0;
  const float2* aX32 = nullptr;          // [r][k][nIx][ny]: aX (kind 1) or alphaX (kind 2)
  const float2* bY32 = nullptr;          // [r][k][nIy][nx]: bY (kind 1) or alphaY (kind 2)
  const float2* wx32 = nullptr;          // kind 1: [nIx][nx]
  const float2* wy32 = nullptr;          // kind 1: [nIy][ny]
  const int* gxl = nullptr; const int* gxr = nullptr;     // kind 2: per i, interface index or -1
  const int* gyl = nullptr; const int* gyr = nullptr;     // kind 2: per j
  const float2* cxl32 = nullptr; const float2* cxr32 = nullptr;   // kind 2: per i
  const float2* cyl32 = nullptr; const float2* cyr32 = nullptr;   // kind 2: per j
  const double* sig = nullptr;           // kind 2: [k] or NULL
};

struct ZSolveArgs {
  const double2* rhs = nullptr;   // mode-layout right-hand side [r][k][i][j]
  double2* out = nullptr;         // mode-layout result [r][k][i][j]
  const double2* P = nullptr;
  const double2* Q = nullptr;
  const double2* cm = nullptr;
  const signed char* skip_i = nullptr;   // 1 at x-interface positions (NULL: sweep every mode)
  const signed char* skip_j = nullptr;
  int nx = 0, ny = 0, nz = 0, nrhs = 0;
  int real_cm = 0;
  // sweep variant: 1 or 2 right-hand sides per thread, 3 one per thread with z taken in
  // register chunks (few sweeps, long z); 0 = chosen from the launch size and sms
  int rhs_per_thread = 0;
  int sms = 0;                           // SM count of the device (automatic choice)
  // complex64 storage (mixed path): when rhs32 is set, the right-hand side is read from
  // rhs32, the result written to out32 (truncated to FP32) and the FP64 forward-sweep
  // values kept in scratch (same layout); the elimination itself stays FP64
  const float2* rhs32 = nullptr;
  float2* out32 = nullptr;
  double2* scratch = nullptr;
  ZRhsGen gen;                           // complex64 storage only: right-hand side formed in the sweep
};
void zsolve(const ZSolveArgs& a, cudaStream_t st);
// Whether zsolve forms a.gen's right-hand side itself (the plain sweep kernels; kind 1 with at
// most kGenMaxIface interfaces per axis).  The chunked sweep reads rhs32: the caller then
// launches global_rhs / boundary_rhs first.
bool zsolve_forms_rhs(const ZSolveArgs& a);

// Step 6 boundary term g~ / M_z added in place to the block right-hand side f~:
// sigma_k (cxl aX[pl] + cxr aX[pr] + cyl aY[ql] + cyr aY[qr]).
struct BoundaryArgs {
  int nx = 0, ny = 0, nz = 0, nrhs = 0, nIx = 0, nIy = 0;
  const signed char* skip_i = nullptr; const signed char* skip_j = nullptr;
  const double* sig = nullptr;           // [k] or NULL
  const double2* alphaX = nullptr;       // [r][k][nIx][ny]
  const double2* alphaY = nullptr;       // [r][k][nIy][nx]
  const int* gxl = nullptr; const int* gxr = nullptr;     // per i: interface index or -1
  const int* gyl = nullptr; const int* gyr = nullptr;     // per j
  const double2* cxl = nullptr; const double2* cxr = nullptr;   // per i
  const double2* cyl = nullptr; const double2* cyr = nullptr;   // per j
  // FP32 copies of the four coefficient arrays: when set, the boundary term is formed in
  // FP32 and added to f~ in FP64 (mixed path)
  const float2* cxl32 = nullptr; const float2* cxr32 = nullptr;
  const float2* cyl32 = nullptr; const float2* cyr32 = nullptr;
  int real_x = 0, real_y = 0;            // FP64: cxl/cxr (cyl/cyr) are real
  // complex64 copies of alphaX / alphaY (mixed path with complex64 f~): read instead of the
  // complex128 arrays, and the sum f~ + g~ is formed in FP32
  const float2* alphaX32 = nullptr; const float2* alphaY32 = nullptr;
};
void boundary_rhs(const BoundaryArgs& a, double2* ft, cudaStream_t st);
// complex64 f~ (mixed path, needs the FP32 coefficient copies): the sum is formed in FP64
// and stored truncated to FP32
void boundary_rhs(const BoundaryArgs& a, float2* ft, cudaStream_t st);

// Step 5 global right-hand side: out = sum_p WgxI[p][i] aX[r][k][p][j] + sum_q WgyI[q][j] bY[r][k][q][i].
struct GlobalRhsArgs {
  int nx = 0, ny = 0, nz = 0, nrhs = 0, nIx = 0, nIy = 0;
  const double2* aX = nullptr;           // [r][k][nIx][ny]
  const double2* bY = nullptr;           // [r][k][nIy][nx]
  const double2* WgxI = nullptr;         // [nIx][nx]
  const double2* WgyI = nullptr;         // [nIy][ny]
  const float2* WgxI32 = nullptr;        // FP32 copies: when set, FP32 arithmetic (mixed path)
  const float2* WgyI32 = nullptr;
  int real_x = 0, real_y = 0;            // FP64: WgxI (WgyI) is real
  const float2* aX32 = nullptr;          // complex64 copies of aX / bY (FP32 arithmetic only)
  const float2* bY32 = nullptr;
};
// out[i] = complex64(in[i]) (truncating conversion), n values.
void to_c64_copy(const double2* in, float2* out, long long n, cudaStream_t st);
void global_rhs(const GlobalRhsArgs& a, double2* out, cudaStream_t st);
// complex64 output (mixed path, needs the FP32 coefficient copies)
void global_rhs(const GlobalRhsArgs& a, float2* out, cudaStream_t st);


// Elimination factors of (Tz + s_ij S_z) for every (i, j) with s_ij = lamx[i] + lamy[j]
// (no pivoting).  fold (may be NULL) scales P by fold[k] (the M_z of the right-hand side).
void zfactor(double2* P, double2* Q, const double2* lamx, const double2* lamy,
             const signed char* skip_i, const signed char* skip_j, const double2* tzd,
             const double2* szs, const double2* coff, const double2* fold, int nx, int ny, int nz,
             unsigned long long* min_pivot_bits, int* status, cudaStream_t st);

// ---------------------------------------------------------------------------
// Interface steps
// ---------------------------------------------------------------------------
// out[plane][s][j] = sum_{i in [lo_s, hi_s)} coef[s][i] V[plane][i][j]  (contraction over rows);
// real_coef: every coefficient is real (2 FMA per term instead of 4)
void contract_rows(const double2* V, double2* out, const double2* coef, const int2* range,
                   int nrows, int ncols, int nslots, long long nplanes, cudaStream_t st, bool real_coef = false);
// out[plane][s][i] = sum_{j in [lo_s, hi_s)} coef[s][j] V[plane][i][j]  (contraction within rows)
void contract_cols(const double2* V, double2* out, const double2* coef, const int2* range,
                   int nrows, int ncols, int nslots, long long nplanes, cudaStream_t st, bool real_coef = false);
// Contractions whose every slot covers the whole row (rows = true: over i, out[plane][s][j];
// false: over j, out[plane][s][i]) in one pass over V; false (nothing launched) unless
// 2 <= nslots <= 8.  FP32 arithmetic (mixed path).
bool contract_all(bool rows, const double2* V, double2* out, const float2* coef, int nrows, int ncols,
                  int nslots, long long nplanes, cudaStream_t st);
// The same contractions with FP32 arithmetic on the FP64 data (mixed path).
void contract_rows(const double2* V, double2* out, const float2* coef, const int2* range,
                   int nrows, int ncols, int nslots, long long nplanes, cudaStream_t st);
void contract_cols(const double2* V, double2* out, const float2* coef, const int2* range,
                   int nrows, int ncols, int nslots, long long nplanes, cudaStream_t st);
// The FP32 contractions on complex64 V (the mixed path's mode-space storage).
bool contract_all(bool rows, const float2* V, double2* out, const float2* coef, int nrows, int ncols,
                  int nslots, long long nplanes, cudaStream_t st);
void contract_rows(const float2* V, double2* out, const float2* coef, const int2* range,
                   int nrows, int ncols, int nslots, long long nplanes, cudaStream_t st);
void contract_cols(const float2* V, double2* out, const float2* coef, const int2* range,
                   int nrows, int ncols, int nslots, long long nplanes, cudaStream_t st);

// ---------------------------------------------------------------------------
// Locally perturbed medium: vector kernels of the GMRES around the layered solve.
// Vectors are [r][n] complex (R right-hand sides of n values); a basis is [i][r][n]
// with vstride = R * n between its vectors.
// ---------------------------------------------------------------------------
constexpr int kMaxVec = 16;     // basis vectors handled per multi_dot / multi_axpy pass
// out[r][n] = d[n] v[r][n]
void pert_mul(const double2* d, const double2* v, double2* out, long long n, int R, cudaStream_t st);
// out = a - b + c (b or c may be NULL), total elements
void vec_lin3(const double2* a, const double2* b, const double2* c, double2* out, long long total,
              cudaStream_t st);
// s[r] = 1 / sqrt(Re d[r]), or 0 where Re d[r] <= 0
void vec_inv_norm(const double2* d, double2* s, int R, cudaStream_t st);
// out[r][n] = s[r] w[r][n]
void vec_scale(const double2* s, const double2* w, double2* out, long long n, int R, cudaStream_t st);
// out[r * cnt + i] = <V_i[r], w[r]> = sum conj(V_i[r][n]) w[r][n], cnt <= kMaxVec; partial needs
// R * multi_dot_parts(n) * cnt entries.  Fixed summation order.
int multi_dot_parts(long long n);
void multi_dot(const double2* V, long long vstride, int cnt, const double2* w, long long n, int R,
               double2* partial, double2* out, cudaStream_t st);
// w[r][n] -= sum_{i < cnt} c[r * cnt + i] V_i[r][n], cnt <= kMaxVec
void multi_axpy(const double2* V, long long vstride, int cnt, const double2* c, double2* w, long long n, int R,
                cudaStream_t st);
// FP32-basis forms (mixed plans): the basis V is complex64, the other vector stays FP64
void pert_mul(const double2* d, const float2* v, double2* out, long long n, int R, cudaStream_t st);
void vec_scale(const double2* s, const double2* w, float2* out, long long n, int R, cudaStream_t st);
void multi_dot(const float2* V, long long vstride, int cnt, const double2* w, long long n, int R,
               double2* partial, double2* out, cudaStream_t st);
void multi_axpy(const float2* V, long long vstride, int cnt, const double2* c, double2* w, long long n, int R,
                cudaStream_t st);

struct IfaceArgs {
  int nx = 0, ny = 0, nz = 0, nrhs = 0, nIx = 0, nIy = 0;
  const int* xif = nullptr; const int* yif = nullptr;          // interface node indices
  const signed char* isx = nullptr; const signed char* isy = nullptr;   // interface flags
  const double2* mx = nullptr; const double2* my = nullptr; const double2* mz = nullptr;
  const double2* ihx = nullptr; const double2* ihy = nullptr;  // 1 / h (N+1 steps)
  const double* sig = nullptr;                                  // sigma per z node
};
// Step 4: residual r = M f - A v on the interfaces from v at the neighbouring nodes.
void iface_residual(const IfaceArgs& a, const double2* f, const double2* vX, const double2* vY,
                    double2* rX, double2* rY, cudaStream_t st);
// Step 7 (interface part): u = w on the interface planes.
void write_iface(const IfaceArgs& a, const double2* wX, const double2* wY, double2* u, int conj_out,
                 int accumulate, cudaStream_t st);

// Adjoint input: out = conj(g) / (mx_i my_j mz_k).
void adjoint_prep(const double2* g, double2* out, const double2* imx, const double2* imy,
                  const double2* imz, int nx, int ny, int nz, int nrhs, cudaStream_t st);

// Right-hand-side gradient: out = conj(mx_i my_j mz_k) lam (out may alias lam).
void grad_rhs(const double2* lam, double2* out, const double2* mx, const double2* my, const double2* mz,
              int nx, int ny, int nz, int nrhs, cudaStream_t st);

// u = conj(u) elementwise.
void conj_inplace(double2* u, long long n, cudaStream_t st);

// Stencil residual (FP64): rho = f - M^{-1} A u and per-RHS sums of |M rho|^2, |M f|^2.
struct StencilArgs {
  int nx = 0, ny = 0, nz = 0, nrhs = 0;
  const double2* kxs = nullptr;   // [nx][3]: (lower, diag, upper) of K_x row i / mx_i
  const double2* kys = nullptr;   // [ny][3]
  const double2* tzs = nullptr;   // [nz][3]: row k of Tz / mz_k
  const double* sig = nullptr;    // [nz]
  const double2* mx = nullptr; const double2* my = nullptr; const double2* mz = nullptr;
  // precomputed by the plan for the residual kernel
  const double2* cxy = nullptr;   // [ny][nx]: kxs[i][1] + kys[j][1]
  const double* w2xy = nullptr;   // [ny][nx]: |mx_i|^2 |my_j|^2
  const double* w2z = nullptr;    // [nz]: |mz_k|^2
  const signed char* rx = nullptr; const signed char* ry = nullptr; const signed char* rz = nullptr;
                                  // 1 where the off-diagonal coefficients of that row are real
};
// rho = f - M^{-1} A u (rho may be NULL) and per-RHS partial sums of |M rho|^2 (and of
// |M f|^2 when fnorm != 0); partial holds stencil_parts(a) * nrhs pairs.
void stencil_residual(const StencilArgs& a, const double2* f, const double2* u, double2* rho,
                      double* partial, int fnorm, cudaStream_t st);
int stencil_parts(const StencilArgs& a);   // number of partial sums per RHS
void finish_norms(const double* partial, int nparts, int nrhs, double* out, cudaStream_t st);

// Layer gradient: G_L = sum_{k in L} mz_k sum_{r,i,j} conj(lam) mx my u.
void grad_layers(const double2* u, const double2* lam, const double2* mx, const double2* my,
                 const double2* mz, const int* z_begin, int nlayers, int nx, int ny, int nz,
                 int nrhs, double2* partial, int nparts, double2* G, cudaStream_t st);
int grad_parts(int nx, int ny, int nrhs);

}  // namespace hz
