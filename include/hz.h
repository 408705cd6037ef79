/*
 * hz.h -- C ABI of the GB300 layered-medium Helmholtz solver.
 *
 * Solves the 7-point finite-volume discretisation (Eq. (fd), Kronecker form
 * Eq. (fdmtr)) of
 *
 *     -sigma(z) (u_xx + u_yy) - (sigma(z) u_z)_z - k^2(z) u = f
 *
 * on a tensor grid S_x x S_y x S_z with homogeneous Dirichlet boundaries, by
 * the block method of Sec. 2: the grid is split into Cartesian blocks
 * S^i_x x S^j_y x S_z; each block is solved with zero Dirichlet data by x/y
 * eigen-transforms and one tridiagonal solve in z per mode (Eq. (fdmtrprjfr));
 * the residual left on the block interfaces is removed with the global
 * eigen-transform (Eq. (fdmtrprjfrerr)) and a second local solve
 * (Eq. (fdmtrprjfrerrloc)); steps 1-7 of the algorithm in Sec. 2.
 *
 * Discretisation conventions (all arrays are host arrays, copied at plan creation):
 *   - An axis with N interior (unknown) nodes has N+1 steps h_0..h_N; step h_n
 *     joins node n-1 to node n and nodes -1 and N carry u = 0.  Steps may be
 *     complex (absorbing "PML" parts of the grid, Sec. 2).
 *   - hhat_i = (h_i + h_{i+1}) / 2 are the control-volume edge lengths, and the
 *     solver returns u = A^{-1} (Mz (x) My (x) Mx) f with M_d = diag(hhat).
 *   - k^2 and sigma are node-based per layer; layer L holds the z nodes
 *     [z_begin[L], z_begin[L+1]).  sigma on a z step inside a layer is the
 *     layer's value, on a step joining two layers the harmonic mean of the two.
 *
 * Device arrays f, u, g, lam are complex128 (interleaved re, im doubles) of
 * shape (nrhs, Nz, Ny, Nx), x fastest, contiguous.  The caller owns them;
 * they are never retained after a call returns.  f == u (in place) is allowed.
 *
 * Errors: every entry point returns an hz_status; nothing is printed and no
 * exception crosses the ABI.  Kernels report a singular pivot (zero, non-finite, or
 * at the rounding level of the terms that formed it) or a non-finite value through a
 * device status word that the call reads back.
 */
#ifndef HZ_H_
#define HZ_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } hz_c128;   /* layout of complex128 */

typedef enum {
  HZ_OK = 0,
  HZ_ERR_ARG = 1,            /* bad size, pointer or option                            */
  HZ_ERR_EIG = 2,            /* a 1D eigen-decomposition failed its identity checks    */
  HZ_ERR_SINGULAR = 3,       /* singular pivot in a z tridiagonal: zero, non-finite, or
                                |d| <= 64 eps x (sum of the 1-norms of the terms of d)  */
  HZ_ERR_NONFINITE = 4,      /* non-finite value in the input or the result            */
  HZ_ERR_NOT_CONVERGED = 5,  /* mixed path: refinement did not reach rtol              */
  HZ_ERR_OOM = 6,            /* device allocation failed                               */
  HZ_ERR_CUDA = 7,           /* a CUDA runtime call failed                             */
  HZ_ERR_TIMEOUT = 8         /* a bounded device-side wait gave up                     */
} hz_status;

/* Precision of a plan (hz_options.precision).  HZ_MIXED is HZ_MIXED_3XTF32. */
enum { HZ_FP64 = 0, HZ_MIXED = 1, HZ_MIXED_3XTF32 = 1, HZ_MIXED_TF32 = 2 };

typedef struct hz_plan_s *hz_plan_t;

/* Grid: nx, ny, nz interior nodes; hx, hy, hz point to nx+1, ny+1, nz+1 steps. */
typedef struct {
  int nx, ny, nz;
  const hz_c128 *hx, *hy, *hz;
} hz_grid;

/* Layers: z_begin has nlayers+1 entries, z_begin[0] = 0, z_begin[nlayers] = nz,
 * strictly increasing.  k2 has nlayers complex entries.  sigma has nlayers
 * positive entries or is NULL (sigma = 1). */
typedef struct {
  int nlayers;
  const int *z_begin;
  const hz_c128 *k2;
  const double *sigma;
} hz_layers;

/* Block partition: nbx x nby blocks.  x_iface lists the nbx-1 interface node
 * indices (strictly increasing, each block keeps >= 1 node); NULL selects the
 * default p_b = floor(b (nx+1) / nbx) - 1, b = 1..nbx-1.  Same for y.  The
 * interface nodes belong to no block (Sec. 2, "the projection operators to
 * interior nodes").  nbx = HZ_BLOCKS_AUTO (x_iface NULL) lets the plan choose the
 * count: the FP64 path balances the dense block transforms (cost ~ N / B per unknown)
 * against the interface steps (cost ~ B), B ~ sqrt(N) as in the cost estimate of Sec. 2,
 * with blocks at least 16 nodes wide; the mixed path, whose block transforms run on
 * the tensor cores (where a wider block costs little more per value), takes blocks
 * about 80 nodes wide.  hz_get_info reports the counts chosen. */
#define HZ_BLOCKS_AUTO 0
typedef struct {
  int nbx, nby;
  const int *x_iface, *y_iface;
} hz_blocks;

/* Options.  precision: HZ_FP64 (all arithmetic FP64) or a mixed precision, HZ_MIXED (=
 * HZ_MIXED_3XTF32: the bulk tensor-core transforms as three TF32 products, A_hi B_hi + A_hi B_lo
 * + A_lo B_hi, about FP32 accuracy) or HZ_MIXED_TF32 (one TF32 product, about 1e-3 relative
 * accuracy per transform, so the refinement needs more corrections) (x/y
 * eigen-transforms in FP32, the bulk ones on the tensor cores; z solves, the interface
 * residual and the refinement residual in FP64; FP64 iterative refinement until the
 * relative residual ||M f - A u|| / ||M f|| <= rtol for every RHS, at most max_refine
 * corrections; HZ_ERR_NOT_CONVERGED otherwise).  The mixed path carries transformed data
 * in FP32 (with tensor-core transforms the mode-space volumes are stored as complex64;
 * the z eliminations keep FP64 values): values below about 1e-30 or above 1e30 lose
 * precision there (the refinement then reports non-convergence rather than a wrong
 * answer), so scale such right-hand sides.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream). */
typedef struct {
  int precision;
  double rtol;
  int max_refine;
  void *cuda_stream;
} hz_options;

/* Per-solve report. */
typedef struct {
  int refinements;           /* corrections applied after the first solve (mixed path)  */
  double rel_residual;       /* max over RHS of ||M f - A u|| / ||M f|| when measured,
                                else -1                                                 */
  double min_abs_pivot;      /* smallest |pivot| over all z eliminations of the plan    */
  double plan_ms;            /* host + device time of the last plan / frequency set-up  */
  double eig_max_residual;   /* largest relative eigen-identity residual of the plan    */
  long long device_bytes;    /* device memory owned by the plan                         */
  long long kernel_launches; /* kernels launched by this plan's solves so far           */
  int nbx, nby;              /* block partition in use                                  */
  int tensor_cores;          /* 1: the mixed path's bulk transforms run on the tensor
                                cores (tcgen05, 3xTF32) with complex64 mode-space data;
                                0: FP32 CUDA-core transforms on complex128 data          */
  int fast_sine;             /* uniform blocks on the FFT-based sine transform: 0 none,
                                1 FP64 path, 2 both paths (hz_plan_set_fast_sine; 0 when
                                the plan has no such block)                              */
  int real_tables;           /* 1 when the mixed path's real block tables run the
                                real-table tensor-core kernel (hz_plan_set_real_tables)  */
  int z_sweep;               /* z sweep variant set (hz_plan_set_z_sweep; 0 automatic)  */
} hz_info;

/* Stage timers: when enabled, every solve records CUDA events on the plan's
 * stream around each stage and accumulates the elapsed milliseconds per stage
 * (HZ_STAGE_*), with the number of launches per stage.  Off by default. */
enum {
  HZ_STAGE_FWD = 0,       /* step 1: bulk forward x/y transforms (2 launches)          */
  HZ_STAGE_PASS_A = 1,    /* step 2: block z solves                                   */
  HZ_STAGE_EDGES = 2,     /* step 3: v next to the interfaces                          */
  HZ_STAGE_IRES = 3,      /* step 4: interface residual                                */
  HZ_STAGE_GLOBAL = 4,    /* step 5: global interface solve                            */
  HZ_STAGE_PASS_B = 5,    /* step 6: boundary terms and block z solves                  */
  HZ_STAGE_INV = 6,       /* step 7: bulk inverse x/y transforms (2 launches)          */
  HZ_STAGE_IFACE_OUT = 7, /* step 7: u = w on the interfaces                           */
  HZ_STAGE_RESID = 8,     /* refinement / residual stencil and norms                    */
  HZ_NSTAGES = 9
};
hz_status hz_set_stage_timing(hz_plan_t plan, int enable);   /* also resets the totals */
/* ms[HZ_NSTAGES] and launches[HZ_NSTAGES] (either may be NULL) receive the totals. */
hz_status hz_get_stage_times(hz_plan_t plan, double *ms, long long *launches);

/* Build a plan: 1D operators, per-block and global generalized eigenpairs
 * (K_d W = M_d W Lambda, W^T M_d W = I; the display after Eq. (fdmtrprj) and
 * before Eq. (fdmtrprjfrerr)), the z elimination factors of every mode, and all
 * device tables (for the tensor-core transforms also one TMA tensor map per tile, encoded
 * through the driver; if the driver offers no encoder, mixed plans use the CUDA-core FP32
 * transforms and hz_get_info reports tensor_cores = 0).  Errors: HZ_ERR_ARG on bad
 * sizes/pointers, HZ_ERR_EIG when an eigen-decomposition fails its checks,
 * HZ_ERR_SINGULAR on a singular pivot, HZ_ERR_OOM / HZ_ERR_CUDA on device failures.
 * *out is NULL on error. */
hz_status hz_plan_create(const hz_grid *grid, const hz_layers *layers, const hz_blocks *blocks,
                         const hz_options *opts, hz_plan_t *out);

/* Scale the base k^2 of every layer by omega^2 and rebuild the z factors
 * (Sec. 2: k^2 enters only the z operator, so the x/y eigen data are kept). */
hz_status hz_plan_set_frequency(hz_plan_t plan, double omega);

/* Replace the base per-layer k^2 (nlayers entries, host array) and rebuild the z
 * factors; the x/y eigen data are kept (k^2 enters only the z operator of
 * Eq. (fdmtrprjfr)).  The current frequency scaling omega^2 still applies. */
hz_status hz_plan_set_k2(hz_plan_t plan, const hz_c128 *k2);

/* Autotuner: times one solve of nrhs right-hand sides (on zero data, in the plan's
 * workspace) for each kernel variant the plan can use -- the three z sweep variants of
 * hz_plan_set_z_sweep, two row tiles of the dense CUDA-core transforms, for mixed plans tensor-core or CUDA-core FP32
 * bulk transforms and the real-table or interleaved tensor-core kernel, for plans with
 * uniform blocks the fast sine transform or the dense product -- and keeps the fastest.
 * *choice_out (may be NULL) receives
 * z_sweep + 10 * tensor_cores + 100 * fast_sine + 1000 * real_tables + 10000 * tile, with tile the
 * data rows per CTA of the dense CUDA-core transforms (FP64, and FP32 interface rows): 1 for 16,
 * 2 for 64 (untuned plans choose by launch size). */
hz_status hz_plan_autotune(hz_plan_t plan, int nrhs, int *choice_out);

/* Transform the uniform blocks (all steps equal and real, so that the block's eigenvectors
 * are the discrete sines and its tables a scaled DST-I) by the FFT-based sine transform, the
 * fast transform of the uniform core in the cost estimate of Sec. 2 (one complex FFT of
 * length n + 1 per row, for blocks whose n + 1 <= 128 has no prime factor above 5), or by
 * the dense product.  enable = 0: dense everywhere (the folded FP64 product on the FP64 path,
 * the tensor cores on the mixed path); 1 (the default): the FP64 path in FP64 through the
 * fast transform, the mixed path on the tensor cores; 2: also the mixed path's bulk
 * transforms through the fast transform, in FP32.  The autotuner times both choices of the
 * plan's path.  HZ_ERR_ARG for other values. */
hz_status hz_plan_set_fast_sine(hz_plan_t plan, int enable);

/* The mode-wise z eliminations of Eq. (fdmtrprjfr) and Eq. (fdmtrprjfrerr) (Thomas sweeps, one
 * thread per mode and right-hand side): variant 1 one right-hand side per thread, 2 two per
 * thread sharing each factor load (the mixed path's step-5/6 sweeps, which form their
 * right-hand side themselves, keep one), 3 one per thread with z taken in register chunks of 16 steps
 * (all loads of a chunk in flight together, one complex multiply-add on the dependency chain:
 * for few modes and long z, where the sweeps cannot fill the GPU); 0 (the default): variant 3
 * when a launch has fewer than 512 sweeps per SM, else 1.  Same elimination in FP64; variant 3
 * rounds the forward step in another order.  HZ_ERR_ARG for other values. */
hz_status hz_plan_set_z_sweep(hz_plan_t plan, int variant);

/* Data rows per CTA of the dense CUDA-core transforms (the FP64 block and whole-axis products of
 * Eq. (fdmtrprjfr) and step 5, and the mixed path's FP32 interface-row transforms): 16 or 64; 0
 * (the default) chooses 64 when a launch has at least two CTAs per SM, else 16.  The autotuner
 * times both.  Same result.  HZ_ERR_ARG for other values. */
hz_status hz_plan_set_dense_tile_rows(hz_plan_t plan, int rows);

/* Mixed path: blocks whose eigenvector tables are real (all their steps real) run the
 * tensor-core transform as two real products, Re C = Re A B and Im C = Im A B, each with K = N =
 * n (enable = 1, the default: 64 data rows per CTA, four CTAs per SM), or as one real GEMM of the
 * interleaved complex matrices with K = N = 2 n (enable = 0).  Same result up to FP32 rounding;
 * the autotuner times both.  Blocks with complex (PML) tables always use the interleaved form. */
hz_status hz_plan_set_real_tables(hz_plan_t plan, int enable);

/* Host-only helper (no device memory is touched): the fast sine transform that the plan
 * runs on the GPU, applied to one row: out[c] = scale sum_j in[g(j)] sin(pi j m / (n + 1)).
 * dir = 1 (forward table of a uniform block): in holds the nodes j = 1..n in order and
 * out the modes m in the symmetric-modes-first order (column c < (n + 1) / 2 is m = 2 c + 1,
 * then the even m); dir = 2 (inverse table): in holds the modes in that order and out the
 * nodes in order.  HZ_ERR_ARG if n + 1 > 128 or has a prime factor above 5, or n < 2. */
hz_status hz_sine_transform_host(int n, int dir, double scale, const hz_c128 *in, hz_c128 *out);

/* Change the options' stream, precision, rtol and max_refine of a plan. */
hz_status hz_plan_set_options(hz_plan_t plan, const hz_options *opts);

/* u = A^{-1} (M f): steps 1-7 of the algorithm in Sec. 2 for nrhs right-hand
 * sides.  f_dev, u_dev: device arrays (see above).  Stream-ordered on the
 * plan's stream; returns after the result is complete. */
hz_status hz_solve(hz_plan_t plan, const hz_c128 *f_dev, hz_c128 *u_dev, int nrhs);

/* The same solve with HOST arrays f_host, u_host (pageable or pinned): the call
 * copies f to the device, solves and copies u back.  With nrhs >= 2 the RHS are solved in
 * up to eight chunks: all uploads are queued at once on one copy stream, each chunk's
 * download starts on a second copy stream when its solve is done, so both overlap the
 * later chunks' solves (pinned buffers make the copies asynchronous).  info.refinements and
 * info.rel_residual are the maxima over the chunks. */
hz_status hz_solve_host(hz_plan_t plan, const hz_c128 *f_host, hz_c128 *u_host, int nrhs);

/* lam = A^{-H} g.  A is complex symmetric (Eq. (fdmtr) with symmetric K_d and
 * diagonal M_d), so A^H = conj(A) and the adjoint reuses the forward path:
 * lam = conj(A^{-1} conj(g)).  g is already in the weighted space (no M is
 * applied to it). */
hz_status hz_solve_adjoint(hz_plan_t plan, const hz_c128 *g_dev, hz_c128 *lam_dev, int nrhs);

/* Layered medium with a local perturbation of k^2 -- the paper's motivating use of the
 * layered solver as a fast preconditioner for media with embedded inhomogeneities (Sec. 1):
 *     -div(sigma grad u) - (k^2(z) + dk2(x, y, z)) u = f,  i.e.  (A - M diag(dk2)) u = M f.
 * Solved by restarted GMRES(restart) on the second-kind form u - S(dk2 u) = S f, where S is
 * this plan's layered solve (FP64 or mixed, per the plan's options; the Born term S f is the
 * initial guess; mixed plans keep the Krylov basis in complex64, combined in FP32 against
 * FP64 vectors, while the restart residuals and the iterate stay FP64).  dk2_dev: device complex [Nz][Ny][Nx], node-based, the same for every RHS;
 * f_dev, u_dev: as hz_solve (distinct buffers).  Stops when every RHS's GMRES residual is
 * <= rtol ||S f||; each iteration is one layered solve of all RHS.  iters_out (may be NULL):
 * iterations used; relres_out (may be NULL, else nrhs doubles): the true relative residual
 * ||M f - (A - M diag(dk2)) u|| / ||M f|| per RHS (FP64 stencil).  The Krylov basis,
 * (restart + 1) volumes of nrhs RHS (restart <= 0: 20), is allocated for the call and freed.
 * Errors: HZ_ERR_ARG; HZ_ERR_NOT_CONVERGED after max_iter iterations (u holds the last
 * iterate); errors of the inner solves. */
hz_status hz_solve_perturbed(hz_plan_t plan, const hz_c128 *dk2_dev, const hz_c128 *f_dev, hz_c128 *u_dev,
                             int nrhs, double rtol, int max_iter, int restart, int *iters_out,
                             double *relres_out);

/* Layer gradient G_L = sum_rhs sum_{k in L} hhat^z_k sum_ij conj(lam_ijk) hhat^x_i hhat^y_j u_ijk
 * for L = 0..nlayers-1, written to G_host (nlayers entries).  For a real misfit J whose
 * adjoint source is g = dJ/du* the result gives dJ/dRe k^2_L = Re G_L and
 * dJ/dIm k^2_L = -Im G_L (derivative of Eq. (fdmtr) in k^2). */
hz_status hz_grad_layers(hz_plan_t plan, const hz_c128 *u_dev, const hz_c128 *lam_dev, int nrhs,
                         hz_c128 *G_host);

/* Gradient in the right-hand side.  The solve is u = A^{-1} M f (Eq. (fdmtr), M = Mz (x)
 * My (x) Mx diagonal), so for a real objective J(u) with adjoint state lam = A^{-H} g,
 * g = dJ/du* (hz_solve_adjoint), the gradient in f is M^H lam:
 *     gf[r][k][j][i] = conj(hhat^x_i hhat^y_j hhat^z_k) lam[r][k][j][i].
 * lam_dev, gf_dev: device arrays of nrhs right-hand sides (layout as f); gf_dev may equal
 * lam_dev (in place).  Stream-ordered on the plan's stream; returns after the result is
 * complete.  Errors: HZ_ERR_ARG, HZ_ERR_CUDA. */
hz_status hz_grad_rhs(hz_plan_t plan, const hz_c128 *lam_dev, hz_c128 *gf_dev, int nrhs);

/* Relative residuals ||M f - A u||_2 / ||M f||_2 per RHS (FP64), into rel_host (nrhs). */
hz_status hz_residual(hz_plan_t plan, const hz_c128 *f_dev, const hz_c128 *u_dev, int nrhs,
                      double *rel_host);

/* Allocation-free residual check (the paper has no counterpart; it serves callers of
 * this library that cannot call cudaMalloc at the time of the check: serving or
 * real-time loops that forbid device allocation, since an allocation can synchronise the
 * device and fragment a memory pool, and frameworks that hand out all device memory
 * themselves).  Same result as hz_residual (per-RHS ||M f - A u||_2 / ||M f||_2 into
 * rel_host, nrhs entries) but all scratch is a fixed 263 KB device array inside the
 * library and no residual field is written; nothing is allocated (no cudaMalloc,
 * cudaFree or allocating library call).  nrhs must be <= 64, and the current device must
 * be the one the plan was created on (HZ_ERR_ARG otherwise).  The array is shared by
 * every call and plan on a device and keeps the last call's contents: calls that overlap
 * on the GPU race on it and must be serialised by the caller.  The first call on a device
 * looks the array's address up (make that first call before any stream capture).
 * Stream-ordered on the plan's stream; the call waits for that stream and returns with
 * the residuals on the host.  Errors as hz_residual. */
hz_status hz_residual_noalloc(hz_plan_t plan, const hz_c128 *f_dev, const hz_c128 *u_dev, int nrhs,
                              double *rel_host);

/* Batches (many independent solves replayed as one CUDA graph).  A batch holds nitems
 * (plan, nrhs) items -- different grids, layers and frequencies (one plan per model and
 * frequency) -- and nlanes concurrent streams (0 = 4), each with one workspace sized for
 * the largest item it runs.  hz_batch_solve captures, on the first call with a given set
 * of pointers, every item's solve into one graph: FP64 plans run steps 1-7 once; mixed
 * plans run the first solve, its FP64 residual, one correction and the final residual
 * (Sec. 2's algorithm per solve; the refinement is the mixed path's).  Later calls with
 * the same pointers replay the graph.  After the replay every item's residual is checked
 * on the host; a mixed item above its rtol gets further corrections eagerly on its plan's
 * own stream.  rel_host (nitems, may be NULL) receives each item's max relative residual.
 * f_dev[i], u_dev[i]: device arrays of item i (must differ).  A plan may appear in one
 * item only.  The batch does not own the plans (destroy the batch first). */
typedef struct hz_batch_s *hz_batch_t;
hz_status hz_batch_create(int nitems, const hz_plan_t *plans, const int *nrhs, int nlanes, hz_batch_t *out);
hz_status hz_batch_solve(hz_batch_t batch, const hz_c128 *const *f_dev, hz_c128 *const *u_dev,
                         double *rel_host);
/* Autotuner: tunes every plan of the batch (hz_plan_autotune), then times graph replays
 * with 1, 2, 4 and 8 lanes on the given inputs and keeps the fastest (*lanes_out). */
hz_status hz_batch_autotune(hz_batch_t batch, const hz_c128 *const *f_dev, hz_c128 *const *u_dev,
                            int *lanes_out);
/* Last replay's CUDA-event time (ms), kernels per replay, lanes in use. */
hz_status hz_batch_info(hz_batch_t batch, double *last_ms, long long *launches_per_replay, int *lanes);
hz_status hz_batch_destroy(hz_batch_t batch);

hz_status hz_get_info(hz_plan_t plan, hz_info *out);

hz_status hz_plan_destroy(hz_plan_t plan);

const char *hz_status_str(hz_status s);

/* Host-only helper (no device memory is touched): the generalised eigenpairs
 * K W = M W Lambda, W^T M W = I of the complex-symmetric tridiagonal pencil with
 * diagonal kd (n), off-diagonal ko (n-1) and diagonal M = diag(m) (n), as used
 * for every block and axis of a plan (display after Eq. (fdmtrprj)).  lam (n)
 * and W (n*n, row-major: W[i*n + l] is node i of mode l) are caller-owned.
 * *residual receives max(||K W - M W Lambda||_F / (||K||_F ||W||_F),
 * max |W^T M W - I|).  HZ_ERR_EIG if the iteration breaks down. */
hz_status hz_tridiag_eig(int n, const hz_c128 *kd, const hz_c128 *ko, const hz_c128 *m, hz_c128 *lam,
                         hz_c128 *W, double *residual);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H_ */
