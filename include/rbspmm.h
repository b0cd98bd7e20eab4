/*
 * rbspmm.h -- C ABI of the repeated-block SpMM library for one GB300 GPU (sm_103a).
 *
 * The library applies the discrete Navier-Stokes operators of arxiv 2508.06710 (the
 * face-to-cell divergence M, the cell-to-face gradient G, the Laplacian L = M G) to a
 * dense block of k right-hand sides at once (SpMM), instead of k separate SpMVs, and
 * builds a batched Jacobi-preconditioned CG Poisson solve on top of spmm, dot, axpy and
 * axty (the four basic operations of Sec. 1).  The k columns are the flow states of an
 * ensemble, the parameters of a multiple-parameter run (Sec. 3), or the identical planes
 * of a mesh extruded along a periodic direction (Sec. 2, repeated geometries).  The same
 * build also assembles on the device the operators those solves and steps need: the FVM
 * operators and their cell/face interpolators, the denser 13p / 27p Laplacians of Sec. 4.1,
 * and the coarse-to-fine maps of inline mesh refinement (Sec. 3.3).
 *
 * Conventions shared by every call
 *   - Dense blocks are row-major with the k columns of one row next to each other (the
 *     array-of-structures layout of Algorithm 1): entry (i, j) of X is X[i * ldx + j],
 *     ldx >= k.  X, Y, B are caller-owned DEVICE pointers unless a call says otherwise.
 *   - Every call is asynchronous on the given stream (0 = the legacy default stream),
 *     except where a call says it synchronises.  Nothing is thrown across the ABI: each
 *     call returns an rb_status; rb_last_error() gives the calling thread's last message.
 *   - rb_operator_create, rb_batch_create and rb_guess_create are the only calls that
 *     allocate device memory; the library owns that memory until the matching destroy.
 *     Every other call allocates nothing: scratch space is a caller-provided workspace
 *     whose size a *_workspace_bytes query returns.
 *   - Invalid arguments (null pointers, negative sizes, ld < k, k > RB_MAX_K, dtype
 *     mismatch) return RB_EINVAL before any work is queued.
 *   - Host threads: calls on different handles may run concurrently from different
 *     threads (the library's launch caches are per thread); calls on the same operator,
 *     batch or guess handle must not overlap (rb_tune_spmm and the solvers update the
 *     handle's state).
 */
#ifndef RBSPMM_H
#define RBSPMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* rb_stream_t; /* the same handle as cudaStream_t */

#define RB_MAX_K 64

typedef enum {
  RB_OK = 0,
  RB_EINVAL = 1,        /* invalid argument; nothing was queued */
  RB_ENOMEM = 2,        /* device allocation failed (only the *_create calls allocate) */
  RB_ECUDA = 3,         /* a CUDA runtime call failed; see rb_last_error() */
  RB_ENOCONV = 4,       /* a CG column reached max_iter before the tolerance */
  RB_EBREAKDOWN = 5,    /* a CG column met p.q <= 0 or a non-finite value */
  RB_ETIMEOUT = 6,      /* a bounded device-side wait gave up (persistent solve) */
  RB_EUNSUPPORTED = 7   /* a valid request this build does not implement */
} rb_status;

/* RB_DF64 ("double-float"): an FP64 number carried as the unevaluated sum hi + lo of two FP32
 * numbers (Dekker 1971), stored as an 8-byte pair {float hi; float lo;} with hi at the lower
 * address, hi = RN32(x), lo = RN32(x - hi).  About 48 significant bits; FP32's exponent range
 * (|x| above ~3.4e38 becomes infinite, |x| below ~1e-30 keeps fewer low bits).  Operators
 * (CSR only) and rb_spmm take it: the FP64 rate of GB300 is 1/64 of its FP32 rate, and the
 * error-free FP32 transformations of a double-float multiply-add take about twelve FP32
 * instructions, so the SpMM's k multiply-adds per entry run at FP32-pipe speed while moving
 * FP64's bytes.  rb_df64_split / rb_df64_join convert FP64 blocks. */
typedef enum { RB_F64 = 0, RB_F32 = 1, RB_DF64 = 2 } rb_dtype;
typedef enum { RB_CSR = 0, RB_SELL = 1, RB_AUTO = 2, RB_STENCIL = 3 } rb_format;

/* Message of the calling thread's last failed call ("" if none). Owned by the library. */
const char* rb_last_error(void);
/* Library version, e.g. "0.1.0". */
const char* rb_version(void);

/* Measured FMA throughput of the current GPU in TFLOP/s (2 flops per FMA) for RB_F64 or
 * RB_F32: eight independent FMA chains per thread on a full-occupancy grid, best of five
 * launches timed with CUDA events.  The arithmetic roof against which the FP64 SpMM and CG
 * kernels are measured (on GB300 they reach the FP64 rate before HBM bandwidth).
 * Synchronises `stream`; allocates nothing; a measurement utility, not part of the method. */
rb_status rb_fma_peak(rb_dtype dtype, double* tflops, rb_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Operator build: staggered symmetry-preserving FVM operators on Cartesian grids
 * (Sec. 3, semi-discrete equations (ns); Sec. 4, symmetry-preserving discretisation).
 *
 * The grid has n[d] cells along axis d (x, y, z), bounded by n[d] + 1 increasing node
 * coordinates nodes[d] (DEVICE pointers, float64).  An axis is periodic or bounded by
 * walls; faces on walls are excluded (no penetration), which gives homogeneous Neumann
 * conditions for the pressure.  Cells are numbered id = i + n[0] (j + n[1] k).  Faces are
 * numbered direction by direction (x, y, z); within a direction lexicographically with
 * x fastest, the face coordinate along its own axis running over 0..n-1 on a periodic
 * axis (face i separates cells i-1 mod n and i) and over 1..n-1 between walls.
 *   A_f = product of the two transverse cell widths, d_f = distance between the two cell
 *   centres adjacent to the face, Omega_s = A_f d_f.
 *   RB_FVM_DIVERGENCE  M (cells x faces):  +A_f in the cell below face f, -A_f above.
 *   RB_FVM_GRADIENT    G = -Omega_s^{-1} M^T (faces x cells): -1/d_f, +1/d_f.
 *   RB_FVM_LAPLACIAN   L = M G (cells x cells): A_f / d_f to each neighbour across f,
 *                      minus their sum on the diagonal (symmetric, zero row sums).
 * Requirements: n[d] >= 3 on a periodic axis, n[d] >= 2 between walls.
 * ------------------------------------------------------------------------------------ */
typedef enum {
  RB_FVM_LAPLACIAN = 0,
  RB_FVM_DIVERGENCE = 1,
  RB_FVM_GRADIENT = 2,
  RB_FVM_INTERP_C2S = 3, /* Gamma_{c->s} (faces x cells): 1/2 on the two cells of each face, the
                            cell-to-face interpolator of Eq. (ns) and of C = M U_s Gamma */
  RB_FVM_INTERP_S2C = 4  /* Gamma_{c->s}^T (cells x faces): 1/2 on each face of a cell; the
                            face-to-cell interpolator on grids with equal cell and face volumes */
} rb_fvm_kind;

typedef struct {
  int32_t n[3];
  int32_t periodic[3];
  const double* nodes[3];
} rb_grid_desc;

/* Rows, columns and nonzeros of the operator `kind` on `grid` (host outputs; no GPU work). */
rb_status rb_fvm_csr_size(const rb_grid_desc* grid, rb_fvm_kind kind, int32_t* n_rows, int32_t* n_cols,
                          int64_t* nnz);

/* Writes the CSR of `kind` times `scale` (e.g. -1 for the SPD Poisson matrix -L) into
 * caller-allocated DEVICE arrays: row_ptr[n_rows + 1], col_idx[nnz], vals[nnz] (float64).
 * Columns are sorted within each row.  Asynchronous on `stream`. */
rb_status rb_fvm_assemble(const rb_grid_desc* grid, rb_fvm_kind kind, double scale, int32_t* row_ptr,
                          int32_t* col_idx, double* vals, rb_stream_t stream);

/* Wider Laplacian stencils on a uniform periodic Cartesian grid (Sec. 4.1: the denser 13p and
 * 27p sparsity patterns measured beside the first-neighbour 7p of RB_FVM_LAPLACIAN).  The paper
 * fixes only the patterns; the values are volume-integrated like the FVM Laplacian (cell
 * volume V = h[0] h[1] h[2] times a pointwise Laplacian), so -L is symmetric positive
 * semi-definite with the constants as null space:
 *   RB_STENCIL_13P  the first and second neighbours along each axis: along axis d the
 *                   fourth-order difference (-u[-2] + 16 u[-1] - 30 u[0] + 16 u[+1] - u[+2])
 *                   / (12 h[d]^2), summed over the axes; needs n[d] >= 5.
 *   RB_STENCIL_27P  the 3 x 3 x 3 block on cubic cells (h[0] == h[1] == h[2] = h): weights
 *                   -128, 14, 3, 1 over 30 h^2 for the centre and the face, edge and corner
 *                   neighbours (leading error isotropic); needs n[d] >= 3.
 * Cells are numbered id = i + n[0] (j + n[1] k).  n and h are HOST arrays.  Writes the CSR
 * times `scale` into caller-allocated DEVICE arrays: row_ptr[N + 1], col_idx[kind N],
 * vals[kind N] (float64), N = n[0] n[1] n[2]; every row has exactly `kind` entries, columns
 * sorted.  RB_EINVAL (nothing launched) for an unknown kind, too few cells, a non-positive or
 * non-finite spacing, unequal spacings for 27p, kind N above 2^31 - 1, or a null output.
 * Asynchronous on `stream`. */
typedef enum { RB_STENCIL_13P = 13, RB_STENCIL_27P = 27 } rb_stencil_kind;
rb_status rb_stencil_assemble(const int32_t n[3], const double h[3], rb_stencil_kind kind, double scale,
                              int32_t* row_ptr, int32_t* col_idx, double* vals, rb_stream_t stream);

/* Coarse-to-fine maps of cell fields for inline mesh refinement (Sec. 3.3: the flow states
 * are developed on a coarser mesh and then mapped onto the target mesh, all k states at once
 * as one rectangular SpMM).  `fine` is a grid as above with an even number n[d] >= 4 of cells
 * along every axis; its coarse grid keeps every other node (coarse cell I = fine cells 2I and
 * 2I + 1 along each axis), so N_c = N / 8 cells, numbered the same way.  The paper does not
 * give the map; the reading here:
 *   RB_REFINE_PROLONG   P (N x N_c): along each axis, linear interpolation in the cell-centre
 *                       coordinate between the two coarse centres nearest to the fine centre
 *                       (across a periodic seam with the period added; next to a wall the two
 *                       coarse cells at the wall, extrapolating); the product of the three
 *                       axis weights, 8 entries per row; reproduces trilinear fields exactly.
 *   RB_REFINE_RESTRICT  R (N_c x N): the volume-weighted mean of the 8 children of each coarse
 *                       cell (keeps the integral of the field).
 *   RB_REFINE_PROLONG_T P^T (N_c x N): the transpose of P, entry for entry (the same values,
 *                       bit for bit); the restriction of residuals in the multigrid cycle of
 *                       the Poisson solve (Sec. 4, Appendix A).  Row lengths vary (8 to 125);
 *                       the total is the same 8 N entries.
 * Writes into caller-allocated DEVICE arrays row_ptr[rows + 1], col_idx[8 N], vals[8 N]
 * (float64), rows = N (P) or N_c (R, P^T); columns sorted.  RB_EINVAL (nothing launched) for
 * an unknown kind, an odd or too small axis, a null array, 8 N > 2^31 - 1, or (P^T) more
 * than 1900 coarse positions summed over the three axes.  Asynchronous on `stream`. */
typedef enum { RB_REFINE_PROLONG = 0, RB_REFINE_RESTRICT = 1, RB_REFINE_PROLONG_T = 2 } rb_refine_kind;
rb_status rb_refine_assemble(const rb_grid_desc* fine, rb_refine_kind kind, int32_t* row_ptr, int32_t* col_idx,
                             double* vals, rb_stream_t stream);

/* Cotangent-weight Laplacian of a triangle mesh (vertex-centred, per unit depth), the
 * unstructured operator of the extruded-airfoil case (Sec. 4.3).  The caller passes the
 * mesh (DEVICE: points[2 n_vert] as x,y pairs, triangles[3 n_tri] counter-clockwise) and
 * the CSR pattern of its vertex adjacency with the diagonal (DEVICE row_ptr, col_idx,
 * columns sorted).  Writes into vals[nnz] (DEVICE float64): off-diagonal
 * w_ij = (cot a_ij + cot b_ij) / 2 over the triangles sharing edge ij, clamped at 0,
 * diagonal -sum_j w_ij; and into area[n_vert] (DEVICE float64, may be NULL) the
 * barycentric dual areas (a third of each incident triangle).  status: DEVICE int64[2],
 * required: status[0] receives the number of clamped edges, status[1] is nonzero when the
 * pattern lacks an edge of a triangle or a diagonal entry (the values are then invalid).
 * Asynchronous on `stream`. */
rb_status rb_mesh_cot_laplacian(int32_t n_vert, const double* points, int32_t n_tri, const int32_t* triangles,
                                const int32_t* row_ptr, const int32_t* col_idx, int64_t nnz, double* vals,
                                double* area, int64_t* status, rb_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Operators: A = I_k (x) A~ stored once (Sec. 2, Eq. (1); memory remark of Sec. 3.1)
 * ------------------------------------------------------------------------------------ */
typedef struct {
  int32_t n_rows, n_cols;
  int64_t nnz;
  const int32_t* row_ptr; /* n_rows + 1, non-decreasing, row_ptr[0] = 0 */
  const int32_t* col_idx; /* nnz, each in [0, n_cols) */
  const double* vals;     /* nnz, finite */
  int32_t on_device;      /* 1: the three arrays are device memory; 0: host memory */
} rb_csr_desc;

/* Repeated-block descriptor.  k_max: the largest k that will be applied (<= RB_MAX_K).
 * extruded_nz > 0 marks an operator extruded along a periodic direction into Nz identical
 * planes: L3D = dz (I_Nz (x) A~) + T_z (x) diag(z_weight), T_z the periodic [1 -2 1]
 * across planes; rb_spmm then takes k == extruded_nz columns (one per plane) and applies
 * the whole L3D.  z_weight: n_rows weights (a_i / dz for a dual area a_i), device or
 * host as the CSR's on_device says; NULL when extruded_nz == 0.  Every row of an extruded
 * operator must store its diagonal entry (it may be zero; RB_EINVAL otherwise): the library's
 * copy holds dz a_ij with the -2 w_i of T_z folded into the diagonal. */
typedef struct {
  int32_t k_max;
  int32_t extruded_nz;
  const double* z_weight;
  double dz;
} rb_block_desc;

typedef struct rb_op* rb_op_t;

typedef struct {
  int32_t n_rows, n_cols;
  int64_t nnz;
  int32_t dtype, format;   /* rb_dtype, rb_format actually stored */
  int32_t sell_c, sell_sigma;
  int64_t sell_padded_nnz; /* stored entries including SELL padding */
  int64_t device_bytes;    /* device memory owned by the operator */
  int32_t has_diag;        /* every row has a nonzero diagonal entry (square operators) */
  int32_t extruded_nz;
} rb_op_info;

/* Copies and validates the CSR (monotone row_ptr, col_idx in range, finite values;
 * RB_EINVAL otherwise), converts values to `dtype` (RB_F32: round to nearest even; RB_DF64:
 * the pairs of rb_df64_split, CSR layout only, not extruded, values within FP32's range), and
 * lays it out in `format` (RB_SELL: sliced ELL with C = 32 rows per slice and rows sorted
 * by length within windows of sigma = 256 rows; RB_AUTO picks CSR).  Also stores the
 * inverse diagonal for Jacobi preconditioning when the operator is square.  Allocates;
 * synchronises `stream`. */
rb_status rb_operator_create(const rb_csr_desc* csr, const rb_block_desc* block, rb_dtype dtype, rb_format format,
                             rb_stream_t stream, rb_op_t* out);
/* The Laplacian of rb_fvm_assemble (RB_FVM_LAPLACIAN, times `scale`) as a matrix-free operator
 * (format RB_STENCIL): the repeated-block reuse of Sec. 2 taken to the structure of a Cartesian
 * grid, where every coefficient A_f / d_f is a product of per-axis quantities (two cell widths
 * and one inverse centre distance), so the operator is held as 2 (n_x + n_y + n_z) + 3 numbers
 * and an SpMM reads only X and writes only Y.  The coefficients are formed in `dtype`
 * arithmetic from the tables (FP32: the tables rounded to nearest, so entries can differ from
 * RNE(FP64 entries) by a few ulp; RB_DF64: blocks of pairs, the entries factorised as
 * V_ijk c_nb with V = w_x w_y w_z and per-axis tables c = ic / w formed in FP64 and split, the
 * products and sums in double-float arithmetic).  The handle works with rb_spmm, rb_tune_spmm,
 * rb_operator_info/check/destroy and every call built on rb_spmm (e.g. rb_galerkin_guess); the
 * CG solves take it (RB_F32) as their inner operator (A_inner of rb_cg_solve, ops_inner of
 * rb_batch_create) and their FP64 operator as CSR.  grid as for rb_fvm_assemble (DEVICE nodes).
 * Allocates; synchronises `stream`. */
rb_status rb_fvm_stencil_create(const rb_grid_desc* grid, double scale, rb_dtype dtype, int32_t k_max,
                                rb_stream_t stream, rb_op_t* out);

rb_status rb_operator_destroy(rb_op_t op);

/* Scheduling hint for a CSR operator whose rows form n_blocks (<= 3) consecutive blocks that
 * address the same columns in the same order: the x-, y- and z-face rows of the gradient G, each
 * block sweeping all cells.  The SpMM without staging then takes row tiles from the blocks in
 * turn, so that the tiles gathering one region of X run together and X is read from HBM about
 * once instead of once per block.  starts: HOST array of the blocks' first rows (starts[0] = 0,
 * increasing, < n_rows).  n_blocks = 1 removes the hint.  Results do not change (each row's
 * sum is the same); RB_EINVAL for invalid starts or a non-CSR operator. */
rb_status rb_operator_set_row_blocks(rb_op_t op, int32_t n_blocks, const int32_t* starts);
rb_status rb_operator_info(rb_op_t op, rb_op_info* info);
/* Synchronises `stream` and reports whether a kernel applying `op` since the last check gave
 * up a bounded wait on its shared-memory pipeline (RB_ETIMEOUT; the affected outputs are
 * invalid).  Clears the condition. */
rb_status rb_operator_check(rb_op_t op, rb_stream_t stream);

/* Y = A~ X with a per-column scale:  Y[i, j] = c[j] * sum_p val[p] X[idx[p], j]  (Algorithm 1).
 * X: n_cols x k (ldx), Y: n_rows x k (ldy), both of the operator's dtype (RB_DF64: pairs,
 * the CSR kernel without staging, each row's sum formed with TwoProd/TwoSum and within about
 * 2^-46 sum_p |val[p] X[idx[p], j]| of the exact value); c: k float64
 * DEVICE values or NULL (= 1).  For an extruded operator k must equal extruded_nz and
 * the full L3D is applied (c is then applied to the whole row).  X and Y must not
 * overlap.  Vector width, rows per block and lanes per row are chosen per (operator, k)
 * from the tuning table (rb_tune_spmm). */
rb_status rb_spmm(rb_op_t A, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t k, const double* c,
                  rb_stream_t stream);

/* FP64 block <-> double-float block (RB_DF64 pairs), n x k, leading dimensions in elements
 * (pairs count as one element):  rb_df64_split: D[i, j] = (RN32(x), RN32(x - RN32(x))) for
 * x = X[i, j] (|x| above FP32's range gives infinite pairs);  rb_df64_join: X[i, j] =
 * RN64(hi + lo).  DEVICE blocks, 8-byte aligned, not overlapping; RB_EINVAL otherwise. */
rb_status rb_df64_split(int64_t n, int32_t k, const double* X, int64_t ldx, void* D, int64_t ldd, rb_stream_t stream);
rb_status rb_df64_join(int64_t n, int32_t k, const void* D, int64_t ldd, double* X, int64_t ldx, rb_stream_t stream);

/* Times the candidate SpMM schedules for (A, k) on scratch copies of X/Y shapes and
 * stores the fastest in A's tuning table (synchronises; X, Y as for rb_spmm, their
 * contents are overwritten: Y only). */
rb_status rb_tune_spmm(rb_op_t A, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t k, rb_stream_t stream);

/* Schedule of the SpMM kernels for k columns (what rb_tune_spmm chooses among):
 *   vec      columns per thread (1, 2, 3 or 4; 8- and 16-byte groups are vector accesses)
 *   lpr      lanes sharing one row's nonzeros (1, 2, 4, 8), reduced with warp shuffles
 *   stage    0: indices and values read by the row's lanes directly; 1: a block's nonzeros
 *            staged in shared memory by its threads; 2: a producer warp streams each tile's
 *            row pointers, indices and values into a 3-stage shared-memory ring with TMA bulk
 *            copies (cp.async.bulk + mbarrier) while eight consumer warps compute
 *   grid_cap -1: one resident wave of persistent blocks; 0: one block per row block; > 0: cap
 * rb_set_spmm_schedule pins a schedule for (A, k) (RB_EINVAL if it is not valid for A);
 * rb_get_spmm_schedule reports the one rb_spmm will use for k with the given layout. */
typedef struct {
  int32_t vec, lpr, stage, grid_cap;
} rb_spmm_schedule;
rb_status rb_set_spmm_schedule(rb_op_t A, int32_t k, const rb_spmm_schedule* sched);
rb_status rb_get_spmm_schedule(rb_op_t A, int32_t k, int64_t ldx, int64_t ldy, const void* X, const void* Y,
                               rb_spmm_schedule* sched);

/* ------------------------------------------------------------------------------------
 * The other basic operations, per column of an n x k block (Sec. 1: dot, axpy, axty)
 * ------------------------------------------------------------------------------------ */
/* Workspace (device bytes) that rb_dot needs for (n, k). */
size_t rb_dot_workspace_bytes(int64_t n, int32_t k);
/* out[j] = sum_i X[i, j] Y[i, j] (float64 accumulation, fixed summation order: the result
 * is bit-reproducible for a given n, k).  out: k float64 DEVICE values.  work: device
 * scratch of rb_dot_workspace_bytes(n, k) bytes, 16-byte aligned, contents ignored. */
rb_status rb_dot(int64_t n, int32_t k, rb_dtype dtype, const void* X, int64_t ldx, const void* Y, int64_t ldy,
                 double* out, void* work, size_t work_bytes, rb_stream_t stream);
/* rb_dot without a workspace, for callers that cannot give the library device memory (a
 * plain C program or a plugin that does not own the GPU's memory pool, or a code path that
 * must not call cudaMalloc / cudaFree because they can synchronise the device).  The paper
 * has no counterpart: this is a property of the library, not of the method.  Same result and
 * arguments as rb_dot minus the workspace; it allocates nothing and keeps its partial sums in
 * a fixed 128 KiB array (256 blocks x RB_MAX_K columns) in the library's device memory,
 * which every GPU that loads the library holds until the process exits.  k > RB_MAX_K is
 * rejected with RB_EINVAL.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call outside any stream capture.
 * All calls share the array: calls whose kernels can overlap on the GPU (other streams,
 * other host threads) race on it and must be ordered by the caller. */
rb_status rb_dot_noalloc(int64_t n, int32_t k, rb_dtype dtype, const void* X, int64_t ldx, const void* Y,
                         int64_t ldy, double* out, rb_stream_t stream);
/* Y[:, j] += alpha[j] X[:, j]; alpha: k float64 DEVICE values. */
rb_status rb_axpy(int64_t n, int32_t k, rb_dtype dtype, const double* alpha, const void* X, int64_t ldx, void* Y,
                  int64_t ldy, rb_stream_t stream);
/* Y[i, j] = alpha X[i, j] Y[i, j]  (the element-wise product of Sec. 1 and Sec. 3.1), each
 * entry rounded as (alpha x) y; alpha == 1 (after conversion to the block's type) computes the
 * single product x y, which is the same value. */
rb_status rb_axty(int64_t n, int32_t k, rb_dtype dtype, double alpha, const void* X, int64_t ldx, void* Y,
                  int64_t ldy, rb_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Poisson solve: Jacobi-preconditioned CG on k independent columns sharing one operator
 * (the pressure solve of the projection method, Sec. 4; the k flow states of Sec. 3).
 * ------------------------------------------------------------------------------------ */
typedef struct {
  double rtol;           /* stop when ||b - A x||_2 <= rtol ||b||_2 (true residual, FP64) */
  int32_t max_iter;      /* CG iterations (inner iterations summed when mixed) */
  int32_t precond;       /* 0: none, 1: Jacobi */
  int32_t mixed;         /* 0: FP64 CG; 1: FP32-inner CG inside FP64 iterative refinement, each
                            sweep restarting the inner CG; 2: the same refinement with reliable
                            updates: the inner recurrence keeps its search direction across
                            sweeps (rescaled) and only its residual is replaced by the FP64
                            one, which keeps the iteration count near that of FP64 CG */
  double inner_rtol;     /* mixed: the residual reduction of each sweep (e.g. 5e-2 for mixed = 2,
                            1e-4 for mixed = 1); a sweep stops earlier when half of what the
                            outer tolerance still needs is a smaller reduction.  The k columns
                            of a sweep iterate together: one that met its target keeps
                            iterating until all have (its share of the SpMM is paid anyway) */
  int32_t max_sweeps;    /* mixed: refinement sweeps */
  int32_t project_mean;  /* 1: singular periodic/Neumann operator; remove the column mean of
                            every true residual and of the final x (zero-mean solution) */
  int32_t check_every;   /* iterations between host convergence checks (>= 1) */
  int32_t persistent;    /* mixed only: 1 runs each sweep's inner iterations in one cooperative
                            launch (grid-wide barriers instead of kernel boundaries) */
} rb_cg_params;

typedef struct {
  int32_t iters[RB_MAX_K];       /* CG iterations per column (inner iterations when mixed) */
  double true_rel_res[RB_MAX_K]; /* ||b - A x|| / ||b|| at exit, FP64 */
  int32_t status[RB_MAX_K];      /* rb_status per column */
  int32_t spmm_calls;            /* operator applications (all columns at once) */
  int32_t sweeps;                /* refinement sweeps (mixed) */
  int32_t host_syncs;            /* device-to-host convergence reads */
  double ms;                     /* wall time of the call */
} rb_cg_report;

/* Device workspace for rb_cg_solve on (A, k, params). */
size_t rb_cg_workspace_bytes(rb_op_t A, int32_t k, const rb_cg_params* params);

/* Solves A x_j = b_j for the k columns.  A: square FP64 operator with a diagonal.
 * A_inner: the same matrix stored as RB_F32, required when params->mixed (else NULL): a CSR
 * copy, or the matrix-free Laplacian of the same grid (rb_fvm_stencil_create, RB_F32, the same
 * scale), whose inner iterations read no matrix.
 * B (n x k, ldb), X (n x k, ldx; in: initial guess, out: solution): float64 DEVICE.
 * work: device scratch of rb_cg_workspace_bytes bytes.  Synchronises `stream` (the host
 * reads the per-column state every check_every iterations).  Returns the worst column
 * status (RB_OK, RB_ENOCONV or RB_EBREAKDOWN); report (may be NULL) gets per-column
 * details. */
rb_status rb_cg_solve(rb_op_t A, rb_op_t A_inner, const rb_cg_params* params, const double* B, int64_t ldb,
                      double* X, int64_t ldx, int32_t k, void* work, size_t work_bytes, rb_cg_report* report,
                      rb_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Batched Poisson solves of uneven systems in one persistent launch under a CUDA graph
 * (the coarse and fine meshes of the inline mesh refinement of Sec. 3.3, or independent
 * meshes).  Each system s has its own operator (FP64 ops[s] and its FP32 copy
 * ops_inner[s]) and k[s] right-hand sides; the solve is the FP32-inner refinement of
 * rb_cg_solve (params->mixed 1 or 2) for every system at once: per sweep the FP64 residual
 * and the inner set-up run per system, then ONE cooperative kernel performs all inner CG
 * iterations of all systems, with the blocks shared among the systems in proportion to their
 * work and grid-wide barriers between the phases of an iteration.  The whole sequence of
 * max_sweeps sweeps is recorded once as a CUDA graph (per set of B/X pointers) and replayed
 * with one launch per call; systems that have converged skip their work inside the graph.
 * ------------------------------------------------------------------------------------ */
typedef struct rb_batch* rb_batch_t;

/* Allocates the per-system workspaces and the launch state.  n_sys <= 8, sum of k <= 64,
 * every ops[s] square RB_F64 CSR with a diagonal, ops_inner[s] its RB_F32 copy (CSR, or the
 * matrix-free Laplacian of the same grid as for rb_cg_solve). */
rb_status rb_batch_create(int32_t n_sys, const rb_op_t* ops, const rb_op_t* ops_inner, const int32_t* k,
                          const rb_cg_params* params, rb_batch_t* out);
rb_status rb_batch_destroy(rb_batch_t batch);

/* Solves every system: B[s] (n_s x k[s], ldb[s]) and X[s] (initial guess in, solution out,
 * ldx[s]) are float64 DEVICE arrays.  reports: n_sys entries (may be NULL).  Synchronises
 * `stream` once at the end.  Returns the worst status; RB_ETIMEOUT if a grid barrier wait
 * gave up (the solutions are then invalid). */
rb_status rb_batch_solve(rb_batch_t batch, const double* const* B, const int64_t* ldb, double* const* X,
                         const int64_t* ldx, rb_cg_report* reports, rb_stream_t stream);

/* Autotuner: times rb_batch_solve for each candidate launch shape (resident blocks per SM)
 * and inner tolerance on the given right-hand sides, starting each trial from X = 0 (X is
 * overwritten), and keeps the fastest for later solves.  *best_ms (may be NULL) gets its time. */
rb_status rb_batch_tune(rb_batch_t batch, const double* const* B, const int64_t* ldb, double* const* X,
                        const int64_t* ldx, double* best_ms, rb_stream_t stream);

/* Failure-detection knob for tests: the grid barrier waits at most timeout_ms and, with
 * extra_arrivals > 0, for more blocks than the launch has, so that its wait runs out and the
 * solve returns RB_ETIMEOUT.  Defaults: 2000 ms, 0. */
rb_status rb_batch_set_barrier(rb_batch_t batch, double timeout_ms, int32_t extra_arrivals);

/* ------------------------------------------------------------------------------------------
 * Multigrid-preconditioned CG for the Poisson matrix A = -L of a Cartesian FVM grid
 * (Sec. 4: the paper solves the pressure equation by CG with a multigrid preconditioner;
 * Appendix A, Table 9: the SpMMs of its levels, restrictions and prolongations).
 *
 * The paper's hierarchy is algebraic and comes from a closed library; this one is geometric,
 * built on the device from the library's own assemblies: level l + 1 keeps every other node
 * of level l (an axis is halved while its cell count is even and its half is >= min_cells),
 * A_l = -L rediscretised on each level (rb_fvm_assemble), the trilinear prolongation P_l and
 * its transpose as the restriction (rb_refine_assemble: RB_REFINE_PROLONG, _PROLONG_T), and
 * the coarsest level (at most 4096 cells) solved exactly through a dense inverse of
 * A_L + s 1 1^T (s > 0), formed on the device when the hierarchy is built; on the zero-mean
 * right-hand sides of the singular periodic / Neumann operator it gives the zero-mean
 * solution.  The preconditioner z = B r is one V(nu, nu) cycle from a zero guess with damped
 * Jacobi smoothing (weight omega): nu sweeps, residual, restriction, the next level's cycle,
 * prolongation-add, nu sweeps.  All k columns go through each kernel together.
 * ------------------------------------------------------------------------------------------ */
typedef struct rb_mg* rb_mg_t;

typedef struct {
  int32_t nu;         /* Jacobi sweeps before and after the coarse correction (1..16; 2) */
  double omega;       /* Jacobi damping weight in (0, 1] (0.8: the smoothing analysis of damped
                         Jacobi for the 2-D and 3-D Poisson stencils gives 4/5 and 6/7) */
  int32_t min_cells;  /* an axis is halved only if its half keeps >= min_cells cells (>= 2; 4) */
  int32_t flexible;   /* 1: flexible CG beta = -alpha (q . z_new) / (r . z)_old (Notay), robust
                         to an FP32 cycle; 0: beta = (r . z)_new / (r . z)_old (1) */
  int32_t matrix_free; /* 1: the FP32 cycle and the FP32 CG apply -L and the transfers from
                          per-axis tables (rb_fvm_stencil_create; no matrix bytes); 0: the CSR
                          operators (1) */
  int32_t smoother;    /* 0: point Jacobi; 1: line Jacobi along the wall-bounded axis whose
                          couplings exceed the others' by a factor >= 4 somewhere (a grid refined
                          towards its walls: point smoothing stalls there), each grid line along
                          it relaxed at once by a tridiagonal solve; point Jacobi when there is
                          no such axis (1) */
} rb_mg_params;

#define RB_MG_MAX_LEVELS 16
typedef struct {
  int32_t levels;
  int32_t n[RB_MG_MAX_LEVELS][3];  /* cells along x, y, z, level by level (fine first) */
  int64_t nnz_A[RB_MG_MAX_LEVELS]; /* nonzeros of -L on the level */
  int64_t nnz_P[RB_MG_MAX_LEVELS]; /* nonzeros of P from the next level (0 on the coarsest) */
  int64_t device_bytes;            /* device memory the hierarchy holds */
  int32_t line_axis;               /* the line smoother's axis, -1 for point Jacobi */
} rb_mg_info_t;

/* Builds the hierarchy of `grid` (as for rb_fvm_assemble; nodes are DEVICE float64) for up to
 * k_max columns, every level in FP64 and FP32, with level and solve vectors for k_max
 * columns.  params NULL = the defaults above.  Allocates (the library owns the memory until
 * rb_mg_destroy); synchronises `stream`.  RB_EINVAL for invalid parameters, an axis too small
 * for rb_fvm_assemble, or a grid beyond int32 indexing; RB_EINVAL also when the coarsest
 * level would keep more than 4096 cells (the grid does not halve often enough). */
rb_status rb_mg_create(const rb_grid_desc* grid, int32_t k_max, const rb_mg_params* params, rb_stream_t stream,
                       rb_mg_t* out);
rb_status rb_mg_destroy(rb_mg_t mg);
rb_status rb_mg_info(rb_mg_t mg, rb_mg_info_t* info);

/* One V-cycle z = B_l r on level `level` (its cells, numbered as on the grid), in `dtype`
 * arithmetic (RB_F64, or RB_F32: operators and vectors in FP32).  R (in), Z (out): float64
 * DEVICE n_l x k blocks (ldr, ldz >= k), k <= k_max.  level = L - 1 applies the coarsest
 * level's dense inverse.  Calls on one hierarchy must not overlap (it holds the level
 * vectors).  Asynchronous on `stream`; allocates nothing. */
rb_status rb_mg_vcycle(rb_mg_t mg, int32_t level, rb_dtype dtype, const double* R, int64_t ldr, double* Z,
                       int64_t ldz, int32_t k, rb_stream_t stream);

/* Solves A x_j = b_j for k <= k_max columns by PCG (Saad, Alg. 9.1) preconditioned by one
 * V-cycle per iteration.  params: rtol (true relative residual ||b - A x|| / ||b||, the mean
 * removed from both when project_mean), max_iter, check_every (iterations between host
 * reads of the per-column state), project_mean, and
 *   mixed = 0: FP64 CG and cycle; the true residual is checked every check_every iterations
 *              (columns stop at the first check that meets rtol);
 *   mixed != 0: FP64 iterative refinement around the same PCG run in FP32 (operators,
 *              vectors and cycle; dot products summed in FP64 across threads): each sweep
 *              solves A d = r / ||r|| to inner_rtol (or to half of what rtol still needs,
 *              when that is looser) and updates x += ||r|| d in FP64; at most max_sweeps.
 * precond and persistent are ignored.  B (ldb), X (ldx; in: initial guess, out: solution,
 * zero-mean with project_mean): float64 DEVICE.  Synchronises `stream`; allocates nothing
 * (the hierarchy holds the vectors and CUDA graphs of the iterations, recorded on first use
 * for each k).  Returns the worst column status; report (may be NULL) as for rb_cg_solve
 * (iters: CG iterations, over all sweeps when mixed; spmm_calls: FP64 residuals). */
rb_status rb_mg_solve(rb_mg_t mg, const rb_cg_params* params, const double* B, int64_t ldb, double* X, int64_t ldx,
                      int32_t k, rb_cg_report* report, rb_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * The projection step on m stacked flow states (Sec. 3, Eq. (ns) and Eq. (ns-nrhs): every
 * operator acts as I_m (x) A, one SpMM over the states' columns; Sec. 4: Heun's third-order
 * Runge-Kutta scheme, c = (0, 1/3, 2/3), a_21 = 1/3, a_32 = 2/3, b = (1/4, 0, 3/4), with a
 * projection at every stage), sequenced in the library on rb_spmm, rb_axpy, rb_axty and the
 * Poisson solvers.  With cell velocities u_c, face velocities u_s, cell volume V:
 *   derivative  F = (nu L u_c - M (u_s * Gamma u_c)) / V, Gamma the cell-to-face
 *               interpolator (RB_FVM_INTERP_C2S), * the element-wise product (rb_axty);
 *   projection  u~_s = the face-normal component of Gamma u~ on each face, -L p =
 *               -M u~_s / (c dt) solved to zero mean (the previous solve of the same stage is
 *               the initial guess), u_s = u~_s - c dt G p, u_c = u~ - c dt G_c p with G_c p's
 *               component d = Gamma^T (G p on the faces of direction d).
 * Layout (DEVICE float64): u_c n x 3 m (ldu >= 3 m), column i m + s = component i of state
 * s; u_s n_faces x m (lds >= m), n_faces = 3 n, numbered as for rb_fvm_assemble (the x faces
 * first, then y, then z; on a periodic axis n faces per direction).  The grid must be uniform
 * and periodic along every axis (one cell volume; Gamma^T the face-to-cell interpolator).
 * ------------------------------------------------------------------------------------------ */
typedef struct rb_projection* rb_projection_t;
typedef enum { RB_PROJ_JACOBI = 0, RB_PROJ_MG = 1 } rb_proj_solver;

typedef struct {
  int32_t m;          /* stacked states, 3 m <= RB_MAX_K */
  double nu;          /* kinematic viscosity (>= 0) */
  double dt;          /* time step (> 0) */
  int32_t solver;     /* RB_PROJ_JACOBI: rb_cg_solve (mixed 0, 1 or 2); RB_PROJ_MG: rb_mg_solve
                         on the grid's multigrid hierarchy (mixed 0 or nonzero) */
  rb_cg_params cg;    /* the pressure solves' parameters; project_mean must be 1 */
} rb_projection_params;

typedef struct {
  int32_t iters[3];   /* the stages' pressure solves: CG iterations, the largest over the states */
  int32_t status;     /* the worst solve status (RB_OK, RB_ENOCONV, RB_EBREAKDOWN) */
  double poisson_ms;  /* wall time of the solves */
} rb_projection_report;

/* Builds the step's operators (M, G, L, Gamma, Gamma^T, the Poisson matrix -L in FP64 and, for
 * the Jacobi refinement, FP32; or the multigrid hierarchy), work vectors and column scales
 * for `grid` (as for rb_fvm_assemble, DEVICE nodes).  Allocates (the library owns the memory
 * until rb_projection_destroy); synchronises `stream`.  RB_EINVAL for a non-uniform or
 * non-periodic grid, axes below 3 cells, invalid parameters. */
rb_status rb_projection_create(const rb_grid_desc* grid, const rb_projection_params* params, rb_stream_t stream,
                               rb_projection_t* out);
rb_status rb_projection_destroy(rb_projection_t p);
/* One Heun RK3 step of the m states; u_c and u_s are updated in place.  Synchronises `stream`
 * (the solves read their convergence on the host).  Returns the worst solve status; report
 * may be NULL.  Calls on one handle must not overlap. */
rb_status rb_projection_step(rb_projection_t p, double* u_c, int64_t ldu, double* u_s, int64_t lds,
                             rb_projection_report* report, rb_stream_t stream);
/* One projection with time cdt (> 0): u_c becomes divergence-free-consistent cell velocities
 * in place and u_s receives the projected face velocities (the mapping of inline mesh
 * refinement, Sec. 3.3, projects the prolonged velocities this way).  Uses the third stage's
 * pressure as the initial guess; report->iters[0] holds the solve's iterations. */
rb_status rb_projection_project(rb_projection_t p, double cdt, double* u_c, int64_t ldu, double* u_s, int64_t lds,
                                rb_projection_report* report, rb_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Galerkin initial guess: the best combination of candidate starting vectors.
 *
 * Not from the paper, whose solver starts each step from the previous pressure.  For k
 * systems A x_j = b_j sharing A (SPD, or semi-definite with compatible b_j) and n_cand <= 3
 * candidate blocks V_a (say the previous two pressures and the learned guess), column j gets
 * x0_j = sum_a c_aj V_a[:, j] with (V_j^T A V_j) c_j = V_j^T b_j: the Ritz-Galerkin projection
 * (Saad, Iterative Methods, Sec. 5.1), which minimises the A-norm of the error over the span
 * of the candidates, so x0 is never worse than any one of them.  Dependent candidates get
 * coefficient 0 (a Cholesky that skips pivots below 1e-12 of their diagonal); if rounding
 * leaves the combination's energy x^T A x / 2 - b^T x above the best single candidate's, that
 * candidate is taken instead.  One SpMM per candidate, one fused reduction, one
 * elementwise pass.
 * ------------------------------------------------------------------------------------------ */

/* Workspace bytes for n rows, k columns and n_cand candidates (0 for invalid sizes). */
size_t rb_galerkin_workspace_bytes(int64_t n, int32_t k, int32_t n_cand);

/* A: square FP64 operator (n x n).  cand: HOST array of n_cand DEVICE pointers to n x k
 * float64 blocks with leading dimensions ldc[a] (host array); B (ldb), X0 (ldx): float64
 * DEVICE n x k blocks; X0 may be one of the candidates.  coef: DEVICE k x n_cand doubles
 * (column j's coefficients at j * n_cand), or NULL.  work: DEVICE, 256-byte aligned,
 * rb_galerkin_workspace_bytes bytes.  Asynchronous on `stream`; allocates nothing.
 * RB_EINVAL for null pointers, k outside [1, 64], n_cand outside [1, 3], ld < k, a non-square
 * or FP32 operator, or a small workspace. */
rb_status rb_galerkin_guess(rb_op_t A, int32_t k, int32_t n_cand, const double* const* cand, const int64_t* ldc,
                            const double* B, int64_t ldb, double* X0, int64_t ldx, double* coef, void* work,
                            size_t work_bytes, rb_stream_t stream);

/* ------------------------------------------------------------------------------------------
 * Learned initial guess for the pressure Poisson solve.
 *
 * The paper's projection step (Sec. 3; the Poisson solve that dominates Sec. 4) solves
 * A p_t = b_t every time step.  The paper has no learned component: this is an addition on
 * top of it.  A 3-D U-Net maps the right-hand side b_t and the two previous pressures
 * p_{t-1}, p_{t-2} on a Cartesian grid to a guess of p_t; CG then always runs from the
 * better of that guess and p_{t-1} (rb_guess_select) to the same tolerance, so the guess
 * can only change the iteration count, never the answer.
 *
 * Network (levels L, channels c_0..c_{L-1}): at level l (the grid coarsened 2^l times) two
 * 3x3x3 convolutions with bias and ReLU; 2x2x2 average pooling between levels; on the way up
 * a 2x2x2 stride-2 transposed convolution (with bias, no activation) whose c_l outputs are
 * concatenated with the level's encoder output (up-sampled channels first), then two 3x3x3
 * convolutions with ReLU; a 1x1x1 head to one channel.  Padding is circular along periodic
 * axes and zero along walled ones.  Inputs are scaled, x = (b / s_b, p_{t-1} / s_p,
 * p_{t-2} / s_p) with s_b = rms(b), s_p = rms(p_{t-1}) (1 for a zero field), and the guess is
 * p = p_{t-1} - mean(p_{t-1}) + s_p (y - mean(y)) for the head output y.
 *
 * Precision: weights and activations in BF16 (round to nearest even), products accumulated
 * in FP32 on the tensor cores (tcgen05, accumulators in tensor memory); FP32 master weights,
 * gradients and Adam moments; FP64 scalars (scales, means, loss).
 *
 * Parameter vector (FP32, rb_guess_param_count entries), layer by layer in the order
 *   enc0a enc0b enc1a enc1b ... enc{L-1}a enc{L-1}b,
 *   then for l = L-2 down to 0: up{l} dec{l}a dec{l}b, and the head;
 * each layer its weights then its biases; a 3x3x3 convolution's weights as
 * [c_out][dz][dy][dx][c_in] (offsets -1..1, x fastest), a transposed convolution's as
 * [c_out][a][b][c][c_in] (a, b, c the z, y, x offsets 0..1 of the fine cell), the head's as
 * [c_0].  enc0a has c_in = 3.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
  int32_t nx, ny, nz;  /* cells, x fastest; each divisible by 2^(levels-1) */
  int32_t levels;      /* 2 .. 4 */
  int32_t channels[4]; /* c_l per level, multiples of 8; each 3x3x3 convolution's BF16 weights,
                          54 c_in roundup16(c_out) bytes (also with c_in and c_out swapped),
                          must fit in 160 KB of shared memory (e.g. c = 8, 16, 32, 48) */
  int32_t periodic[3]; /* x, y, z: 1 circular padding (periodic axis), 0 zero padding (walls) */
} rb_guess_cfg;

typedef struct rb_guess* rb_guess_t;

typedef struct {
  double lr, beta1, beta2, eps; /* Adam (Kingma and Ba 2015, Algorithm 1) */
} rb_adam_params;

/* Number of FP32 parameters of the network that cfg describes. */
rb_status rb_guess_param_count(const rb_guess_cfg* cfg, int64_t* n);

/* Allocates the network for one grid: parameters (zero until rb_guess_set_params), Adam
 * moments, gradients and every activation buffer (about 40 bytes per cell and channel of
 * level 0).  Synchronises.  RB_EINVAL for a grid or channel list outside the limits above. */
rb_status rb_guess_create(const rb_guess_cfg* cfg, rb_guess_t* out);
rb_status rb_guess_destroy(rb_guess_t g);

/* He initialisation from given N(0, 1) draws (device, rb_guess_param_count floats): every
 * weight = draw * sqrt(2 / fan_in) (fan_in 27 c_in for a 3x3x3 convolution, c_in for the
 * transposed convolution and the head), the head's weights further times head_scale, biases
 * zero; then as rb_guess_set_params. */
rb_status rb_guess_init_params(rb_guess_t g, const float* normals, double head_scale, rb_stream_t stream);

/* Copy the FP32 parameter vector in / out (device pointers, rb_guess_param_count entries).
 * Setting parameters also refreshes the BF16 copies and resets the Adam step count. */
rb_status rb_guess_set_params(rb_guess_t g, const float* theta, rb_stream_t stream);
rb_status rb_guess_get_params(rb_guess_t g, float* theta, rb_stream_t stream);
/* The accumulated parameter gradient (device, rb_guess_param_count entries). */
rb_status rb_guess_get_grad(rb_guess_t g, float* grad, rb_stream_t stream);

/* Guess p_out (device, n = nx ny nz doubles) from b, p1 = p_{t-1}, p2 = p_{t-2}. */
rb_status rb_guess_predict(rb_guess_t g, const double* b, const double* p1, const double* p2, double* p_out,
                           rb_stream_t stream);

/* Forward and backward pass for one training pair with target p (the solver's p_t): the
 * loss is mean_i (y_i - mean(y) - t_i + mean(t))^2 with t = (p - p1) / s_p, and its gradient
 * is added to the gradient buffer (zeroed first when accumulate == 0).  The loss is added
 * to *loss (device, may be NULL), so that one scalar can sum a minibatch or an epoch. */
rb_status rb_guess_loss_grad(rb_guess_t g, const double* b, const double* p1, const double* p2, const double* p,
                             int32_t accumulate, double* loss, rb_stream_t stream);

/* One Adam step on the accumulated gradient times grad_scale (e.g. 1 / batch), then zeroes
 * the gradient and refreshes the BF16 weights. */
rb_status rb_guess_adam_step(rb_guess_t g, const rb_adam_params* h, double grad_scale, rb_stream_t stream);

/* Inspection for tests: the output of layer `index` (flat-parameter order; -1 the scaled
 * input x with its 3 channels) of the last forward pass, as FP32 [cells of its level][c_out]
 * into out (device; NULL to query); *count receives the number of floats. */
rb_status rb_guess_read_activation(rb_guess_t g, int32_t index, float* out, int64_t* count, rb_stream_t stream);

/* The fallback and judge: each candidate (cand0, cand1: device, n doubles, not modified) is
 * first smoothed by `sweeps` damped Jacobi sweeps x <- x + omega D^-1 (b - A x) (D the
 * diagonal of A; 0 sweeps leaves it as is), then x0 = the smoothed candidate with the smaller
 * ||b - A x||_2, all on the device with rb_spmm and FP64 sums.  res[2] (device) receives
 * ||b - A x_i||_2 / ||b||_2 of both, *choice (device) the index taken.  A is the FP64
 * operator of the solve (n x n, with a diagonal when sweeps > 0); uses g's scratch, so calls
 * on one g must not overlap. */
rb_status rb_guess_select(rb_guess_t g, rb_op_t A, const double* b, const double* cand0, const double* cand1,
                          int32_t sweeps, double omega, double* x0, double* res, int32_t* choice,
                          rb_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* RBSPMM_H */
