/*
 * dg.h -- C ABI of the GB300 matrix-free DG operator library (libdg.so).
 *
 * The library applies the weighted symmetric interior penalty (WSIPG) DG
 * operator of Muething, Piatkowski & Bastian, "High-performance
 * Implementation of Matrix-free High-order Discontinuous Galerkin Methods"
 * (arXiv 1711.10885), for the stationary convection-diffusion-reaction problem
 *     -div(D grad u) + div(b u) + c u = f  in Omega,   u = g on dOmega
 * (Sec. 2, eq. modelproblem without the time derivative) on an axis-parallel,
 * uniform cuboid mesh with the tensor-product space Q_k (Sec. 3.1) and the
 * (k+1)^3-point Gauss-Legendre rule (Problem A of Sec. 5.1: q = 2p).
 *
 * Numbering and layouts (all arrays are plain, contiguous, C order):
 *   cells      cell = ix + nx*(iy + ny*iz)                       (x fastest)
 *   DOFs       vector[cell*(k+1)^3 + J],  J = j1 + n*(j2 + n*j3), n = k+1,
 *              coefficients of the ORTHONORMAL shifted Legendre basis on the
 *              reference cell [0,1]^3: phi_J = theta_j1 theta_j2 theta_j3,
 *              theta_j(x) = sqrt(2j+1) P_j(2x-1)  (the "L2-orthogonal
 *              Legendre" basis of Sec. 2; the mass matrix is |T| I).
 *   vol. pts   f_qp[cell*m^3 + q],  q = i1 + m*(i2 + m*i3), m = k+1.
 *   faces      boundary side s = 2*dir + (0: lower, 1: upper), dir 0=x,1=y,2=z;
 *              face f of side s = c_a + n_a*c_b over the two tangential cell
 *              indices (a < b); its m^2 points p = p_a + m*p_b.
 *
 * Operator (Sec. 2, eq. blf):  (A u)_i = a_h(u, phi_i).  Right hand side
 * F_i = l_h(phi_i) with f and Dirichlet data g.  Residual r = A u - F.
 * Jacobian application y = A z (the problem is linear, so this is the
 * operator without f and g).  Readings where the paper is ambiguous:
 * weighted average {v}_w = w- v- + w+ v+; penalty
 *   gamma_F = <D-,D+> * sigma * |F| / min(|T-|,|T+|),  <a,b> = 2ab/(a+b),
 * with the caller's sigma (dg_penalty_sigma gives the two conventions);
 * boundary faces use D- and |T-|; boundary faces are Dirichlet unless
 * dg_setup_ext.bc_type makes a side Neumann or outflow; interior faces are
 * oriented from the lower-index cell T- to T+ along the axis.
 *
 * Ownership: the caller owns every vector it passes (device pointers for the
 * *_dev arguments, in layout above, 8-byte (FP64) or 4-byte (FP32) elements,
 * input and output must not alias).  The library owns the handle and all
 * memory reachable from it (tables, coefficients, right hand side, work
 * buffers) and frees it in dg_destroy.  Host pointers passed to dg_setup are
 * read during the call only.
 *
 * Streams: every `stream` argument is a cudaStream_t passed as void* (NULL =
 * legacy default stream).  Apply calls are asynchronous on that stream.
 *
 * Errors: every call returns DG_OK (0) or a negative DG_ERR_* code and never
 * aborts; dg_last_error() returns a message for the calling thread's last
 * failure.  Calls on one handle must not run concurrently from several host
 * threads (the handle's work buffers are shared by its applies).
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DG_OK = 0,
  DG_ERR_INVALID_ARG = -1, /* bad size, degree, coefficient or pointer         */
  DG_ERR_CUDA = -2,        /* a CUDA runtime call failed (message has details) */
  DG_ERR_OOM = -3,         /* device allocation failed                         */
  DG_ERR_NOT_CONVERGED = -4,
  DG_ERR_TIMEOUT = -5,
  DG_ERR_NAN = -6
};

/* Precision of an apply.  DG_F64 and DG_F32: vectors and arithmetic in FP64 / FP32.  DG_F64X: FP64
 * vectors (double), arithmetic in "double-float" -- each value a pair of FP32 numbers whose sum
 * carries about 48 significand bits, combined with error-free transformations (TwoSum, Fast2Sum,
 * FMA-based TwoProduct).  It gives FP64-level results (checked to <= 1e-12 against the FP64 oracle)
 * on the FP32 pipes, which on GB300 issue 62x more FMAs per clock than the FP64 pipe. */
enum { DG_F64 = 0, DG_F32 = 1, DG_F64X = 2 };

#define DG_MAX_DEGREE 10

typedef struct dg_handle dg_handle;

/* Axis-parallel uniform cuboid mesh [lo, hi] with n[d] cells per axis (Sec. 2, maps mu_T are
 * translations plus axis scalings: S_T = diag(1/h), Delta_T = h_x h_y h_z, Sec. 3.2). */
typedef struct {
  double lo[3], hi[3];
  int32_t n[3];
} dg_mesh;

/* Coefficients of eq. modelproblem: D = D_T * I constant per cell (D_cell[ncells] on the host,
 * or NULL to use D_const everywhere; every D_T must be finite and > 0), constant velocity b,
 * constant reaction c, and the penalty factor sigma of gamma_F (see above). */
typedef struct {
  const double* D_cell;
  double D_const;
  double b[3];
  double c;
  double sigma;
} dg_coeffs;

/* Boundary data at the boundary face points: g_qp[s] is a host array of
 * (faces of side s) * m^2 values, or NULL for zero data on that side: the
 * Dirichlet value g, or on a Neumann side (dg_setup_ext.bc_type) the total
 * flux j = (b u - D grad u) . nu (nu the outer unit normal). */
typedef struct {
  const double* g_qp[6];
} dg_bc;

/* Penalty factor sigma for degree k.  mode 0: 2k(k+1) (the benchmark convention "2k(k+1)/h"
 * for D = 1); mode 1: alpha*k*(k+d-1) with alpha = 2, d = 3, as printed in Sec. 2. */
double dg_penalty_sigma(int32_t k, int32_t mode);

/* Build a handle for degree k in [1, DG_MAX_DEGREE] (k = 0 is rejected: the paper's penalty
 * p(p+d-1) vanishes).  f_qp: host array [ncells][(k+1)^3] of f at the volume points, or NULL
 * (f = 0).  bc may be NULL (g = 0).  Computes the right hand side F = l_h(phi_i) (Sec. 2) on
 * the device.  Synchronises `stream` before returning. */
int dg_setup(const dg_mesh* mesh, int32_t k, const dg_coeffs* coeffs, const dg_bc* bc, const double* f_qp,
             void* stream, dg_handle** out);

int dg_destroy(dg_handle* h);

/* Sizes of the handle's problem: number of cells, DOFs per cell, total DOFs. */
int dg_sizes(const dg_handle* h, int64_t* ncells, int32_t* dofs_per_cell, int64_t* ndofs);

/* Physical coordinates of the quadrature points, written to a host array (m = k+1, or the handle's m):
 * which = 0: volume points [ncells][m^3][3]; which = 1+s: boundary side s [faces][m^2][3]; which = 7:
 * the points of all 6 faces of every cell [ncells][6][m^2][3] (face 2*dir+side, points as for
 * dg_setup_ext.D_face).  Use them to sample f, g and point-wise coefficients for dg_setup_ex. */
int dg_quadrature_points(const dg_handle* h, int32_t which, double* xyz_host);

/* y = A z: matrix-free application of eq. blf by sum factorisation (Algorithm 1 of Sec. 3.6:
 * volume terms, interior faces, boundary faces).  precision DG_F64 (double vectors) or DG_F32
 * (float vectors, the same algorithm in single precision). */
int dg_apply_jacobian(dg_handle* h, const void* z_dev, void* y_dev, int32_t precision, void* stream);

/* r = A u - F (residual evaluation, Sec. 1 and Sec. 2), same precisions as above. */
int dg_apply_residual(dg_handle* h, const void* u_dev, void* r_dev, int32_t precision, void* stream);

/* One of the two kernels of an apply, for per-kernel timing and profiling.  stage 0 runs the
 * cell kernel (volume terms and face traces, Algorithm 1 steps 1-3 and the evaluation halves of
 * steps 4 and 8) from `in` into the handle's work buffers; stage 1 runs the face kernel (face
 * fluxes, lifting and the final contraction, the integration halves of steps 4-10) from the work
 * buffers into `out`, subtracting F when `residual` is non-zero.  Stage 0 followed by stage 1 on
 * the same stream is exactly dg_apply_jacobian (residual = 0) or dg_apply_residual (residual = 1).
 * The pointer a stage does not use is ignored. */
int dg_apply_stage(dg_handle* h, int32_t stage, const void* in, void* out, int32_t precision, int32_t residual,
                   void* stream);

/* Copy the right hand side F = l_h(phi_i) into F_dev (device, given precision). */
int dg_rhs(dg_handle* h, void* F_dev, int32_t precision, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Solvers.  The paper measures operator application only and leaves solvers to future work
 * (Sec. 1, Sec. 6); the solvers below use that operator as their only access to A.
 * --------------------------------------------------------------------------------------------- */

enum { DG_SOLVE_FP64 = 0, DG_SOLVE_MIXED = 1 };
/* DG_PRECOND_MLP: z = network(r); DG_PRECOND_BJ_MLP: z = block-Jacobi(r) + network(r), the network
 * trained on the part of the error that block-Jacobi misses (needs dg_precond_setup).  DG_PRECOND_RB_GS:
 * red-black block Gauss-Seidel (dg_precond_apply_rbgs; needs dg_precond_setup): one operator application more
 * per preconditioner application than block-Jacobi, about half the Krylov iterations. */
enum { DG_PRECOND_NONE = 0, DG_PRECOND_BLOCK_JACOBI = 1, DG_PRECOND_MLP = 2, DG_PRECOND_BJ_MLP = 3,
       DG_PRECOND_RB_GS = 4 };

typedef struct dg_mlp dg_mlp; /* learned per-element preconditioner, see below */

typedef struct {
  int32_t mode;           /* DG_SOLVE_FP64: FGMRES(restart) in FP64 on the FP64 operator.
                             DG_SOLVE_MIXED: FGMRES(outer_restart) in FP64 (true residual, defect update
                             and orthogonalisation in FP64) whose preconditioner is one cycle of an FP32
                             FGMRES(restart) on the FP32 operator, stopped at inner_rtol.             */
  int32_t preconditioner; /* DG_PRECOND_NONE, DG_PRECOND_BLOCK_JACOBI (FP64 blocks in FP64 mode, FP32
                             blocks inside the FP32 inner solve), DG_PRECOND_RB_GS (in the precision of the
                             solve it preconditions) or an MLP mode; needs dg_precond_setup first      */
  int32_t restart;        /* FGMRES restart length (inner length in MIXED mode), 1..60, 0 = 30        */
  int32_t outer_restart;  /* MIXED: outer restart length, 1..60, 0 = 20                               */
  int32_t max_iterations; /* cap on (outer) iterations, 0 = 10000                                      */
  double rtol;            /* stop when ||b - A x||_2 <= rtol ||b||_2, checked on the FP64 residual     */
  double inner_rtol;      /* MIXED: relative residual reduction of each inner solve, in (0, 1)         */
  const dg_mlp* mlp;      /* DG_PRECOND_MLP: the trained network (degree must match the handle)       */
  int32_t mlp_placement;  /* MLP modes: 0 = the network acts in every preconditioner application;
                             1 = only on the first direction of each (outer) FGMRES cycle, whose input is
                             the true residual r/||r|| like its training data; the other directions use
                             block-Jacobi (DG_PRECOND_BJ_MLP) or none (DG_PRECOND_MLP)              */
  double fallback_ratio;  /* DG_PRECOND_MLP: if one inner cycle (MIXED) or restart cycle (FP64) reduces
                             its residual by less than this factor (e.g. 0.5), the rest of the solve
                             uses block-Jacobi when dg_precond_setup was called; 0 = never          */
  int32_t inner_block_precision; /* MIXED with block-Jacobi, the block inverse applied in the inner FP32
                             solve: 0 = by fast diagonalisation (each diagonal block is a Kronecker sum of
                             three 1D cell operators; six complex FP32 1D contractions per cell), or the
                             FP16 blocks if it could not be built; 1 = the FP32 dense blocks; 2 = FP16
                             copies of the dense blocks, each divided by its largest |entry| (half the
                             bytes of that bandwidth-bound product).  A flexible method tolerates the
                             rounding of the preconditioner.                                           */
  int32_t outer_precision; /* MIXED: arithmetic of the operator in the outer FGMRES (its vectors,
                             orthogonalisation and defect updates are FP64 either way): 0 = double-float
                             (DG_F64X: FP64-level results on the FP32 pipes, about 4x faster on GB300),
                             with the stopping test confirmed by a true FP64 residual and the solve
                             finished in FP64 if that residual is still above rtol; 1 = FP64      */
  int32_t inner_basis_precision; /* MIXED: storage of the inner FP32 FGMRES's orthonormal basis (its arithmetic
                             stays FP32): 0 = FP32; 1 = FP16, each entry stored times 2^8 (the rows have unit
                             length), which halves the bytes of the basis passes; applies when the vector
                             length is a multiple of 8 (always for odd k), else FP32.  The rounding of the
                             rows (2^-11 relative) perturbs the inner Arnoldi relation at that level, which
                             the flexible outer method absorbs like any other inexact preconditioner.  */
} dg_solve_opts;

typedef struct {
  int32_t status;           /* DG_OK or the returned error code                                    */
  int32_t iterations;       /* FGMRES iterations (outer iterations in MIXED mode)                    */
  int32_t inner_iterations; /* FP32 inner iterations (MIXED), else equal to iterations              */
  int32_t applies_f64;      /* operator applications on FP64 vectors (FP64 or double-float)         */
  int32_t applies_f32;      /* FP32 operator applications                                           */
  double rel_residual;      /* final ||b - A x||_2 / ||b||_2 (true FP64 residual at exit)           */
  double seconds;           /* wall time of the call                                                */
  int32_t fallback;         /* 1 if an MLP-preconditioned solve switched to block-Jacobi            */
} dg_solve_stats;

/* Kinds of dg_precond_setup.  DG_BJ_DENSE: the dense inverse blocks below (FP64, FP32, FP16) and the
 * fast-diagonalisation tables.  DG_BJ_FAST_DIAG: only the fast-diagonalisation tables (FP32 and FP64, real or
 * complex, 3 (2 (k+1)^2 + k+1) + 1 numbers per cell; any degree): every diagonal block is a Kronecker sum of three
 * 1D cell operators A_TT = I (x) I (x) A_x + I (x) A_y (x) I + A_z (x) I (x) I + c |T| I, inverted exactly
 * through their eigen-decompositions (computed on the host).  Both need the scalar axis-parallel kernels. */
enum { DG_BJ_DENSE = 1, DG_BJ_FAST_DIAG = 2 };

/* Build the block-Jacobi preconditioner (kind = DG_BJ_DENSE): for every cell the
 * diagonal block A_TT ((k+1)^3 x (k+1)^3: the cell's volume term plus the self-coupling of its
 * faces) is assembled on the device by running the operator's own kernels on unit vectors, then
 * inverted in a batch (Gauss-Jordan, partial pivoting) and kept in FP64 and FP32 (FP32 rows padded
 * to a multiple of 4).  Memory: about ncells * (k+1)^6 * 12 bytes, owned by the handle.  Requires (k+1)^3 <= 512.  Returns
 * DG_ERR_NAN if a block is singular.  Synchronises `stream`. */
int dg_precond_setup(dg_handle* h, int32_t kind, void* stream);

/* What dg_precond_setup built, as bits of *info: DG_PRECOND_HAS_DENSE the dense inverse blocks,
 * DG_PRECOND_HAS_FAST_DIAG the fast-diagonalisation tables, DG_PRECOND_FAST_DIAG_REAL all of them in real
 * arithmetic.  A cell whose three 1D operators have real eigenvalues and eigenvectors (diffusion-dominated
 * cells) gets real tables: half the bytes and a quarter of the multiply-adds of the complex form, which the
 * other cells keep (e.g. convection-dominated ones); *complex_cells (may be NULL) receives their number.
 * 0 before set-up. */
enum { DG_PRECOND_HAS_DENSE = 1, DG_PRECOND_HAS_FAST_DIAG = 2, DG_PRECOND_FAST_DIAG_REAL = 4 };
int dg_precond_info(const dg_handle* h, int32_t* info, int64_t* complex_cells);

/* z = M^{-1} r with the block-Jacobi preconditioner (r, z device vectors of the given precision).  DG_F64
 * applies the dense FP64 inverse blocks (or, after DG_BJ_FAST_DIAG, the fast diagonalisation in complex FP64);
 * DG_F32 the exact block inverse by fast diagonalisation with complex FP32 contractions, or the FP32 dense
 * blocks where the 1D operators could not be diagonalised. */
int dg_precond_apply(dg_handle* h, const void* r_dev, void* z_dev, int32_t precision, void* stream);

/* z = M^{-1} r with red-black block Gauss-Seidel.  The cells are coloured by the parity of ix + iy + iz, so the
 * face neighbours of a red cell are black (on a periodic axis with an odd number of cells the two cells across
 * the wrap share a colour; their coupling is then left out as in block-Jacobi).  M is the block lower-triangular
 * part of A in red-before-black order:
 *   z_red = A_rr^{-1} r_red,   z_black = A_bb^{-1} (r - A z_red)_black,
 * the diagonal blocks inverted by fast diagonalisation (any degree; dg_precond_setup first; in dg_solve
 * whatever dg_solve_opts.inner_block_precision says) and A z_red the operator applied to z_red (zero on the
 * black cells).  r, z and work are distinct device vectors of the given
 * precision (DG_F64 or DG_F32), work is scratch; asynchronous on `stream`. */
int dg_precond_apply_rbgs(dg_handle* h, const void* r_dev, void* z_dev, void* work_dev, int32_t precision,
                          void* stream);

/* Solve A x = b (b_dev NULL: b = F, the right hand side of dg_setup) with FGMRES; x_dev holds the
 * initial guess and receives the solution (FP64, device).  Fills *stats (may be NULL).  Returns
 * DG_OK when the FP64 relative residual reached opts->rtol, DG_ERR_NOT_CONVERGED when the iteration
 * cap was hit first, DG_ERR_NAN on a non-finite residual.  Synchronises `stream` (once per Arnoldi
 * step).  Workspace is allocated on first use and kept by the handle. */
int dg_solve(dg_handle* h, const double* b_dev, double* x_dev, const dg_solve_opts* opts, dg_solve_stats* stats,
             void* stream);

/* ---------------------------------------------------------------------------------------------
 * Learned per-element preconditioner.  The paper has no solver or preconditioner (Sec. 1, Sec. 6
 * leave them to future work); this network is trained on (residual, error) pairs produced by the
 * solver above on the operator above, and used as the preconditioner M inside FGMRES.
 *
 * For a cell T with residual block r_T ((k+1)^3 values) the network input is
 *   x = [r_T / s, log D_T, log D of the 6 face neighbours (x-, x+, y-, y+, z-, z+; the cell's own
 *        value where the neighbour is missing)],  s = ||r_T||_2,  zero-padded to kin_padded,
 * two ReLU layers of 256 units, and an output layer of (k+1)^3 units; the correction is
 *   z_T = s * t_scale * y(x),
 * which makes the preconditioner positively homogeneous in r.  Weights are FP32 masters rounded to
 * BF16 for the GEMMs of the forward and the backward pass (tensor cores, FP32 accumulation); bias
 * gradients and Adam run in FP32.  Rows of X are BF16 [rows][kin_padded]; targets T are FP32
 * [rows][(k+1)^3].
 * --------------------------------------------------------------------------------------------- */
typedef struct {
  int32_t epochs;   /* passes over the rows                    */
  int32_t batch;    /* rows per Adam step (rows / batch steps)   */
  double lr;        /* Adam step size (beta1 0.9, beta2 0.999)   */
} dg_mlp_train_opts;

typedef struct {
  double first_epoch_loss; /* mean squared error over the first epoch  */
  double last_epoch_loss;  /* mean squared error over the last epoch   */
  int64_t steps;           /* Adam steps taken by this network so far  */
} dg_mlp_train_stats;

/* New network for degree k in [1, 7], He-uniform weights from `seed`, zero biases, t_scale 1. */
int dg_mlp_create(int32_t k, uint64_t seed, dg_mlp** out);
int dg_mlp_destroy(dg_mlp* m);
int dg_mlp_dims(const dg_mlp* m, int32_t* k, int32_t* kin, int32_t* kin_padded, int32_t* out_padded,
                int64_t* nparam);
/* Parameter block (FP32, nparam values: W1 [256][kin_padded], b1, W2 [256][256], b2,
 * W3 [out_padded][256], b3 at the offsets of dg_mlp_param_offsets).  direction 0: copy weights to
 * host; 1: copy weights from host (BF16 copy refreshed, t_scale set if non-NULL); 2: copy the
 * gradient of the last dg_mlp_loss_grad / training step to host.  Synchronous. */
int dg_mlp_params(dg_mlp* m, float* host, int32_t direction, float* t_scale);
int dg_mlp_param_offsets(const dg_mlp* m, int64_t* offsets6);
int dg_mlp_set_target_scale(dg_mlp* m, float t_scale);
/* Feature rows X (device, BF16) and scales s * t_scale (device) for the listed cells of the handle's
 * mesh (cells_dev = NULL: all cells in order, rows = ncells), from the residual r_dev (device, given
 * precision). */
int dg_mlp_features(const dg_mlp* m, const dg_handle* h, const void* r_dev, int32_t precision,
                    const int32_t* cells_dev, int64_t rows, void* X_dev, float* scale_dev, void* stream);
/* Training pairs of the learned preconditioner from a solver state of the handle's problem (the method's own
 * data).  With r = F - A x (x_dev, FP64), for sample i < count with cell = cells_dev[i] and output row
 * row = rows_dev[i] (int32 device arrays; rows may be any permutation, e.g. to shuffle the set):
 *   X[row] = the feature row of r on the cell (as dg_mlp_features), BF16 [*][kin_padded];
 *   E[row][j] = e_j / ||r_cell||_2, e = (xstar - x) on the cell, minus the block-Jacobi correction of r when
 *   subtract_block_jacobi (needs dg_precond_setup), FP32 [*][(k+1)^3]; zero where r_cell = 0.
 * Uses the network's device work space for r.  Asynchronous on `stream`. */
int dg_mlp_pairs(dg_mlp* m, dg_handle* h, const double* x_dev, const double* xstar_dev, const int32_t* cells_dev,
                 const int32_t* rows_dev, int64_t count, int32_t subtract_block_jacobi, void* X_dev, float* E_dev,
                 void* stream);
/* t = RMS of E_dev (rows x (k+1)^3 FP32 targets); E_dev /= t in place and t becomes the network's target scale
 * (as dg_mlp_set_target_scale).  *t_scale (host, may be null) receives it.  Synchronises `stream`. */
int dg_mlp_normalize_targets(dg_mlp* m, float* E_dev, int64_t rows, float* t_scale, void* stream);
/* Y = network(X) for `rows` rows: Y device FP32 [rows][out_padded]. */
int dg_mlp_forward(const dg_mlp* m, const void* X_dev, int64_t rows, float* Y_dev, void* stream);
/* Mean squared error of network(X) against T and its gradient (kept in the network). */
int dg_mlp_loss_grad(dg_mlp* m, const void* X_dev, const float* T_dev, int64_t rows, double* loss, void* stream);
/* Adam training on the rows in order (batches of opts->batch rows); synchronises `stream`. */
int dg_mlp_train(dg_mlp* m, const void* X_dev, const float* T_dev, int64_t rows, const dg_mlp_train_opts* opts,
                 dg_mlp_train_stats* stats, void* stream);
/* The preconditioner: z = M(r) for every cell of the handle (r, z device vectors, given precision). */
int dg_mlp_apply(dg_mlp* m, const dg_handle* h, const void* r_dev, void* z_dev, int32_t precision, void* stream);
/* z += M(r): the network's correction added to z (used with block-Jacobi in DG_PRECOND_BJ_MLP). */
int dg_mlp_apply_add(dg_mlp* m, const dg_handle* h, const void* r_dev, void* z_dev, int32_t precision,
                     void* stream);
/* Checkpoint: weights, Adam moments and step count, t_scale (binary, host file). */
int dg_mlp_save(const dg_mlp* m, const char* path);
int dg_mlp_load(const char* path, dg_mlp** out);

/* ---------------------------------------------------------------------------------------------
 * Batched application of many uneven problems.  The paper applies one operator per process
 * (Sec. 5); a batch runs the applies of many handles (different meshes and degrees 1..8, FP64) in
 * one CUDA graph launch: each of the two kernels of Algorithm 1's split (cell kernel, face kernel)
 * runs as one persistent kernel that takes tiles of cells of all problems from a work queue
 * (heaviest tiles first).  At creation an autotuner times, per degree, two cells-per-CTA choices
 * (so two CTA thread layouts) on that degree's problems and keeps the faster.
 * --------------------------------------------------------------------------------------------- */
typedef struct dg_batch dg_batch;

/* Create a batch over `count` handles (not owned: they must outlive the batch, and must not be
 * applied on their own while a batch apply that uses them is in flight, since the batch uses their
 * work buffers).  Runs the autotuner on `stream` and synchronises it. */
int dg_batch_create(dg_handle* const* handles, int32_t count, void* stream, dg_batch** out);

/* For every problem i: out_dev[i] = A_i in_dev[i] (residual = 0) or A_i in_dev[i] - F_i (residual = 1),
 * FP64 device vectors, as one graph launch on `stream`.  The first call captures the graph; later
 * calls with the same vectors and mode launch it directly (no host synchronisation). */
int dg_batch_apply(dg_batch* b, const double* const* in_dev, double* const* out_dev, int32_t residual,
                   void* stream);

/* Autotuner result for degree k.  At dg_batch_create every degree present is timed alone (its counter reset,
 * cell kernel and face kernel over all its problems, best of three after a warm-up) with each of the
 * DG_BATCH_CANDIDATES thread layouts, with F = floor(256 / (k+1)^2) cells per CTA of the standalone kernels:
 *   0: F cells per CTA, one line per thread (the standalone layout)   1: F/2 cells, one line per thread
 *   2: F cells, two lines per thread                                    3: 2F cells, two lines per thread
 * and the fastest is used.  Outputs (host, may be null): the chosen cells per CTA and lines per thread, and
 * the time (ms) of every candidate (DG_BATCH_CANDIDATES floats); zeros for a degree not in the batch. */
#define DG_BATCH_CANDIDATES 4
int dg_batch_tuning(const dg_batch* b, int32_t k, int32_t* cells_per_cta, int32_t* lines_per_thread,
                    float* ms_candidates);

int dg_batch_destroy(dg_batch* b);

/* ---------------------------------------------------------------------------------------------
 * Arithmetic throughput probes: the denominators of the roofline of the cost model (Sec. 3.6), measured
 * on the device the library runs on.  kind DG_PROBE_DFMA runs chains of FP64 FMAs, DG_PROBE_DMMA FP64
 * tensor-core products (mma.sync m8n8k4, 512 flops per warp instruction), DG_PROBE_FFMA chains of FP32
 * FMAs, on every warp slot of every SM, `iterations` rounds each.  *flops (host) receives the floating-point
 * operations of the launch; the caller times it with events on `stream`.  sink_dev is a device double that
 * is written only by an impossible outcome (it keeps the work from being removed).  Asynchronous.
 * --------------------------------------------------------------------------------------------- */
enum { DG_PROBE_DFMA = 0, DG_PROBE_DMMA = 1, DG_PROBE_FFMA = 2 };
int dg_peak_probe(int32_t kind, int64_t iterations, double* sink_dev, double* flops, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Allocation-free Jacobian application.  The paper has no counterpart of this entry point.
 *
 * dg_setup obtains its tables, coefficients and work buffers from cudaMalloc.  Some callers cannot
 * allocate device memory at the point where they apply the operator: a host application that owns
 * all device memory through its own pool and forbids other allocators, or a latency-critical loop
 * where cudaMalloc, which can synchronise the whole device, is not allowed after start-up.
 * dg_apply_jacobian_static serves them.  It computes y = A z in FP64 exactly like
 * dg_apply_jacobian (same kernels, same operator), and it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Its work space (point-space residual, face traces, face coefficients) is a fixed device array
 * of DG_STATIC_SCRATCH_BYTES inside libdg.so.  The array is reserved on a device together with
 * the library's kernel images: with CUDA's lazy module loading (the default of current toolkits)
 * that happens at the first call of this entry point (or the first kernel launch of the library) on
 * that device, otherwise when the library is loaded; from then on the device holds it until the
 * process exits.  Callers that must not allocate after start-up should therefore make one call at
 * start-up on each device they use.  A problem needs
 *     256-byte-rounded ncells*(k+1)^3*8  +  ncells*12*(k+1)^2*8  +  ncells*18*8  bytes,
 * for example at most about 3200 cells at k = 7 or 15000 cells at k = 3.  Larger problems are
 * rejected with DG_ERR_INVALID_ARG and a message; use dg_setup / dg_apply_jacobian for them.
 *
 * Arguments: the mesh and degree as in dg_setup; D_dev is a device array of ncells diffusion
 * values (finite, > 0, not checked on the device); b, c and sigma are as in dg_coeffs.  z_dev and
 * y_dev are FP64 device vectors in the DOF layout above and must not alias.  The call is
 * asynchronous on `stream`.
 *
 * Set-up: the first call on each device looks up the device address of the array
 * (cudaGetSymbolAddress) with that device current, so make this first call before any stream
 * capture.  Sharing: all calls in the process use the same array, and a call leaves its contents
 * behind.  Every byte a call reads has been written earlier in that call, so nothing has to start
 * at zero.  Calls whose kernels overlap on the GPU (different streams or host threads without
 * ordering) race on the array and give wrong results; order them on one stream.
 * --------------------------------------------------------------------------------------------- */
#define DG_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

int dg_apply_jacobian_static(const dg_mesh* mesh, int32_t k, const double* D_dev, const double b[3], double c,
                             double sigma, const double* z_dev, double* y_dev, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Transport problems (Sec. 5.3): periodic axes, a flow field b(x), the q = 2p+4 quadrature rule,
 * and explicit strong-stability-preserving Runge-Kutta time stepping (Sec. 2, "ODE": the basis is
 * L2-orthogonal, so the mass matrix is |T| I and M^{-1} is a scaling).
 * --------------------------------------------------------------------------------------------- */
enum { DG_VELOCITY_CONSTANT = 0, DG_VELOCITY_POINTS = 1, DG_VELOCITY_TAYLOR_GREEN = 2 };

typedef struct {
  int32_t periodic[3];  /* 1: the axis wraps around; its two end faces are one interior face between the
                           last and the first cell (no Dirichlet data there)                          */
  int32_t m;            /* Gauss points per direction: 0 or k+1 (q = 2p), or k+3 (q = 2p+4, Sec. 5.3).
                           f_qp, g_qp and dg_quadrature_points then use m points per direction.        */
  int32_t velocity;     /* DG_VELOCITY_CONSTANT: coeffs->b.
                           DG_VELOCITY_POINTS: b_qp and b_face below (coeffs->b is ignored).
                           DG_VELOCITY_TAYLOR_GREEN: the fixed flow field of Sec. 5.3,
                             b = (cos x1 sin(-x2) sin(-x3), sin x1 cos(-x2) sin(-x3) / 2,
                                  sin x1 sin(-x2) cos(-x3) / 2),
                           evaluated on the device at the quadrature points with CUDA's sin and cos.  */
  const double* b_qp;   /* POINTS: host [ncells][m^3][3], b at the volume points (layout of f_qp)      */
  const double* b_face; /* POINTS: host [ncells][6][m^2], b . e_dir at the points of face 2*dir+side
                           of each cell (points p = p_a + m*p_b over the tangential axes a < b).  An
                           interior face uses the value given for its lower cell's upper face for both
                           cells, so the two sides see one flux.                                       */
  const double* D_tensor; /* host [ncells][6] = (xx, yy, zz, xy, xz, yz): a symmetric positive definite
                           diffusion tensor per cell (Sec. 5.1: "tensor-valued diffusion coefficients"),
                           replacing coeffs->D_cell / D_const; NULL: D_T * I.  delta = nu^T D nu enters
                           the face weights and the penalty.                                          */
  const double* jacobian; /* host [9], row-major J: the cells are lo + J (ic + [0,1]^3), an affine image
                           of the structured grid (Problem B of Sec. 5.1); mesh->hi is then unused and
                           the quadrature points follow the map.  NULL: the axis-parallel [lo, hi] grid.
                           With D_tensor or jacobian the tensor-diffusion kernels run (m = k+1, constant
                           velocity, degrees 1..8, DG_F64 and DG_F64X applies).                       */
  /* Coefficients given at the quadrature points (Problem B of Sec. 5.1: affine cells and coefficients that
     are polynomials in the coordinates, integrated with q = 2p+4, i.e. m = k+3).  The caller evaluates them
     at the points of dg_quadrature_points (which = 0 for the volume, 7 for every cell's faces).  Given D_qp
     and D_face, the point-wise kernels run: they replace coeffs->D_cell / D_const and D_tensor, work with
     m = k+1 or k+3, a constant velocity or DG_VELOCITY_POINTS (b_face is then the normal velocity b . nu
     along +reference axis dir, nu the unit normal), periodic axes and the jacobian, for degrees 1..8 and
     DG_F64 / DG_F64X applies.  On an interior face the weights w+-, delta = nu^T D nu and the penalty are
     formed point by point from both cells' D_face values at that point (Sec. 2, with readings 1-3 above). */
  const double* D_qp;   /* host [ncells][m^3][6] (xx, yy, zz, xy, xz, yz): D at the volume points, every
                           point symmetric positive definite; with D_face, or NULL                    */
  const double* D_face; /* host [ncells][6][m^2][6]: D at the points of face 2*dir+side of each cell
                           (points p = p_a + m*p_b over the tangential axes a < b)                    */
  const double* c_qp;   /* host [ncells][m^3]: c at the volume points (point-wise kernels only), or NULL
                           for coeffs->c                                                               */
  int32_t bc_type[6];   /* boundary type of side 2*dir+side (Sec. 2, eq. modelproblem; ignored on periodic
                           axes): DG_BC_DIRICHLET (0, u = g), DG_BC_NEUMANN (total flux (b u - D grad u) . nu
                           = j: no term in a_h, -(j, v) in l_h, j given in dg_bc.g_qp of that side), or
                           DG_BC_OUTFLOW ((D grad u) . nu = 0: only the upwind flux Phi(u, 0, b . nu) in a_h,
                           meant for sides with b . nu >= 0; nothing in l_h)                         */
  const double* vertices; /* host [(n0+1)(n1+1)(n2+1)][3], vertex (i, j, l) at i + (n0+1)(j + (n1+1) l), or
                           NULL.  Multilinear cells (Problem C of Sec. 5.1): cell (ix, iy, iz) is the trilinear
                           image of [0,1]^3 through its 8 corner vertices; mesh->lo/hi and jacobian are unused.
                           The point-wise kernels run (coefficients from D_qp/D_face/c_qp when given, else from
                           coeffs / D_tensor), with J taken at every quadrature point; the penalty's |F| and |T|
                           are the face area and cell volume.  No periodic axes; degrees 1..8; dg_project and the
                           Runge-Kutta calls reject such a handle (its mass matrix is not |T| I). */
} dg_setup_ext;

enum { DG_BC_DIRICHLET = 0, DG_BC_NEUMANN = 1, DG_BC_OUTFLOW = 2 };

/* dg_setup with the options above (ext = NULL is dg_setup).  A field b(x) or m = k+3 selects the
 * velocity field kernels, which support degrees 1..8 and DG_F64 and DG_F64X applies (DG_F32 applies,
 * the mixed-precision solver, block-Jacobi and batches reject such a handle).  On a periodic
 * axis with a single cell the cell is its own neighbour.  Synchronises `stream`. */
int dg_setup_ex(const dg_mesh* mesh, int32_t k, const dg_coeffs* coeffs, const dg_bc* bc, const double* f_qp,
                const dg_setup_ext* ext, void* stream, dg_handle** out);

/* L2 projection of a function given at the volume points onto the DG space (the initial value of a
 * time-dependent run): z_i = (u0, phi_i)_T / |T|, computed with the handle's quadrature rule.
 * u_qp_dev: device [ncells][m^3]; z_dev: device FP64 DOF vector. */
int dg_project(dg_handle* h, const double* u_qp_dev, double* z_dev, void* stream);

/* One explicit Runge-Kutta stage (Sec. 2, "ODE", with M = |T| I):
 *     y = cz * z0 + cu * u - cdt * M^{-1} (A u - F)
 * fused into the operator's face kernel.  F is the right hand side of the handle (f and g do not
 * depend on time here).  u, z0, y are FP64 device vectors; y may alias u or z0 (every element is
 * read before it is written, by the same thread).  precision: DG_F64, or DG_F64X (A u - F in
 * double-float; the update itself is FP64 in both). */
int dg_rk_stage(dg_handle* h, const double* u_dev, const double* z0_dev, double* y_dev, double cz, double cu,
                double cdt, int32_t precision, void* stream);

/* nsteps steps of Heun's method, the second-order strong-stability-preserving Runge-Kutta scheme of
 * Sec. 5.3, on z_dev in place:  z1 = z - dt M^{-1}(A z - F);  z <- (z + z1 - dt M^{-1}(A z1 - F)) / 2.
 * Four kernel launches per step; the stage vector is kept by the handle (allocated on the first
 * call, which then synchronises `stream`).  precision as in dg_rk_stage. */
int dg_ssprk2(dg_handle* h, double* z_dev, double dt, int32_t nsteps, int32_t precision, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Matrix-based comparison (Sec. 5.2, table of matrix-free vs matrix-based application and matrix
 * assembly).  The operator's matrix in block compressed row storage: block row T holds one
 * (k+1)^3 x (k+1)^3 block A_{T,S} for S = T and each face neighbour of T (sorted by S; on a periodic
 * axis with one or two cells, coinciding neighbours share one block), nb = (k+1)^3.  On the device the
 * blocks are column-major with each column padded to an even length; dg_matrix_export returns them
 * column-major without padding: entry (i, j) of block b at vals[(b*nb + j)*nb + i].
 * --------------------------------------------------------------------------------------------- */
typedef struct dg_matrix dg_matrix;

/* Assemble the FP64 matrix of the handle's operator (A of dg_apply_jacobian) on the device, by applying
 * the matrix-free operator to colour-class probe vectors: cells are coloured so that no two cells of a
 * colour share a face neighbour (27 colours on a non-periodic mesh), and each (colour, basis index)
 * pair costs one operator application.  Needs (k+1)^3 <= 512.  Memory: about nnzb * (k+1)^6 * 8 bytes,
 * owned by the matrix.  Synchronises `stream`. */
int dg_assemble(dg_handle* h, void* stream, dg_matrix** out);

/* Block rows, stored blocks, block size, and the assembly time in seconds (device events). */
int dg_matrix_info(const dg_matrix* m, int64_t* nrows, int64_t* nnzb, int32_t* block, double* assemble_seconds);

/* Copy the structure (host arrays of nrows+1 and nnzb entries) and the values (host, nnzb*nb*nb) out;
 * any pointer may be NULL.  Synchronous. */
int dg_matrix_export(const dg_matrix* m, int32_t* rowptr_host, int32_t* colidx_host, double* vals_host);

/* y = A x, block sparse matrix-vector product (FP64 device vectors, x != y), asynchronous on `stream`. */
int dg_spmv(const dg_matrix* m, const double* x_dev, double* y_dev, void* stream);

int dg_matrix_destroy(dg_matrix* m);

/* Message for the calling thread's last error ("" if none). */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
