/*
 * iskra_gb300.h -- C ABI of the GB300 (sm_103a) implicit mesh-smoothing library.
 *
 * The library computes one step of the paper's inverse mean-curvature flow (§7.1) and its
 * gradient by the adjoint rule for linear solves (§5.2, "Differentiating linear solvers",
 * which applies Eq. 3 of §3.1 to f(A, b; y) = A y - b):
 *
 *   assemble : per-face cotangents and areas of the triangle mesh (V, F) give the cotangent
 *              Laplacian L(V) and the diagonal (barycentric, area/3) mass M(V), and the
 *              operator A = M + t L. L uses the positive-semidefinite sign convention
 *              (L_ab = -(cot alpha_ab + cot beta_ab)/2, L_aa = -sum_b L_ab), so A is the
 *              paper's M - tau L_paper with L_paper = -L and tau = t.
 *   solve    : A U = M B, the paper's (M - tau L) v' = M v when B = V (§7.1).
 *   adjoint  : A Lambda = G with G = dl/dU (A is symmetric), then the vector-Jacobian product
 *              dl/dV = <Lambda, d(M B)/dV - (dA/dV) U> gathered per face, plus
 *              dl/dB = M Lambda and dl/dt = -<Lambda, L U>.
 *
 * Conventions for every call:
 *   - All array arguments are DEVICE pointers on the context's device, contiguous, row-major.
 *     V is [n][3] double; F is [m][3] int32 (counter-clockwise faces); B, U, G, Lambda are
 *     [n][k] double with 1 <= k <= 4; gV is [n][3] double.
 *   - The caller owns every array it passes and must keep it alive and unchanged until the
 *     work queued on the context's stream has finished. The library owns every object it
 *     creates (contexts, meshes, batches) and all memory behind them; free them with the
 *     matching *_free / ig_destroy call.
 *   - Every call is asynchronous on the context's stream unless its description says it
 *     synchronises. Calls that fill an ig_solve_info synchronise.
 *   - Errors are reported by the return code (never by exceptions or aborts);
 *     ig_last_error() gives a one-line description of the last failure on a context.
 *   - Integer offsets are 32-bit: n, m and nnz must each stay below 2^31 - 1.
 */
#ifndef ISKRA_GB300_H
#define ISKRA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IG_OK = 0,
  IG_ERR_INVALID_ARG = 1,        /* bad size, null pointer, unsupported k or option, unused vertex */
  IG_ERR_INDEX_OUT_OF_RANGE = 2, /* a face index outside [0, n) */
  IG_ERR_DEGENERATE_FACE = 3,    /* a face repeats a vertex or has zero area */
  IG_ERR_NOT_CONVERGED = 4,      /* a solve reached max_iter above rel_tol; the best iterate is written */
  IG_ERR_NONFINITE = 5,          /* a NaN/Inf in the inputs or a breakdown of the iteration */
  IG_ERR_OOM = 6,                /* device allocation failed */
  IG_ERR_CUDA = 7,               /* any other CUDA runtime error */
  IG_ERR_STATE = 8               /* call out of order (e.g. solve before assemble) */
} ig_status;

/* Precision of the assembled operator and of the solves (ig_assemble):
 *   IG_PRECISION_FP64        FP64 geometry, FP64 operator, FP64 Jacobi-PCG.
 *   IG_PRECISION_MIXED       FP64 geometry and FP64 operator; the solves iterate in FP32 on an
 *                            FP32 copy inside FP64 residual refinement against the FP64 operator,
 *                            so they reach the FP64 solution (same accuracy as FP64).
 *   IG_PRECISION_MIXED_GEOM32  FP32 face geometry as well: cotangents, areas and the per-face
 *                            gradient in FP32, FP64 only for near-degenerate faces (smallest
 *                            corner with sin < 1e-2); the operator is the FP32 one (A32), and the
 *                            FP64 refinement solves it to rel_tol exactly. Results differ from the
 *                            FP64 path by the FP32 rounding of the operator (about 1e-7 relative
 *                            in its entries, amplified by its condition number). For the smoothing
 *                            step (ig_solve, ig_adjoint, ig_vjp and the batch and serving calls)
 *                            only. */
enum { IG_PRECISION_FP64 = 0, IG_PRECISION_MIXED = 1, IG_PRECISION_MIXED_GEOM32 = 2 };
enum { IG_LAUNCH_GRAPH = 0, IG_LAUNCH_HOST = 1 };

typedef struct ig_ctx ig_ctx;
typedef struct ig_mesh ig_mesh;
typedef struct ig_batch ig_batch;

/* Solver options. ig_default_opts() fills the defaults shown. */
typedef struct {
  double rel_tol;   /* stop when, for every column, ||rhs - A x||_2 / ||rhs||_2 <= rel_tol (1e-10) */
  int max_iter;     /* cap on conjugate-gradient iterations per solve (20000) */
  int launch;       /* IG_LAUNCH_GRAPH: device-side loop in a CUDA graph (default);
                       IG_LAUNCH_HOST: the host launches every iteration and polls every 16 */
  double inner_tol; /* mixed precision: relative tolerance of each FP32 inner solve (1e-5) */
  int max_refine;   /* mixed precision: cap on FP64 residual refinements (30) */
} ig_solve_opts;

/* Per-solve report (filled only when a non-NULL pointer is passed; the call then synchronises). */
typedef struct {
  int status;                /* ig_status of the solve */
  int k;                     /* number of right-hand-side columns */
  int iterations;            /* conjugate-gradient iterations performed (all refinements) */
  int refinements;           /* FP64 residual refinements performed (mixed precision) */
  double rel_residual[4];    /* final relative residual per column as seen by the stopping test */
  double true_rel_residual[4]; /* ||rhs - A x|| / ||rhs|| recomputed in FP64 after the solve */
} ig_solve_info;

/* One-line description of a status code (static storage). */
const char* ig_status_str(ig_status s);

/* Fill opts with the defaults listed in ig_solve_opts. */
void ig_default_opts(ig_solve_opts* opts);

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream` (a cudaStream_t;
 * NULL means the legacy default stream). The context owns its scratch buffers.
 * Errors: IG_ERR_INVALID_ARG (ctx NULL), IG_ERR_CUDA (bad device). */
ig_status ig_create(ig_ctx** ctx, int device, void* cuda_stream);

/* Change the stream later calls are issued on. Work already queued stays on the old stream. */
ig_status ig_set_stream(ig_ctx* ctx, void* cuda_stream);

/* Destroy a context. Every mesh created on it must have been freed first. */
ig_status ig_destroy(ig_ctx* ctx);

/* Last error message recorded on ctx (empty string if none). */
const char* ig_last_error(ig_ctx* ctx);

/* Upload the topology of a triangle mesh and build, on the device, everything that depends
 * on it alone (the paper reuses the sparsity pattern across iterations because it does not
 * change with V, §7.1): the CSR pattern of L (sorted columns, diagonal included), the
 * vertex->(face, corner) incidence used by the atomic-free assembly and gradient gathers.
 * F_dev is [m][3] int32 on the device; the library copies it (the caller keeps F_dev).
 * Synchronises (the pattern size must be known before allocating).
 * Errors: IG_ERR_INVALID_ARG (n < 3, m < 1, a vertex used by no face, a vertex with more
 * than 65535 neighbours), IG_ERR_INDEX_OUT_OF_RANGE, IG_ERR_DEGENERATE_FACE (repeated vertex),
 * IG_ERR_OOM, IG_ERR_CUDA. On error *out is NULL. */
ig_status ig_mesh_upload(ig_ctx* ctx, const int32_t* F_dev, int64_t m, int64_t n, ig_mesh** out);

/* Release a mesh and all device memory it owns (after the stream's queued work on it). */
ig_status ig_mesh_free(ig_mesh* mesh);

/* Sizes of a mesh: vertices, faces, stored nonzeros of L / A, device bytes owned. Any output
 * pointer may be NULL. */
ig_status ig_mesh_info(ig_mesh* mesh, int64_t* n, int64_t* m, int64_t* nnz, int64_t* device_bytes);

/* Copy the CSR pattern into caller device buffers rowptr_dev [n+1] and col_dev [nnz] (int32). */
ig_status ig_mesh_pattern(ig_mesh* mesh, int32_t* rowptr_dev, int32_t* col_dev);

/* Assemble A = M(V) + t L(V) for positions V_dev [n][3] (§7.1: L(v), M(v) recomputed
 * whenever v changes). precision = IG_PRECISION_FP64 keeps A in FP64; IG_PRECISION_MIXED also
 * keeps an FP32 copy of A and its diagonal for the inner iterations (the FP64 operator is
 * still the one every residual is measured against); IG_PRECISION_MIXED_GEOM32 computes the
 * face geometry in FP32 (FP64 for faces whose smallest corner has sin < 1e-2) and keeps only
 * the FP32 operator, which ig_operator then returns (its values are exact in FP64); positions
 * must lie within the float range in this mode. Asynchronous; a zero-area face or a
 * non-finite coordinate is reported by the next synchronising call (ig_solve with info, or
 * ig_check), as IG_ERR_DEGENERATE_FACE / IG_ERR_NONFINITE.
 * Errors: IG_ERR_INVALID_ARG (t < 0 or not finite, bad precision), IG_ERR_OOM, IG_ERR_CUDA. */
ig_status ig_assemble(ig_mesh* mesh, const double* V_dev, double t, int precision);

/* Cotangent clamp: with enable != 0, every corner's cotangent enters L as max(cot, clamp_min) --
 * the cotangent weights with a minimum (clamp_min) of the paper's §4 ARAP listing, applied per
 * corner before the two corners of an edge are added -- and a clamped corner (cot < clamp_min)
 * adds nothing to dl/dV (the clamp is constant there), while dl/dt uses clamp_min for it. With
 * clamp_min >= 0 every off-diagonal entry of L is <= -clamp_min / 2. enable = 0 restores the
 * plain cotangents. It applies to every later assembly of this mesh, in every precision, and to
 * the gradients of those assemblies; the mesh must be assembled again after the call
 * (IG_ERR_STATE otherwise). The geodesic calls (ig_rgd_*), whose identity L = D G needs the plain
 * cotangents, return IG_ERR_STATE on a mesh with the clamp on.
 * Errors: IG_ERR_INVALID_ARG (NULL mesh, clamp_min not finite). */
ig_status ig_mesh_set_cot_clamp(ig_mesh* mesh, int enable, double clamp_min);

/* Synchronise and return the first error the device recorded for this mesh since upload
 * (assembly or solve), or IG_OK. */
ig_status ig_check(ig_mesh* mesh);

/* Copy the assembled operator: Aval_dev [nnz] (values of A on the pattern, FP64) and
 * M_dev [n] (the lumped mass). Either pointer may be NULL. */
ig_status ig_operator(ig_mesh* mesh, double* Aval_dev, double* M_dev);

/* Copy the FP32 operator of a mixed-precision assembly (IG_PRECISION_MIXED or
 * IG_PRECISION_MIXED_GEOM32) on the pattern: Aval_dev [nnz] floats, in the order of ig_operator.
 * With IG_PRECISION_MIXED each value is the FP64 value rounded to nearest (ties to even).
 * Errors: IG_ERR_INVALID_ARG (NULL mesh or pointer), IG_ERR_STATE (no mixed-precision
 * assembly). */
ig_status ig_operator32(ig_mesh* mesh, float* Aval_dev);

/* Solve A U = M B (the forward smoothing step of §7.1) by Jacobi-preconditioned conjugate
 * gradients, x0 = 0, every column to opts->rel_tol (FP64 operator; in mixed precision the
 * iterations run in FP32 and the residual is recomputed in FP64 between refinements).
 * B_dev, U_dev are [n][k], 1 <= k <= 4, and may not overlap. opts may be NULL (defaults).
 * Errors: IG_ERR_STATE (not assembled), IG_ERR_INVALID_ARG, and -- only when info is given --
 * IG_ERR_NOT_CONVERGED / IG_ERR_NONFINITE / IG_ERR_DEGENERATE_FACE from the device. */
ig_status ig_solve(ig_mesh* mesh, const double* B_dev, int k, double* U_dev, const ig_solve_opts* opts,
                   ig_solve_info* info);

/* Reverse pass of ig_solve for the loss l(U): solves A Lambda = G_dev (G = dl/dU, [n][k]) and
 * writes the vector-Jacobian products
 *   gV_dev [n][3] : dl/dV (NULL not allowed),
 *   gB_dev [n][k] : dl/dB = M Lambda (may be NULL),
 *   gt_dev [1]    : dl/dt = -<Lambda, L U> (device double; may be NULL).
 * V_dev must hold the positions the operator was assembled with, U_dev the forward solution.
 * b_is_V != 0 means the forward right-hand side was B = V itself (k must be 3): the explicit
 * term M Lambda is then added to gV and B_dev is ignored. The gradient is gathered per vertex
 * from per-face contributions, without atomics. Errors as for ig_solve. */
ig_status ig_adjoint(ig_mesh* mesh, const double* V_dev, const double* B_dev, int b_is_V, const double* U_dev,
                     const double* G_dev, int k, double* gV_dev, double* gB_dev, double* gt_dev,
                     const ig_solve_opts* opts, ig_solve_info* info);

/* ---- batches ------------------------------------------------------------------------------ */
/* A batch runs the assembly, the solves and the gradient of many meshes in the same kernel
 * launches: the block-diagonal system of independent smoothing steps (§7.1 applied to each
 * mesh), every mesh with its own t, its own conjugate-gradient scalars and its own convergence
 * test. A mesh gives the same bits alone and inside a batch. Array-of-pointer arguments are HOST
 * arrays with one device pointer per mesh, in the order the meshes were given; per-mesh arrays
 * follow the single-mesh conventions. A mesh may belong to several batches but must not be used
 * by two calls at once. */

/* Create a batch over count (1..1024) meshes of ctx. The batch does not own the meshes; free the
 * batch before them. Errors: IG_ERR_INVALID_ARG (bad count, repeated or foreign mesh), IG_ERR_OOM. */
ig_status ig_batch_create(ig_ctx* ctx, ig_mesh* const* meshes, int count, ig_batch** out);

/* Release a batch (not its meshes). */
ig_status ig_batch_free(ig_batch* batch);

/* Assemble every mesh: V_dev[i] [n_i][3] and t[i] (host array of doubles). Same semantics and
 * errors as ig_assemble, for all meshes in two launches. */
ig_status ig_batch_assemble(ig_batch* batch, const double* const* V_dev, const double* t, int precision);

/* Solve A_i U_i = M_i B_i for every mesh (k columns each, shared options). infos, if given, is
 * a host array of count records; the call then synchronises and returns the first failing
 * status (or IG_OK). Errors as ig_solve. */
ig_status ig_batch_solve(ig_batch* batch, const double* const* B_dev, int k, double* const* U_dev,
                         const ig_solve_opts* opts, ig_solve_info* infos);

/* Reverse pass of ig_batch_solve (as ig_adjoint, per mesh): G_dev[i] = dl/dU_i; writes gV_dev[i],
 * gB_dev[i] (gB_dev may be NULL) and gt_dev[i] (gt_dev is a DEVICE array of count doubles or
 * NULL). */
ig_status ig_batch_adjoint(ig_batch* batch, const double* const* V_dev, const double* const* B_dev, int b_is_V,
                           const double* const* U_dev, const double* const* G_dev, int k, double* const* gV_dev,
                           double* const* gB_dev, double* gt_dev, const ig_solve_opts* opts, ig_solve_info* infos);

/* ---- continuous batching (serving) ------------------------------------------------------- */
/* A served request is one forward + adjoint solve whose iterations interleave with those of the
 * other requests in flight. ig_solve_begin starts a solve on a mesh (its state stays on the
 * device), ig_batch_iterate advances every running solve of a batch by up to max_iters
 * iterations in shared launches, and ig_solve_end writes a finished solve's result. Members may
 * be at different stages (forward or adjoint, any iteration, any refinement). */

/* Start solving A X = M in (rhs_mass != 0) or A X = in (rhs_mass == 0) on one mesh: the
 * initialisation kernel only. in_dev [n][k] must stay valid until ig_solve_end. */
ig_status ig_solve_begin(ig_mesh* mesh, const double* in_dev, int k, int rhs_mass, const ig_solve_opts* opts);

/* Advance the running solves of the batch's meshes by at most max_iters iterations (all k
 * columns; meshes already done are skipped). The loop returns early as soon as one of the solves
 * that were running finishes. Synchronises; done_host (host array of count ints, may be NULL)
 * receives 1 for each mesh whose solve is finished. */
ig_status ig_batch_iterate(ig_batch* batch, int k, int max_iters, int* done_host);

/* Write the result of a finished (or interrupted) solve: X into out_dev [n][k], or, when out_dev
 * is NULL, into the mesh's adjoint buffer used by ig_vjp. info as for ig_solve (synchronises). */
ig_status ig_solve_end(ig_mesh* mesh, int k, double* out_dev, ig_solve_info* info);

/* The gradient half of ig_adjoint: after an adjoint solve ended with out_dev == NULL, gather
 * dl/dV (and dl/dB, dl/dt) as ig_adjoint does. Same arguments and layouts. */
ig_status ig_vjp(ig_mesh* mesh, const double* V_dev, const double* B_dev, int b_is_V, const double* U_dev, int k,
                 double* gV_dev, double* gB_dev, double* gt_dev);

/* ---- mass gradient and the inverse-fairing loop (§7.1) --------------------------------------- */

/* gV_dev [n][3] = d( sum_i M_i(V) w_i )/dV for positions V_dev [n][3] and per-vertex weights
 * w_dev [n] (the lumped mass M_i = sum of area/3 over the faces at vertex i). This is the
 * part of a loss that depends on V through the mass directly, e.g. the M-norm loss
 * 1/2 ||T - U||_M^2 of the inverse-fairing objective of §7.1, with w = |T - U|^2 / 2.
 * Needs only ig_mesh_upload. Asynchronous. Errors: IG_ERR_INVALID_ARG (NULL pointer). */
ig_status ig_mass_vjp(ig_mesh* mesh, const double* V_dev, const double* w_dev, double* gV_dev);

/* One step of the inverse-fairing optimisation of §7.1, every part on the device:
 *   assemble A = M(V) + t L(V); U = A^-1 M V (the fairing of V);
 *   loss = 1/2 sum_i M_i |T_i - U_i|^2 (the M-norm objective against targets T_dev [n][3]);
 *   g = dloss/dV by the adjoint rule (Eq. 3; with B = V) plus the direct mass term;
 *   Sobolev H^1 preconditioning with the same operator, g~ = A^-1 g; V <- V - eta g~.
 * V_dev [n][3] is updated in place. precision: IG_PRECISION_FP64 or IG_PRECISION_MIXED. loss_host (may be NULL)
 * receives the loss at the positions the step started from (synchronises). info3 (may be NULL)
 * is an array of 3 ig_solve_info for the forward, adjoint and preconditioning solves
 * (synchronises). Workspace (13 n doubles) is allocated on the mesh at the first call.
 * Errors: IG_ERR_INVALID_ARG (NULL pointer, eta < 0 or not finite, bad t or precision),
 * the errors of ig_assemble and ig_solve, IG_ERR_OOM, IG_ERR_CUDA. */
ig_status ig_fairing_step(ig_mesh* mesh, double* V_dev, const double* T_dev, double t, double eta, int precision,
                          const ig_solve_opts* opts, double* loss_host, ig_solve_info* info3);

/* ---- Laplacian eigenvectors by shift-invert subspace iteration (Eq. eigiter of §5) ------------ */

/* The lowest k eigenpairs of the pencil L u = lambda M u of the assembled mesh, by the
 * fixed-point iteration U <- Q((L - sigma M)^-1 M U) of Eq. eigiter (§5) with the shift
 * sigma = -1/t of the assembled operator: (L - sigma M)^-1 M = t (M + t L)^-1 M, so each of the
 * `iters` steps is the smoothing solve (M + tL) Y = M U (k columns together, to opts->rel_tol, in
 * the assembled precision) followed by Q: the M-orthonormal basis of Y's columns in Gram-Schmidt
 * order (Y = Q R, R upper triangular from the Cholesky factor of Y^T M Y). A larger t separates
 * the lowest eigenvalues more per step: the error of column c shrinks by about
 * (1 + t lambda_c) / (1 + t lambda_{c+1}) per step.
 * After the last step every column gets a canonical sign: its first entry, in vertex order, whose
 * magnitude is within a relative 1e-6 of the column's largest magnitude is made positive.
 * U_dev: [n][k] row-major device buffer: the start basis on entry (linearly independent
 * columns, e.g. random), the M-orthonormal result on return. k in 1..4, iters >= 1.
 * lambda_host (may be NULL): k doubles, lambda_c = u_c^T L u_c, computed from the FP64 operator as
 * (u_c^T A u_c - u_c^T M u_c) / t. info (may be NULL): status and iteration count of the last
 * solve. Either synchronises the stream; without both the call is asynchronous.
 * Workspace (17 n + 16 ceil(n / 256) doubles and a few bytes, shared with ig_eigs_vjp) is
 * allocated on the mesh at the first call. Errors: IG_ERR_STATE (not assembled), IG_ERR_INVALID_ARG (NULL U_dev, k or iters
 * out of range), IG_ERR_NONFINITE (a Gram matrix was not positive definite: the start columns
 * were dependent or not finite; reported when lambda_host or info is given), the errors of
 * ig_solve, IG_ERR_OOM, IG_ERR_CUDA; IG_ERR_STATE also for a mesh assembled with
 * IG_PRECISION_MIXED_GEOM32. The gradient through this fixed point: ig_eigs_vjp. */
ig_status ig_eigs(ig_mesh* mesh, int k, int iters, double* U_dev, double* lambda_host, const ig_solve_opts* opts,
                  ig_solve_info* info);

/* Gradient of a loss l(U*) with respect to the positions through the fixed point of ig_eigs,
 * U* = Q((M + tL)^-1 M U*) (Eq. eigiter, §5), by the implicit-function rule for fixed points:
 * w = gU + J^T w with J = dQ((M + tL)^-1 M U)/dU at U*, solved by `iters` terms of its Neumann
 * series (each one k-column solve with the assembled operator; the series contracts at the rate
 * of the forward iteration, so about as many terms as forward steps are needed, and it converges
 * only when the k lowest eigenvalues are distinct), then dl/dV = (df/dV)^T w: the adjoint-solve
 * term <Lambda, d(M U*)/dV - dA/dV Y> (Y = (M + tL)^-1 M U*, Lambda = (M + tL)^-1 Ybar) and the
 * mass term of the orthonormalization's Gram matrix Y^T M Y. The converged eigenvectors do not
 * depend on t, nor does this gradient.
 * V_dev [n][3]: the positions the mesh was assembled at. U_dev [n][k]: the result of ig_eigs.
 * gU_dev [n][k]: dl/dU*. gV_dev [n][3]: the result. k in 1..4, iters >= 1.
 * Synchronises. Uses ig_eigs's workspace and the mesh's adjoint buffer.
 * Errors: IG_ERR_STATE (not assembled), IG_ERR_INVALID_ARG (NULL pointer, k or iters out of range),
 * IG_ERR_NONFINITE (the Gram matrix of (M + tL)^-1 M U* is not positive definite), the errors of
 * ig_solve, IG_ERR_OOM, IG_ERR_CUDA. */
ig_status ig_eigs_vjp(ig_mesh* mesh, const double* V_dev, int k, int iters, const double* U_dev, const double* gU_dev,
                      double* gV_dev, const ig_solve_opts* opts);

/* ---- regularized geodesic distances: the ADMM u-step --------------------------------------- */

/* The u-step of the ADMM scheme for regularized geodesic distances (the geodesics application,
 * formulation eq. edelstein: minimise -m^T u + beta/2 u^T L u subject to |(G u)_f| <= 1 and
 * u_s = 0 on the sources): with per-face iterates y_dev and z_dev [m][3] (the dual variable and
 * z = G u),
 *   b = m - D y + rho D z,   L u = b / (beta + rho) on the non-source vertices,   u = 0 on the sources,
 * with m the lumped vertex areas, G the face gradient of piecewise-linear functions, D = G^T A_F its
 * area-weighted adjoint (L = D G is the cotangent Laplacian). The solve is the Jacobi-PCG of
 * ig_solve on the Laplacian whose source rows and columns are the identity, in FP64, to
 * opts->rel_tol. V_dev [n][3]: positions. sources_host: nsrc >= 1 vertex indices in host memory
 * (every connected part of the mesh needs one, or the system is singular and the solve reports
 * IG_ERR_NOT_CONVERGED). u_dev [n]: the result. rho, beta >= 0, rho + beta > 0.
 * The call assembles the mesh at V (t = 1) and then rewrites its operator, so the mesh must be
 * assembled again before any other solve. info as for ig_solve (synchronises).
 * Errors: IG_ERR_INVALID_ARG (NULL pointer, no source, a source out of range, bad rho or beta),
 * the errors of ig_assemble and ig_solve, IG_ERR_OOM, IG_ERR_CUDA. */
ig_status ig_rgd_u_step(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc, const double* y_dev,
                        const double* z_dev, double rho, double beta, double* u_dev, const ig_solve_opts* opts,
                        ig_solve_info* info);

/* Gradients of a loss l(u) through the u-step of ig_rgd_u_step, for its result u_dev [n] and
 * gu_dev = dl/du [n], with the same V, sources, y, z, rho and beta: with lam = L_D^-1 gu (the same
 * source-constrained Laplacian; lam = 0 on the sources) and s = 1 / (beta + rho),
 *   gy_dev [m][3] = dl/dy = -s area_f grad(lam)_f,   gz_dev [m][3] = dl/dz = rho s area_f grad(lam)_f,
 *   gV_dev [n][3] = dl/dV = s <lam, dm/dV> - <lam, dL/dV u> + s <lam, dD/dV (rho z - y)>.
 * gy_dev and gz_dev may be NULL. Asynchronous. Like ig_rgd_u_step it assembles the mesh at V and
 * rewrites the operator, and it uses the mesh's adjoint buffer.
 * Errors: as ig_rgd_u_step (a solve that does not converge is not reported; use ig_rgd_u_step's
 * info on the same inputs). */
ig_status ig_rgd_u_step_vjp(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc,
                            const double* y_dev, const double* z_dev, double rho, double beta, const double* u_dev,
                            const double* gu_dev, double* gV_dev, double* gy_dev, double* gz_dev,
                            const ig_solve_opts* opts);

/* Rounds of the ADMM scheme for regularized geodesic distances (formulation eq. edelstein and its
 * listing), every part on the device: the u-step of ig_rgd_u_step; the z-step
 * z_f = P(y_f / rho + (G u)_f), P the projection onto the unit ball; the dual step
 * y_f += rho (beta_k (G u)_f + (1 - beta_k) z_f,old - z_f). With beta = 0 and enough rounds u
 * approaches the geodesic distance from the sources (under the constraint |G u| <= 1).
 * Residuals of a round: primal = max_f |(G u)_f - z_f|, dual = rho max_i |(D (z - z_old))_i| / m_i
 * over the non-source vertices. With tol > 0 the rounds stop once both are <= tol; with adapt_rho
 * rho is doubled after a round whose primal exceeds 10 x its dual, halved in the opposite case
 * (residual balancing; y is the unscaled dual, so it needs no rescaling). Either setting reads the
 * residuals after every round (one synchronisation per round); with neither, exactly max_rounds
 * rounds run without synchronising.
 * y_dev and z_dev [m][3]: the start (e.g. zeros) on entry, the last iterates on return. u_dev [n]:
 * the last u. stats_host (may be NULL): 5 doubles, the rounds run, the primal and dual residuals
 * of the last round, the final rho, and the rounds that needed no solve (below). rho > 0,
 * beta >= 0, beta_k in [0, 2] (over-relaxation), max_rounds >= 1, tol >= 0. The operator is built
 * once (as in ig_rgd_u_step); each round after the first warm-starts its Laplacian solve from the
 * previous round's u (it solves A d = b - A u for the correction, to the tolerance that leaves
 * |b - A (u + d)| <= opts->rel_tol |b|, the criterion of a cold solve, and skips the solve when u
 * already meets it), which reads one scalar back per round (the call synchronises every round).
 * The mesh must be assembled again before other solves.
 * Errors: as ig_rgd_u_step, and IG_ERR_INVALID_ARG for max_rounds, rho, beta_k or tol out of
 * range. IG_ERR_NOT_CONVERGED / IG_ERR_NONFINITE when a round's solve ended so (the worst over the
 * rounds); the rounds still run to the end and every output is written. */
ig_status ig_rgd_admm(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc, double rho, double beta,
                      double beta_k, int max_rounds, double tol, int adapt_rho, double* u_dev, double* y_dev,
                      double* z_dev, double* stats_host, const ig_solve_opts* opts);

/* Gradient through the converged ADMM (the framework's fixed-point implicit layer, section on
 * implicit differentiation, applied to the geodesics application): for l(u*) with u* the u-step
 * at a fixed point (y*, z*) = T(y*, z*) of one round T of ig_rgd_admm (fixed rho), and
 * gu_dev [n] = dl/du*, it writes
 *   gV_dev [n][3] = dl/dV = gV0 + (dT/dV)^T w,   where (I - J^T) w = (gy0, gz0),
 * J = dT/d(y, z) and (gV0, gy0, gz0) is the u-step's VJP of gu (ig_rgd_u_step_vjp). The adjoint
 * system is solved by restarted GMRES (restart vectors of 6 m doubles each, 1 <= restart <= 100;
 * at most max_iter Arnoldi steps; stop when the residual estimate is <= tol |(gy0, gz0)|), and
 * each product with J^T is the round's backward pass: per face through the projection and the dual
 * step, G^T, and one constrained Laplacian solve to opts->rel_tol.
 * y_dev, z_dev [m][3]: the fixed point, e.g. the iterates ig_rgd_admm returned with its final rho
 * (y is the unscaled dual, so (y*, z*) is a fixed point of T for every rho). w_dev [2][m][3] (may
 * be NULL): receives w = (w_y, w_z). stats_host (may be NULL): 3 doubles, the Arnoldi steps
 * taken, the final relative residual estimate and 1 if it met tol, else 0. Synchronises; the
 * GMRES basis ((restart + 1) x 6 m doubles) is allocated for the call. Like ig_rgd_u_step it
 * assembles the mesh at V, rewrites the operator and uses the mesh's adjoint buffer.
 * Errors: as ig_rgd_admm; IG_ERR_INVALID_ARG for restart or max_iter out of range;
 * IG_ERR_NOT_CONVERGED when GMRES stops at max_iter above tol (gV is still written from its best
 * iterate); IG_ERR_NONFINITE for a non-finite residual. */
ig_status ig_rgd_admm_vjp(ig_mesh* mesh, const double* V_dev, const int32_t* sources_host, int nsrc, double rho,
                          double beta, double beta_k, const double* y_dev, const double* z_dev, const double* gu_dev,
                          int restart, int max_iter, double tol, double* gV_dev, double* w_dev, double* stats_host,
                          const ig_solve_opts* opts);

/* ---- allocation-free solve ----------------------------------------------------------------- */

/* Largest number of rows ig_solve_csr_noalloc accepts. */
#define IG_NOALLOC_MAX_ROWS 65536

/* Solve A X = M B (or A X = B when M_dev is NULL) for a CSR operator the caller already holds,
 * by the same Jacobi-preconditioned conjugate gradients as ig_solve, WITHOUT ALLOCATING: no
 * cudaMalloc, cudaFree, graph or other allocating call is made. It is meant for callers that
 * cannot allocate device memory -- a host running under a fixed memory plan or pre-reserved
 * arena that forbids new device allocations after start-up, or a process whose device memory
 * belongs to another framework's allocator. The paper has no counterpart to this call; it is a
 * service of this library.
 *
 * Inputs (device pointers on the CURRENT CUDA device): rowptr_dev [n+1] and col_dev [nnz] int32
 * (CSR, each row holding its diagonal), Aval_dev [nnz] double (symmetric positive definite
 * values, e.g. from ig_operator), M_dev [n] double or NULL, B_dev [n][k] double. Output: U_dev
 * [n][k] double (must not overlap B). 1 <= k <= 4, 1 <= n <= IG_NOALLOC_MAX_ROWS. Work goes on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream). The call SYNCHRONISES that stream:
 * its loop is driven from the host, which waits for a 4-byte flag every 16 iterations and for
 * the error word at the end, so it returns only after the solve has finished and it must never
 * be made while the stream (or any stream, in global capture mode) is being captured into a
 * CUDA graph. opts may be NULL (defaults; the launch mode is always one launch per kernel).
 * info, if given, is filled as by ig_solve.
 *
 * Scratch: all workspace lives in one static device array of about 9 MB, which every GPU that
 * loads this library holds until the process exits. The first call on a device looks up that
 * array's device address (once per device). Every call reuses the same array and overwrites
 * what the previous call left there (the call clears its counters itself); two calls that
 * overlap on the GPU -- on different streams or from different host threads -- race on the
 * array and give wrong results.
 *
 * Before solving, a set-up kernel checks the caller's pattern on the device (the call reads the
 * result back and returns without solving, U untouched, when it fails):
 * IG_ERR_INDEX_OUT_OF_RANGE for a row range outside [0, nnz) or a column outside [0, n);
 * IG_ERR_INVALID_ARG for a missing or non-positive (or non-finite) diagonal entry. These are
 * reported with or without info (info->status carries them too).
 * Other errors: IG_ERR_INVALID_ARG for a NULL pointer, n > IG_NOALLOC_MAX_ROWS, nnz < n, k
 * outside [1, 4], overlapping B and U or bad options; IG_ERR_CUDA for a failed launch; with info,
 * IG_ERR_NOT_CONVERGED / IG_ERR_NONFINITE as for ig_solve. */
ig_status ig_solve_csr_noalloc(const int32_t* rowptr_dev, const int32_t* col_dev, const double* Aval_dev,
                               const double* M_dev, int64_t n, int64_t nnz, const double* B_dev, int k,
                               double* U_dev, void* cuda_stream, const ig_solve_opts* opts, ig_solve_info* info);

/* ---- kernel timing (tracing) -------------------------------------------------------------- */

/* Per-kernel device time accumulated while profiling is on. */
typedef struct {
  char name[48];      /* kernel name */
  int64_t launches;   /* launches timed */
  double total_ms;    /* summed device time between the CUDA events around each launch */
} ig_kernel_stat;

/* Turn process-wide kernel timing on (enable != 0) or off, clearing the accumulated figures.
 * While it is on, every launch is bracketed by CUDA events on the stream it is issued on, and
 * the conjugate-gradient loop is launched from the host (one launch per kernel) so that each
 * iteration's kernels are timed individually. It changes no result. */
ig_status ig_profile_enable(int enable);

/* Synchronise on the recorded events and copy up to max per-kernel records into out; returns
 * the number of kernel names recorded (which may exceed max). */
int ig_profile_read(ig_kernel_stat* out, int max);

/* ---- measured arithmetic peak ------------------------------------------------------------- */

/* Measure the device's fused multiply-add throughput, the ceiling of kernels bound by arithmetic
 * instructions rather than by memory (on this GPU the FP64 ones: assembly, the per-face gradient
 * and the FP64 solver loop). A grid of one wave of resident CTAs on every SM (current device) runs
 * 8 independent FMA chains per thread for `steps` steps (2 flops per FMA) after a short warm-up,
 * timed with CUDA events on cuda_stream. precision: IG_PRECISION_FP64 for double FMA,
 * IG_PRECISION_MIXED for float FMA. flops_per_s receives the measured rate, seconds (may be NULL)
 * the kernel's duration. Synchronises; allocates a small output buffer for the call. The rate
 * follows the SM clock: sample the clock alongside it.
 * Errors: IG_ERR_INVALID_ARG (NULL flops_per_s, steps < 1, bad precision), IG_ERR_OOM, IG_ERR_CUDA. */
ig_status ig_measure_fma_peak(int precision, int steps, void* cuda_stream, double* flops_per_s, double* seconds);

#ifdef __cplusplus
}
#endif

#endif /* ISKRA_GB300_H */
