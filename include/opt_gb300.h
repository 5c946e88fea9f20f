/*
 * opt_gb300.h -- C ABI of the GB300 (sm_103a) Gauss-Newton / Levenberg-Marquardt
 * PCG solver for sum-of-squares energies E(x) = sum_r f_r(x)^2 (Sec. 2, Sec. 4).
 *
 * The shape follows the paper's split of a solve into define / plan / solve
 * (Fig. 4 and Sec. 3 "API": compile, allocate and run are separate calls so
 * that set-up is amortised over many solves).  The energy templates are fixed
 * and hand-derived (no DSL): ARAP image warping (Fig. 24), Poisson image
 * editing (Fig. 27), ARAP mesh deformation (Fig. 25), the warp on an
 * explicit graph (Fig. 18), volumetric ARAP (Fig. 31) and embedded
 * deformation (Fig. 28).
 *
 * Conventions for every call:
 *  - Pointers named "device" point to CUDA global memory on the current
 *    device; pointers named "host" point to host memory.  No call takes
 *    ownership of a caller pointer.
 *  - Unknown arrays are owned by the caller.  A call that evaluates at x reads
 *    them when it starts; opt_solve_gn / opt_solve_lm write the solution back
 *    into them when they finish.  Constant arrays (rest shape, guidance image,
 *    mask, handles) are copied into the problem when it is created.
 *  - The library owns its scratch (PCG vectors, reduction slots, CSR arrays)
 *    and frees it in opt_problem_destroy.
 *  - All device work is ordered on the stream given in opt_solve_params
 *    (NULL = the legacy default stream).  Calls that return results to the
 *    host synchronise that stream.  One problem must not be used from two
 *    host threads or two streams at once.
 *  - Arithmetic: residuals, Jacobian entries, J^T J p and vector updates run
 *    in float32; PCG dot products (alpha, beta), energies and the LM gain
 *    ratio run in float64.
 *  - Errors: every call returns an opt_status; no exception crosses the ABI.
 *    OPT_ERR_INVALID_ARG leaves the problem unchanged.  OPT_ERR_CUDA means a
 *    CUDA call failed (the message is in opt_last_error()).
 */
#ifndef OPT_GB300_H
#define OPT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OPT_OK = 0,
    OPT_ERR_INVALID_ARG = 1,  /* bad shape, null pointer, index out of range, non-finite input */
    OPT_ERR_OOM = 2,          /* device allocation failed */
    OPT_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    OPT_ERR_NUMERIC = 4,      /* non-finite energy or PCG scalar produced by a solve */
    OPT_ERR_TIMEOUT = 5,      /* a bounded device-side wait expired */
    OPT_ERR_BUDGET = 6,       /* admission refused: the memory budget is exhausted */
    OPT_ERR_NOT_READY = 7     /* the batched / served solve has not finished yet */
} opt_status;

typedef enum {
    OPT_ARAP_WARP_2D = 0,     /* Fig. 24: unknowns dx, dy, theta per pixel */
    OPT_POISSON_2D = 1,       /* Fig. 27: unknowns X (4 channels) per pixel */
    OPT_ARAP_MESH = 2,        /* Fig. 25: unknowns dx, dy, dz, ax, ay, az per vertex */
    OPT_ARAP_WARP_GRAPH = 3,  /* Fig. 24 on an explicit graph (Fig. 18): dx, dy, theta per vertex */
    OPT_ARAP_VOLUME = 4,      /* Fig. 31: dx, dy, dz, ax, ay, az per voxel of a 3-D grid */
    OPT_EMBEDDED_DEFORMATION = 5  /* Fig. 28: dx, dy, dz and a 3x3 matrix per vertex */
} opt_energy;

typedef struct opt_problem opt_problem;

/* Grid (image) problem, Sec. 4.1 "Stencil-based Array Access".
 * Every plane is W*H float32 (or uint8) values, row-major, index y*W + x.
 *   OPT_ARAP_WARP_2D (Fig. 24):
 *     unknowns[0..2] = dx, dy, theta (device).  Offset = UrShape + (dx, dy).
 *     consts[0..1]   = UrShape x, y (device).
 *     mask           = nonzero marks an excluded pixel (device, may be NULL).
 *     handle_idx     = n_handles distinct pixel indices (device).
 *     handle_target  = n_handles (tx, ty) target displacements, interleaved (device).
 *     Residuals: for every pixel k and direction d in {+x,-x,+y,-y} with k+d in
 *     the image and both pixels unmasked,
 *       sqrt(w_reg) * ((O_k - O_{k+d}) - R(theta_k)(U_k - U_{k+d})),
 *     R counter-clockwise; for every handle h, sqrt(w_fit) * (O_h - C_h)
 *     with C_h = U_h + target.
 *   OPT_POISSON_2D (Fig. 27):
 *     unknowns[0..3] = X channels (device); consts[0..3] = guidance T (device);
 *     mask = nonzero marks a fixed pixel (device, may be NULL = all free).
 *     Residuals: for every free pixel k and direction d with k+d in the image,
 *       (X_k - X_{k+d}) - (T_k - T_{k+d}) per channel; fixed neighbours are
 *     constants.  Handles and weights are ignored. */
typedef struct {
    int32_t kind;
    int32_t W, H;
    float* unknowns[4];
    const float* consts[4];
    const uint8_t* mask;
    const int32_t* handle_idx;
    const float* handle_target;
    int32_t n_handles;
    float w_reg, w_fit;
} opt_grid_desc;

/* Graph (mesh) problem, Sec. 4.1 "Graph-based Array Access", Fig. 25.
 *   v0, v1      = E directed edges (device int32, any order; the library
 *                 keeps a copy sorted by (v0, v1)).
 *   unknowns[6] = dx, dy, dz (displacement from UrShape) and Euler angles
 *                 ax, ay, az in radians, V floats each (device).
 *   urshape[3]  = rest positions x, y, z (device).
 *   handle_idx / handle_target = n_handles distinct vertices and (x, y, z)
 *                 target displacements, interleaved (device).
 *   Residuals: for every edge (a, b),
 *     sqrt(w_reg) * ((O_a - O_b) - Rz(az_a) Ry(ay_a) Rx(ax_a) (U_a - U_b));
 *   for every handle, sqrt(w_fit) * (O_h - C_h), C_h = U_h + target. */
typedef struct {
    int32_t V, E;
    const int32_t* v0;
    const int32_t* v1;
    float* unknowns[6];
    const float* urshape[3];
    const int32_t* handle_idx;
    const float* handle_target;
    int32_t n_handles;
    float w_reg, w_fit;
} opt_graph_desc;

/* Volumetric ARAP deformation (Fig. 31, Appendix A.2.5): a W x H x D voxel
 * grid, voxel index (z*H + y)*W + x, every plane W*H*D float32 values.
 *   unknowns[6] = dx, dy, dz (Offset - UrShape) and Euler angles ax, ay, az
 *                 (device).
 *   urshape[3]  = rest positions x, y, z (device).
 *   handle_idx / handle_target = n_handles distinct constrained voxels and
 *                 their (x, y, z) target displacements, interleaved (device).
 *   Residuals: for every voxel k and direction d in {+-x, +-y, +-z} with k+d
 *   in the grid, sqrt(w_reg) * ((O_k - O_{k+d}) - Rz Ry Rx(A_k) (U_k - U_{k+d}));
 *   for every constrained voxel, sqrt(w_fit) * (O_h - C_h), C_h = U_h + target. */
typedef struct {
    int32_t W, H, D;
    float* unknowns[6];
    const float* urshape[3];
    const int32_t* handle_idx;
    const float* handle_target;
    int32_t n_handles;
    float w_reg, w_fit;
} opt_volume_desc;

/* Embedded deformation (Fig. 28, Appendix A.2.1): per vertex a displacement
 * and a full 3x3 matrix R instead of Euler angles, with soft constraints
 * that keep R a rotation.
 *   v0, v1       = E directed edges (device, any order; as opt_graph_desc).
 *   unknowns[12] = dx, dy, dz (Offset - UrShape), then R row-major R00, R01,
 *                  R02, R10, ..., R22, V floats each (device).  Identity
 *                  matrices and zero displacement are the rest state.
 *   urshape[3], handle_idx, handle_target: as opt_graph_desc.
 *   Residuals: for every edge (a, b),
 *     sqrt(w_reg) * ((O_a - O_b) - R_a (U_a - U_b));
 *   for every vertex, with c_k = (R[k], R[3+k], R[6+k]) the columns of R,
 *     sqrt(w_rot) * (c0.c1), (c0.c2), (c1.c2), (c0.c0 - 1), (c1.c1 - 1), (c2.c2 - 1);
 *   for every handle, sqrt(w_fit) * (O_h - C_h), C_h = U_h + target. */
typedef struct {
    int32_t V, E;
    const int32_t* v0;
    const int32_t* v1;
    float* unknowns[12];
    const float* urshape[3];
    const int32_t* handle_idx;
    const float* handle_target;
    int32_t n_handles;
    float w_reg, w_fit, w_rot;
} opt_embedded_desc;

/* Solver parameters (Sec. 4, Sec. 7 "LM vs. GN", "Matrix-free vs.
 * Materialized").  opt_solve_params_default fills the values used by the
 * paper-shaped configurations; lambda0 is the inverse initial trust radius. */
typedef struct {
    int32_t outer;            /* GN / LM outer iterations (>= 1) */
    int32_t inner;            /* PCG iterations per outer iteration (>= 0) */
    double lambda0;           /* LM initial damping (default 1e-3) */
    double lambda_min;        /* LM damping clamp (default 1e-16) */
    double lambda_max;        /* (default 1e32) */
    double diag_min;          /* LM clamp of diag(J^T J) entries (default 1e-6) */
    double diag_max;          /* (default 1e32) */
    double eta;               /* LM acceptance threshold on the gain ratio (default 1e-3) */
    double rel_tol;           /* LM: stop after an accepted step with |dE|/E < rel_tol (0 = off) */
    int32_t use_precond;      /* 1 = Jacobi preconditioner (default), 0 = plain CG */
    int32_t materialized;     /* 0 = matrix-free (default); 1 = materialized CSR J, q = J^T (J p)
                                 (Sec. 7); 2 = J^T J assembled once per outer iteration, q = A p
                                 (the paper's materialized form, Fig. 16).  Grid warp, Poisson,
                                 mesh and volume problems. */
    int32_t use_graph;        /* 1 = replay the solve as one CUDA graph (default) */
    int32_t tile_w;           /* grid planning only: tile width 32 or 128, 0 = automatic
                                 (128 for grids at least 128 pixels wide, else 32) */
    int32_t persistent;       /* 1 = run each outer iteration's PCG loop as one cooperative
                                 launch with grid-wide barriers when the problem is a wide-tile
                                 warp, matrix-free, and all its blocks fit on the device at once;
                                 0 (default) = one launch per PCG kernel, measured faster on
                                 GB300 (a barrier costs more than a kernel boundary with
                                 programmatic dependent launch).  Same arithmetic either way.  A
                                 barrier wait is bounded (1 s): OPT_ERR_TIMEOUT. */
    void* stream;             /* cudaStream_t; NULL = legacy default stream */
    int32_t pcg_form;         /* 0 (default) = the two-pass Jacobi-PCG iteration of Sec. 4.1
                                 (applyJTJ with p.q, then the vector update with r.z: two
                                 grid-wide reductions, two launches per iteration).
                                 1 = single-reduction iteration, taken by matrix-free solves of
                                 OPT_ARAP_WARP_2D and OPT_POISSON_2D grids planned with 128-pixel
                                 tiles (other problems run form 0): it carries z = M^-1 r and
                                 w = M^-1 q instead of r and q, and one launch per iteration
                                 reduces p.q, q.z, q.M^-1 q and r.z together: alpha = r.z / p.q
                                 as in form 0, and the next r.z, which sets beta, by
                                 r.z' = r.z - 2 alpha q.z + alpha^2 q.M^-1 q.  The same iterates
                                 in exact arithmetic; in float32 they differ from form 0 by
                                 rounding.  Batches (and the server) apply it to their members of
                                 those kinds, the others run form 0.  Other values:
                                 OPT_ERR_INVALID_ARG. */
} opt_solve_params;

/* Result of a solve.  E_history, when not NULL, is a host array of at least
 * outer + 1 doubles that receives E(x_k) at the start of every executed outer
 * iteration followed by the final energy. */
typedef struct {
    int32_t outer_done;       /* outer iterations executed (LM: including rejected ones) */
    int32_t pcg_done;         /* PCG iterations completed over the whole solve */
    int32_t accepted;         /* LM: accepted steps (GN: = outer_done) */
    int32_t converged;        /* LM: stopped by rel_tol */
    double E0;                /* energy at the initial x */
    double E_final;           /* energy at the returned x */
    double lambda_final;      /* LM damping after the last update (GN: 0) */
    double* E_history;        /* host, caller-owned, or NULL */
    float ms;                 /* device time of the solve (CUDA events) */
} opt_report;

/* Fills *p with the defaults listed above (outer = 10, inner = 10, GN). */
opt_status opt_solve_params_default(opt_solve_params* p);

/* Plan a grid problem: validates the descriptor (OPT_ERR_INVALID_ARG on a bad
 * kind, W or H outside [1, 32768), null planes, handle index out of range or a
 * non-finite constant), copies the constants, and allocates the PCG scratch
 * (and the CSR arrays when params->materialized).  params may be NULL.
 * *out receives the problem; it stays NULL on error. */
opt_status opt_problem_create_grid(const opt_grid_desc* desc, const opt_solve_params* params,
                                   opt_problem** out);

/* Plan a graph problem (edges: 0 <= v0, v1 < V, v0 != v1, else
 * OPT_ERR_INVALID_ARG).  Same ownership rules as opt_problem_create_grid.
 * The library keeps its vertices in its own (locality) order; the caller's
 * planes stay in the caller's order. */
opt_status opt_problem_create_graph(const opt_graph_desc* desc, const opt_solve_params* params,
                                    opt_problem** out);

/* Plan ARAP image warping written on an explicit graph (OPT_ARAP_WARP_GRAPH:
 * Sec. 4.1 "Graph-based Array Access", the explicit side of the implicit
 * grid vs explicit graph comparison of Fig. 18), with opt_graph_desc read as
 *   unknowns[0..2] = dx, dy, theta per vertex (unknowns[3..5] unused);
 *   urshape[0..1]  = rest positions x, y (urshape[2] unused);
 *   handle_target  = n_handles (tx, ty) target displacements, interleaved.
 *   Residuals: for every edge (a, b),
 *     sqrt(w_reg) * ((O_a - O_b) - R(theta_a) (U_a - U_b)), R counter-clockwise;
 *   for every handle, sqrt(w_fit) * (O_h - C_h), C_h = U_h + target.
 * With the stencil neighbour pairs of an image as edges this is the
 * OPT_ARAP_WARP_2D energy.  Solves as a graph problem; there is no
 * materialized form (params.materialized = 1 gives OPT_ERR_INVALID_ARG at
 * solve time).  Errors as opt_problem_create_graph. */
opt_status opt_problem_create_graph2d(const opt_graph_desc* desc, const opt_solve_params* params,
                                      opt_problem** out);

/* Plan a volumetric ARAP problem (OPT_ARAP_VOLUME).  The voxel grid is the
 * implicit structure: the kernels take each voxel's neighbours from the
 * 7-point stencil (the mesh energy's gather kernels otherwise).  W, H, D >= 1
 * with W*H*D <= 2^27, same validation and ownership as
 * opt_problem_create_graph.  Solves like a graph problem, including the
 * materialized form. */
opt_status opt_problem_create_volume(const opt_volume_desc* desc, const opt_solve_params* params,
                                     opt_problem** out);

/* Plan an embedded deformation problem (OPT_EMBEDDED_DEFORMATION).  Same
 * validation (plus a finite w_rot >= 0), ownership and vertex ordering as
 * opt_problem_create_graph.  Solves as a graph problem, also in batches;
 * there is no materialized form (params.materialized != 0 gives
 * OPT_ERR_INVALID_ARG at solve time).  The paper solves this energy with
 * LM: GN is not robust on it (Appendix A.2.1). */
opt_status opt_problem_create_embedded(const opt_embedded_desc* desc, const opt_solve_params* params,
                                       opt_problem** out);

/* Frees everything the problem owns.  NULL is accepted. */
opt_status opt_problem_destroy(opt_problem* prob);

/* Gauss-Newton (Sec. 4): outer x inner iterations from the caller's current
 * unknowns, x written back at the end.  report may be NULL. */
opt_status opt_solve_gn(opt_problem* prob, const opt_solve_params* params, opt_report* report);

/* Levenberg-Marquardt (Sec. 4): as opt_solve_gn with damping
 * (J^T J + lambda D) d = -J^T F, D = clamp(diag(J^T J), diag_min, diag_max),
 * gain-ratio acceptance and Nielsen's damping update; everything stays on the
 * device. */
opt_status opt_solve_lm(opt_problem* prob, const opt_solve_params* params, opt_report* report);

/* PCGInit (Sec. 4.1, Sec. 4.2 evalJTF): reads the caller's unknowns, evaluates
 * F, b = -J^T F, the Jacobi preconditioner 1 / diag(J^T J + lambda D), sets
 * delta = 0, r = b, p = z = M^-1 r.  energy (host, may be NULL) receives E(x). */
opt_status opt_pcg_init(opt_problem* prob, double lambda, double* energy);

/* Runs n_iters PCG iterations (PCGStep kernels of Sec. 4.1: applyJTJ with the
 * direction update, then the vector update) on the state left by
 * opt_pcg_init or a previous opt_pcg_step.  Stream-ordered; no host sync. */
opt_status opt_pcg_step(opt_problem* prob, int32_t n_iters);

/* Copies the PCG state to caller device buffers in the dense layout of the
 * unknowns (any pointer may be NULL): delta, r, and the direction p. */
opt_status opt_pcg_get_state(opt_problem* prob, float* delta, float* r, float* p,
                             int32_t* iters_done);

/* q = (J^T J + lambda * D) p at the caller's current unknowns (Sec. 4.2
 * applyJTJ without the factor 2 that cancels).  p, q: device, dense layout of
 * the unknowns (excluded Poisson pixels must hold p = 0).  pq (host, may be
 * NULL) receives p.q in float64. */
opt_status opt_apply_jtj(opt_problem* prob, const float* p, float* q, double lambda, double* pq);

/* J^T F and diag(J^T J) at the caller's current unknowns (Sec. 4.2 evalJTF).
 * jtf, diag: device, dense layout (either may be NULL); energy: host (may be
 * NULL) receives E(x) = sum f_r^2 in float64. */
opt_status opt_eval_jtf(opt_problem* prob, float* jtf, float* diag, double* energy);

/* E(x) = sum f_r(x)^2 at the caller's current unknowns (Sec. 4.2 evalF). */
opt_status opt_eval_energy(opt_problem* prob, double* energy);

/* Measurement hook: runs PCGInit, then n_iters PCG iterations, with a CUDA
 * event pair around every launch on `stream` (cudaStream_t, NULL = legacy
 * default stream), synchronises, and writes the mean device time per launch
 * in milliseconds: ms[0] = PCGInit, ms[1] = applyJTJ (with the fused
 * direction update), ms[2] = vector update.  ms: host, 3 floats.  Leaves the
 * PCG state as opt_pcg_init + opt_pcg_step would (lambda = 0). */
opt_status opt_profile_pcg(opt_problem* prob, int32_t n_iters, void* stream, float* ms);

/* Measurement hook of the single-reduction PCG iteration (pcg_form = 1 of
 * opt_solve_params; the Jacobi-PCG of Sec. 4.1 with one reduction per
 * iteration): PCGInit, n_iters (>= 2) single-reduction iterations and the
 * final step, each launch bracketed by CUDA events on `stream`; writes ms[0]
 * = PCGInit, ms[1] = mean of iterations 1 .. n_iters - 1 (iteration 0 reads
 * r and M^-1 instead of z and w), ms[2] = the final step (host, 3 floats).
 * OPT_ERR_INVALID_ARG unless the problem is an OPT_ARAP_WARP_2D or
 * OPT_POISSON_2D grid planned with 128-pixel tiles, or n_iters < 2.  Leaves delta = the PCG step after
 * n_iters iterations (lambda = 0). */
opt_status opt_profile_pcg_fused(opt_problem* prob, int32_t n_iters, void* stream, float* ms);

/* Work granularity of the problem's kernels.  units_per_block > 0: that many
 * consecutive tiles (grid) or 256-vertex tiles and units_per_block * 256 edges
 * (graph) per block; units_per_block < 0: the work split into
 * (-units_per_block) x (number of SMs) balanced blocks (grid; graph: 4x that;
 * sizes differ by at most one unit, the larger blocks first);
 * 0 restores the default (balanced, 2 blocks per SM for grids, 8 for graphs).
 * Drops the cached solve graph.  Synchronises the device. */
opt_status opt_problem_set_chunking(opt_problem* prob, int32_t units_per_block);

/* Autotuner: times one PCG iteration -- the single-reduction iteration
 * (opt_profile_pcg_fused) on warp and Poisson layouts with 128-pixel tiles,
 * applyJTJ + vector update (opt_profile_pcg) elsewhere -- for each
 * candidate granularity {-1, -2, -3, -4, -6, -8, 1, 4} (see
 * opt_problem_set_chunking) and, beside it, each apply form of an ARAP mesh
 * with tile tables and each tile width (32, 128) of a grid (see
 * opt_problem_get_config); keeps the fastest combination and returns its
 * granularity in *chosen and its per-iteration time in *best_ms (host, either
 * may be NULL).  Leaves the PCG state of its last timed run.  A grid whose
 * other tile width wins is re-planned in place: autotune a problem before
 * building a batch over it, not while a batch holds it. */
opt_status opt_problem_autotune(opt_problem* prob, int32_t* chosen, float* best_ms);

/* Number of unknowns (elements per plane x planes) and of planes. */
opt_status opt_problem_info(const opt_problem* prob, int64_t* n_unknowns, int32_t* n_planes,
                            int64_t* plane_len);

/* The launch configuration in use (host outputs, each may be NULL):
 * tile_w = tile width of a grid problem (32 or 128 pixels; 0 for graphs),
 * chunking = granularity as passed to opt_problem_set_chunking (0 = the
 * default), apply_form = how an ARAP mesh forms J^T J p (1: one block per
 * vertex tile with the tile's halo staged in shared memory, every residual of
 * the tile evaluated once; 0: the two-pass vertex gather; -1: not an ARAP mesh
 * with tile tables).  opt_problem_autotune chooses all three: the form and
 * granularity of a mesh, the granularity and tile width of a grid (the other
 * width is planned afresh from the creation descriptor, whose arrays must
 * still be valid, and kept if faster).  Results agree across configurations
 * to float rounding (the sums are compensated, see Sec. 4.1 PCG). */
opt_status opt_problem_get_config(const opt_problem* prob, int32_t* tile_w, int32_t* chunking,
                                  int32_t* apply_form);

/* Forces the ARAP-mesh apply form (1 tiled, 0 two-pass gather; see
 * opt_problem_get_config).  OPT_ERR_INVALID_ARG for other values, for a NULL
 * problem or for form 1 on a problem without tile tables (graphs whose
 * vertex tiles exceed 384 out-of-tile neighbours or 2,304 edge slots, other
 * energies). */
opt_status opt_problem_set_apply_form(opt_problem* prob, int32_t form);

/* ---------------------------------------------------------------------------
 * Batched solves: many planned problems of uneven sizes advanced together,
 * one launch per solver phase for the whole batch.  The paper solves one
 * problem at a time; the batch runs, for every member, exactly the sequence of
 * opt_solve_gn / opt_solve_lm (same outer / inner counts for all members), so
 * each member's result equals its solo solve up to float rounding.
 * ------------------------------------------------------------------------- */
typedef struct opt_batch opt_batch;

/* Builds a batch over n distinct planned problems (any mix of kinds; probs:
 * host array).  The problems must outlive the batch and must not be solved
 * on their own while a batched solve is in flight.  OPT_ERR_INVALID_ARG on a
 * null or repeated problem or n < 1. */
opt_status opt_batch_create(opt_problem* const* probs, int32_t n, opt_batch** out);

/* Frees the batch (not its problems).  NULL is accepted. */
opt_status opt_batch_destroy(opt_batch* batch);

/* Work granularity: tiles_per_chunk consecutive 32x8 tiles of one problem per
 * block (0 = each problem's own default, about 8 blocks per SM per problem). */
opt_status opt_batch_set_chunking(opt_batch* batch, int32_t tiles_per_chunk);

/* Autotuner: times one outer iteration (<= 4 PCG iterations) of the batch for
 * each candidate granularity {default, 1, 2, 4, 8, 16} without writing the
 * unknowns back, keeps the fastest and returns it in *chosen (host, may be
 * NULL) and its time in *best_ms (host, may be NULL). */
opt_status opt_batch_autotune(opt_batch* batch, const opt_solve_params* params, int32_t* chosen,
                              float* best_ms);

/* Batched Gauss-Newton / Levenberg-Marquardt over every member (Sec. 4), the
 * whole batched solve replayed as one CUDA graph.  reports: host array of n
 * opt_report (each E_history may be NULL), or NULL.  ms (host, may be NULL):
 * device time of the batched solve.  params->materialized must be 0. */
opt_status opt_batch_solve_gn(opt_batch* batch, const opt_solve_params* params, opt_report* reports, float* ms);
opt_status opt_batch_solve_lm(opt_batch* batch, const opt_solve_params* params, opt_report* reports, float* ms);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over LM solves with continuous batching.  The paper
 * solves one problem per call; the server keeps every admitted request's
 * unknowns and PCG state on the device, admits queued requests in arrival
 * order while their estimated device footprint fits in hbm_budget_bytes, and
 * advances all admitted requests together one LM outer iteration per
 * opt_server_step (Sec. 4 LM, exactly the sequence of opt_solve_lm), so work of
 * requests admitted at different times overlaps on the GPU.
 * ------------------------------------------------------------------------- */
typedef struct opt_server opt_server;

/* params: outer = cap on LM outer iterations per request, inner = PCG
 * iterations per outer iteration, rel_tol = convergence test (Sec. 4 LM;
 * see opt_solve_params), lambda0 / clamps / eta as for opt_solve_lm;
 * params->stream is ignored (the server owns a non-blocking stream).
 * OPT_ERR_INVALID_ARG on a zero budget or invalid parameters. */
opt_status opt_server_create(size_t hbm_budget_bytes, const opt_solve_params* params, opt_server** out);

/* Waits for the server's stream and frees every request it still holds. */
opt_status opt_server_destroy(opt_server* server);

/* Queues a request.  The descriptor is copied; the device arrays it points to
 * must stay valid until the request is polled as finished (the solution is
 * written into its unknowns).  *ticket (host) identifies the request.
 * OPT_ERR_BUDGET if the request alone exceeds the budget.  Planning errors
 * (invalid descriptors) are reported by opt_server_poll. */
opt_status opt_server_submit_grid(opt_server* server, const opt_grid_desc* desc, uint64_t* ticket);
opt_status opt_server_submit_graph(opt_server* server, const opt_graph_desc* desc, uint64_t* ticket);

/* Admits, runs one LM outer iteration of every admitted request (or more
 * when no request is waiting, see opt_server_set_max_rounds), retires the
 * finished ones (synchronises the server's stream).  n_active / n_queued
 * (host, may be NULL) receive the counts after the step.  If rebuilding the
 * batch after an admission or a retirement fails (e.g. OPT_ERR_OOM), or the
 * round itself fails, every request active at that moment ends with that
 * status (opt_server_poll returns it), its memory returns to the budget, the
 * step returns the status, and later steps go on with the queue. */
opt_status opt_server_step(opt_server* server, int32_t* n_active, int32_t* n_queued);

/* Failure-path test hook (host only, no device work): the next batch rebuild
 * of opt_server_step fails with `status` instead of planning the batch, as an
 * allocation failure would.  OPT_ERR_INVALID_ARG for a NULL server or
 * status == OPT_OK. */
opt_status opt_server_inject_rebuild_failure(opt_server* server, opt_status status);

/* Caps the number of requests admitted at once (0, the default: admission by
 * the budget alone).  Admission stays in arrival order; under a cap, requests
 * that arrive faster than they are served wait in the queue instead of all
 * sharing the device, so the early ones finish first (a FIFO of batches).
 * Takes effect at the next opt_server_step.  OPT_ERR_INVALID_ARG on a NULL
 * server or a negative cap. */
opt_status opt_server_set_max_active(opt_server* server, int32_t max_active);

/* LM outer iterations per opt_server_step when no request is waiting after
 * admission: as many as the admitted request closest to its iteration cap
 * has left, at most max_rounds (1 .. 64; 1, the default, is one per step).
 * With max_rounds > 1 a lightly loaded server synchronises once per step
 * instead of once per outer iteration; a request that converges earlier idles
 * through the rest of the step, and requests arriving meanwhile wait for the
 * next step.  Results are the same either way.  Takes effect at the next
 * step.  OPT_ERR_INVALID_ARG on a NULL server or a value outside 1 .. 64. */
opt_status opt_server_set_max_rounds(opt_server* server, int32_t max_rounds);

/* OPT_OK and the report (E_history, if not NULL, receives outer_done + 1
 * values) once the request finished; the ticket is then forgotten.
 * OPT_ERR_NOT_READY while queued or running; OPT_ERR_INVALID_ARG for an
 * unknown ticket; the request's own error status if its planning or solve
 * failed. */
opt_status opt_server_poll(opt_server* server, uint64_t ticket, opt_report* report);

/* Allocation-free variant of the warp J^T J p (no counterpart in the paper).
 * For callers that cannot call cudaMalloc: interactive loops on a fixed frame
 * budget that must not stall on an allocation, and host applications or
 * plug-in hosts that own all device memory and hand a component only its
 * buffers.  Computes q = J^T J p (lambda = 0) for an OPT_ARAP_WARP_2D energy
 * at x -- the product opt_apply_jtj computes, equal to it within 1e-5
 * relative error but not bitwise (cos / sin are evaluated per call and the
 * sums are rounded in another order) -- and p.q in float64, without any
 * allocation: its only scratch (float64 reduction partials, an arrival
 * counter) is a file-scope device array of 262,400 bytes that every device
 * loading the library holds until the process exits.
 *   x        device, 3*W*H floats: dx, dy, theta planes (row-major, y*W + x)
 *   urshape  device, 2*W*H floats: UrShape x, y planes
 *   mask     device, W*H bytes (nonzero = excluded) or NULL
 *   handle_idx device, n_handles pixel indices y*W + x in any order (may be
 *            NULL if n_handles = 0).  Unlike opt_problem_create_grid, repeated
 *            indices are not rejected: each entry adds its own fit residual
 *            (a pixel listed twice gets twice the fit weight).  Every block
 *            scans the whole list, so the cost grows as tiles x n_handles:
 *            cheap for the few handles of an interactive warp, about 0.7 G
 *            index loads per call at 2048 x 2048 with 40k handles.
 *   p        device, 3*W*H floats (input direction)
 *   q        device, 3*W*H floats (output)
 *   pq       device, one double (output p.q) or NULL
 *   stream   cudaStream_t (NULL = legacy default stream); the call only
 *            enqueues work and does not synchronise.
 * Limits: ceil(W/32) * ceil(H/8) <= OPT_NOALLOC_MAX_TILES (e.g. 2048 x 2048);
 * larger grids, W or H outside [1, 32768), null inputs or negative weights
 * return OPT_ERR_INVALID_ARG before any device work.  The first call made
 * with a given device current looks up the array's device address
 * (cudaGetSymbolAddress), so make it before any stream capture.  All calls
 * share the array and each clears its counter on entry: calls whose work
 * overlaps on the GPU race and must be serialised by the caller. */
#define OPT_NOALLOC_MAX_TILES 16384
opt_status opt_warp_apply_jtj_noalloc(int32_t W, int32_t H, const float* x, const float* urshape,
                                      const uint8_t* mask, const int32_t* handle_idx, int32_t n_handles,
                                      float w_reg, float w_fit, const float* p, float* q, double* pq,
                                      void* stream);

/* ---------------------------------------------------------------------------
 * Full float64 solver (Sec. 7 "Numerical Precision": the solver runs in
 * single or double precision; Fig. 14 compares the two).  Same energies,
 * conventions and algorithm as the float32 calls above (matrix-free GN / LM
 * with Jacobi PCG, the whole solve one CUDA graph), with every quantity in
 * float64: unknowns, constants, residuals, J^T J p, PCG vectors, dot
 * products, energies.  Planes are dense: grid index y*W + x, graph index =
 * vertex.  The grid energies are OPT_ARAP_WARP_2D and OPT_POISSON_2D, the
 * graph energy is OPT_ARAP_MESH.  Not supported here: materialized forms
 * (params.materialized must be 0), batches and the server.
 * ------------------------------------------------------------------------- */
typedef struct opt_problem_f64 opt_problem_f64;

/* As opt_grid_desc with float64 planes, handle targets and weights. */
typedef struct {
    int32_t kind;                 /* OPT_ARAP_WARP_2D or OPT_POISSON_2D */
    int32_t W, H;
    double* unknowns[4];          /* device: warp dx, dy, theta; Poisson X (4 channels) */
    const double* consts[4];      /* device: warp UrShape x, y; Poisson guidance T (4) */
    const uint8_t* mask;          /* device W*H bytes or NULL (as opt_grid_desc) */
    const int32_t* handle_idx;    /* device, warp only */
    const double* handle_target;  /* device, 2 per handle, warp only */
    int32_t n_handles;
    double w_reg, w_fit;          /* warp only */
} opt_grid_desc_f64;

/* As opt_graph_desc (ARAP mesh, Fig. 25) with float64 planes. */
typedef struct {
    int32_t V, E;
    const int32_t* v0;            /* device, E directed edges, 0 <= v < V, v0 != v1 */
    const int32_t* v1;
    double* unknowns[6];          /* device: dx, dy, dz, ax, ay, az (V each) */
    const double* urshape[3];     /* device: rest positions x, y, z */
    const int32_t* handle_idx;    /* device, distinct vertices */
    const double* handle_target;  /* device, 3 per handle */
    int32_t n_handles;
    double w_reg, w_fit;
} opt_graph_desc_f64;

/* Planning: validates (OPT_ERR_INVALID_ARG on a bad kind, size, null plane,
 * handle index out of range or repeated, edge out of range or a loop,
 * non-finite constant or weight), copies the constants and allocates the
 * float64 scratch (about 8 * (8 nx + 2) bytes per pixel / vertex).  params
 * is unused (may be NULL).  *out stays NULL on error. */
opt_status opt_problem_create_grid_f64(const opt_grid_desc_f64* desc, const opt_solve_params* params,
                                       opt_problem_f64** out);
opt_status opt_problem_create_graph_f64(const opt_graph_desc_f64* desc, const opt_solve_params* params,
                                        opt_problem_f64** out);
opt_status opt_problem_destroy_f64(opt_problem_f64* prob);

/* GN / LM exactly as opt_solve_gn / opt_solve_lm (params->materialized must
 * be 0; tile_w and persistent are ignored). */
opt_status opt_solve_gn_f64(opt_problem_f64* prob, const opt_solve_params* params, opt_report* report);
opt_status opt_solve_lm_f64(opt_problem_f64* prob, const opt_solve_params* params, opt_report* report);

/* Hooks as opt_apply_jtj / opt_eval_jtf / opt_eval_energy, synchronous, on
 * the legacy default stream.  p, q, jtf, diag: device, nx dense planes
 * (diag: one entry per unknown). */
opt_status opt_apply_jtj_f64(opt_problem_f64* prob, const double* p, double* q, double lambda, double* pq);
opt_status opt_eval_jtf_f64(opt_problem_f64* prob, double* jtf, double* diag, double* energy);
opt_status opt_eval_energy_f64(opt_problem_f64* prob, double* energy);

/* Measurement hook as opt_profile_pcg: ms[0] PCGInit (with the cos / sin
 * pass), ms[1] applyJTJ with the direction update (two launches from the
 * second PCG iteration on), ms[2] vector update (mean device ms). */
opt_status opt_profile_pcg_f64(opt_problem_f64* prob, int32_t n_iters, void* stream, float* ms);

/* Number of unknowns, planes and plane length. */
opt_status opt_problem_info_f64(const opt_problem_f64* prob, int64_t* n_unknowns, int32_t* n_planes,
                                int64_t* plane_len);

/* Measured float64 fused multiply-add throughput of the current device in
 * GFLOP/s (2 flops per FMA): one launch of independent FMA chains on every
 * SM, timed with CUDA events on `stream` (cudaStream_t, NULL = legacy
 * default stream).  The denominator of the float64 kernels' arithmetic
 * roofline.  Synchronises the stream. */
opt_status opt_measure_fp64_fma_rate(void* stream, double* gflops);

/* Self-test of the bounded grid-wide barrier used by the persistent PCG loop
 * (opt_solve_params.persistent).  Runs one cooperative launch of 2 blocks that
 * meet at the barrier `rounds` times while the barrier awaits 2 + extra
 * blocks.  extra = 0: a working barrier, *timed_out = 0.  extra > 0: the wait
 * cannot complete; every block gives up after 50 ms, the launch ends and
 * *timed_out = 1 (the bounded wait leaves the context usable).  Synchronous.
 * OPT_ERR_INVALID_ARG for extra outside [0, 64], rounds outside [1, 1000] or a
 * NULL pointer. */
opt_status opt_selftest_grid_barrier(int32_t extra, int32_t rounds, int32_t* timed_out);

/* Self-test of the bounded wait behind the tensor-copy (TMA) staging of the
 * wide grid kernels: each thread of 2 blocks waits on a shared-memory
 * mbarrier phase, as the kernels wait for a tile.  complete = 1: one thread
 * arrives first, the phase completes, *timed_out = 0.  complete = 0: nothing
 * arrives; every wait gives up after 50 ms (the solver kernels allow 1 s, then
 * flag the problem and the solve returns OPT_ERR_TIMEOUT), the launch ends
 * and *timed_out = 1, leaving the context usable.  Synchronous.
 * OPT_ERR_INVALID_ARG for complete outside {0, 1} or a NULL pointer. */
opt_status opt_selftest_staging_wait(int32_t complete, int32_t* timed_out);

/* Human-readable name of a status code; never NULL. */
const char* opt_status_str(opt_status s);

/* Message of the last CUDA error seen on this host thread ("" if none). */
const char* opt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OPT_GB300_H */
