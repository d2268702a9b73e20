/*
 * hmg.h -- C ABI of the GB300 tensor-product multigrid solver for the lumped
 * pressure-Helmholtz operator of the lowest-order (RT0 x DG0) mixed finite
 * element discretisation on an extruded icosahedral shell.
 *
 * Method: Mitchell & Mueller, "High level implementation of geometric
 * multigrid solvers for finite element problems: applications in atmospheric
 * modelling".  The operator is H^ of Sec. 4.2, Eq. (Preconditioner); the
 * preconditioner is the horizontal-only V-cycle of Sec. 4.2.1 (vertical line
 * relaxation, Eq. (BlockJacobi) in the form of Sec. 5.4, DG0 transfers of
 * Sec. 3.2, Algorithm 1), wrapped in a Krylov solve (Sec. 5).
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Every function returns an hmg_status; none aborts or exits.
 * - Device pointers are CUDA device (or managed) memory owned by the caller
 *   unless stated otherwise; host pointers are ordinary host memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   All GPU work is enqueued on it.  Argument errors are reported
 *   synchronously; errors raised by kernels are reported by the next call
 *   that synchronises (hmg_solve, hmg_solve_host) or by hmg_sync.
 * - Vectors are FP64 (or FP32 where a dtype argument says so) over the cells
 *   of one level.  Layout HMG_LAYOUT_COLUMN numbers cell (column c, layer l)
 *   as c * nlayers + l, all unknowns of a column consecutive (Sec. 4.3).
 *   Layout HMG_LAYOUT_TILED is the library's working layout: columns in
 *   tiles of 32, layer-major inside a tile,
 *       index = (c / 32) * 32 * nlayers + l * 32 + (c % 32),
 *   over ncols_padded = 32 * ceil(ncols / 32) columns; padding entries are
 *   written as zero and must be zero on input.
 * - Level 0 is the finest mesh; level k has 20 * 4^(refinement - k) columns
 *   and the parent of column c on level k is column c / 4 on level k + 1.
 * - A context is not thread safe; calls on one context must be ordered.
 */
#ifndef HMG_H
#define HMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMG_OK = 0,
  HMG_ERR_INVALID_ARG = 1,   /* bad pointer, size, level or parameter */
  HMG_ERR_CUDA = 2,          /* a CUDA runtime call or kernel failed */
  HMG_ERR_OOM = 3,           /* device or host allocation failed */
  HMG_ERR_NOT_CONVERGED = 4, /* max_iter reached; info is filled in */
  HMG_ERR_BREAKDOWN = 5,     /* Krylov breakdown (p.q <= 0 or r.z <= 0) */
  HMG_ERR_NONFINITE = 6,     /* NaN or Inf in the right-hand side or residual */
  HMG_ERR_STATE = 7          /* call out of order (e.g. solve before assemble) */
} hmg_status;

typedef enum { HMG_FP64 = 0, HMG_FP32 = 1 } hmg_dtype;
typedef enum { HMG_LAYOUT_COLUMN = 0, HMG_LAYOUT_TILED = 1 } hmg_layout;
typedef enum { HMG_PRECISION_FP64 = 0, HMG_PRECISION_MIXED = 1 } hmg_precision;
typedef enum { HMG_KRYLOV_CG = 0, HMG_KRYLOV_FCG = 1, HMG_KRYLOV_GMRES = 2 } hmg_krylov;

/* Largest GMRES restart length (basis vectors kept per cycle). */
#define HMG_GMRES_MAX_RESTART 32

/* Shell and hierarchy (Sec. 3.1, Sec. 4.1, Table "Grid setup"). */
typedef struct {
  int refinement;       /* finest icosahedral refinement r >= 0 (20 * 4^r columns) */
  int nlayers;          /* vertical layers, 1 <= nlayers <= 256 */
  int nlevels;          /* multigrid levels, 1 <= nlevels <= refinement + 1 */
  double radius_m;      /* inner radius R of the shell, > 0 (6.371e6) */
  double thickness_m;   /* shell thickness H, > 0 (1.0e4) */
} hmg_mesh_params;

/* Operator parameters (Sec. 4.1, Eq. HelmholtzOperator, Eq.
 * PressureVelocitySystem, Sec. 5).  dt = nu_cfl * dx_m / c, w_c = c dt / 2,
 * w_N = N dt / 2.  dx_m <= 0 selects 90 km * 2^(6 - refinement). */
typedef struct {
  double c;             /* speed of sound, m/s (300) */
  double N;             /* buoyancy frequency, 1/s (0.01), >= 0 */
  double nu_cfl;        /* horizontal acoustic Courant number (8) */
  double dx_m;          /* horizontal grid spacing defining dt; <= 0: default */
  double omega;         /* smoother over-relaxation, 0 < omega < 2 (0.8) */
} hmg_op_params;

typedef struct {
  int precision;        /* hmg_precision */
  int krylov;           /* hmg_krylov; MIXED runs flexible CG for CG and FCG */
  double rtol;          /* stop when ||r_k||_2 / ||b||_2 < rtol (1e-8) */
  int max_iter;         /* >= 1; for GMRES, Arnoldi steps over all restart cycles */
  int nu_pre;           /* pre-smoothing sweeps per level, >= 1 (2) */
  int nu_post;          /* post-smoothing sweeps per level, >= 1 (2) */
  int n_coarse;         /* smoother iterations on the coarsest level, >= 1 (2) */
  int restart;          /* GMRES restart length m, 1..HMG_GMRES_MAX_RESTART (30);
                           ignored by CG and FCG */
  int levels;           /* multigrid levels used, 0 (all) or 1..nlevels; 1 is the
                           single-level method of Sec. 6: n_coarse block-Jacobi
                           vertical line relaxations on the finest level */
  int orth;             /* GMRES orthogonalisation: 0 or 1 = classical Gram-Schmidt
                           once (as PETSc's GMRES does by default), 2 = twice */
} hmg_solve_params;

typedef struct {
  int iterations;           /* Krylov iterations performed */
  int converged;            /* 1 if ||r||/||b|| < rtol */
  double rel_residual;      /* recursive residual ||r_k|| / ||b|| */
  double true_rel_residual; /* ||b - H^ x|| / ||b||, recomputed at the end */
  double solve_ms;          /* device time of the solve (CUDA events) */
} hmg_solve_info;

typedef struct {
  int refinement;       /* icosahedral refinement of this level */
  int ncols;            /* columns 20 * 4^refinement */
  int ncols_padded;     /* ncols rounded up to a multiple of 32 */
  int nlayers;
  int64_t ncells;       /* ncols * nlayers (COLUMN layout length) */
  int64_t ncells_padded;/* ncols_padded * nlayers (TILED layout length) */
} hmg_level_info;

typedef struct hmg_ctx hmg_ctx;

/* Build the mesh hierarchy (Sec. 3.1): the icosahedron refined `refinement`
 * times by edge bisection with midpoints projected to the sphere, children of
 * column c at 4c..4c+3, three neighbours per column, radial extrusion into
 * `nlayers` uniform layers (Sec. 4.1).  Allocates all device memory of the
 * hierarchy on the current device.  *out receives a new context, owned by the
 * caller and released with hmg_destroy.  Errors: INVALID_ARG, OOM, CUDA. */
hmg_status hmg_build_hierarchy(const hmg_mesh_params* params, hmg_ctx** out);

/* Device memory through the caller's allocator.  alloc(bytes, user) returns
 * device memory of the current device (at least `bytes`, 256-byte aligned),
 * or NULL when it cannot; release(ptr, user) takes back what alloc returned.
 * The callbacks are called from the thread that calls into the library,
 * only while no kernel of the context reads or writes that memory. */
typedef void* (*hmg_alloc_fn)(size_t bytes, void* user);
typedef void (*hmg_release_fn)(void* ptr, void* user);

/* hmg_build_hierarchy with every device allocation of the context (levels,
 * Krylov and GMRES vectors, the velocity-pressure and next-to-lowest-order
 * tables, built later on first use) taken from alloc and returned with
 * release by hmg_destroy, so a framework's memory pool (for instance a
 * caching allocator) backs the context.  alloc returning NULL makes the call
 * that needed the memory fail with HMG_ERR_OOM; the build releases what it
 * had taken.  Page-locked host copies of the solver's scalars still come
 * from the CUDA runtime.  Errors: INVALID_ARG (NULL callbacks), OOM, CUDA. */
hmg_status hmg_build_hierarchy_with_allocator(const hmg_mesh_params* params, hmg_alloc_fn alloc,
                                              hmg_release_fn release, void* user, hmg_ctx** out);

/* Release every resource of a context: its device memory (through the
 * caller's release callback when it was built with one), page-locked host
 * buffers, events, its capture stream and captured graphs.  Synchronises
 * the current device first (all its work, not only the context's).  NULL is
 * accepted (no-op).  Always returns HMG_OK. */
hmg_status hmg_destroy(hmg_ctx* ctx);

/* Sizes of one level of the hierarchy (level 0 = finest, refinement
 * `refinement` of the build; level k has refinement - k) into *out:
 * columns 20 * 4^refinement, their count padded to a multiple of 32 (the
 * TILED layout), layers, and cells in both layouts.  Host only, no device
 * work.  Errors: INVALID_ARG (ctx or out NULL, level outside [0, nlevels)). */
hmg_status hmg_get_level_info(const hmg_ctx* ctx, int level, hmg_level_info* out);

/* Copy one level's mesh to caller-owned host buffers (any may be NULL):
 * centroids[3 * ncols] = flat-triangle centroids on the unit sphere,
 * nbr[3 * ncols] = column across the edge opposite vertex k of each column.
 * Used to match cells with an independent implementation. */
hmg_status hmg_export_mesh(const hmg_ctx* ctx, int level, double* centroids, int32_t* nbr);

/* Assemble H^ and H^_z on every level (Sec. 4.2, Eq. Preconditioner and
 * Eq. HHgeneralbanded; coarse levels rediscretised, Sec. 3.3) and factorise
 * H^_z = L D L^T per column for the Thomas solve (Sec. 4.3.1).  Builds FP64
 * and FP32 copies of all coefficients.
 * theta: NULL, or a device FP64 vector (COLUMN layout, finest level) of
 * positive coefficients dividing each cell's share of the vertical lumped
 * mass; coarse levels use the mean over the four children.  The values are
 * copied; the pointer is read during this call only.
 * Errors: INVALID_ARG (bad parameters), STATE (no hierarchy), CUDA. */
hmg_status hmg_assemble_helmholtz(hmg_ctx* ctx, const hmg_op_params* params,
                                  const double* theta, void* stream);

/* y = H^ x on `level` (Sec. 5.4, "operator application").  x and y are
 * device vectors of type `dtype` in `layout`; x != y.  FP32 uses the FP32
 * copy of the coefficients.  Errors: INVALID_ARG, STATE, CUDA. */
hmg_status hmg_apply(hmg_ctx* ctx, int level, int dtype, int layout,
                     const void* x, void* y, void* stream);

/* z = V r: one V-cycle from a zero initial guess on the finest level
 * (Algorithm 1 applied recursively; line relaxation of Sec. 4.2.1 with
 * nu_pre / nu_post sweeps per level and n_coarse sweeps on the coarsest
 * level).  r and z are FP64 device vectors in `layout`; precision
 * HMG_PRECISION_MIXED runs levels 0..nlevels-2 in FP32 and the coarsest level
 * in FP64.  r != z.  Errors: INVALID_ARG, STATE, CUDA. */
hmg_status hmg_vcycle(hmg_ctx* ctx, int precision, int layout, const void* r,
                      void* z, int nu_pre, int nu_post, int n_coarse, void* stream);

/* Solve H^ x = b on the finest level with a Krylov method preconditioned by
 * one V-cycle per iteration, x_0 = 0 (Sec. 5): CG (H^ is symmetric positive
 * definite), flexible CG, or restarted GMRES(m), the paper's outer method, in
 * its flexible right-preconditioned form (Saad, Algorithm 9.6: Arnoldi with
 * classical Gram-Schmidt once or twice (params->orth), Givens rotations, the iterate formed
 * at the end of each restart cycle, stopping on the least-squares residual
 * ||r_k|| / ||b|| < rtol).  GMRES keeps 2m + 1 finest-level FP64 vectors,
 * allocated by the first GMRES solve that needs them.  b, x: FP64 device
 * vectors, COLUMN layout, ncells.  Blocks until the solve has finished.
 * Returns NOT_CONVERGED (info filled in) when max_iter is reached, NONFINITE
 * for a non-finite b or residual, BREAKDOWN when p.q <= 0 or r.z <= 0 (CG)
 * or a zero rotation (GMRES), OOM when the GMRES basis cannot be allocated. */
hmg_status hmg_solve(hmg_ctx* ctx, const double* b, double* x,
                     const hmg_solve_params* params, hmg_solve_info* info, void* stream);

/* hmg_solve with HOST buffers (b_host, x_host: ncells doubles in the COLUMN
 * layout), all on `stream`, synchronising before it returns.  Page-locked
 * buffers that the device can address (cudaHostAlloc'd or registered) are read
 * and written in place by the layout kernels over the host link; any other
 * host memory is copied through a device buffer with cudaMemcpyAsync. */
hmg_status hmg_solve_host(hmg_ctx* ctx, const double* b_host, double* x_host,
                          const hmg_solve_params* params, hmg_solve_info* info, void* stream);

/* The velocity-pressure system of Sec. 4.1 (Eq. PressureVelocitySystem) on
 * the finest level, lowest order (RT0 x DG0, no orography):
 *   A (U, P) = ( M2~ U - dt/2 D^T P ,  dt/2 c^2 D U + M3 P ),
 *   M2~ = M2^h (+) (1 + w_N^2) M2^z  (full, not lumped, velocity mass),
 * with unit-flux bases, the prism geometry of hmg_assemble_helmholtz and its
 * parameters (c, N, nu_cfl, dx_m).  Vectors in COLUMN layouts:
 *   U: horizontal faces e * nlayers + l (edge e of hmg_export_edges, layer l;
 *      positive flux from column t into column tn), then vertical faces
 *      c * (nlayers - 1) + l (between layers l and l + 1, positive upwards);
 *   P: cells c * nlayers + l.
 * Sizes from hmg_mixed_sizes.  The coefficient tables are built by the first
 * call that needs them (device memory of about 9 vectors of ncells doubles,
 * plus the GMRES basis of 2m + 1 vectors of the system's size). */
hmg_status hmg_mixed_sizes(const hmg_ctx* ctx, int64_t* n_hfaces, int64_t* n_vfaces, int64_t* n_cells);

/* edges[4 e + 0..3] = (t, k, tn, kn): edge e is local edge k (opposite vertex
 * k) of column t and local edge kn of column tn, t < tn; edges are ordered by
 * t, then k.  Host buffer of 4 * (n_hfaces / nlayers) int32. */
hmg_status hmg_export_edges(hmg_ctx* ctx, int32_t* edges);

/* (yu, yp) = A (u, p), device FP64 vectors.  Errors: INVALID_ARG, STATE, CUDA. */
hmg_status hmg_mixed_apply(hmg_ctx* ctx, const double* u, const double* p, double* yu, double* yp, void* stream);

/* Solve A (u, p) = (bu, bp) with restarted flexible GMRES(params->restart),
 * x_0 = 0, preconditioned on the right by the Schur-complement factorisation
 * of Sec. 4.2 (Eq. SchurComplement) with the diagonal velocity-mass inverse
 * of Eq. LumpedMass and one V-cycle (params: precision, nu_pre, nu_post,
 * n_coarse, levels) for H^^-1; stops when ||r|| / ||(bu, bp)|| < rtol (the
 * paper uses 1e-5).  params->krylov is ignored.  Status as hmg_solve. */
hmg_status hmg_mixed_solve(hmg_ctx* ctx, const double* bu, const double* bp, double* u, double* p,
                           const hmg_solve_params* params, hmg_solve_info* info, void* stream);

/* ---- Next-to-lowest order (NLO): Table "FiniteElements" -------------------
 * Pressure in DG1(T) x DG1(z) (6 unknowns per cell), horizontal velocity in
 * BDFM1(T) x DG1(z), vertical velocity in DG1(T) x P2(z); H^ is Eq.
 * (Preconditioner) for these spaces with the lumped masses of Eq.
 * (LumpedMass), evaluated on the finest mesh of the context with the
 * parameters of the last hmg_assemble_helmholtz (theta = 1).  Unknown order
 * (NLO COLUMN layout): ((c * nlayers + l) * 3 + j) * 2 + m for column c,
 * layer l, vertex j of the column's triangle (hmg_export_vertices; DG1 nodal
 * at the vertices) and m = 0 / 1 for the bottom / top of the layer.  The
 * BDFM1 degrees of freedom are the length-scaled normal components at the
 * points 1/3 and 2/3 of each edge and the moments against the three Whitney
 * functions.  The V-cycle (Sec. 4.2.1) smooths with the column block solve of
 * Eq. (HHgeneralbanded) (block tridiagonal, 6 x 6 blocks, factorised once),
 * p-coarsens DG1 -> DG0 on the same mesh by the natural embedding and runs
 * the lowest-order V-cycle of the context below.  The coefficient tables
 * (about 1.7 KB per cell) are built on the host by the first NLO call after
 * each hmg_assemble_helmholtz. */

/* Length of an NLO vector: 6 * ncols * nlayers of the finest level. */
hmg_status hmg_nlo_size(const hmg_ctx* ctx, int64_t* n);

/* verts[9 c + 3 j + x]: coordinate x of vertex j of column c's triangle on
 * the unit sphere (the order that numbers the DG1 unknowns).  Host buffer of
 * 9 * ncols doubles.  Errors: INVALID_ARG. */
hmg_status hmg_export_vertices(const hmg_ctx* ctx, int level, double* verts);

/* ---- Horizontal domain decomposition (Sec. 5: the paper splits the
 * horizontal domain over MPI processes, exchanges the halo columns before
 * each parallel loop and reduces the Krylov dot products over processes).
 * Parts are contiguous ranges of the hierarchical column order, cut in whole
 * tiles of 32 columns on the coarsest partitioned level and inherited by the
 * finer levels (the children 4C..4C+3 of an owned column C are owned by the
 * same part).  Levels 0 .. nlevels - 2 are partitioned; the coarsest level is
 * gathered on one part (a one-level hierarchy partitions its only level).
 * In a part's local numbering, owned column c is c - col_begin, the owned
 * columns are padded to ncols_padded (a multiple of 32), and ghost i (a
 * column the part's stencils read but another part owns) is
 * ncols_padded + i.  Ghosts are ordered by (owner part, global column). */
typedef struct {
  int32_t col_begin, col_end; /* owned columns [col_begin, col_end), global numbering of the level */
  int32_t ncols_padded;       /* col_end - col_begin rounded up to 32: local index of ghost 0 */
  int32_t n_ghost;            /* ghost columns */
  int32_t n_send;             /* entries of the send list: owned columns that are ghosts of other parts */
} hmg_part_info;

/* Host only (no context, no GPU): the partition of the hierarchy of
 * `refinement` and `nlevels` levels into `nparts` parts, for one part and one
 * partitioned level.  Errors: INVALID_ARG (bad sizes; nparts larger than the
 * tiles of the coarsest partitioned level; level not partitioned). */
hmg_status hmg_partition_info(int refinement, int nlevels, int nparts, int part, int level, hmg_part_info* out);

/* Host only: the tables of that part and level, into caller-owned host
 * buffers (sizes from hmg_partition_info; any pointer may be NULL):
 *   ghost_col[n_ghost]          global column of each ghost
 *   ghost_owner[n_ghost]        the part that owns it
 *   ghost_owner_local[n_ghost]  its local index in the owner
 *   local_nbr[3 n_own]          the three neighbours of each owned column, local indices
 *   send_col[n_send], send_to[n_send]: the owned columns other parts read, grouped by
 *                               the receiving part and, within a group, in that part's
 *                               ghost order (so a receiver unpacks its halo in order).
 * Errors: as hmg_partition_info. */
hmg_status hmg_partition_tables(int refinement, int nlevels, int nparts, int part, int level, int32_t* ghost_col,
                                int32_t* ghost_owner, int32_t* ghost_owner_local, int32_t* local_nbr,
                                int32_t* send_col, int32_t* send_to);

/* Run this context as `nparts` parts of the horizontal domain decomposition
 * above, emulated on its one device (nparts = 1: unpartitioned, the
 * default).  From then on every V-cycle (hmg_vcycle, and the preconditioner
 * of hmg_solve in every Krylov method and precision) and every level-0 FP64
 * operator application (hmg_apply, and the solves' operator) runs as the
 * parts would on `nparts` devices: each sweep, residual and prolongation
 * pass once per part on its owned columns, every pass that reads neighbour
 * columns after a halo exchange (each part packs its send list, the
 * (sender, receiver) segments are moved, each part unpacks its ghosts), the
 * coarsest level gathered from the parts, solved once and scattered back,
 * and the solves' dot products reduced over all parts.  The per-cell
 * arithmetic is that of the unpartitioned context, so results agree with it
 * (V-cycles to rounding, solves to the Krylov tolerance).  The velocity-
 * pressure and NLO systems keep their unpartitioned outer operators.
 * Allocates each part's local vectors (owned and ghost columns) and tables
 * through the context's allocator; drops the context's captured graphs.
 * Errors: INVALID_ARG (nparts outside [1, 16] or above the tiles of the
 * coarsest partitioned level), OOM, CUDA. */
hmg_status hmg_partition(hmg_ctx* ctx, int nparts);

/* Host-only assembly of the NLO operator on the finest mesh of `mesh` (no
 * context, no GPU): diag[36 (c nlayers + l) + 6 u + u'] = H^[(c,l,u),(c,l,u')],
 * sub[36 (c nlayers + l) + 6 u + u'] = H^[(c,l,u),(c,l-1,u')] (zero for l = 0),
 * nbr_blocks[36 (3 c + k) + 6 u + u'] = H^[(c,l,u),(n,l,u')] for the
 * neighbour n = nbr[3 c + k] across the edge opposite vertex k (the same for
 * every layer), with u = 2 j + m.  Output host buffers of 36 ncols nlayers,
 * 36 ncols nlayers, 108 ncols doubles; nbr (3 ncols int32) and verts
 * (9 ncols doubles) may be NULL.  Errors: INVALID_ARG. */
hmg_status hmg_nlo_host_blocks(const hmg_mesh_params* mesh, const hmg_op_params* op, double* diag, double* sub,
                               double* nbr_blocks, int32_t* nbr, double* verts);

/* y = H^ x for NLO COLUMN-layout FP64 device vectors (x != y).
 * Errors: INVALID_ARG, STATE (not assembled), CUDA. */
hmg_status hmg_nlo_apply(hmg_ctx* ctx, const double* x, double* y, void* stream);

/* z = V r: one NLO V-cycle from zero (NLO COLUMN layout, FP64 device
 * vectors).  nu_pre / nu_post sweeps on the NLO level and on every
 * lowest-order level, n_coarse on the coarsest; levels = 0 uses the NLO level
 * and all lowest-order levels, 1 the NLO smoother alone (n_coarse sweeps),
 * k > 1 the NLO level and k - 1 lowest-order levels.  precision MIXED runs
 * the lowest-order levels in FP32 (the NLO level stays FP64).
 * Errors: INVALID_ARG, STATE, CUDA. */
hmg_status hmg_nlo_vcycle(hmg_ctx* ctx, int precision, const double* r, double* z, int nu_pre, int nu_post,
                          int n_coarse, int levels, void* stream);

/* Solve H^ x = b (NLO COLUMN layout) with restarted flexible GMRES(restart)
 * from x = 0, right-preconditioned by one NLO V-cycle (params as for
 * hmg_nlo_vcycle; levels counts as there); params->krylov must be
 * HMG_KRYLOV_GMRES.  Status and info as hmg_solve. */
hmg_status hmg_nlo_solve(hmg_ctx* ctx, const double* b, double* x, const hmg_solve_params* params,
                         hmg_solve_info* info, void* stream);

/* ---- NLO velocity-pressure system: Eq. (PressureVelocitySystem) with the NLO
 * spaces above, full (consistent) velocity masses of BDFM1(T) x DG1(z) and
 * DG1(T) x P2(z), the divergence pairings of H^ and the DG1 pressure mass,
 * assembled on the host as CSR by the first call after each assembly.  NLO
 * mixed COLUMN layout, in this order: horizontal edge velocity
 * ((E nlayers + l) 2 + q) 2 + b (edge E of hmg_export_edges, points q = 0, 1
 * at 1/3 and 2/3 along local edge k of its first column t with t's outward
 * normal, b = bottom / top DG1 node of the layer); interior horizontal
 * velocity ((c nlayers + l) 3 + k) 2 + b (the Whitney moment of local edge
 * k); vertical velocity (c 3 + i) (2 nlayers - 1) + n - 1 (vertex i, P2 node
 * n = 1 .. 2 nlayers - 1 counted from the bottom); pressure in the NLO COLUMN
 * layout.  Size: about 30 matrix entries per unknown (232 M for the 7.85 M
 * unknowns of 5,120 columns x 64 layers); A, D and D^T take 12 B per entry
 * on the device, and the host assembly holds 16 B per entry while it runs. */

/* Block lengths of an NLO velocity-pressure vector.  Errors: INVALID_ARG. */
hmg_status hmg_nlo_mixed_sizes(const hmg_ctx* ctx, int64_t* n_hedge, int64_t* n_hint, int64_t* n_vert,
                               int64_t* n_p);

/* Host-only assembly of the NLO velocity-pressure matrix A on the finest
 * mesh of `mesh` (no context, no GPU): *n and *nnz always; the CSR arrays
 * ptr (n + 1 int64), col (nnz int32, ascending in each row), val (nnz
 * doubles) and the edge list (3 ncols / 2 x 4 int32, as hmg_export_edges)
 * when non-NULL.  refinement <= 5.  Errors: INVALID_ARG. */
hmg_status hmg_nlo_mixed_host_csr(const hmg_mesh_params* mesh, const hmg_op_params* op, int64_t* n, int64_t* nnz,
                                  int64_t* ptr, int32_t* col, double* val, int32_t* edges);

/* y = A x for FP64 device vectors in the NLO mixed COLUMN layout (x != y).
 * Errors: INVALID_ARG, STATE, CUDA. */
hmg_status hmg_nlo_mixed_apply(hmg_ctx* ctx, const double* x, double* y, void* stream);

/* Solve A x = b (NLO mixed COLUMN layout) with restarted flexible
 * GMRES(params->restart) from x = 0, preconditioned on the right by Eq.
 * (SchurComplement) with the lumped velocity-mass inverse and one NLO
 * V-cycle (params as for hmg_nlo_vcycle) for H^^-1.  params->krylov is
 * ignored.  Status and info as hmg_solve. */
hmg_status hmg_nlo_mixed_solve(hmg_ctx* ctx, const double* b, double* x, const hmg_solve_params* params,
                               hmg_solve_info* info, void* stream);

/* Adjoint face contraction: grad_theta_K = -lambda^T (dH^/dtheta_K) p for the
 * theta given to the last hmg_assemble_helmholtz (all ones if NULL).  Only
 * the vertical term of Eq. (Preconditioner) depends on theta, through the two
 * vertical faces of K.  p, lambda, grad: FP64 device vectors, COLUMN layout,
 * finest level.  Errors: INVALID_ARG, STATE, CUDA. */
hmg_status hmg_theta_grad(hmg_ctx* ctx, const double* p, const double* lambda,
                          double* grad, void* stream);

/* Convert a finest-level (or any level) FP64 vector between layouts. */
hmg_status hmg_to_layout(hmg_ctx* ctx, int level, int src_layout, const double* src,
                         int dst_layout, double* dst, void* stream);

/* Element-wise conversions used by the mixed-precision cycle, done with
 * integer operations on the bit patterns (on GB300 the hardware conversion
 * issues on the slow FP64 pipe): FP64 -> FP32 rounds to nearest, ties to even
 * (IEEE 754 roundTiesToEven); FP32 -> FP64 is exact.  n elements, device
 * pointers, src and dst must not overlap.  Errors: INVALID_ARG, CUDA. */
hmg_status hmg_convert_fp64_to_fp32(const double* src, float* dst, int64_t n, void* stream);
hmg_status hmg_convert_fp32_to_fp64(const float* src, double* dst, int64_t n, void* stream);

/* Synchronise `stream` and report any pending device error. */
hmg_status hmg_sync(hmg_ctx* ctx, void* stream);

/* Largest level (padded TILED length, ncells_padded) hmg_apply_noalloc accepts. */
#define HMG_NOALLOC_MAX_CELLS 524288

/* hmg_apply with COLUMN-layout FP64 vectors, for callers that may not
 * allocate device memory at the point of the call: code running while another
 * component captures a CUDA graph (an allocation there is either refused or
 * becomes part of the graph), code inside a framework that owns the whole
 * device memory pool and forbids side allocations, and latency-bound loops
 * where cudaMalloc / cudaFree would synchronise the device.  The paper has no
 * counterpart: this is an interface convenience, not part of the method.
 * y = H^ x on `level`, the same result as hmg_apply(ctx, level, HMG_FP64,
 * HMG_LAYOUT_COLUMN, x, y, stream).  The two staging vectors that hmg_apply
 * takes from the context live instead in one fixed array of
 * 2 * HMG_NOALLOC_MAX_CELLS doubles (8 MiB) inside the library, which every
 * device that loads the library keeps until the process exits; the call
 * allocates nothing.  The first call on a device looks up the array's device
 * address (with that device current); make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on
 * the GPU (other streams, other threads) race and must be ordered by the
 * caller.  Each call overwrites every staging entry it reads.  Its three
 * launches (layout, operator, layout) are traced and counted like
 * hmg_apply's.  Errors: INVALID_ARG (bad level or pointers, or
 * ncells_padded of the level above HMG_NOALLOC_MAX_CELLS), STATE (not
 * assembled), OOM (host allocation of an error message), CUDA. */
hmg_status hmg_apply_noalloc(hmg_ctx* ctx, int level, const double* x, double* y, void* stream);

/* Kernel classes reported by the tracing calls below. */
typedef enum {
  HMG_K_SWEEP0 = 0,          /* first line relaxation from u = 0 */
  HMG_K_SWEEP = 1,           /* line relaxation (with fused prolongation in FP32) */
  HMG_K_PROLONG = 2,         /* u += P e_c (FP64 cycle) */
  HMG_K_RESID_RESTRICT = 3,  /* b_c = P^T (b - H^ u) */
  HMG_K_APPLY = 4,           /* H^ x (outer operator, optionally with p.q) */
  HMG_K_DOT = 5,
  HMG_K_UPDATE_XR = 6,       /* x += alpha p, r -= alpha q, r.r */
  HMG_K_UPDATE_P = 7,        /* p = z + beta p */
  HMG_K_LAYOUT = 8,          /* COLUMN <-> TILED */
  HMG_K_RESID_SQ = 9,        /* |b - H^ x|^2 */
  HMG_K_ASSEMBLY = 10,
  HMG_K_THETA_GRAD = 11,
  HMG_K_ORTHO = 12,          /* GMRES: Gram-Schmidt passes, basis start, iterate update */
  HMG_K_NLO_SWEEP = 13,      /* NLO column block relaxation (after the first) */
  HMG_K_NLO_RESID = 14,      /* NLO b_c = P^T (b - H^ u) into the lowest-order level */
  HMG_K_NLO_APPLY = 15,      /* NLO H^ x */
  HMG_K_NLO_SWEEP0 = 16,     /* NLO first column block relaxation from u = 0 */
  HMG_K_COARSE = 17,         /* the coarse end of the V-cycle as one cooperative kernel
                                (level = its first level) */
  HMG_K_HALO = 18,           /* domain decomposition: halo pack / unpack, coarsest-level gather and scatter */
  HMG_K_COUNT = 19
} hmg_kernel_id;

typedef struct {
  int kernel;       /* hmg_kernel_id */
  int level;        /* multigrid level (0 = finest) */
  int launches;
  double total_ms;  /* sum of CUDA-event durations of those launches */
} hmg_kernel_stat;

/* Measures the FP64 FMA throughput of the context's device (the bound of the
 * FP64 cycle's kernels, Sec. 5.4's performance model on this hardware): a
 * kernel of 8 independent FMA chains per thread on 8 CTAs of 256 threads per
 * SM, timed with CUDA events on `stream` after a warm-up launch.  Writes
 * TFLOP/s (2 flops per FMA) to *tflops; synchronises the stream.
 * Errors: INVALID_ARG, CUDA. */
hmg_status hmg_measure_fp64_rate(hmg_ctx* ctx, double* tflops, void* stream);

/* Whether V-cycles run their coarse end (Algorithm 1 from the first level
 * below the finest with at most 160 tiles of 32 columns, down to the
 * coarsest and back) as one cooperative kernel with a grid-wide barrier
 * between its sweep and residual passes (enable != 0), or as one kernel per
 * pass (0, the default).  Both run the same arithmetic in the same order and
 * give identical results.  The fused form removes the launches of the small
 * levels, but on GB300 its passes take as long as the separate kernels and
 * solves that use it measured 4 % (FP64) to 10 % (mixed) slower, so it is
 * off unless asked for.  Applies to later calls on this context.  Errors: INVALID_ARG (ctx
 * NULL). */
hmg_status hmg_set_coarse_fusion(hmg_ctx* ctx, int enable);

/* Tracing (the per-level kernel breakdown of Sec. 5.4): from this call on,
 * every launch of a kernel class whose bit is set in kernel_mask, on a level
 * whose bit is set in level_mask, is bracketed by CUDA events on its stream.
 * Any previous records are discarded.  Errors: INVALID_ARG, CUDA. */
hmg_status hmg_profile_start(hmg_ctx* ctx, unsigned kernel_mask, unsigned level_mask);

/* Stop tracing, synchronise the recorded events and write up to `capacity`
 * aggregated (kernel, level) records to `out`; *count receives the number of
 * records available.  Errors: INVALID_ARG, STATE (not started), CUDA. */
hmg_status hmg_profile_stop(hmg_ctx* ctx, hmg_kernel_stat* out, int capacity, int* count);

/* Convergence history of the last solve on this context (Sec. 6,
 * convergence histories): after each Krylov iteration, the relative residual
 * the stopping test used: ||r_k|| / ||b|| of the recursive residual for CG
 * and flexible CG, the least-squares residual estimate for GMRES.  Up to
 * `capacity` values are copied to the host buffer `out`; *count receives how
 * many there are (the iteration count of the last solve).
 * Errors: INVALID_ARG. */
hmg_status hmg_residual_history(const hmg_ctx* ctx, double* out, int capacity, int* count);

/* Number of kernels this context has launched since it was built. */
hmg_status hmg_launch_count(const hmg_ctx* ctx, int64_t* count);

/* Name of a kernel class ("?" if out of range). */
const char* hmg_kernel_name(int kernel);

/* Human-readable description of the last error on this context ("" if none),
 * or of the last build failure when ctx is NULL.  Owned by the library. */
const char* hmg_last_error(const hmg_ctx* ctx);

const char* hmg_status_string(hmg_status s);

#ifdef __cplusplus
}
#endif

#endif /* HMG_H */
