/*
 * lbmg.h -- C ABI of the GB300 library for the connectivity-aware multi-level
 * finite-element system of Chuang & Kazhdan (arXiv 1505.03615).
 *
 * The library builds, for a triangle mesh, the hierarchy of connectivity-split
 * trilinear B-spline spaces of Sections 3.2 and 4 (one function b_k^i per
 * connected component C_k^i of supp(b_k) restricted to the mesh, on grids of
 * depth min_depth..depth), assembles the mass matrix M and the stiffness matrix L
 * of every level (Eq. 2 and Section 5.1), and solves the screened system
 * (M + t L) x = rhs with multigrid V-cycles (Section 4.3) whose relaxation,
 * residual, restriction and prolongation run as CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status (LBMG_OK = 0 or one of the codes
 *    below); no exception or abort crosses the ABI.  lbmg_status_string()
 *    names a code.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; functions return without synchronizing
 *    unless their comment says otherwise.
 *  - Vector arguments are dense row-major arrays [n][nrhs] of double, with
 *    1 <= nrhs <= 4.  Each may be a device pointer (the caller owns it and it
 *    must stay valid until the stream reaches the call) or a host pointer, in
 *    which case the library copies through pinned staging memory and the call
 *    synchronizes the stream before returning.
 *  - Levels are addressed by depth d, min_depth <= d <= depth; the finest
 *    level (d = depth) carries right-hand sides and solutions.
 *  - Dof order on the device: by colour (corner parity (k mod 2)^3), then Morton
 *    order of the corner, then the smallest triangle index of the component.
 *    lbmg_get_dofs() gives, per dof, its corner and that triangle, so results
 *    can be matched with any other numbering of the same functions.
 *  - A handle is not thread-safe: calls on one handle must be serialized, and
 *    all its device work must be on one stream at a time.
 */
#ifndef LBMG_H
#define LBMG_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBMG_OK = 0,
    LBMG_INVALID_ARG = 1,      /* NaN/inf coordinates, index out of range, bad depth or nrhs, NULL pointer */
    LBMG_DEGENERATE_MESH = 2,  /* no triangle of positive area inside the grid */
    LBMG_OUT_OF_MEMORY = 3,    /* host or device allocation failed; the handle is left unchanged */
    LBMG_NOT_CONVERGED = 4,    /* solve reached max_cycles; x holds the last iterate, stats say how far */
    LBMG_NOT_ASSEMBLED = 5,    /* solve/vcycle before lbmg_assemble */
    LBMG_COARSE_FACTOR = 6,    /* coarsest-level Cholesky met a non-positive pivot */
    LBMG_CUDA_ERROR = 7,       /* a CUDA call failed; lbmg_last_cuda_error() names it */
    LBMG_DIVERGED = 8,         /* residual became NaN or grew by 1e6 */
    LBMG_DEVICE_TIMEOUT = 9    /* a bounded device-side wait (grid barrier, or the bottom kernel's copy of
                                  its static data) expired; results are invalid */
};

enum { LBMG_FP64 = 0, LBMG_MIXED = 1 };          /* precision of the V-cycle */
enum { LBMG_GS_COLOURED = 0, LBMG_JACOBI = 1 };  /* smoother */

typedef struct lbmg_options {
    int min_depth;      /* coarsest depth; < 0: deepest level with at most coarse_max functions */
    int coarse_max;     /* default 160 */
    int nu1, nu2;       /* pre/post smoothing sweeps per level, default 2/2 */
    int smoother;       /* LBMG_GS_COLOURED (default) or LBMG_JACOBI */
    double jacobi_omega;/* damping of the weighted Jacobi smoother, default 0.6 */
    int split;          /* 1 (default): connectivity-aware split of Section 4.2; 0: unsplit space of Section 3.2 */
    int threads;        /* host threads for the hierarchy build; 0 = all cores */
    int persistent;     /* 1: whole solve in one cooperative launch (grid barriers between phases,
                           bounded waits; always used for batches); 0 (default): one graph launch
                           per cycle */
    int narrow_max;     /* bottom levels with at most this many rows run inside one block, with
                           block barriers between their phases (default 2048) */
    int barrier_phantoms; /* fault injection for tests, default 0: the persistent solve's grid barrier
                           waits for this many extra arrivals that never come, so its bounded wait
                           (about one second) expires and lbmg_solve returns LBMG_DEVICE_TIMEOUT */
    int use_graphs;     /* per-cycle path: 1 (default) replays a captured CUDA graph per cycle; 0
                           launches the cycle's kernels directly (same kernels, e.g. for profilers) */
    int pdl;            /* per-cycle path: 1 (default) chains the cycle's kernels with programmatic
                           dependent launch, so each kernel loads its static matrix rows while the
                           previous one finishes; 0 launches them with plain stream order.  Direct
                           launches (use_graphs = 0) on the legacy or per-thread default stream
                           always use plain stream order */
    int copy_phantom_bytes; /* fault injection for tests, default 0 (0..65536): the shared-memory bottom
                           kernel's copy of its static data waits for this many extra bytes that never
                           arrive, so its bounded wait (about one second) expires, the kernel sets a
                           status word and returns, and lbmg_solve returns LBMG_DEVICE_TIMEOUT at the
                           end of that cycle */
    int host_alloc_fail; /* fault injection for tests, default 0: 1 makes the host hierarchy builder fail
                           as an exhausted host allocation does, once the triangles are cut into voxel
                           pieces, so the build returns LBMG_OUT_OF_MEMORY and creates no handle */
    int host_check;     /* graph path: 0 (default) runs a whole solve as one graph launch whose
                           conditional loop is stopped by a device-side test of the residual norms, and
                           the host synchronizes once, at the end; 1 launches one graph per iteration
                           and reads the norms back after each one (the only mode in which
                           lbmg_stats.ms_fine_smooth is measured) */
    int cycle;          /* 0 (default): V-cycle; 1: W-cycle, two visits of each coarser level per cycle
                           (the cycle of the convergence experiment of Section 5.2).  Single meshes,
                           not with persistent (LBMG_INVALID_ARG) */
    int coarse_smooth;  /* 0 (default): the coarsest level is solved with its dense factor; 1: it is
                           relaxed by nu1 + nu2 coloured Gauss-Seidel sweeps like the other levels (the
                           minimum-depth sweep of Section 5.2, where the minimum depth is the coarsest
                           level a cycle visits).  Single meshes, not with persistent */
    int gpu_clip;       /* 0 (default): the hierarchy build runs on the host cores; 1: two of its steps
                           run on the GPU: the cut of the triangles into finest-voxel pieces (one thread
                           per triangle, the same sweep of axis planes) and, on every level, the sorted
                           (corner, triangle) pairs and the split labelling of each corner's support
                           into connected components (Section 4.2; one thread per corner of up to 255
                           triangles, one thread per (corner, triangle) pair with a shared lock-free
                           union-find for larger corners).  The dof numbering, prolongation and
                           contribution lists stay on the host.  The pieces agree with the host's up to
                           FMA contraction in the plane intersections, the labels exactly.  Needs a GPU
                           (LBMG_CUDA_ERROR otherwise), also for lbmg_host_build */
} lbmg_options;

typedef struct lbmg_stats {
    int cycles;              /* V-cycles applied */
    int converged;           /* 1 if every right-hand side met tol */
    double rel_residual[4];  /* final ||rhs - A x||_2 / ||rhs||_2 per right-hand side (FP64) */
    double initial_residual[4];
    float ms_total;          /* device time of the solve, CUDA events */
    float ms_fine_smooth;    /* device time of the finest-level smoothing sweeps summed over all cycles
                                (events in the per-cycle graph; %globaltimer in the persistent solve) */
    int learned;             /* 1 if the learned correction preceded the cycles (lbmg_learned_enable) */
    int learned_fallback;    /* 1 if an iteration with it raised a residual and the solve went on with
                                plain cycles (the acceptance test) */
    int host_syncs;          /* times the call waited for the device: 1 for a solve run as one graph
                                launch or one persistent launch (the final status read); one more per
                                iteration with host_check = 1 or without graphs */
} lbmg_stats;

typedef struct lbmg_ctx *lbmg_handle;

const char *lbmg_status_string(int code);
/* message of the last failure on this thread: the CUDA call that failed, or, after a
   failed lbmg_build_hierarchy / lbmg_build_batch, the host builder's reason */
const char *lbmg_last_cuda_error(void);
void lbmg_default_options(lbmg_options *o);

/*
 * Build the hierarchy (host, then upload).  Sections 3.2, 4.1-4.3.
 *  V: host double[nv][3] vertex positions; F: host int[nt][3] triangle indices.
 *  depth: finest grid depth, 1..12 (2^depth voxels per axis).
 * The mesh's bounding box is centred in a cube of side 1.1 x its largest extent.
 * For every level: fragments of triangles cut by the voxels (area above
 * 1e-12 finest voxel faces), the split functions (one per connected component
 * of supp(b_k) /\ M, two triangles being joined through a shared edge meeting
 * the open support cube or a shared vertex inside it), the prolongation of
 * Eq. 4 (parent component via chi, weights from the trilinear stencil
 * 1/2(1 2 1)), and the contribution lists used by lbmg_assemble.
 * Synchronous.  *out receives a new handle owned by the caller (lbmg_destroy).
 */
int lbmg_build_hierarchy(const double *V, int nv, const int *F, int nt, int depth,
                         const lbmg_options *opt, lbmg_handle *out);
void lbmg_destroy(lbmg_handle h);

/*
 * Build one hierarchy for a batch of meshes solved together (many meshes of
 * uneven size, each with its own embedding and depth).  V[i], F[i], nv[i],
 * nt[i], depth[i] describe mesh i as for lbmg_build_hierarchy.  Levels are
 * aligned at the finest: batch depth d holds level depth[i] - (D - d) of every
 * mesh, where D = (largest level count) - 1 and the coarsest batch depth is 0.
 * The finest-level vectors of a batch are the meshes' own finest vectors
 * concatenated in mesh order (see lbmg_instance_info); vertex arrays likewise.
 * A batch always uses the persistent solve; it stops when every mesh meets tol.
 * The meshes are built concurrently, one per host thread (opt->threads of them,
 * 0 = all cores), so the host memory held at once grows with the thread count.
 * Errors: LBMG_INVALID_ARG for a NULL array, ninst < 1 or a bad mesh (the first
 * failing mesh is named in lbmg_last_cuda_error), LBMG_DEGENERATE_MESH,
 * LBMG_OUT_OF_MEMORY, LBMG_CUDA_ERROR.
 */
int lbmg_build_batch(const double *const *V, const int *nv, const int *const *F, const int *nt, const int *depth,
                     int ninst, const lbmg_options *opt, lbmg_handle *out);
/* number of meshes in the hierarchy (1 for lbmg_build_hierarchy) */
int lbmg_instances(lbmg_handle h, int *ninst);
/* mesh `inst`: its finest and coarsest depth, finest function count, and the offsets of its rows in
   finest-level vectors and of its vertices in vertex arrays */
int lbmg_instance_info(lbmg_handle h, int inst, int *depth, int *min_depth, long *nfine, long *row_offset,
                       long *vertex_offset);
/* inst int[n_d]: the mesh of every row of level d, in the device dof order (all 0 for a
   single mesh).  Host only. */
int lbmg_row_instances(lbmg_handle h, int d, int *inst);
/* relative residual ||rhs - A x|| / ||rhs|| of every mesh and right-hand side after the last
   persistent solve, rel[ninst][nrhs] (host) */
int lbmg_instance_residuals(lbmg_handle h, int nrhs, double *rel);

/* min_depth and depth of the hierarchy. */
int lbmg_levels(lbmg_handle h, int *min_depth, int *depth);
/* functions (dofs), stored non-zeros and, for the finest level, fragments of level d */
int lbmg_level_info(lbmg_handle h, int d, long *ndof, long *nnz, long *nfrag);
/* cube side S and centre of the embedding (host double[3]) */
int lbmg_embedding(lbmg_handle h, double *cube_side, double *center);

/*
 * Per-triangle area weights for the mass matrix and the right-hand side
 * (Section 5.3, conformalized mean-curvature flow).  A cMCF step solves
 * (M_t + delta L_0) u_{t+1} = M_t u_t on the build-time function space: the
 * surface has moved by an affine map per triangle, so triangle T's area element
 * is the build-time one times w[T] = A_t(T) / A_0(T).  After this call,
 * lbmg_assemble forms A = M_w + t L with M_w,ij = sum_T w[T] int_T b_i b_j and L
 * unchanged, and lbmg_project_rhs integrates with the same weights.
 *  w: host double[nt] (the meshes' triangles in order, concatenated for a
 *     batch), each finite and >= 0; NULL restores the build-time metric (all 1).
 * Synchronizes `stream` first (the kernels that read the weights must have
 * finished) and copies synchronously.  Takes effect at the next lbmg_assemble /
 * lbmg_project_rhs.  Errors: LBMG_INVALID_ARG (NULL handle, a negative or
 * non-finite weight), LBMG_CUDA_ERROR.
 */
int lbmg_set_area_weights(lbmg_handle h, const double *w, void *stream);

/*
 * Assemble A_d = M_d + t L_d for every level (Eq. 2, Section 5.1; positive
 * stiffness L_ij = int <grad_M b_i, grad_M b_j>).  The finest level is
 * integrated exactly over each fragment (Gauss-Legendre product rule on a fan
 * of sub-triangles, exact to degree 6); every coarser level is the Galerkin
 * product P^T A_{d+1} P, which equals its own quadrature because the spaces nest
 * (Claim of Section 4.1).  Sums use precomputed contribution lists, no atomics.
 * Also factors the coarsest level (FP64 Cholesky of A + eps Id, eps =
 * 1e-12 mean diag, Discussion of Section 5).  Asynchronous on `stream`; a
 * non-positive pivot of that factorisation is kept in a device flag and reported
 * by the next solve (LBMG_COARSE_FACTOR).
 */
int lbmg_assemble(lbmg_handle h, double t, void *stream);

/*
 * rhs_i = int_M f b_i over the finest level, f linear on each triangle from
 * per-vertex values f_vertex[nv][nrhs] (Section 5.2, s_i; Section 5.3, M_t u_t).
 * rhs: [n_depth][nrhs].  Needs lbmg_assemble (it reuses the fragment moments).
 */
int lbmg_project_rhs(lbmg_handle h, const double *f_vertex, int nrhs, double *rhs, void *stream);

/*
 * Solve (M + t L) x = rhs by V-cycles: each cycle is ν1 smoothing sweeps per
 * level on the way down, residual, restriction P^T r, the coarsest solve, then
 * prolongation x += P e and ν2 sweeps on the way up (Section 4.3).  precision:
 * LBMG_FP64 runs the whole cycle in FP64; LBMG_MIXED runs it in FP32 inside an
 * FP64 defect-correction loop (residual and update in FP64).  Stops when
 * ||rhs - A x||_2 <= tol ||rhs||_2 for every right-hand side (||rhs - A x||_2 <=
 * tol when rhs = 0), or after max_cycles.  x: [n_depth][nrhs], in/out (warm
 * start).  stats may be NULL.
 * The default path runs the whole solve as one CUDA-graph launch: a conditional
 * WHILE node whose body is one cycle and a one-thread kernel that tests the norms
 * on the device and ends the loop; the call synchronizes once, to read the final
 * status.  With options.persistent (and for batches) the cycle loop runs in one
 * cooperative kernel launch, also with one synchronization.  With
 * options.host_check = 1 (lbmg_set_host_check) or use_graphs = 0 each cycle is one
 * launch and the call reads the norms back after each.  A coarsest-level
 * factorisation that failed in lbmg_assemble is reported here as
 * LBMG_COARSE_FACTOR.
 */
int lbmg_solve(lbmg_handle h, const double *rhs, double *x, int nrhs, double tol, int max_cycles,
               int precision, lbmg_stats *stats, void *stream);

/*
 * Conjugate gradients on (M + t L) x = rhs, preconditioned by one V-cycle of
 * Section 4.3 per iteration.  The cycle is symmetric (colours 0..7 on the way
 * down, 7..0 on the way up, nu1 = nu2, exact dense solve of A + eps I at the
 * coarsest level), so it is an SPD preconditioner; the iteration takes the
 * flexible (Polak-Ribiere) form, in which the nearly linear FP32 cycle of
 * LBMG_MIXED keeps it stable.  Every right-hand side has its own step lengths;
 * vectors, dot products and the operator are FP64, the cycle runs in `precision`.
 * Arguments, stopping rule (per right-hand side, recursively updated FP64
 * residual) and statistics as for lbmg_solve; stats->cycles counts iterations,
 * one V-cycle each.  Near-null modes that plain V-cycles reduce slowly (nearly
 * axis-aligned sheets, Discussion of Section 5) are taken out by the Krylov
 * recurrence.  Only with the coloured Gauss-Seidel smoother (LBMG_INVALID_ARG
 * otherwise); the persistent option does not apply.  On a batch every mesh has its
 * own step lengths (per-mesh dot products), the solve stops when every mesh and
 * right-hand side meets tol, stats->rel_residual holds the worst mesh per right-hand
 * side, and lbmg_instance_residuals reports each mesh afterwards.
 */
int lbmg_solve_pcg(lbmg_handle h, const double *rhs, double *x, int nrhs, double tol, int max_iters,
                   int precision, lbmg_stats *stats, void *stream);

/*
 * One step of conformalized mean-curvature flow (Section 5.3) on the build-time
 * function space: (M_t + delta L_0) x = M_t u_t, u_t the current vertex positions X
 * (linear per triangle), M_t the mass matrix with every triangle weighted by its
 * current over its build-time area, L_0 the build-time stiffness; then the new
 * positions X_next(v) = sum_i x_i b_i(v).  On `stream`: the area weights from X
 * (device kernels), lbmg_assemble(h, delta), the projection of X, lbmg_solve
 * (solver 0) or lbmg_solve_pcg (solver 1) warm-started from x, and vertex
 * evaluation; the call synchronizes once (the solve's status read).
 *  X, X_next: device double[nv][3] (may not alias); x: device double[n_depth][3],
 *  in/out: the previous step's solution as warm start (zeros at the first step).
 * Single meshes only.  Leaves the area weights of X in the handle (the next
 * lbmg_assemble uses them; lbmg_set_area_weights(h, NULL) restores the build-time
 * metric).  The first call allocates the step's weight and right-hand-side buffers.
 * Returns the solve's status (LBMG_NOT_CONVERGED still evaluates X_next); host
 * pointers or a batch give LBMG_INVALID_ARG.
 */
int lbmg_cmcf_step(lbmg_handle h, const double *X, double delta, double *x, double tol, int max_cycles,
                   int precision, int solver, double *X_next, lbmg_stats *stats, void *stream);

/*
 * The k smallest eigenpairs of L x = lambda M x on the finest level (the spectral analysis
 * of Section 5.1: M and L of Eq. 2 on the split space), by LOBPCG (locally optimal block
 * preconditioned conjugate gradients) preconditioned by one FP64 V-cycle of the assembled
 * A = M + t L per residual (t from the last lbmg_assemble; a t near 1 / lambda_k suits the
 * wanted end of the spectrum).  Each iteration does the block products, V-cycles and
 * Gram matrices on the device and the Rayleigh-Ritz step on the host (at most 48 x 48),
 * which reads the Gram matrices and residual norms back (two synchronizations per
 * iteration).  Stops when ||L x_j - lambda_j M x_j|| <= tol ||M x_j|| for every j.
 *  k: 1..16, 3k <= functions; X0: device double[n_depth][k], the start (e.g. random,
 *  columns independent); X: device double[n_depth][k], M-orthonormal eigenvectors
 *  (X may alias X0); lambda: host double[k], ascending; residuals: host double[k] or NULL;
 *  *iters: iterations taken.  The call allocates and frees its work blocks (about
 *  9 k n doubles).  Errors: LBMG_NOT_ASSEMBLED, LBMG_INVALID_ARG (sizes, host pointers, a
 *  batch), LBMG_DIVERGED (the block lost rank), LBMG_NOT_CONVERGED (x, lambda hold the last
 *  iterate), LBMG_CUDA_ERROR.
 */
int lbmg_eigs(lbmg_handle h, int k, double tol, int max_iters, const double *X0, double *lambda, double *X,
              double *residuals, int *iters, void *stream);

/* Number of kernels each call launches: lbmg_assemble, lbmg_project_rhs, one
   V-cycle step of lbmg_solve/lbmg_vcycles in `precision` (cycle + FP64 residual
   + norms; 0 for the persistent solve, whose cycles run inside its one launch),
   and the fixed part of lbmg_solve around its cycles.  Host only. */
int lbmg_launch_counts(lbmg_handle h, int precision, int *assemble, int *project_rhs, int *per_cycle,
                       int *solve_fixed);

/*
 * Launch-shape autotuner (throughput layer; the paper fixes no launch shapes).
 * For every level above the coarsest, times the coloured Gauss-Seidel sweep and
 * the residual kernel of `precision` for nrhs right-hand sides (1..4) with each of
 * nine launch shapes -- 4, 8 or 16 threads per matrix row x 128, 256 or 512 threads
 * per block -- as a captured graph of `reps` (1..64) sweeps replayed three times, and
 * keeps the fastest in the handle (the default 4 x 256 unless another shape is at
 * least 2% faster).  Threads per row 8 and 16 read the matrix in CSR order; 4 reads
 * a packed copy in which groups of 8 rows of one colour with equal quad counts
 * ceil(len / 4) store their entries quad-interleaved, so that each warp load is 256
 * aligned contiguous bytes.  Results are also kept in a process-wide cache
 * keyed by (device name, precision, kernel, lanes, rows, non-zeros): levels of
 * any handle that match an entry are not timed again.  The levels' cycle work
 * vectors are overwritten; they carry no state between calls.  Captured cycle
 * graphs are rebuilt at the next solve.  Needs lbmg_assemble first
 * (LBMG_NOT_ASSEMBLED).  Synchronous.  *timed (may be NULL) receives how many
 * (level, kernel) pairs were timed rather than taken from the cache.
 */
int lbmg_autotune(lbmg_handle h, int nrhs, int precision, int reps, int *timed, void *stream);
/* launch shapes of level d for `precision`: out[4] = Gauss-Seidel sweep (threads per row,
   threads per block), residual (threads per row, threads per block).  Host only. */
int lbmg_launch_shape(lbmg_handle h, int d, int precision, int *out);
/* device time (ms) that the last lbmg_autotune measured on this handle for level d's chosen
   shapes: ms[0] one Gauss-Seidel sweep (8 chained colour launches), ms[1] one residual
   launch; 0 where the shape came from the cache or was set by hand.  Host only. */
int lbmg_tuned_times(lbmg_handle h, int d, int precision, float *ms);
/* set a launch shape of level d by hand: kind 0 = Gauss-Seidel sweep, 1 = residual;
   tpr in {4, 8, 16} (see lbmg_autotune); tpb a multiple of 32 in [32, 512], or, for an
   LBMG_MIXED sweep with tpr = 4, tpb = 1024: the whole sweep (all colour steps of the
   sweeps of one smoothing) in one cooperative launch of the packed-copy kernel, whose
   blocks meet at a bounded grid barrier between colours (a timeout gives
   LBMG_DEVICE_TIMEOUT); it computes exactly what the colour launches of tpr = 4 compute.
   LBMG_INVALID_ARG otherwise.  Results change only by the summation order inside a row.
   Host only. */
int lbmg_set_launch_shape(lbmg_handle h, int d, int precision, int kind, int tpr, int tpb);
/* options.host_check of an existing handle (0 or 1; LBMG_INVALID_ARG otherwise).  Host only. */
int lbmg_set_host_check(lbmg_handle h, int on);
/* write / read the process-wide tuning cache as text, one entry per line:
   device fp64 kind lanes rows nnz threads_per_row threads_per_block.
   Load merges valid lines and returns LBMG_INVALID_ARG if the file cannot be
   opened or a line is malformed (valid lines are still taken). */
int lbmg_tune_cache_save(const char *path);
int lbmg_tune_cache_load(const char *path);

/* Exactly `cycles` V-cycles in the same defect-correction form, with no norm
   read-back (used for throughput measurement).  x in/out. */
int lbmg_vcycles(lbmg_handle h, const double *rhs, double *x, int nrhs, int cycles, int precision,
                 void *stream);

/* r = rhs - A_d x on level d in FP64 (Eq. 2 operator); all [n_d][nrhs]. */
int lbmg_residual(lbmg_handle h, int d, const double *rhs, const double *x, double *r, int nrhs,
                  void *stream);
/* The mixed solve's outer residual r = rhs - A_d x (Section 4.3's defect correction) as
   lbmg_residual computes it, arguments and layout the same, with FP64 values carried as
   pairs of FP32 numbers (value = hi + lo): every product a x = ah xh + (ah xl + al xh + the
   exact rounding error of ah xh) and every partial sum is an FP32 pair (Knuth's two-sum),
   and rhs - sum is formed in FP64.  The result agrees with the FP64 residual to about 2^-44
   of sum_j |a_ij x_j| (the dropped al xl term and FP32 rounding of the small terms).  Why:
   GB300 executes FP64 arithmetic at a small fraction of its FP32 rate, which made the FP64
   residual of the finest level compute-bound.  Levels with a packed copy only (not the
   coarsest): LBMG_INVALID_ARG there. */
int lbmg_residual_split(lbmg_handle h, int d, const double *rhs, const double *x, double *r, int nrhs,
                        void *stream);

/* `sweeps` smoothing sweeps of the configured smoother on level d, in the
   given precision, on A_d x = rhs; x in/out.  Colour order 0..7. */
int lbmg_smooth(lbmg_handle h, int d, const double *rhs, double *x, int nrhs, int sweeps,
                int precision, void *stream);

/*
 * ||rhs_q - A_d x_q||_2 for each right-hand side q < nrhs of level d (FP64), the
 * norms of lbmg_residual's output, computed without allocating anything.  The
 * paper has no counterpart.  It is for callers that cannot allocate device memory
 * while they run: a time-critical loop cannot afford cudaMalloc's implicit device
 * synchronisation or an out-of-memory failure midway, and a plug-in inside an
 * application that owns the device memory budget may not grow it.  The call's only
 * scratch, the partial sums of a two-pass reduction, is a file-scope device array
 * of 512 x 4 doubles (16 KiB) that every GPU loading the library keeps until the
 * process exits.
 *  rhs, x: device double[n_d][nrhs] in the library's dof order of level d;
 *  norms: device double[nrhs]; 1 <= nrhs <= 4.  Host pointers, memory of another
 *  device, a level outside [min_depth, depth] or more than 4 right-hand sides are
 *  rejected with LBMG_INVALID_ARG, a handle not yet assembled with
 *  LBMG_NOT_ASSEMBLED (lbmg_last_cuda_error names the reason).  Asynchronous on
 *  `stream`.
 *  The first call on each device looks up the array's device address with that
 *  device current and keeps it; make that first call before any stream capture.
 *  Each call overwrites the whole array before reading it; calls that overlap on
 *  the GPU (other streams or host threads) share the array and race, so serialize
 *  them.
 */
int lbmg_residual_norms_noalloc(lbmg_handle h, int d, const double *rhs, const double *x, int nrhs, double *norms,
                                void *stream);

/* r_c = P^T r_f from level d to d-1 (FP64). r_f: [n_d][nrhs], r_c: [n_{d-1}][nrhs]. */
int lbmg_restrict(lbmg_handle h, int d, const double *r_fine, double *r_coarse, int nrhs, void *stream);
/* x_f += P x_c from level d-1 to d (FP64). */
int lbmg_prolong_add(lbmg_handle h, int d, const double *x_coarse, double *x_fine, int nrhs, void *stream);

/* u(v) = sum_i x_i b_i(v) at every mesh vertex; x: [n_depth][nrhs], u: [nv][nrhs]. */
int lbmg_eval_vertices(lbmg_handle h, const double *x, int nrhs, double *u, void *stream);

/*
 * Host copies for inspection and testing (synchronous).
 *  lbmg_get_dofs: corner int[n][3] (grid corner index at depth d), mintri int[n].
 *  lbmg_get_matrix: CSR of level d, rowptr int[n+1], col int[nnz] (sorted per
 *    row), M, L double[nnz] (either may be NULL); needs lbmg_assemble.
 *  lbmg_get_prolongation: parents int[n_d][8] (coarse dofs at depth d-1, -1 =
 *    none) and weights double[n_d][8].
 */
int lbmg_get_dofs(lbmg_handle h, int d, int *corner, int *mintri);
int lbmg_get_matrix(lbmg_handle h, int d, int *rowptr, int *col, double *M, double *L);
int lbmg_get_prolongation(lbmg_handle h, int d, int *parents, double *weights);

/*
 * Host-only hierarchy: the construction of lbmg_build_hierarchy (Sections 3.2,
 * 4.1-4.3: voxel pieces, split functions, the Eq. 4 prolongation, the sparsity
 * pattern of every level) without any device memory or CUDA call, so that the
 * split space can be built and inspected on a machine without a GPU.  Arguments
 * and errors of lbmg_host_build are those of lbmg_build_hierarchy (no
 * LBMG_CUDA_ERROR); the other calls read the result in the same layout and dof
 * order as the device handle's lbmg_levels, lbmg_level_info, lbmg_get_dofs,
 * lbmg_get_matrix (pattern only) and lbmg_get_prolongation.  LBMG_INVALID_ARG
 * for a NULL handle or a level outside [min_depth, depth] (outside
 * (min_depth, depth] for the prolongation).  The handle is owned by the caller
 * and released with lbmg_host_destroy; a host handle is not an lbmg_handle.
 */
typedef struct lbmg_host_ctx *lbmg_host_handle;
int lbmg_host_build(const double *V, int nv, const int *F, int nt, int depth, const lbmg_options *opt,
                    lbmg_host_handle *out);
void lbmg_host_destroy(lbmg_host_handle h);
int lbmg_host_levels(lbmg_host_handle h, int *min_depth, int *depth);
int lbmg_host_level_info(lbmg_host_handle h, int d, long *ndof, long *nnz, long *nfrag);
int lbmg_host_get_dofs(lbmg_host_handle h, int d, int *corner, int *mintri);
int lbmg_host_get_pattern(lbmg_host_handle h, int d, int *rowptr, int *col);
int lbmg_host_get_prolongation(lbmg_host_handle h, int d, int *parents, double *weights);
/*
 * Host-only batch: the construction of lbmg_build_batch (same arguments and
 * errors, no LBMG_CUDA_ERROR), read with the calls above.
 *  lbmg_host_instances: number of meshes and, per mesh (arrays [ninst], may be
 *    NULL), its finest and coarsest depth.
 *  lbmg_host_row_instances: inst int[n_d], the mesh of every row of level d.
 * A single-mesh host handle reports one instance.
 */
int lbmg_host_build_batch(const double *const *V, const int *nv, const int *const *F, const int *nt,
                          const int *depth, int ninst, const lbmg_options *opt, lbmg_host_handle *out);
int lbmg_host_instances(lbmg_host_handle h, int *ninst, int *depth, int *min_depth);
int lbmg_host_row_instances(lbmg_host_handle h, int d, int *inst);

/*
 * Learned residual correction in front of each cycle.  The paper has no counterpart:
 * its solver iterates the plain cycle on the residual (Section 4.3, Gauss-Seidel
 * smoothing of Section 5.2), which is also the fallback here and the yardstick of the
 * learned form.  Before each cycle of lbmg_solve / lbmg_vcycles the residual r gets
 * delta_i = omega_i r_i / a_ii (every lane; 0 on rows under the relaxation floor) and
 * the cycle starts from delta instead of zero.  omega_i = 1 + y_i / (1 + |y_i|) in
 * (0, 2) comes from a network 30 -> 64 (ReLU) -> 1 of node i's features: 27
 * neighbour-offset sums of a_ij / a_ii (centre: a_ii / mean diagonal), the entry
 * count / 27, and two residual features, q / (1 + |q|) with q_i = r_i.z_i / z_i.z_i,
 * z = A D^-1 r, and e_i / (e_i + mean e) with e_i = r_i.r_i (sums over the lanes).
 * The dense layer runs on the tensor cores (BF16 inputs and weights, FP32
 * accumulation).  Training minimises log(||C (r - A delta)||^2 / ||r||^2), C = I - A V
 * (the residual reduction of one learned iteration, V the plain V-cycle), in FP64 by the
 * exact adjoint, with Adam on FP32 master weights.  Acceptance test: once an
 * iteration with the correction leaves a larger relative residual than the one
 * before in some lane, the solve drops it and runs plain cycles (the host loop
 * without a stopping test does not apply it).  Conjugate gradients and the
 * persistent solve do not use the correction (lbmg_solve returns
 * LBMG_INVALID_ARG for a persistent handle with it on).  Single-mesh hierarchies
 * with at least two levels; lbmg_assemble first (else LBMG_NOT_ASSEMBLED).
 *  lbmg_learned_nparams: length P of the flat parameter vector: W1 [32][64]
 *    row-major (rows 30, 31 unused, zero), b1 [64], w2 [64], b2 [1].
 *  lbmg_learned_params: get (host double[P], may be NULL) and/or set (host
 *    double[P], may be NULL; resets the Adam moments).
 *  lbmg_learned_state: get and/or set (host double[3 P + 1], may be NULL) the
 *    optimiser state: parameters, Adam's first and second moments, its step count;
 *    carries training from one handle (mesh) to the next.
 *  lbmg_learned_collect: runs plain FP64 V-cycles from x = 0 on rhs [n_depth][ns]
 *    (user order, ns <= 4 lanes) and stores the residual block before cycles
 *    skip .. skip + keep - 1 as `keep` training samples (appended to the bank).
 *  lbmg_learned_loss_grad: loss and gradient (host double[P], may be NULL) at the
 *    current parameters for one residual sample r0 [n_depth][ns], ns <= 4.
 *  lbmg_learned_train: `steps` Adam steps with learning rate lr; order (host
 *    int[steps][batch], batch <= 8) lists the bank samples of each step, whose
 *    mean gradient the step takes; loss_hist (host double[steps], may be NULL)
 *    receives each step's mean loss.
 *  lbmg_learned_enable: on = 1 puts the correction in front of every cycle of this
 *    handle's solves (its stencil features follow each lbmg_assemble); 0 removes it.
 *  lbmg_learned_apply: the correction of one residual r [n_depth][ns] (ns <= 4) by
 *    the solve's own kernels in the given precision (LBMG_MIXED: FP32 features and
 *    start, LBMG_FP64: FP64): omega [n_depth] and delta [n_depth][ns], user order.
 *    r, omega and delta are device pointers (else LBMG_INVALID_ARG).
 */
int lbmg_learned_nparams(void);
int lbmg_learned_params(lbmg_handle h, double *get, const double *set, void *stream);
int lbmg_learned_state(lbmg_handle h, double *get, const double *set, void *stream);
int lbmg_learned_collect(lbmg_handle h, const double *rhs, int ns, int skip, int keep, void *stream);
int lbmg_learned_loss_grad(lbmg_handle h, const double *r0, int ns, double *loss, double *grad, void *stream);
int lbmg_learned_train(lbmg_handle h, int steps, double lr, const int *order, int batch, double *loss_hist,
                       void *stream);
int lbmg_learned_enable(lbmg_handle h, int on, void *stream);
int lbmg_learned_apply(lbmg_handle h, const double *r, int ns, int precision, double *omega, double *delta,
                       void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBMG_H */
