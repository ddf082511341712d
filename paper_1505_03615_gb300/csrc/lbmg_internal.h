// lbmg_internal.h -- device-side state of a hierarchy and kernel launch wrappers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "hier.h"

namespace lbmg {

constexpr int kNQ = 4;            // Gauss-Legendre points per direction of the collapsed triangle rule
constexpr int kMaxCoarse = 2048;  // largest coarsest level factored densely
constexpr int kNormBlocks = 256;  // partial sums of the two-pass norm reduction

// Launch shape of the row-parallel kernels (Gauss-Seidel colour sweep, residual):
// tpr threads share one matrix row (4, 8 or 16), tpb threads per block (128-512).  With
// 4 threads per row the kernels read the packed copy of the matrix (packed.cu).
struct LaunchShape {
    int tpr = 4, tpb = 256;   // Gauss-Seidel with tpb = 1024: the whole-sweep cooperative kernel (packed.cu)
    int grid = 0;             // its blocks (0: one per SM; fewer make the grid barrier cheaper on small levels)
};
constexpr int kSweepShapeTpb = 1024;
enum { kShapeSmooth = 0, kShapeResidual = 1 };

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may begin while the kernel before it in the
// stream is still running; it reads only data that no kernel of the chain writes
// (the matrices, transfer tables) until grid_dep_wait() returns, which happens
// once the predecessor has finished and its writes are visible.  Each kernel
// calls grid_dep_launch() right after its own wait, so at most two kernels of a
// chain are resident at once.  Without the launch attribute both are no-ops.
#ifdef __CUDACC__
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif

// The kernels of one V-cycle form a chain: a launch gets the programmatic
// attribute only when the operation just before it in the stream is a kernel of
// the same chain (an event record, memset or copy in between cuts it).
struct Chain {
    bool on = false, prev = false;
    bool capturing = false;   // the stream is being captured into a graph
    void cut() { prev = false; }
};

// cudaLaunchKernelEx with the programmatic attribute when the chain allows it;
// marks the chain as ending in a kernel.
template <class... KArgs, class... Args>
inline void klaunch(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, Chain *ch,
                    Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (ch && ch->on && ch->prev) ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    if (ch) ch->prev = true;
}

// The groups of one colour of the packed copy, sorted by quad count, as runs of equal quads: group g of
// run k (g[k] <= g < g[k + 1]) starts at entry 32 (b[k] + (g - g[k]) q[k]) and has q[k] quads.  Passed to
// the colour kernel by value, so that a group's position needs no load (n = 0: read the group header).
constexpr int kPkRuns = 12;
struct PkRuns {
    int n = 0;
    int g[kPkRuns] = {0}, b[kPkRuns] = {0}, q[kPkRuns] = {0};
};

struct DevLevel {
    int d = 0, n = 0;
    int ns = 0;                            // rows [0, ns) are smoothed; [ns, n) belong to coarsest blocks
    int cb0 = 0, ncb = 0;                  // this level's coarsest blocks in Ctx::cblk
    int64_t nnz = 0;
    int cs[9] = {0};                       // colour ranges
    int cs_all[9] = {0};                   // colour ranges of all rows (the coarsest level relaxed)
    int *rp = nullptr, *ci = nullptr;
    double *M = nullptr, *L = nullptr, *A64 = nullptr;
    float *A32 = nullptr;
    double *dinv64 = nullptr;
    float *dinv32 = nullptr;
    int *par = nullptr;                    // [n*8] parents at depth d-1, -1 pad
    int8_t *npl2 = nullptr;                // log2 #parents
    int *crp = nullptr;                    // children lists (this level as coarse)
    uint32_t *cch = nullptr;
    int64_t *grp = nullptr;                // Galerkin lists (this level as coarse)
    uint32_t *gidx = nullptr;
    // V-cycle work vectors, room for [n][4]
    double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;
    float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr;
    // packed copy of A for the row kernels (packed.cu): per colour, 8-row groups of rows with
    // equal quad counts, entries quad-interleaved across the group; null pk_map when not built
    int2 *pk_gq = nullptr;                 // [ngroups] (base / 32, quads)
    int *pk_rows = nullptr;                // [ngroups * 8] rows of the slots, -1 none
    int *pk_map = nullptr;                 // [total] packed position -> CSR position, -1 pad
    int *pk_col = nullptr;                 // [total] columns in packed order, -1 pad (FP64 kernels)
    int2 *pk_e32 = nullptr;                // [total] (column, FP32 value bits)
    double *pk_v64 = nullptr;              // [total] FP64 values
    float2 *pk_v2 = nullptr;               // [total] FP64 values as FP32 pairs (hi, lo = value - hi)
    int64_t pk_total = 0;
    int pk_gs[10] = {0};                   // group ranges of colours 0..7, then rows [ns, n)
    int64_t pk_es[10] = {0};               // entry offset of the first group of each range (pk_es[9]: total)
    PkRuns pk_runs[8];                     // per colour (n = 0 when a colour has more than kPkRuns runs)
    LaunchShape shape[2][2];               // [FP64][kShapeSmooth / kShapeResidual], set by the autotuner
    float tuned_ms[2][2] = {{0, 0}, {0, 0}};   // device time of the chosen shape when the tuner timed it
};

struct Learned;

constexpr int kMaxNarrow = 6;     // bottom levels that can live in shared memory
struct NarrowLevel {
    int n = 0, ns = 0, nnz = 0, cb0 = 0, ncb = 0;
    int cs[9] = {0};
    // byte offsets in shared memory (blob part, then vectors); -1 = absent
    // (parents: o_pof [n + 1] offsets into o_par, the parents of each row in order; r: one
    // buffer shared by all levels, live only between a level's residual and its restriction)
    int o_rp = -1, o_ci = -1, o_A = -1, o_dinv = -1, o_par = -1, o_pof = -1, o_crp = -1, o_cch = -1;
    int o_x = -1, o_b = -1, o_r = -1;
};
struct NarrowParams {
    int d0 = 0, dn = -1, nu1 = 2, nu2 = 2;
    NarrowLevel lev[kMaxNarrow];
};
struct NarrowState {
    int dn = -1;                      // top level held in shared memory (< d0: none)
    NarrowParams p;
    unsigned char *blob = nullptr;    // packed static data (device)
    int *status = nullptr;            // device word (beside the norms the solve reads back every cycle):
                                      // 1 after a bounded wait of the bottom kernel gave up
    int blob_bytes = 0, vec_bytes = 0;
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int R = 0, precision = -1, nu1 = -1, nu2 = -1, smoother = -1, pcg = -1;
    int cond = -1;   // 1: the whole solve (conditional WHILE node), 0: one iteration
    int learned = -1;   // the learned correction in front of each cycle
};

// Device-side control of a solve that runs as one graph launch: a conditional WHILE node
// whose body is one iteration followed by a check kernel that decides, from the residual
// norms the iteration leaves in device memory, whether another iteration follows.
struct SolveCtl {
    double tol;
    int max_cycles, cycles, status, fixed;   // fixed: run exactly max_cycles iterations
    int nrhs;
    int learned_off;                         // a learned iteration raised a residual: plain cycles from now on
    int pad[2];
    double nb[4], r0[4], rel[4];            // ||b||^2, initial and current relative residual per lane
};
enum { kCtlRunning = 0, kCtlConverged = 1, kCtlDiverged = 2, kCtlTimeout = 3, kCtlMaxCycles = 4, kCtlCoarse = 5 };

struct Ctx {
    HostHierarchy host;
    int D = 0, d0 = 0, nv = 0, nt = 0, nfrag = 0;
    int ninst = 1, nu = 0;                 // meshes; rows of a user finest vector
    double *frag_scale = nullptr;          // [nfrag] physical area per finest-unit area
    // the pieces' moments and local (M, L) integrals in finest-unit area depend only on the
    // build-time geometry: computed by the first assembly, reused by the next (frag_scale enters
    // in fine_gather_kernel)
    bool moments_ready = false;
    int *fperm = nullptr;                  // [nu] user finest index -> finest row
    int *fiperm = nullptr;                 // [n_D] finest row -> user index
    // coarsest blocks, one per mesh: (level, mesh, first row, rows, inverse offset), sorted by level
    std::vector<int> cblk_host;
    int *cblk = nullptr;
    int ncblk = 0, n0max = 0;
    // finest-level norm work items: (mesh, first row, end row), chunks of (colour, mesh) segments
    std::vector<int> nitem_host;
    int *nitem = nullptr;
    int nnitem = 0;
    double *item_part = nullptr;           // [nnitem][8]
    double *inst_norm = nullptr;           // [ninst][12]: ||r||^2, ||b||^2, initial ||r||^2 per rhs
    int nu1 = 2, nu2 = 2, smoother = 0;
    int gamma = 1;                         // coarse visits per level: 1 V-cycle, 2 W-cycle
    int coarse_smooth = 0;                 // 1: the coarsest level is relaxed, not solved
    double omega = 0.6;
    DevLevel lev[kMaxDepth + 1];
    // finest-level geometry
    double *poly = nullptr;
    int *forder = nullptr;       // [nfrag] fragments by vertex count (moment kernel order)
    int *pstart = nullptr, *ftri = nullptr, *fvox = nullptr, *fdof = nullptr;
    double *tnormal = nullptr, *Vg = nullptr;
    int *F = nullptr;
    int64_t *arp = nullptr, *rrp = nullptr;
    uint32_t *aidx = nullptr, *ridx = nullptr;
    double *moments = nullptr;   // [nfrag*27]
    double *stage = nullptr;     // [nfrag*36*2]  (M, L) per local pair
    double *stage_rhs = nullptr; // [nfrag*8*4]
    int *vdof = nullptr;
    double *vw = nullptr;
    // coarsest level
    double *cdense = nullptr;    // factor workspace n0*n0
    double *cinv64 = nullptr;
    float *cinv32 = nullptr;
    int *flag = nullptr;         // device status word (coarse factor)
    // a flow step's triangle weights [nt] and right-hand side [n_D][3] (allocated at the first step)
    double *cmcf_w = nullptr, *cmcf_rhs = nullptr;
    // finest FP64 solve vectors, room for [n][4]
    double *xs = nullptr, *bs = nullptr, *rs = nullptr;
    double *norm_part = nullptr, *norm_out = nullptr;
    double *diag_part = nullptr;   // [256] per-block sums of a level's diagonal
    // preconditioned conjugate gradients: z, p, q = -A p and a zero vector ([n][4] FP64), scalars, partials
    double *pcg_z = nullptr, *pcg_p = nullptr, *pcg_q = nullptr, *pcg_zero = nullptr;
    double *pcg_s = nullptr, *pcg_part = nullptr;
    // batches: per-mesh scalars [ninst][kPcgScalars], the first work item of each mesh, finest row -> mesh
    double *pcg_si = nullptr;
    double *pcg_tol = nullptr;     // [1] tolerance of the running batch solve
    int *item_start = nullptr, *row_inst = nullptr;
    double *h_norm = nullptr;    // pinned [8]
    SolveCtl *ctl = nullptr;     // device control block of the running solve
    SolveCtl *h_ctl = nullptr;   // pinned copy read after the solve
    double *norm_b = nullptr;    // [4] ||b||^2 per lane of the running solve
    int host_check = 0;          // 1: the host reads the norms after every iteration (events time
                                 // the finest smoothing); 0: one graph launch per solve
    bool cond_failed = false;    // the conditional graph could not be built: the host loop is used
    // staging of user vectors (device [n][nrhs]) and pinned host mirrors
    double *dev_io = nullptr;
    size_t dev_io_bytes = 0;
    double *pin_io = nullptr;
    size_t pin_io_bytes = 0;
    bool assembled = false;
    double t = 0;
    cudaStream_t capture_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_smooth[4] = {nullptr, nullptr, nullptr, nullptr};   // around finest-level smoothing in the cycle graph
    GraphCache graph;
    // persistent cooperative solve
    int persistent = 1;           // use the one-launch solve when the device allows it
    int use_graphs = 1;           // per-cycle path: replay a captured graph (1) or launch directly (0)
    int pdl = 1;                  // chain the kernels of a cycle with programmatic dependent launch
    int persist_ok = 0;
    int persist_blocks = 0, persist_dn = 0, persist_narrow = 2048;
    int barrier_phantoms = 0;        // fault injection: extra arrivals a grid barrier waits for
    int copy_phantoms = 0;           // fault injection: extra bytes the bottom kernel's copy waits for
    void *persist_views = nullptr;
    void *views32 = nullptr, *views64 = nullptr;   // level views for the one-block bottom cycle
    size_t persist_view_bytes = 0;
    double *persist_part = nullptr;   // [blocks][8]
    double *persist_norm = nullptr;   // [16]
    void *persist_state = nullptr;    // 64 bytes: barrier, status, cycles, timer
    void *h_state = nullptr;          // pinned mirror: 64 bytes state + 16 doubles norms
    NarrowState narrow;               // shared-memory bottom of the V-cycle (narrow.cu)
    // the mixed solve's iterate as FP32 pairs for its outer residual (packed.cu)
    float *xs_hi = nullptr, *xs_lo = nullptr;
    // whole-sweep cooperative kernel (packed.cu): arrival counter and grid per lane count
    unsigned *sweep_bar = nullptr;
    int sweep_blocks[5] = {0, 0, 0, 0, 0};
    // learned residual correction in front of each cycle (learned.cu)
    Learned *learned = nullptr;
    int learned_on = 0;
};

// ----- shared-memory bottom cycle (narrow.cu) -----
int narrow_smem_setup(Ctx &c, size_t smem_budget);
size_t narrow_smem_budget();   // dynamic shared memory a block of the bottom kernel may take
void narrow_smem_refresh(const Ctx &c, cudaStream_t s);
void launch_narrow_smem(const Ctx &c, int R, cudaStream_t s, Chain *ch = nullptr);

// ----- launch-shape autotuner (tune.cu) -----
int autotune(Ctx &c, int R, int precision, int reps, cudaStream_t s, int *timed);
int tune_cache_save(const char *path);
int tune_cache_load(const char *path);

// ----- learned residual correction (learned.cu) -----
int learned_setup(Ctx &c, cudaStream_t s);
void learned_free(Ctx &c);
int learned_params(Ctx &c, double *get, const double *set, cudaStream_t s);
int learned_state(Ctx &c, double *get, const double *set, cudaStream_t s);
int learned_collect(Ctx &c, const double *rhs_user, int ns, int skip, int keep, cudaStream_t s);
int learned_loss_grad(Ctx &c, const double *r0_user, int ns, double *loss, double *grad, cudaStream_t s);
int learned_train(Ctx &c, int steps, double lr, const int *order, int batch, double *loss_hist, cudaStream_t s);
int learned_enable(Ctx &c, int on, cudaStream_t s);
void learned_refresh(Ctx &c, cudaStream_t s);
void learned_enqueue(Ctx &c, int R, int precision, cudaStream_t s, Chain *ch);
int learned_apply(Ctx &c, const double *r_user, int ns, int precision, double *omega_dev, double *delta_dev,
                  cudaStream_t s);
int learned_nparams();

// ----- persistent solve (persist.cu) -----
int persist_setup(Ctx &c);
int narrow_views_setup(Ctx &c);
void launch_narrow_cycle(const Ctx &c, int precision, int R, int top, cudaStream_t s);
int persist_solve(Ctx &c, int precision, int R, int nrhs, double tol, int max_cycles, cudaStream_t s);
size_t persist_view_bytes();

// ----- conformalized mean-curvature flow (cmcf.cu) -----
// per-triangle area ratios of the positions X (device [nv][3]) to the build-time surface, and
// the fragments' mass scales sigma^2 w_T; tri_w: device [nt] scratch
void launch_cmcf_weights(const Ctx &c, const double *X, double *tri_w, cudaStream_t s);

// ----- smallest eigenpairs of L x = lambda M x (lobpcg.cu) -----
// 0 converged, 1 bad size, 2 CUDA failure, 3 the block lost rank, 4 not converged in max_iters
int lobpcg(Ctx &c, int k, double tol, int max_iters, const double *X_user, double *lambda, double *X_out, double *res,
           int *iters, cudaStream_t s, std::string &err);

// ----- kernels (assemble.cu) -----
void launch_fragment_moments(const Ctx &c, cudaStream_t s);
void launch_fine_gather(const Ctx &c, double t, cudaStream_t s);
void launch_galerkin(const Ctx &c, int dc, double t, cudaStream_t s);
// FP64 and FP32 inverse diagonals, 0 for rows below 1e-20 of the level's mean diagonal;
// part: 256 doubles of scratch (per-block sums of the diagonal)
void launch_inverse_diag(const DevLevel &L, double *part, cudaStream_t s);
void launch_project_rhs(const Ctx &c, const double *fv, int nrhs, double *rhs_out, cudaStream_t s);
void launch_eval_vertices(const Ctx &c, const double *x, int nrhs, double *u, cudaStream_t s);

// ----- packed matrix layout of the row kernels (packed.cu) -----
// host: groups, slot rows, packed -> CSR position map and columns of one level (rows of
// colours 0..7, then [ns, n)); false when the packed positions would not fit 32 bits
bool packed_layout(const HostLevel &hl, std::vector<int32_t> &gq, std::vector<int32_t> &rows,
                   std::vector<int32_t> &map, std::vector<int32_t> &col, int gs[10], int64_t *total);
// refresh the packed FP32 and FP64 values from the level's CSR A32 / A64 (after assembly)
void launch_packed_fill(const DevLevel &L, cudaStream_t s);
// packed Gauss-Seidel colour / residual over rows [0, nrows); false when the level or the
// matrix has no packed copy (the caller then uses the CSR kernels)
template <class T> bool launch_packed_smooth(const DevLevel &L, int colour, const T *A, const T *dinv, const T *b,
                                             T *x, int R, int tpb, cudaStream_t s, Chain *ch, int next = -1);
template <class T> bool launch_packed_residual(const DevLevel &L, const T *A, const T *b, const T *x, T *r, int R,
                                               int nrows, int tpb, cudaStream_t s, Chain *ch);
// r = b - A x at all rows of level L for the mixed solve's outer residual: x given as FP32 pairs
// (xh + xl), the matrix as FP32 pairs, products and sums in pairs of FP32 (about 44 significant
// bits) and b - sum in FP64; false when the level has no packed copy
bool launch_packed_residual_split(const DevLevel &L, const double *b, const float *xh, const float *xl, double *r,
                                  int R, cudaStream_t s, Chain *ch);
// xh, xl of an FP64 vector; x = xh + xl in FP64; x += e on the pair (FP32 two-sum)
void launch_split(const double *x, float *xh, float *xl, int64_t n, cudaStream_t s);
void launch_join(const float *xh, const float *xl, double *x, int64_t n, cudaStream_t s);
void launch_add_pair(const float *e, float *xh, float *xl, int64_t n, cudaStream_t s, Chain *ch);
// a colour sequence (FP32) in one cooperative launch; bar: a device counter, status: the
// bounded-wait word; false if the level has no packed copy or the launch is refused
bool launch_packed_sweep(const DevLevel &L, const int *seq, int nseq, const float *dinv, const float *b, float *x,
                         int R, unsigned *bar, int *status, int blocks, cudaStream_t s);
int packed_sweep_blocks(int R);   // the grid of the sweep kernel (resident blocks per SM x SMs)

// ----- kernels (relax.cu) -----
// vectors below are [n][R] with stride R in {1, 2, 4} (3 right-hand sides padded to 4)
// `sweeps` Gauss-Seidel sweeps of level L (colours 0..7, or 7..0 backwards): one cooperative
// launch per call when the level's tuned shape is the whole-sweep kernel (FP32), else one
// launch per colour, each prefetching the next colour's entries.  skip: colour steps of the
// first sweep already done (1: the restriction applied colour 0's step from a zero start)
template <class T> void launch_sweeps(const Ctx &c, const DevLevel &L, int sweeps, bool forward, const T *A,
                                      const T *dinv, const T *b, T *x, int R, cudaStream_t s, Chain *ch,
                                      int skip = 0);
// next: the colour launched after this one on the same level (-1: none); its packed entries
// are prefetched into L2 while this colour runs
template <class T> void launch_smooth_colour(const DevLevel &L, int colour, const T *A, const T *dinv,
                                             const T *b, T *x, int R, cudaStream_t s, Chain *ch = nullptr,
                                             int next = -1);
template <class T> void launch_residual(const DevLevel &L, const T *A, const T *b, const T *x, T *r, int R,
                                        cudaStream_t s, int nrows = -1, Chain *ch = nullptr);
template <class T> void launch_jacobi_update(const DevLevel &L, const T *dinv, const T *r, T *x, T omega, int R,
                                             cudaStream_t s);
// bc = P^T rf; when xc is given, the coarse correction xc is zeroed in the same pass, or, with
// first_colour, given the first Gauss-Seidel colour step from zero: x_i = 0 + b_i / a_ii on the rows
// of colour 0 (the colour kernels' arithmetic with x = 0, bit for bit), zero elsewhere
template <class T> void launch_restrict(const DevLevel &Lc, const T *rf, T *bc, int R, cudaStream_t s,
                                        T *xc = nullptr, Chain *ch = nullptr, bool first_colour = false);
template <class T> void launch_prolong_add(const DevLevel &Lf, const T *xc, T *xf, int R, cudaStream_t s,
                                           Chain *ch = nullptr);
struct Ctx;
template <class T> void launch_coarse_apply(const Ctx &c, const DevLevel &L, const T *inv, const T *b, T *x, int R,
                                            cudaStream_t s, Chain *ch = nullptr);
void launch_coarse_factor(const Ctx &c, const int *const *rps, const int *const *cis, const double *const *As,
                          cudaStream_t s);
void launch_norms(const double *v, int n, int R, double *part, double *out, cudaStream_t s, Chain *ch = nullptr);
// conjugate-gradient scalars in Ctx::pcg_s, four lanes each
enum { kPcgRz = 0, kPcgS1 = 4, kPcgS2 = 8, kPcgAlpha = 12, kPcgBeta = 16, kPcgRz0 = 20, kPcgScalars = 24 };
// a lane whose r.z has fallen below this fraction of its first value is converged to
// rounding level (residual about 1e-14 of the start): its step lengths stay 0
constexpr double kPcgStop = 1e-28;
void launch_pcg_dot(const double *a, const double *b, int n, int R, double *part, double *sc, int mode,
                    cudaStream_t s);
void launch_pcg_direction(const double *z, double *p, const double *sc, int n, int R, cudaStream_t s);
void launch_pcg_update(double *x, double *r, const double *p, const double *q, const double *sc, int n, int R,
                       cudaStream_t s);
// batches: per-mesh dot products over the finest-level work items
void launch_item_dot2(const int *items, int nitems, const double *a, const double *b, const double *c,
                      const double *d, int R, double *part, cudaStream_t s);
void launch_inst_sum(const int *istart, int ninst, const double *part, double *out, int ostride, cudaStream_t s);
void launch_inst_pcg_scalar(const int *istart, int ninst, int R, const double *part, double *sc, int mode,
                            const double *norms, const double *tol, cudaStream_t s);
void launch_inst_pcg_direction(const double *z, double *p, const double *sc, const int *row_inst, int n, int R,
                               cudaStream_t s);
void launch_inst_pcg_update(double *x, double *r, const double *p, const double *q, const double *sc,
                            const int *row_inst, int n, int R, cudaStream_t s);
void launch_pack(const double *user, int n, int nrhs, int R, double *v, cudaStream_t s, const int *perm = nullptr);
void launch_unpack(const double *v, int n, int nrhs, int R, double *user, cudaStream_t s, const int *perm = nullptr);
void launch_to_float(const double *a, float *b, int64_t n, cudaStream_t s, float *zero = nullptr, Chain *ch = nullptr);
void launch_add_float(double *x, const float *e, int64_t n, cudaStream_t s, Chain *ch = nullptr);
void launch_add_double(double *x, const double *e, int64_t n, cudaStream_t s);

}  // namespace lbmg
