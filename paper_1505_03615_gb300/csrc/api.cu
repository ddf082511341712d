// api.cu -- C ABI of the library (declared in include/lbmg.h): handle lifetime,
// device upload of the hierarchy, assembly, V-cycles and the defect-correction
// solve loop (Chuang & Kazhdan, Sections 4.3 and 5).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "../../include/lbmg.h"
#include "lbmg_internal.h"

using namespace lbmg;

namespace {

thread_local std::string g_cuda_err;

#define LBMG_CK(call)                                                                 \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            g_cuda_err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return e_ == cudaErrorMemoryAllocation ? LBMG_OUT_OF_MEMORY : LBMG_CUDA_ERROR; \
        }                                                                             \
    } while (0)

#define LBMG_TRY(expr)          \
    do {                        \
        int st_ = (expr);       \
        if (st_) return st_;    \
    } while (0)

int check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_cuda_err = std::string("kernel launch: ") + cudaGetErrorString(e);
        return LBMG_CUDA_ERROR;
    }
    return LBMG_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int stride_for(int nrhs) { return nrhs == 1 ? 1 : (nrhs == 2 ? 2 : 4); }

__global__ void to_double_kernel(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) b[q] = (double)a[q];
}

// ---- stopping test of a solve on the device (one graph launch per solve) ----
// relative residual from squared norms, the rule every solve path uses: non-finite norms
// give infinity (never convergence); a zero right-hand side is judged by the absolute
// residual ||r||, so a warm start on b = 0 still iterates towards x = 0
__device__ __forceinline__ double ctl_rel(double r2, double b2) {
    if (!isfinite(r2) || !isfinite(b2)) return __longlong_as_double(0x7ff0000000000000ll);
    return sqrt(r2 / (b2 > 0.0 ? b2 : 1.0));
}

__global__ void ctl_setup_kernel(SolveCtl *ctl, double tol, int max_cycles, int fixed, int nrhs, double *pcg_tol) {
    if (threadIdx.x != 0) return;
    ctl->tol = tol;
    ctl->max_cycles = max_cycles;
    ctl->cycles = 0;
    ctl->status = kCtlRunning;
    ctl->fixed = fixed;
    ctl->nrhs = nrhs;
    ctl->learned_off = 0;
    if (pcg_tol) *pcg_tol = tol;
}

// worst relative residual per lane: one mesh (nr: ||r||^2, ctl->nb: ||b||^2) or a batch
// (inst: per mesh ||r||^2 at [16 m + q] and ||b||^2 at [16 m + 4 + q])
__device__ void ctl_worst(const SolveCtl &c, const double *nr, const double *inst, int ninst, double (&rel)[4]) {
    for (int q = 0; q < 4; q++) rel[q] = 0.0;
    if (inst) {
        for (int m = 0; m < ninst; m++)
            for (int q = 0; q < c.nrhs; q++) rel[q] = fmax(rel[q], ctl_rel(inst[16 * m + q], inst[16 * m + 4 + q]));
    } else {
        for (int q = 0; q < c.nrhs; q++) rel[q] = ctl_rel(nr[q], c.nb[q]);
    }
}

// status after a check: device timeout (a bounded wait gave up), failed coarse factor,
// divergence (non-finite, or growth by 1e6 over the initial residual), convergence of
// every lane, or the iteration cap; the loop continues only while running
__device__ void ctl_decide(SolveCtl &c, const double (&rel)[4], const int *tstat, const int *cflag,
                           cudaGraphConditionalHandle h) {
    bool conv = true, bad = false;
    for (int q = 0; q < c.nrhs; q++) {
        c.rel[q] = rel[q];
        if (!(rel[q] <= c.tol)) conv = false;
        if (!isfinite(rel[q]) || rel[q] > 1e6 * fmax(c.r0[q], 1e-300)) bad = true;
    }
    int st = kCtlRunning;
    if (*tstat != 0) st = kCtlTimeout;
    else if (*cflag != 0) st = kCtlCoarse;
    else if (!c.fixed && bad) st = kCtlDiverged;
    else if (!c.fixed && conv) st = kCtlConverged;
    else if (c.cycles >= c.max_cycles) st = kCtlMaxCycles;
    c.status = st;
    cudaGraphSetConditional(h, st == kCtlRunning ? 1u : 0u);
}

__global__ void ctl_begin_kernel(SolveCtl *ctl, const double *nb, const double *nr, const double *inst, int ninst,
                                 const int *tstat, const int *cflag, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    SolveCtl &c = *ctl;
    if (!inst)
        for (int q = 0; q < 4; q++) c.nb[q] = nb[q];
    double rel[4];
    ctl_worst(c, nr, inst, ninst, rel);
    for (int q = 0; q < 4; q++) c.r0[q] = rel[q];
    ctl_decide(c, rel, tstat, cflag, h);
}

__global__ void ctl_step_kernel(SolveCtl *ctl, const double *nr, const double *inst, int ninst, const int *tstat,
                                const int *cflag, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    SolveCtl &c = *ctl;
    c.cycles++;
    double rel[4];
    ctl_worst(c, nr, inst, ninst, rel);
    // acceptance test of the learned correction: a residual that grew drops it for good
    for (int q = 0; q < c.nrhs; q++)
        if (rel[q] > c.rel[q]) c.learned_off = 1;
    ctl_decide(c, rel, tstat, cflag, h);
}

}  // namespace

struct lbmg_ctx {
    Ctx c;
    std::vector<void *> allocs;
    const int **lev_rp = nullptr, **lev_ci = nullptr;   // device arrays of per-level pointers
    const double **lev_A = nullptr;
    std::vector<double> inst_norm_host;                 // last solve: [ninst][12]
    size_t io_cap = 0;   // doubles per io slot
    int *h_flag = nullptr;
    double pcg_tol_host = 0.0;   // source of the tolerance copy of a running batch solve
    int syncs = 0;               // host synchronizations of the running solve
    double *h_inst = nullptr;    // pinned [ninst][16]: per-mesh norms read after a solve

    template <class T>
    int alloc(T **p, size_t count) {
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
        if (e != cudaSuccess) {
            g_cuda_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            cudaGetLastError();
            *p = nullptr;
            return LBMG_OUT_OF_MEMORY;
        }
        allocs.push_back((void *)*p);
        return LBMG_OK;
    }
    template <class T>
    int upload(T **p, const std::vector<T> &v) {
        LBMG_TRY(alloc(p, v.size()));
        if (!v.empty()) LBMG_CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return LBMG_OK;
    }
    ~lbmg_ctx() {
        if (c.graph.exec) cudaGraphExecDestroy(c.graph.exec);
        for (void *p : allocs) cudaFree(p);
        if (c.h_norm) cudaFreeHost(c.h_norm);
        if (h_flag) cudaFreeHost(h_flag);
        if (c.h_state) cudaFreeHost(c.h_state);
        if (c.h_ctl) cudaFreeHost(c.h_ctl);
        if (h_inst) cudaFreeHost(h_inst);
        if (c.capture_stream) cudaStreamDestroy(c.capture_stream);
        if (c.ev0) cudaEventDestroy(c.ev0);
        if (c.ev1) cudaEventDestroy(c.ev1);
        learned_free(c);
        if (c.narrow.blob) cudaFree(c.narrow.blob);
        for (int q = 0; q < 4; q++) if (c.ev_smooth[q]) cudaEventDestroy(c.ev_smooth[q]);
    }
};

namespace {

// device pointer for a user input: copies host data into io slot `slot`
int input_ptr(lbmg_handle h, const double *user, size_t count, int slot, cudaStream_t s, const double **out) {
    if (on_device(user)) { *out = user; return LBMG_OK; }
    if (count > h->io_cap) return LBMG_INVALID_ARG;
    double *dst = h->c.dev_io + (size_t)slot * h->io_cap;
    LBMG_CK(cudaMemcpyAsync(dst, user, count * sizeof(double), cudaMemcpyHostToDevice, s));
    *out = dst;
    return LBMG_OK;
}

// device pointer for a user output; *host tells whether finish_output must copy back
int output_ptr(lbmg_handle h, double *user, size_t count, int slot, double **out, bool *host) {
    if (on_device(user)) { *out = user; *host = false; return LBMG_OK; }
    if (count > h->io_cap) return LBMG_INVALID_ARG;
    *out = h->c.dev_io + (size_t)slot * h->io_cap;
    *host = true;
    return LBMG_OK;
}

int finish_output(double *user, const double *dev, size_t count, bool host, cudaStream_t s, int *syncs = nullptr) {
    if (host) {
        LBMG_CK(cudaMemcpyAsync(user, dev, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        LBMG_CK(cudaStreamSynchronize(s));
        if (syncs) (*syncs)++;
    }
    return check_launch();
}

template <class T> struct P;
template <> struct P<float> {
    static float *x(DevLevel &L) { return L.x32; }
    static float *b(DevLevel &L) { return L.b32; }
    static float *r(DevLevel &L) { return L.r32; }
    static const float *A(DevLevel &L) { return L.A32; }
    static const float *dinv(DevLevel &L) { return L.dinv32; }
    static const float *inv(Ctx &c) { return c.cinv32; }
};
template <> struct P<double> {
    static double *x(DevLevel &L) { return L.x64; }
    static double *b(DevLevel &L) { return L.b64; }
    static double *r(DevLevel &L) { return L.r64; }
    static const double *A(DevLevel &L) { return L.A64; }
    static const double *dinv(DevLevel &L) { return L.dinv64; }
    static const double *inv(Ctx &c) { return c.cinv64; }
};

template <class T>
void enqueue_smooth(Ctx &c, DevLevel &L, int R, int sweeps, bool forward, cudaStream_t s, Chain *ch, int skip = 0) {
    if (c.smoother == LBMG_JACOBI) {
        for (int sw = 0; sw < sweeps; sw++) {
            launch_residual<T>(L, P<T>::A(L), P<T>::b(L), P<T>::x(L), P<T>::r(L), R, s, L.ns, ch);
            launch_jacobi_update<T>(L, P<T>::dinv(L), P<T>::r(L), P<T>::x(L), (T)c.omega, R, s);
            if (ch) ch->cut();
        }
    } else {
        launch_sweeps<T>(c, L, sweeps, forward, P<T>::A(L), P<T>::dinv(L), P<T>::b(L), P<T>::x(L), R, s, ch, skip);
    }
}

// event record inside the cycle (an external event node when captured into a graph,
// which a plain record outside capture must not ask for); it ends the chain of
// dependent launches
inline void record(cudaEvent_t e, cudaStream_t s, Chain *ch) {
    if (ch->capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
    ch->cut();
}

// one V-cycle on A e = b at the finest level; e (finest x) must be zero on entry.
// Every coarser correction is zeroed by the restriction that fills its right-hand
// side, so the kernels of the cycle follow one another with no memset between
// them and run as one chain of dependent launches.
template <class T>
void enqueue_vcycle(Ctx &c, int R, cudaStream_t s, bool timed, Chain *ch, int top = -1) {
    if (top < 0) top = c.D;
    // bottom levels: from shared memory in one block (FP32), from global memory in
    // one block (levels of at most narrow_max rows), or one launch per phase down to d0
    // (a single SM's FP64 rate makes the one-block bottom slower than per-phase launches)
    int dn = c.d0;
    enum { kPlain, kSmem, kL2 } bottom = kPlain;
    if (sizeof(T) == 4 && c.smoother != LBMG_JACOBI) {
        if (c.narrow.dn >= c.d0 && c.narrow.dn <= top) { bottom = kSmem; dn = c.narrow.dn; }
        else if (std::min(c.persist_dn, top) >= c.d0) { bottom = kL2; dn = std::min(c.persist_dn, top); }
    }
    int skip = 0;   // colour steps of the next level's first sweep that its restriction did
    for (int d = top; d > dn; d--) {
        DevLevel &L = c.lev[d], &Lc = c.lev[d - 1];
        launch_coarse_apply<T>(c, L, P<T>::inv(c), P<T>::b(L), P<T>::x(L), R, s, ch);
        if (timed && d == top) record(c.ev_smooth[0], s, ch);
        enqueue_smooth<T>(c, L, R, c.nu1, true, s, ch, skip);
        if (timed && d == top) record(c.ev_smooth[1], s, ch);
        launch_residual<T>(L, P<T>::A(L), P<T>::b(L), P<T>::x(L), P<T>::r(L), R, s, L.ns, ch);
        // the shared-memory bottom starts level dn from zero itself; the dense solve overwrites d0
        const bool zero = bottom == kSmem ? d - 1 > dn : (bottom == kL2 || d - 1 > c.d0);
        // a level that this loop smooths next (Gauss-Seidel, from zero) gets its first colour step
        // from the restriction that zeroes it
        const bool fuse = zero && d - 1 > dn && c.smoother != LBMG_JACOBI && c.nu1 > 0;
        launch_restrict<T>(Lc, P<T>::r(L), P<T>::b(Lc), R, s, zero ? P<T>::x(Lc) : (T *)nullptr, ch, fuse);
        skip = fuse ? 1 : 0;
    }
    if (bottom == kSmem) launch_narrow_smem(c, R, s, ch);
    else if (bottom == kL2) { launch_narrow_cycle(c, 1, R, dn, s); ch->cut(); }
    else {
        DevLevel &L0 = c.lev[c.d0];
        launch_coarse_apply<T>(c, L0, P<T>::inv(c), P<T>::b(L0), P<T>::x(L0), R, s, ch);
    }
    for (int d = dn + 1; d <= top; d++) {
        DevLevel &L = c.lev[d];
        launch_prolong_add<T>(L, P<T>::x(c.lev[d - 1]), P<T>::x(L), R, s, ch);
        if (timed && d == top) record(c.ev_smooth[2], s, ch);
        enqueue_smooth<T>(c, L, R, c.nu2, false, s, ch);
        if (timed && d == top) record(c.ev_smooth[3], s, ch);
    }
}

// The general multigrid cycle of Section 4.3, level by level: nu1 sweeps, residual,
// restriction (which zeroes the coarse correction), gamma visits of the next coarser level
// (gamma = 2: the W-cycle of the convergence experiment of Section 5.2), prolongation and nu2
// sweeps in the reverse colour order.  The coarsest level is solved by the dense factor, or
// (coarse_smooth) relaxed by nu1 + nu2 sweeps like the others.  Used for the W-cycle and for
// the relaxed coarsest level; the plain V-cycle with a solved coarsest level takes
// enqueue_vcycle and its one-block bottom.
template <class T>
void enqueue_cycle_level(Ctx &c, int d, int R, cudaStream_t s, Chain *ch) {
    DevLevel &L = c.lev[d];
    if (d == c.d0) {
        if (c.coarse_smooth) {
            DevLevel L0 = L;   // the coarsest level's rows, smoothed by colour like any level
            for (int q = 0; q < 9; q++) L0.cs[q] = L0.cs_all[q];
            L0.ns = L0.n;
            enqueue_smooth<T>(c, L0, R, c.nu1, true, s, ch);
            enqueue_smooth<T>(c, L0, R, c.nu2, false, s, ch);
        } else {
            launch_coarse_apply<T>(c, L, P<T>::inv(c), P<T>::b(L), P<T>::x(L), R, s, ch);
        }
        return;
    }
    DevLevel &Lc = c.lev[d - 1];
    enqueue_smooth<T>(c, L, R, c.nu1, true, s, ch);
    launch_residual<T>(L, P<T>::A(L), P<T>::b(L), P<T>::x(L), P<T>::r(L), R, s, L.ns, ch);
    launch_restrict<T>(Lc, P<T>::r(L), P<T>::b(Lc), R, s, P<T>::x(Lc), ch);
    for (int g = 0; g < c.gamma; g++) enqueue_cycle_level<T>(c, d - 1, R, s, ch);
    launch_prolong_add<T>(L, P<T>::x(Lc), P<T>::x(L), R, s, ch);
    enqueue_smooth<T>(c, L, R, c.nu2, false, s, ch);
}

// one cycle on A e = b at the finest level, e zero on entry
template <class T>
void enqueue_cycle(Ctx &c, int R, cudaStream_t s, bool timed, Chain *ch) {
    if (c.gamma == 1 && !c.coarse_smooth) enqueue_vcycle<T>(c, R, s, timed, ch);
    else enqueue_cycle_level<T>(c, c.D, R, s, ch);
}

Chain make_chain(const Ctx &c, cudaStream_t s) {
    Chain ch;
    // the legacy and per-thread default streams take no programmatic serialization
    ch.on = c.pdl != 0 && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ch.capturing = cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusActive;
    return ch;
}

// the mixed V-cycle iteration keeps its iterate as an FP32 pair (c.xs_hi + c.xs_lo, updated by
// an FP32 two-sum) and forms the outer residual from it; c.xs holds it in FP64 only before and
// after the solve (split at the start, joined at the end)
inline bool pair_iterate(const Ctx &c, int precision, bool pcg) {
    return precision == LBMG_MIXED && !pcg && c.lev[c.D].pk_v2 != nullptr;
}

// one defect-correction step: x += Vcycle(r); r = b - A x; norms(r)
// timed: events around the finest smoothing (not inside the body of a conditional node)
void enqueue_iteration(Ctx &c, int R, int precision, cudaStream_t s, bool timed = true) {
    DevLevel &F = c.lev[c.D];
    const int64_t m = (int64_t)F.n * R;
    Chain ch = make_chain(c, s);
    if (precision == LBMG_MIXED) {
        if (c.learned_on) learned_enqueue(c, R, precision, s, &ch);   // the cycle starts from the correction
        else launch_to_float(c.rs, F.b32, m, s, F.x32, &ch);
        enqueue_cycle<float>(c, R, s, timed, &ch);
        // x += e, and the outer residual with FP64 values carried as FP32 pairs (GB300's FP64
        // rate would bound an FP64 residual of the finest level)
        if (pair_iterate(c, precision, false)) {
            launch_add_pair(F.x32, c.xs_hi, c.xs_lo, m, s, &ch);
            launch_packed_residual_split(F, c.bs, c.xs_hi, c.xs_lo, c.rs, R, s, &ch);
            launch_norms(c.rs, F.n, R, c.norm_part, c.norm_out, s, &ch);
            return;
        }
        launch_add_float(c.xs, F.x32, m, s, &ch);
    } else {
        if (c.learned_on) {
            learned_enqueue(c, R, precision, s, &ch);
        } else {
            cudaMemcpyAsync(F.b64, c.rs, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
            cudaMemsetAsync(F.x64, 0, m * sizeof(double), s);
        }
        enqueue_cycle<double>(c, R, s, timed, &ch);
        launch_add_double(c.xs, F.x64, m, s);
        ch.cut();
    }
    launch_residual<double>(F, F.A64, c.bs, c.xs, c.rs, R, s, -1, &ch);
    launch_norms(c.rs, F.n, R, c.norm_part, c.norm_out, s, &ch);
}

// q = -A p of a CG step: in mixed precision with p's FP64 values carried as FP32 pairs
// (the product of the outer residual), else in FP64
void enqueue_pcg_product(Ctx &c, DevLevel &F, int R, int precision, int64_t m, cudaStream_t s) {
    if (precision == LBMG_MIXED && F.pk_v2) {
        launch_split(c.pcg_p, c.xs_hi, c.xs_lo, m, s);
        if (launch_packed_residual_split(F, c.pcg_zero, c.xs_hi, c.xs_lo, c.pcg_q, R, s, nullptr)) return;
    }
    launch_residual<double>(F, F.A64, c.pcg_zero, c.pcg_p, c.pcg_q, R, s);
}

// one step of conjugate gradients preconditioned by the V-cycle, in the flexible
// (Polak-Ribiere) form, each right-hand side lane with its own step lengths:
//   s2 = r.z_old;  z = Vcycle(r);  s1 = r.z;  beta = (s1 - s2) / rz;  rz = s1;
//   p = z + beta p;  q = -A p;  alpha = s1 / (p.A p);  x += alpha p;  r -= alpha A p;  norms(r)
void enqueue_pcg_iteration(Ctx &c, int R, int precision, cudaStream_t s, bool timed = true) {
    DevLevel &F = c.lev[c.D];
    const int64_t m = (int64_t)F.n * R;
    launch_pcg_dot(c.rs, c.pcg_z, F.n, R, c.pcg_part, c.pcg_s, 0, s);
    Chain ch = make_chain(c, s);
    if (precision == LBMG_MIXED) {
        launch_to_float(c.rs, F.b32, m, s, F.x32, &ch);
        enqueue_cycle<float>(c, R, s, timed, &ch);
        to_double_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(F.x32, c.pcg_z, m);
    } else {
        cudaMemcpyAsync(F.b64, c.rs, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(F.x64, 0, m * sizeof(double), s);
        enqueue_cycle<double>(c, R, s, timed, &ch);
        cudaMemcpyAsync(c.pcg_z, F.x64, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
    launch_pcg_dot(c.rs, c.pcg_z, F.n, R, c.pcg_part, c.pcg_s, 1, s);
    launch_pcg_direction(c.pcg_z, c.pcg_p, c.pcg_s, F.n, R, s);
    enqueue_pcg_product(c, F, R, precision, m, s);
    launch_pcg_dot(c.pcg_p, c.pcg_q, F.n, R, c.pcg_part, c.pcg_s, 2, s);
    launch_pcg_update(c.xs, c.rs, c.pcg_p, c.pcg_q, c.pcg_s, F.n, R, s);
    launch_norms(c.rs, F.n, R, c.norm_part, c.norm_out, s);
}

// the same step for a batch: every mesh has its own step lengths (per-mesh dot products
// over the finest-level work items), and the per-mesh norms of r and b end the step
void enqueue_pcg_batch_iteration(Ctx &c, int R, int precision, cudaStream_t s) {
    DevLevel &F = c.lev[c.D];
    const int64_t m = (int64_t)F.n * R;
    launch_item_dot2(c.nitem, c.nnitem, c.rs, c.pcg_z, nullptr, nullptr, R, c.item_part, s);
    launch_inst_pcg_scalar(c.item_start, c.ninst, R, c.item_part, c.pcg_si, 0, c.inst_norm, c.pcg_tol, s);
    Chain ch = make_chain(c, s);
    if (precision == LBMG_MIXED) {
        launch_to_float(c.rs, F.b32, m, s, F.x32, &ch);
        enqueue_vcycle<float>(c, R, s, false, &ch);
        to_double_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(F.x32, c.pcg_z, m);
    } else {
        cudaMemcpyAsync(F.b64, c.rs, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(F.x64, 0, m * sizeof(double), s);
        enqueue_vcycle<double>(c, R, s, false, &ch);
        cudaMemcpyAsync(c.pcg_z, F.x64, m * sizeof(double), cudaMemcpyDeviceToDevice, s);
    }
    launch_item_dot2(c.nitem, c.nnitem, c.rs, c.pcg_z, nullptr, nullptr, R, c.item_part, s);
    launch_inst_pcg_scalar(c.item_start, c.ninst, R, c.item_part, c.pcg_si, 1, c.inst_norm, c.pcg_tol, s);
    launch_inst_pcg_direction(c.pcg_z, c.pcg_p, c.pcg_si, c.row_inst, F.n, R, s);
    enqueue_pcg_product(c, F, R, precision, m, s);
    launch_item_dot2(c.nitem, c.nnitem, c.pcg_p, c.pcg_q, nullptr, nullptr, R, c.item_part, s);
    launch_inst_pcg_scalar(c.item_start, c.ninst, R, c.item_part, c.pcg_si, 2, c.inst_norm, c.pcg_tol, s);
    launch_inst_pcg_update(c.xs, c.rs, c.pcg_p, c.pcg_q, c.pcg_si, c.row_inst, F.n, R, s);
    launch_item_dot2(c.nitem, c.nnitem, c.rs, c.rs, c.bs, c.bs, R, c.item_part, s);
    launch_inst_sum(c.item_start, c.ninst, c.item_part, c.inst_norm, 16, s);
}

int get_graph(lbmg_handle h, int R, int precision, bool pcg, cudaGraphExec_t *out) {
    Ctx &c = h->c;
    GraphCache &g = c.graph;
    if (g.exec && g.R == R && g.precision == precision && g.nu1 == c.nu1 && g.nu2 == c.nu2 && g.smoother == c.smoother &&
        g.pcg == (int)pcg && g.cond == 0 && g.learned == c.learned_on) {
        *out = g.exec;
        return LBMG_OK;
    }
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    LBMG_CK(cudaStreamBeginCapture(c.capture_stream, cudaStreamCaptureModeThreadLocal));
    if (pcg && c.ninst > 1) enqueue_pcg_batch_iteration(c, R, precision, c.capture_stream);
    else if (pcg) enqueue_pcg_iteration(c, R, precision, c.capture_stream);
    else enqueue_iteration(c, R, precision, c.capture_stream);
    cudaGraph_t graph = nullptr;
    LBMG_CK(cudaStreamEndCapture(c.capture_stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g_cuda_err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        g.exec = nullptr;
        return LBMG_CUDA_ERROR;
    }
    g.R = R; g.precision = precision; g.nu1 = c.nu1; g.nu2 = c.nu2; g.smoother = c.smoother; g.pcg = pcg;
    g.cond = 0;
    g.learned = c.learned_on;
    *out = g.exec;
    return LBMG_OK;
}

// The whole solve as one graph: a check of the initial residual, then a conditional WHILE
// node whose body is one iteration (V-cycle step, or CG step preconditioned by one V-cycle)
// and the check kernel that sets the loop condition.  The parameters (tolerance, cycle
// cap) and the initial norms are written by ordinary launches before each graph launch.
int build_cond_graph(Ctx &c, int R, int precision, bool pcg, cudaGraphExec_t *out) {
    cudaStream_t cs = c.capture_stream;
    const bool batch = c.ninst > 1;
    cudaGraph_t g = nullptr;
    LBMG_CK(cudaGraphCreate(&g, 0));
    // on an error return: end a capture still open into the graph or its body, then free the graph
    struct GraphGuard {
        cudaGraph_t g;
        cudaStream_t cs;
        ~GraphGuard() {
            cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(cs, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
                cudaGraph_t part = nullptr;   // the captured-to graph itself: owned by g
                cudaStreamEndCapture(cs, &part);
            }
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
        }
    } guard{g, cs};
    cudaGraphConditionalHandle hc;
    LBMG_CK(cudaGraphConditionalHandleCreate(&hc, g, 0, cudaGraphCondAssignDefault));
    LBMG_CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctl_begin_kernel<<<1, 32, 0, cs>>>(c.ctl, c.norm_b, c.norm_out, batch ? c.inst_norm : nullptr, c.ninst,
                                       c.narrow.status, c.flag, hc);
    cudaGraph_t gc = nullptr;
    LBMG_CK(cudaStreamEndCapture(cs, &gc));
    cudaGraphNode_t begin = nullptr;
    size_t nn = 1;
    LBMG_CK(cudaGraphGetNodes(g, &begin, &nn));
    if (nn != 1) return LBMG_CUDA_ERROR;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    LBMG_CK(cudaGraphAddNode(&loop, g, &begin, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    LBMG_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (pcg && batch) enqueue_pcg_batch_iteration(c, R, precision, cs);
    else if (pcg) enqueue_pcg_iteration(c, R, precision, cs, false);
    else enqueue_iteration(c, R, precision, cs, false);
    ctl_step_kernel<<<1, 32, 0, cs>>>(c.ctl, c.norm_out, batch ? c.inst_norm : nullptr, c.ninst, c.narrow.status,
                                      c.flag, hc);
    cudaGraph_t bc = nullptr;
    LBMG_CK(cudaStreamEndCapture(cs, &bc));
    LBMG_CK(cudaGraphInstantiate(out, g, 0));
    return LBMG_OK;
}

int get_cond_graph(lbmg_handle h, int R, int precision, bool pcg, cudaGraphExec_t *out) {
    Ctx &c = h->c;
    GraphCache &g = c.graph;
    if (g.exec && g.R == R && g.precision == precision && g.nu1 == c.nu1 && g.nu2 == c.nu2 && g.smoother == c.smoother &&
        g.pcg == (int)pcg && g.cond == 1 && g.learned == c.learned_on) {
        *out = g.exec;
        return LBMG_OK;
    }
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    int e = build_cond_graph(c, R, precision, pcg, &g.exec);
    if (e != LBMG_OK) {
        // (the builder has ended any capture it left open)
        cudaGetLastError();
        g.exec = nullptr;
        return e;
    }
    g.R = R; g.precision = precision; g.nu1 = c.nu1; g.nu2 = c.nu2; g.smoother = c.smoother; g.pcg = pcg;
    g.cond = 1;
    g.learned = c.learned_on;
    *out = g.exec;
    return LBMG_OK;
}

int read_norms(lbmg_handle h, int R, cudaStream_t s, double *out4) {
    // four norms, then the bottom kernel's status word
    LBMG_CK(cudaMemcpyAsync(h->c.h_norm, h->c.norm_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LBMG_CK(cudaStreamSynchronize(s));
    h->syncs++;
    for (int r = 0; r < 4; r++) out4[r] = r < R ? h->c.h_norm[r] : 0.0;
    int st = 0;
    std::memcpy(&st, &h->c.h_norm[4], sizeof st);
    if (st != 0) {
        // a bounded wait in the bottom kernel gave up: the cycle's result is invalid
        LBMG_CK(cudaMemsetAsync(h->c.norm_out + 4, 0, sizeof(double), s));
        return LBMG_DEVICE_TIMEOUT;
    }
    return LBMG_OK;
}

int check_level(lbmg_handle h, int d) {
    if (!h) return LBMG_INVALID_ARG;
    if (d < h->c.d0 || d > h->c.D) return LBMG_INVALID_ARG;
    return LBMG_OK;
}

int upload_hierarchy(lbmg_handle h) {
    Ctx &c = h->c;
    HostHierarchy &H = c.host;
    c.D = H.D; c.d0 = H.d0; c.nv = H.nv; c.nt = H.nt; c.nfrag = H.nfrag;
    c.ninst = H.ninst;
    c.nu = (int)H.fperm.size();
    // coarsest blocks, sorted by level
    c.cblk_host.clear();
    c.n0max = 0;
    int64_t inv_total = 0;
    for (int d = c.d0; d <= c.D; d++) {
        HostLevel &hl = H.lev[d];
        c.lev[d].cb0 = (int)(c.cblk_host.size() / 5);
        // a relaxed coarsest level has no dense block (and no size limit)
        c.lev[d].ncb = c.coarse_smooth ? 0 : (int)(hl.coarse.size() / 3);
        for (size_t q = 0; q < hl.coarse.size() && !c.coarse_smooth; q += 3) {
            const int n0 = hl.coarse[q + 2];
            if (n0 > kMaxCoarse) return LBMG_INVALID_ARG;
            c.cblk_host.insert(c.cblk_host.end(), {d, hl.coarse[q], hl.coarse[q + 1], n0, (int)inv_total});
            inv_total += (int64_t)n0 * n0;
            c.n0max = std::max(c.n0max, n0);
            if (inv_total > INT32_MAX) return LBMG_INVALID_ARG;
        }
    }
    c.ncblk = (int)(c.cblk_host.size() / 5);
    LBMG_TRY(h->upload(&c.cblk, c.cblk_host));
    for (int d = c.d0; d <= c.D; d++) {
        HostLevel &hl = H.lev[d];
        DevLevel &L = c.lev[d];
        L.d = d;
        L.n = hl.ndof;
        L.ns = hl.ns;
        L.nnz = hl.rp.empty() ? 0 : hl.rp[hl.ndof];
        for (int q = 0; q < 9; q++) L.cs[q] = hl.colour_start[q];
        for (int q = 0; q < 9; q++) L.cs_all[q] = hl.colour_all[q];
        LBMG_TRY(h->upload(&L.rp, hl.rp));
        LBMG_TRY(h->upload(&L.ci, hl.ci));
        LBMG_TRY(h->alloc(&L.M, L.nnz));
        LBMG_TRY(h->alloc(&L.L, L.nnz));
        LBMG_TRY(h->alloc(&L.A64, L.nnz));
        LBMG_TRY(h->alloc(&L.A32, L.nnz));
        LBMG_TRY(h->alloc(&L.dinv64, L.n));
        LBMG_TRY(h->alloc(&L.dinv32, L.n));
        if (!hl.par.empty()) {
            LBMG_TRY(h->upload(&L.par, hl.par));
            LBMG_TRY(h->upload(&L.npl2, hl.npar_log2));
        }
        if (d < c.D) {
            LBMG_TRY(h->upload(&L.crp, hl.crp));
            LBMG_TRY(h->upload(&L.cch, hl.cch));
            LBMG_TRY(h->upload(&L.grp, hl.grp));
            LBMG_TRY(h->upload(&L.gidx, hl.gidx));
        }
        if (d > c.d0 && L.nnz > 0) {
            // packed copy of A for the smoothing and residual kernels (packed.cu)
            std::vector<int32_t> gq, rows, map, col;
            if (packed_layout(hl, gq, rows, map, col, L.pk_gs, &L.pk_total)) {
                std::vector<int2> gq2(gq.size() / 2);
                for (size_t g = 0; g < gq2.size(); g++) gq2[g] = make_int2(gq[2 * g], gq[2 * g + 1]);
                for (int q = 0; q < 10; q++)
                    L.pk_es[q] = L.pk_gs[q] < (int)gq2.size() ? (int64_t)(unsigned)gq2[L.pk_gs[q]].x * 32 : L.pk_total;
                for (int col = 0; col < 8; col++) {
                    PkRuns &pr = L.pk_runs[col];
                    pr = PkRuns();
                    for (int g = L.pk_gs[col]; g < L.pk_gs[col + 1]; g++) {
                        if (pr.n > 0 && gq2[g].y == pr.q[pr.n - 1] &&
                            gq2[g].x == pr.b[pr.n - 1] + (g - pr.g[pr.n - 1]) * pr.q[pr.n - 1])
                            continue;   // continues the run
                        if (pr.n == kPkRuns) { pr.n = -1; break; }
                        pr.g[pr.n] = g; pr.b[pr.n] = gq2[g].x; pr.q[pr.n] = gq2[g].y;
                        pr.n++;
                    }
                    if (pr.n < 0) pr = PkRuns();   // too many runs: the kernel reads the headers
                }
                LBMG_TRY(h->upload(&L.pk_gq, gq2));
                LBMG_TRY(h->upload(&L.pk_rows, rows));
                LBMG_TRY(h->upload(&L.pk_map, map));
                LBMG_TRY(h->upload(&L.pk_col, col));
                LBMG_TRY(h->alloc(&L.pk_e32, (size_t)L.pk_total));
                LBMG_TRY(h->alloc(&L.pk_v64, (size_t)L.pk_total));
                LBMG_TRY(h->alloc(&L.pk_v2, (size_t)L.pk_total));
            }
        }
        const size_t v4 = 4 * (size_t)L.n;
        LBMG_TRY(h->alloc(&L.x64, v4));
        LBMG_TRY(h->alloc(&L.b64, v4));
        LBMG_TRY(h->alloc(&L.r64, v4));
        LBMG_TRY(h->alloc(&L.x32, v4));
        LBMG_TRY(h->alloc(&L.b32, v4));
        LBMG_TRY(h->alloc(&L.r32, v4));
    }
    LBMG_TRY(h->upload(&c.poly, H.frag_poly));
    LBMG_TRY(h->upload(&c.pstart, H.frag_pstart));
    {
        // fragments by vertex count, so that the threads of a warp integrate equally many sub-triangles
        std::vector<int32_t> order(c.nfrag), cnt(64, 0);
        auto nv = [&](int f) { return std::min(63, (int)(H.frag_pstart[f + 1] - H.frag_pstart[f])); };
        for (int f = 0; f < c.nfrag; f++) cnt[nv(f)]++;
        for (int k = 1; k < 64; k++) cnt[k] += cnt[k - 1];
        for (int f = c.nfrag - 1; f >= 0; f--) order[--cnt[nv(f)]] = f;
        LBMG_TRY(h->upload(&c.forder, order));
    }
    LBMG_TRY(h->upload(&c.ftri, H.frag_tri));
    LBMG_TRY(h->upload(&c.fvox, H.frag_vox));
    LBMG_TRY(h->upload(&c.fdof, H.frag_dof));
    LBMG_TRY(h->upload(&c.tnormal, H.tri_normal));
    LBMG_TRY(h->upload(&c.Vg, H.Vg));
    LBMG_TRY(h->upload(&c.F, H.F));
    LBMG_TRY(h->upload(&c.arp, H.arp));
    LBMG_TRY(h->upload(&c.aidx, H.aidx));
    LBMG_TRY(h->upload(&c.rrp, H.rrp));
    LBMG_TRY(h->upload(&c.ridx, H.ridx));
    LBMG_TRY(h->upload(&c.frag_scale, H.frag_scale));
    LBMG_TRY(h->upload(&c.fperm, H.fperm));
    {
        std::vector<int32_t> inv(H.fperm.size()), vdu(H.vdof.size());
        for (size_t u = 0; u < H.fperm.size(); u++) inv[H.fperm[u]] = (int32_t)u;
        for (size_t q = 0; q < H.vdof.size(); q++) vdu[q] = H.vdof[q] >= 0 ? inv[H.vdof[q]] : -1;
        LBMG_TRY(h->upload(&c.fiperm, inv));
        LBMG_TRY(h->upload(&c.vdof, vdu));   // vertex evaluation reads user-ordered vectors
    }
    LBMG_TRY(h->upload(&c.vw, H.vw));
    // finest-level norm work items: chunks of each (colour, mesh) segment
    c.nitem_host.clear();
    for (int m = 0; m < c.ninst; m++)
        for (int q = 0; q < 8; q++) {
            const int s0 = H.seg[2 * (8 * m + q)], s1 = H.seg[2 * (8 * m + q) + 1];
            for (int r = s0; r < s1; r += 2048) c.nitem_host.insert(c.nitem_host.end(), {m, r, std::min(s1, r + 2048)});
        }
    c.nnitem = (int)(c.nitem_host.size() / 3);
    LBMG_TRY(h->upload(&c.nitem, c.nitem_host));
    {
        // the items are generated mesh by mesh: mesh m owns items [start[m], start[m + 1])
        std::vector<int32_t> start(c.ninst + 1, 0);
        for (int it = 0; it < c.nnitem; it++) start[c.nitem_host[3 * it] + 1]++;
        for (int m = 0; m < c.ninst; m++) start[m + 1] += start[m];
        LBMG_TRY(h->upload(&c.item_start, start));
        LBMG_TRY(h->upload(&c.row_inst, H.lev[H.D].inst));
        LBMG_TRY(h->alloc(&c.pcg_si, (size_t)kPcgScalars * c.ninst));
        LBMG_TRY(h->alloc(&c.pcg_tol, 1));
    }
    LBMG_TRY(h->alloc(&c.item_part, 8 * (size_t)std::max(c.nnitem, 1)));
    LBMG_TRY(h->alloc(&c.inst_norm, 16 * (size_t)c.ninst));
    {
        std::vector<const int *> rps(kMaxDepth + 1, nullptr), cis(kMaxDepth + 1, nullptr);
        std::vector<const double *> As(kMaxDepth + 1, nullptr);
        for (int d = c.d0; d <= c.D; d++) { rps[d] = c.lev[d].rp; cis[d] = c.lev[d].ci; As[d] = c.lev[d].A64; }
        LBMG_TRY(h->upload(&h->lev_rp, rps));
        LBMG_TRY(h->upload(&h->lev_ci, cis));
        LBMG_TRY(h->upload(&h->lev_A, As));
    }
    LBMG_TRY(h->alloc(&c.moments, 27 * (size_t)c.nfrag));
    LBMG_TRY(h->alloc(&c.stage, 72 * (size_t)c.nfrag));
    LBMG_TRY(h->alloc(&c.stage_rhs, 32 * (size_t)c.nfrag));
    LBMG_TRY(h->alloc(&c.cdense, (size_t)std::max<int64_t>(inv_total, 1)));
    LBMG_TRY(h->alloc(&c.cinv64, (size_t)std::max<int64_t>(inv_total, 1)));
    LBMG_TRY(h->alloc(&c.cinv32, (size_t)std::max<int64_t>(inv_total, 1)));
    LBMG_TRY(h->alloc(&c.flag, 1));
    const size_t nD = (size_t)c.lev[c.D].n;
    LBMG_TRY(h->alloc(&c.xs, 4 * nD));
    LBMG_TRY(h->alloc(&c.bs, 4 * nD));
    LBMG_TRY(h->alloc(&c.rs, 4 * nD));
    LBMG_TRY(h->alloc(&c.xs_hi, 4 * nD));
    LBMG_TRY(h->alloc(&c.xs_lo, 4 * nD));
    LBMG_TRY(h->alloc(&c.norm_part, 4 * (size_t)kNormBlocks));
    LBMG_TRY(h->alloc(&c.pcg_z, 4 * nD));
    LBMG_TRY(h->alloc(&c.pcg_p, 4 * nD));
    LBMG_TRY(h->alloc(&c.pcg_q, 4 * nD));
    LBMG_TRY(h->alloc(&c.pcg_zero, 4 * nD));
    LBMG_CK(cudaMemset(c.pcg_zero, 0, 4 * nD * sizeof(double)));
    LBMG_TRY(h->alloc(&c.pcg_s, (size_t)kPcgScalars));
    LBMG_TRY(h->alloc(&c.pcg_part, 4 * (size_t)kNormBlocks));
    LBMG_TRY(h->alloc(&c.diag_part, 256));
    LBMG_TRY(h->alloc(&c.norm_out, 8));
    LBMG_CK(cudaMemset(c.norm_out, 0, 8 * sizeof(double)));
    c.narrow.status = reinterpret_cast<int *>(c.norm_out + 4);
    LBMG_TRY(h->alloc(&c.sweep_bar, 1));
    for (int r : {1, 2, 4}) c.sweep_blocks[r] = packed_sweep_blocks(r);
    cudaGetLastError();
    h->io_cap = 4 * std::max(std::max(nD, (size_t)c.nv), (size_t)c.nu);
    LBMG_TRY(h->alloc(&c.dev_io, 2 * h->io_cap));
    LBMG_CK(cudaMallocHost((void **)&c.h_norm, 8 * sizeof(double)));
    LBMG_TRY(h->alloc((char **)&c.ctl, sizeof(SolveCtl)));
    LBMG_CK(cudaMemset(c.ctl, 0, sizeof(SolveCtl)));
    LBMG_CK(cudaMallocHost((void **)&c.h_ctl, sizeof(SolveCtl)));
    LBMG_TRY(h->alloc(&c.norm_b, 4));
    LBMG_CK(cudaMallocHost((void **)&h->h_inst, 16 * sizeof(double) * (size_t)c.ninst));
    LBMG_CK(cudaMallocHost((void **)&h->h_flag, sizeof(int)));
    LBMG_CK(cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking));
    LBMG_CK(cudaEventCreate(&c.ev0));
    LBMG_CK(cudaEventCreate(&c.ev1));
    for (int q = 0; q < 4; q++) LBMG_CK(cudaEventCreate(&c.ev_smooth[q]));
    c.persist_view_bytes = persist_view_bytes();
    LBMG_TRY(h->alloc((char **)&c.persist_views, c.persist_view_bytes));
    LBMG_TRY(h->alloc((char **)&c.persist_state, 64));
    LBMG_CK(cudaMallocHost(&c.h_state, 64 + 16 * sizeof(double)));
    // the one-launch solve and the one-block bottom cycles end in the coarsest level's dense
    // solve: a relaxed coarsest level runs the general cycle with neither
    c.persist_ok = !c.coarse_smooth && persist_setup(c) == 0 && c.persist_blocks <= 1024;
    cudaGetLastError();
    if (!c.persist_ok) {   // no narrow levels either: the persistent set-up also picks them
        c.persist_dn = c.d0 - 1;
        for (int d = c.d0; d <= c.D; d++) {
            if (c.lev[d].n <= c.persist_narrow) c.persist_dn = d; else break;
        }
    }
    LBMG_TRY(h->alloc((char **)&c.views32, c.persist_view_bytes));
    LBMG_TRY(h->alloc((char **)&c.views64, c.persist_view_bytes));
    if (c.coarse_smooth) {
        c.persist_dn = c.d0 - 1;
        c.narrow.dn = c.d0 - 1;
        return LBMG_OK;
    }
    if (narrow_views_setup(c) != 0) return LBMG_CUDA_ERROR;
    if (c.ninst == 1 && narrow_smem_setup(c, narrow_smem_budget()) != 0) {
        cudaGetLastError();
        c.narrow.dn = c.d0 - 1;   // the bottom then runs from global memory
    }
    return LBMG_OK;
}

}  // namespace

namespace lbmg {
void enqueue_vcycle64_from(Ctx &c, int top, int R, cudaStream_t s) {
    Chain ch;   // plain launches
    enqueue_vcycle<double>(c, R, s, false, &ch, top);
}

// level d of an assembled handle, for entry points defined in other files: LBMG_INVALID_ARG for
// a null handle or a level outside [min_depth, depth], LBMG_NOT_ASSEMBLED before lbmg_assemble,
// each with its reason in the error string
int noalloc_level(lbmg_handle h, int d, const DevLevel **out) {
    *out = nullptr;
    if (!h) { g_cuda_err = "null handle"; return LBMG_INVALID_ARG; }
    if (d < h->c.d0 || d > h->c.D) { g_cuda_err = "level outside [min_depth, depth]"; return LBMG_INVALID_ARG; }
    if (!h->c.assembled) { g_cuda_err = "the handle is not assembled (lbmg_assemble)"; return LBMG_NOT_ASSEMBLED; }
    *out = &h->c.lev[d];
    return LBMG_OK;
}
void noalloc_set_error(const std::string &msg) { g_cuda_err = msg; }

// relative residual sqrt(r2 / b2) from squared norms: a non-finite norm (NaN or inf in the
// right-hand side or the iterate) gives infinity, so it can never pass for convergence; a zero
// right-hand side is judged by the absolute residual sqrt(r2) (the rule of the device-side
// stopping test and of the persistent solve)
static double rel_residual(double r2, double b2) {
    if (!std::isfinite(r2) || !std::isfinite(b2)) return INFINITY;
    return std::sqrt(r2 / (b2 > 0 ? b2 : 1.0));
}

static int check_build_options(const lbmg_options &o) {
    if (o.host_check != 0 && o.host_check != 1) return LBMG_INVALID_ARG;
    if ((o.cycle != 0 && o.cycle != 1) || (o.coarse_smooth != 0 && o.coarse_smooth != 1)) return LBMG_INVALID_ARG;
    // the persistent solve runs the V-cycle with a solved coarsest level only
    if (o.persistent && (o.cycle != 0 || o.coarse_smooth != 0)) return LBMG_INVALID_ARG;
    if (o.nu1 < 0 || o.nu2 < 0 || o.coarse_max < 1 || o.coarse_max > kMaxCoarse) return LBMG_INVALID_ARG;
    if (o.smoother != LBMG_GS_COLOURED && o.smoother != LBMG_JACOBI) return LBMG_INVALID_ARG;
    if (o.narrow_max < 0 || o.barrier_phantoms < 0 || o.barrier_phantoms > 1024) return LBMG_INVALID_ARG;
    if (o.copy_phantom_bytes < 0 || o.copy_phantom_bytes > 65536) return LBMG_INVALID_ARG;
    if (o.host_alloc_fail != 0 && o.host_alloc_fail != 1) return LBMG_INVALID_ARG;
    if (o.gpu_clip != 0 && o.gpu_clip != 1) return LBMG_INVALID_ARG;
    return LBMG_OK;
}

// host hierarchy of one mesh in the layout the device handle uploads; on failure the
// reason goes to the thread's error string
static int build_single_host(const double *V, int nv, const int *F, int nt, int depth, const lbmg_options &o,
                      HostHierarchy &out) {
    std::string err;
    int st;
    try {
        std::vector<HostHierarchy> parts(1);
        st = build_host_hierarchy(V, nv, F, nt, depth, o.min_depth, o.coarse_max, o.split, o.threads, parts[0], err,
                                  o.host_alloc_fail != 0, o.gpu_clip != 0);
        if (st == 0) st = combine_batch(parts, out, err);
    } catch (const std::bad_alloc &) {
        st = LBMG_OUT_OF_MEMORY;
        err = "host memory exhausted";
    } catch (const BuildCudaError &e) {
        st = LBMG_CUDA_ERROR;
        err = e.what();
    } catch (const std::exception &e) {
        st = LBMG_INVALID_ARG;
        err = e.what();
    } catch (...) {
        st = LBMG_INVALID_ARG;
    }
    if (st != 0) g_cuda_err = "hierarchy build: " + err;
    return st;
}

static void copy_dofs(const HostLevel &L, int *corner, int *mintri) {
    if (corner) std::memcpy(corner, L.corner.data(), L.corner.size() * sizeof(int));
    if (mintri) std::memcpy(mintri, L.mintri.data(), L.mintri.size() * sizeof(int));
}

static void copy_pattern(const HostLevel &L, int *rowptr, int *col) {
    if (rowptr) std::memcpy(rowptr, L.rp.data(), L.rp.size() * sizeof(int));
    if (col) std::memcpy(col, L.ci.data(), L.ci.size() * sizeof(int));
}

static void copy_prolongation(const HostLevel &L, int *parents, double *weights) {
    for (int i = 0; i < L.ndof; i++) {
        const int np = 1 << L.npar_log2[i];
        for (int q = 0; q < 8; q++) {
            if (parents) parents[8 * (size_t)i + q] = q < np ? L.par[8 * (size_t)i + q] : -1;
            if (weights) weights[8 * (size_t)i + q] = q < np ? 1.0 / np : 0.0;
        }
    }
}

// host hierarchy of a batch in the layout the device handle uploads; on failure the reason
// goes to the thread's error string
static int build_batch_host(const double *const *V, const int *nv, const int *const *F, const int *nt,
                            const int *depth, int ninst, const lbmg_options &o, HostHierarchy &out) {
    std::string err;
    int st = 0;
    try {
        std::vector<HostHierarchy> parts(ninst);
        for (int i = 0; i < ninst && st == 0; i++)
            if (!V[i] || !F[i]) { st = LBMG_INVALID_ARG; err = "null mesh pointer"; }
        if (st == 0) {
            // Meshes are built concurrently, one per thread; the builder's own parallel loops
            // then run on that thread alone.  Each mesh's hierarchy is independent of the
            // schedule.
            std::vector<int> sti(ninst, 0);
            std::vector<std::string> erri(ninst);
#ifdef _OPENMP
            if (o.threads > 0) omp_set_num_threads(o.threads);
#endif
#pragma omp parallel for schedule(dynamic, 1)
            for (int i = 0; i < ninst; i++) {
                try {
                    sti[i] = build_host_hierarchy(V[i], nv[i], F[i], nt[i], depth[i], o.min_depth, o.coarse_max,
                                                  o.split, 0, parts[i], erri[i], o.host_alloc_fail != 0,
                                                  o.gpu_clip != 0);
                } catch (const std::bad_alloc &) {
                    sti[i] = LBMG_OUT_OF_MEMORY;
                    erri[i] = "host memory exhausted";
                } catch (const BuildCudaError &e) {
                    sti[i] = LBMG_CUDA_ERROR;
                    erri[i] = e.what();
                } catch (const std::exception &e) {
                    sti[i] = LBMG_INVALID_ARG;
                    erri[i] = e.what();
                } catch (...) {
                    sti[i] = LBMG_INVALID_ARG;
                }
            }
            for (int i = 0; i < ninst && st == 0; i++)
                if (sti[i] != 0) { st = sti[i]; err = "mesh " + std::to_string(i) + ": " + erri[i]; }
        }
        if (st == 0) st = combine_batch(parts, out, err);
    } catch (const std::bad_alloc &) {
        st = LBMG_OUT_OF_MEMORY;
        err = "host memory exhausted";
    } catch (const std::exception &e) {
        st = LBMG_INVALID_ARG;
        err = e.what();
    } catch (...) {
        st = LBMG_INVALID_ARG;
    }
    if (st != 0) g_cuda_err = "hierarchy build: " + err;
    return st;
}

static int check_batch_options(const lbmg_options &o) {
    if (o.nu1 < 0 || o.nu2 < 0 || o.coarse_max < 1 || o.coarse_max > kMaxCoarse) return LBMG_INVALID_ARG;
    if (o.smoother != LBMG_GS_COLOURED || o.narrow_max < 0 || o.barrier_phantoms < 0) return LBMG_INVALID_ARG;
    if (o.host_alloc_fail != 0 && o.host_alloc_fail != 1) return LBMG_INVALID_ARG;
    if (o.gpu_clip != 0 && o.gpu_clip != 1) return LBMG_INVALID_ARG;
    if (o.cycle != 0 || o.coarse_smooth != 0 || o.host_check < 0 || o.host_check > 1) return LBMG_INVALID_ARG;
    return LBMG_OK;
}

}  // namespace lbmg

// host-only hierarchy (no device memory)
struct lbmg_host_ctx {
    lbmg::HostHierarchy H;
};

extern "C" {

const char *lbmg_status_string(int code) {
    switch (code) {
        case LBMG_OK: return "ok";
        case LBMG_INVALID_ARG: return "invalid argument";
        case LBMG_DEGENERATE_MESH: return "degenerate mesh";
        case LBMG_OUT_OF_MEMORY: return "out of memory";
        case LBMG_NOT_CONVERGED: return "not converged";
        case LBMG_NOT_ASSEMBLED: return "not assembled";
        case LBMG_COARSE_FACTOR: return "coarse factorisation failed";
        case LBMG_CUDA_ERROR: return "CUDA error";
        case LBMG_DIVERGED: return "diverged";
        case LBMG_DEVICE_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char *lbmg_last_cuda_error(void) { return g_cuda_err.c_str(); }

void lbmg_default_options(lbmg_options *o) {
    if (!o) return;
    o->min_depth = -1;
    o->coarse_max = 160;
    o->nu1 = 2;
    o->nu2 = 2;
    o->smoother = LBMG_GS_COLOURED;
    o->jacobi_omega = 0.6;
    o->split = 1;
    o->threads = 0;
    o->persistent = 0;
    o->narrow_max = 2048;
    o->barrier_phantoms = 0;
    o->use_graphs = 1;
    o->pdl = 1;
    o->copy_phantom_bytes = 0;
    o->host_alloc_fail = 0;
    o->host_check = 0;
    o->cycle = 0;
    o->coarse_smooth = 0;
    o->gpu_clip = 0;
}

int lbmg_build_hierarchy(const double *V, int nv, const int *F, int nt, int depth, const lbmg_options *opt,
                         lbmg_handle *out) {
    if (!out || !V || !F) return LBMG_INVALID_ARG;
    *out = nullptr;
    lbmg_options o;
    lbmg_default_options(&o);
    if (opt) o = *opt;
    LBMG_TRY(check_build_options(o));
    lbmg_ctx *h = new (std::nothrow) lbmg_ctx();
    if (!h) return LBMG_OUT_OF_MEMORY;
    int st = build_single_host(V, nv, F, nt, depth, o, h->c.host);
    if (st != 0) {
        delete h;
        return st;
    }
    h->c.nu1 = o.nu1;
    h->c.nu2 = o.nu2;
    h->c.smoother = o.smoother;
    h->c.omega = o.jacobi_omega;
    h->c.persistent = o.persistent;
    h->c.use_graphs = o.use_graphs;
    h->c.pdl = o.pdl;
    h->c.copy_phantoms = o.copy_phantom_bytes;
    h->c.persist_narrow = o.narrow_max;
    h->c.barrier_phantoms = o.barrier_phantoms;
    h->c.host_check = o.host_check;
    h->c.gamma = o.cycle == 1 ? 2 : 1;
    h->c.coarse_smooth = o.coarse_smooth;
    st = upload_hierarchy(h);
    if (st != 0) { delete h; return st; }
    *out = h;
    return LBMG_OK;
}

int lbmg_build_batch(const double *const *V, const int *nv, const int *const *F, const int *nt, const int *depth,
                     int ninst, const lbmg_options *opt, lbmg_handle *out) {
    if (!out || !V || !nv || !F || !nt || !depth || ninst < 1) return LBMG_INVALID_ARG;
    *out = nullptr;
    lbmg_options o;
    lbmg_default_options(&o);
    if (opt) o = *opt;
    LBMG_TRY(check_batch_options(o));
    lbmg_ctx *h = new (std::nothrow) lbmg_ctx();
    if (!h) return LBMG_OUT_OF_MEMORY;
    int st = build_batch_host(V, nv, F, nt, depth, ninst, o, h->c.host);
    if (st != 0) {
        delete h;
        return st;
    }
    h->c.nu1 = o.nu1; h->c.nu2 = o.nu2; h->c.smoother = o.smoother; h->c.omega = o.jacobi_omega;
    h->c.persistent = 1; h->c.persist_narrow = o.narrow_max; h->c.barrier_phantoms = o.barrier_phantoms;
    h->c.host_check = o.host_check;
    st = upload_hierarchy(h);
    if (st != 0) { delete h; return st; }
    if (!h->c.persist_ok) { delete h; return LBMG_CUDA_ERROR; }
    *out = h;
    return LBMG_OK;
}

int lbmg_instances(lbmg_handle h, int *ninst) {
    if (!h || !ninst) return LBMG_INVALID_ARG;
    *ninst = h->c.ninst;
    return LBMG_OK;
}

int lbmg_instance_info(lbmg_handle h, int inst, int *depth, int *min_depth, long *nfine, long *row_offset,
                       long *vertex_offset) {
    if (!h || inst < 0 || inst >= h->c.ninst) return LBMG_INVALID_ARG;
    const HostHierarchy &H = h->c.host;
    if (depth) *depth = H.inst_D[inst];
    if (min_depth) *min_depth = H.inst_d0[inst];
    if (nfine) *nfine = H.inst_nfine[inst];
    if (row_offset) *row_offset = H.inst_uoff[inst];
    if (vertex_offset) *vertex_offset = H.inst_voff[inst];
    return LBMG_OK;
}

int lbmg_row_instances(lbmg_handle h, int d, int *inst) {
    LBMG_TRY(check_level(h, d));
    if (!inst) return LBMG_INVALID_ARG;
    const HostLevel &hl = h->c.host.lev[d];
    for (int i = 0; i < hl.ndof; i++) inst[i] = hl.inst.empty() ? 0 : hl.inst[i];
    return LBMG_OK;
}

int lbmg_instance_residuals(lbmg_handle h, int nrhs, double *rel) {
    if (!h || !rel || nrhs < 1 || nrhs > 4) return LBMG_INVALID_ARG;
    if (h->inst_norm_host.size() != 16 * (size_t)h->c.ninst) return LBMG_NOT_ASSEMBLED;
    for (int m = 0; m < h->c.ninst; m++)
        for (int r = 0; r < nrhs; r++) {
            const double *nm = &h->inst_norm_host[16 * (size_t)m];
            rel[(size_t)m * nrhs + r] = rel_residual(nm[r], nm[4 + r]);
        }
    return LBMG_OK;
}

void lbmg_destroy(lbmg_handle h) { delete h; }

int lbmg_levels(lbmg_handle h, int *min_depth, int *depth) {
    if (!h) return LBMG_INVALID_ARG;
    if (min_depth) *min_depth = h->c.d0;
    if (depth) *depth = h->c.D;
    return LBMG_OK;
}

int lbmg_level_info(lbmg_handle h, int d, long *ndof, long *nnz, long *nfrag) {
    LBMG_TRY(check_level(h, d));
    if (ndof) *ndof = h->c.lev[d].n;
    if (nnz) *nnz = (long)h->c.lev[d].nnz;
    if (nfrag) *nfrag = d == h->c.D ? h->c.nfrag : 0;
    return LBMG_OK;
}

int lbmg_embedding(lbmg_handle h, double *cube_side, double *center) {
    if (!h) return LBMG_INVALID_ARG;
    if (cube_side) *cube_side = h->c.host.S;
    if (center) for (int a = 0; a < 3; a++) center[a] = h->c.host.center[a];
    return LBMG_OK;
}

int lbmg_set_area_weights(lbmg_handle h, const double *w, void *stream) {
    if (!h) return LBMG_INVALID_ARG;
    const HostHierarchy &H = h->c.host;
    std::vector<double> fs(H.frag_scale);
    if (w) {
        for (int t = 0; t < H.nt; t++)
            if (!(w[t] >= 0.0) || !std::isfinite(w[t])) return LBMG_INVALID_ARG;
        for (int f = 0; f < H.nfrag; f++) fs[f] *= w[H.frag_tri[f]];
    }
    // the assembly and projection kernels read the scales: none may still be running
    LBMG_CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (!fs.empty())
        LBMG_CK(cudaMemcpy(h->c.frag_scale, fs.data(), fs.size() * sizeof(double), cudaMemcpyHostToDevice));
    return LBMG_OK;
}

int lbmg_assemble(lbmg_handle h, double t, void *stream) {
    if (!h || !(t >= 0) || !std::isfinite(t)) return LBMG_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx &c = h->c;
    if (!c.moments_ready) {   // build-time geometry: once per hierarchy
        launch_fragment_moments(c, s);
        c.moments_ready = true;
    }
    launch_fine_gather(c, t, s);
    for (int d = c.D - 1; d >= c.d0; d--) launch_galerkin(c, d, t, s);
    for (int d = c.d0; d <= c.D; d++) launch_inverse_diag(c.lev[d], c.diag_part, s);
    for (int d = c.d0 + 1; d <= c.D; d++) launch_packed_fill(c.lev[d], s);
    cudaMemsetAsync(c.flag, 0, sizeof(int), s);
    launch_coarse_factor(c, h->lev_rp, h->lev_ci, h->lev_A, s);
    narrow_smem_refresh(c, s);
    LBMG_TRY(check_launch());
    // the coarse-factor flag stays on the device: the next solve reports a failed factor
    c.assembled = true;
    c.t = t;
    learned_refresh(c, s);   // stencil features of the new matrix for the learned correction
    return LBMG_OK;
}

int lbmg_project_rhs(lbmg_handle h, const double *f_vertex, int nrhs, double *rhs, void *stream) {
    if (!h || !f_vertex || !rhs || nrhs < 1 || nrhs > 4) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    cudaStream_t s = (cudaStream_t)stream;
    const double *fv;
    double *out;
    bool host_out;
    const size_t nD = (size_t)h->c.lev[h->c.D].n;
    LBMG_TRY(input_ptr(h, f_vertex, (size_t)h->c.nv * nrhs, 0, s, &fv));
    LBMG_TRY(output_ptr(h, rhs, nD * nrhs, 1, &out, &host_out));
    launch_project_rhs(h->c, fv, nrhs, out, s);
    return finish_output(rhs, out, nD * nrhs, host_out, s);
}

int lbmg_eval_vertices(lbmg_handle h, const double *x, int nrhs, double *u, void *stream) {
    if (!h || !x || !u || nrhs < 1 || nrhs > 4) return LBMG_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nD = (size_t)h->c.lev[h->c.D].n;
    const double *xd;
    double *ud;
    bool host_out;
    LBMG_TRY(input_ptr(h, x, nD * nrhs, 0, s, &xd));
    LBMG_TRY(output_ptr(h, u, (size_t)h->c.nv * nrhs, 1, &ud, &host_out));
    launch_eval_vertices(h->c, xd, nrhs, ud, s);
    return finish_output(u, ud, (size_t)h->c.nv * nrhs, host_out, s);
}

// A solve as one graph launch (conditional WHILE node, see build_cond_graph): packing, the
// initial residual and norms and the graph go out on `stream`, and the host synchronizes once,
// to read the final status (and the solution, for a host output buffer).
static int solve_cond(lbmg_handle h, cudaGraphExec_t exec, const double *rd, const double *xin, double *xout,
                      bool host_out, double *x, size_t cnt, int nrhs, int R, double tol, int max_cycles, bool pcg,
                      bool check, int precision, lbmg_stats *stats, cudaStream_t s) {
    Ctx &c = h->c;
    DevLevel &Fl = c.lev[c.D];
    const bool batch = c.ninst > 1;
    h->syncs = 0;
    LBMG_CK(cudaEventRecord(c.ev0, s));
    launch_pack(rd, Fl.n, nrhs, R, c.bs, s, c.fperm);
    launch_pack(xin, Fl.n, nrhs, R, c.xs, s, c.fperm);
    launch_residual<double>(Fl, Fl.A64, c.bs, c.xs, c.rs, R, s);
    const size_t m = (size_t)Fl.n * R;
    const bool pairs = pair_iterate(c, precision, pcg);
    if (pairs) launch_split(c.xs, c.xs_hi, c.xs_lo, (int64_t)m, s);
    if (pcg) {
        LBMG_CK(cudaMemsetAsync(c.pcg_z, 0, m * sizeof(double), s));
        LBMG_CK(cudaMemsetAsync(c.pcg_p, 0, m * sizeof(double), s));
        if (batch) LBMG_CK(cudaMemsetAsync(c.pcg_si, 0, sizeof(double) * kPcgScalars * c.ninst, s));
        else LBMG_CK(cudaMemsetAsync(c.pcg_s, 0, kPcgScalars * sizeof(double), s));
    }
    ctl_setup_kernel<<<1, 32, 0, s>>>(c.ctl, check ? tol : 0.0, max_cycles, check ? 0 : 1, nrhs,
                                      batch ? c.pcg_tol : nullptr);
    if (batch) {
        launch_item_dot2(c.nitem, c.nnitem, c.rs, c.rs, c.bs, c.bs, R, c.item_part, s);
        launch_inst_sum(c.item_start, c.ninst, c.item_part, c.inst_norm, 16, s);
    } else {
        launch_norms(c.bs, Fl.n, R, c.norm_part, c.norm_b, s);
        launch_norms(c.rs, Fl.n, R, c.norm_part, c.norm_out, s);
    }
    LBMG_CK(cudaGraphLaunch(exec, s));
    if (pairs) launch_join(c.xs_hi, c.xs_lo, c.xs, (int64_t)m, s);
    launch_unpack(c.xs, Fl.n, nrhs, R, xout, s, c.fperm);
    LBMG_CK(cudaEventRecord(c.ev1, s));
    LBMG_CK(cudaMemcpyAsync(c.h_ctl, c.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
    if (batch)
        LBMG_CK(cudaMemcpyAsync(h->h_inst, c.inst_norm, 16 * sizeof(double) * c.ninst, cudaMemcpyDeviceToHost, s));
    LBMG_TRY(finish_output(x, xout, cnt, host_out, s, &h->syncs));
    if (!host_out) {
        LBMG_CK(cudaStreamSynchronize(s));
        h->syncs++;
    }
    const SolveCtl &hc = *c.h_ctl;
    if (batch) h->inst_norm_host.assign(h->h_inst, h->h_inst + 16 * (size_t)c.ninst);
    int status = LBMG_OK;
    switch (hc.status) {
        case kCtlConverged: status = LBMG_OK; break;
        case kCtlMaxCycles: status = check ? LBMG_NOT_CONVERGED : LBMG_OK; break;
        case kCtlDiverged: status = LBMG_DIVERGED; break;
        case kCtlCoarse: status = LBMG_COARSE_FACTOR; break;
        case kCtlTimeout:
            // a bounded wait gave up: the results are invalid; clear the word for the next solve
            status = LBMG_DEVICE_TIMEOUT;
            LBMG_CK(cudaMemsetAsync(c.norm_out + 4, 0, sizeof(double), s));
            break;
        default: g_cuda_err = "solve ended with an unknown control status"; status = LBMG_CUDA_ERROR;
    }
    if (stats) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c.ev0, c.ev1);
        stats->cycles = hc.cycles;
        stats->converged = hc.status == kCtlConverged ? 1 : 0;
        for (int r = 0; r < 4; r++) {
            stats->rel_residual[r] = r < nrhs ? hc.rel[r] : 0.0;
            stats->initial_residual[r] = r < nrhs ? hc.r0[r] : 0.0;
        }
        stats->ms_total = ms;
        stats->ms_fine_smooth = 0.f;
        stats->learned = (!pcg && c.learned_on) ? 1 : 0;
        stats->learned_fallback = stats->learned && hc.learned_off ? 1 : 0;
        stats->host_syncs = h->syncs;
    }
    return status;
}

// V-cycle-preconditioned conjugate gradients on a batch: per-mesh step lengths and norms;
// stops when every mesh meets tol (or after max_iters iterations)
static int solve_pcg_batch(lbmg_handle h, const double *rd, const double *xin, double *xout, bool host_out,
                           double *x, size_t cnt, int nrhs, int R, double tol, int max_iters, int precision,
                           lbmg_stats *stats, cudaStream_t s) {
    Ctx &c = h->c;
    DevLevel &Fl = c.lev[c.D];
    cudaGraphExec_t exec = nullptr;
    if (c.use_graphs) LBMG_TRY(get_graph(h, R, precision, true, &exec));
    LBMG_CK(cudaEventRecord(c.ev0, s));
    launch_pack(rd, Fl.n, nrhs, R, c.bs, s, c.fperm);
    launch_pack(xin, Fl.n, nrhs, R, c.xs, s, c.fperm);
    launch_residual<double>(Fl, Fl.A64, c.bs, c.xs, c.rs, R, s);
    const size_t m = (size_t)Fl.n * R;
    LBMG_CK(cudaMemsetAsync(c.pcg_z, 0, m * sizeof(double), s));
    LBMG_CK(cudaMemsetAsync(c.pcg_p, 0, m * sizeof(double), s));
    LBMG_CK(cudaMemsetAsync(c.pcg_si, 0, sizeof(double) * kPcgScalars * c.ninst, s));
    h->pcg_tol_host = tol;
    LBMG_CK(cudaMemcpyAsync(c.pcg_tol, &h->pcg_tol_host, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_item_dot2(c.nitem, c.nnitem, c.rs, c.rs, c.bs, c.bs, R, c.item_part, s);
    launch_inst_sum(c.item_start, c.ninst, c.item_part, c.inst_norm, 16, s);
    std::vector<double> &nh = h->inst_norm_host;
    nh.assign(16 * (size_t)c.ninst, 0.0);
    h->syncs = 0;
    auto read = [&]() -> int {
        LBMG_CK(cudaMemcpyAsync(nh.data(), c.inst_norm, nh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        LBMG_CK(cudaStreamSynchronize(s));
        h->syncs++;
        return check_launch();
    };
    auto worst = [&](const std::vector<double> &v, double *w) {
        for (int r = 0; r < 4; r++) w[r] = 0.0;
        for (int mm = 0; mm < c.ninst; mm++)
            for (int r = 0; r < nrhs; r++) {
                const double *nm = &v[16 * (size_t)mm];
                w[r] = std::max(w[r], rel_residual(nm[r], nm[4 + r]));
            }
    };
    LBMG_TRY(read());
    double w0[4], w[4];
    worst(nh, w0);
    int it = 0, status = LBMG_OK;
    bool conv = false;
    for (;;) {
        worst(nh, w);
        conv = true;
        bool bad = false;
        for (int r = 0; r < nrhs; r++) {
            if (!(w[r] <= tol)) conv = false;
            if (!std::isfinite(w[r]) || w[r] > 1e6 * std::max(w0[r], 1e-300)) bad = true;
        }
        if (bad) { status = LBMG_DIVERGED; break; }
        if (conv || it >= max_iters) break;
        if (exec) LBMG_CK(cudaGraphLaunch(exec, s));
        else enqueue_pcg_batch_iteration(c, R, precision, s);
        LBMG_TRY(read());
        it++;
    }
    if (!conv && status == LBMG_OK) status = LBMG_NOT_CONVERGED;
    launch_unpack(c.xs, Fl.n, nrhs, R, xout, s, c.fperm);
    LBMG_CK(cudaEventRecord(c.ev1, s));
    LBMG_TRY(finish_output(x, xout, cnt, host_out, s, &h->syncs));
    if (stats) {
        LBMG_CK(cudaEventSynchronize(c.ev1));
        if (!host_out) h->syncs++;
        float ms = 0;
        cudaEventElapsedTime(&ms, c.ev0, c.ev1);
        stats->host_syncs = h->syncs;
        stats->cycles = it;
        stats->converged = conv ? 1 : 0;
        for (int r = 0; r < 4; r++) {
            stats->rel_residual[r] = r < nrhs ? w[r] : 0.0;
            stats->initial_residual[r] = r < nrhs ? w0[r] : 0.0;
        }
        stats->ms_total = ms;
        stats->ms_fine_smooth = 0.f;
        stats->learned = 0;
        stats->learned_fallback = 0;
    }
    return status;
}

static int solve_impl(lbmg_handle h, const double *rhs, double *x, int nrhs, double tol, int max_cycles,
                      int precision, lbmg_stats *stats, void *stream, bool check, bool pcg = false) {
    if (!h || !rhs || !x || nrhs < 1 || nrhs > 4 || max_cycles < 0) return LBMG_INVALID_ARG;
    if (precision != LBMG_FP64 && precision != LBMG_MIXED) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    Ctx &c = h->c;
    cudaStream_t s = (cudaStream_t)stream;
    const int R = stride_for(nrhs);
    DevLevel &Fl = c.lev[c.D];
    const size_t cnt = (size_t)Fl.n * nrhs;
    const double *rd, *xin;
    double *xout;
    bool host_out;
    LBMG_TRY(input_ptr(h, rhs, cnt, 0, s, &rd));
    LBMG_TRY(input_ptr(h, x, cnt, 1, s, &xin));
    LBMG_TRY(output_ptr(h, x, cnt, 1, &xout, &host_out));
    if (!pcg && c.persistent && c.persist_ok && c.smoother == LBMG_GS_COLOURED) {
        if (c.learned_on) {
            g_cuda_err = "the learned correction runs on the graph and host-loop solves, not the persistent one";
            return LBMG_INVALID_ARG;
        }
        LBMG_CK(cudaEventRecord(c.ev0, s));
        launch_pack(rd, Fl.n, nrhs, R, c.bs, s, c.fperm);
        launch_pack(xin, Fl.n, nrhs, R, c.xs, s, c.fperm);
        const int e = persist_solve(c, precision, R, nrhs, check ? tol : 0.0, max_cycles, s);
        if (e) {
            g_cuda_err = std::string("cooperative launch: ") + cudaGetErrorString((cudaError_t)e);
            cudaGetLastError();
            return LBMG_CUDA_ERROR;
        }
        unsigned char *hs = reinterpret_cast<unsigned char *>(c.h_state);
        LBMG_CK(cudaMemcpyAsync(hs, c.persist_state, 64, cudaMemcpyDeviceToHost, s));
        LBMG_CK(cudaMemcpyAsync(h->h_inst, c.inst_norm, 16 * sizeof(double) * c.ninst, cudaMemcpyDeviceToHost, s));
        LBMG_CK(cudaMemcpyAsync(h->h_flag, c.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        launch_unpack(c.xs, Fl.n, nrhs, R, xout, s, c.fperm);
        LBMG_CK(cudaEventRecord(c.ev1, s));
        h->syncs = 0;
        LBMG_TRY(finish_output(x, xout, cnt, host_out, s, &h->syncs));
        LBMG_CK(cudaEventSynchronize(c.ev1));
        if (!host_out) h->syncs++;
        h->inst_norm_host.assign(h->h_inst, h->h_inst + 16 * (size_t)c.ninst);
        int dstat, dcyc, dfall;
        std::memcpy(&dfall, hs + 32, sizeof(int));
        unsigned long long sns;
        std::memcpy(&dstat, hs + 16, sizeof(int));
        std::memcpy(&dcyc, hs + 20, sizeof(int));
        std::memcpy(&sns, hs + 24, sizeof(sns));
        bool conv = true;
        double worst[4] = {0, 0, 0, 0}, worst0[4] = {0, 0, 0, 0};
        for (int m = 0; m < c.ninst; m++)
            for (int r = 0; r < nrhs; r++) {
                const double *nm = &h->inst_norm_host[16 * (size_t)m];
                const double rel = rel_residual(nm[r], nm[4 + r]);
                const double rel0 = rel_residual(nm[8 + r], nm[4 + r]);
                if (!(rel <= tol)) conv = false;
                worst[r] = std::max(worst[r], rel);
                worst0[r] = std::max(worst0[r], rel0);
            }
        int status = LBMG_OK;
        if (dstat == 1) status = LBMG_DEVICE_TIMEOUT;
        else if (*h->h_flag != 0) status = LBMG_COARSE_FACTOR;
        else if (dstat == 2) status = LBMG_DIVERGED;
        else if (check && !conv) status = LBMG_NOT_CONVERGED;
        if (stats) {
            stats->host_syncs = h->syncs;
            stats->cycles = dcyc;
            stats->converged = (check && conv && dstat == 0) ? 1 : 0;
            for (int r = 0; r < 4; r++) {
                stats->rel_residual[r] = r < nrhs ? worst[r] : 0.0;
                stats->initial_residual[r] = r < nrhs ? worst0[r] : 0.0;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, c.ev0, c.ev1);
            stats->ms_total = ms;
            stats->ms_fine_smooth = (float)(sns * 1e-6);
            stats->learned = 0;
            stats->learned_fallback = 0;
            (void)dfall;
        }
        return status;
    }
    if (pcg && c.smoother != LBMG_GS_COLOURED) return LBMG_INVALID_ARG;   // the preconditioner must be symmetric
    if (!pcg && c.ninst > 1) return LBMG_INVALID_ARG;   // batch V-cycles need the persistent solve (per-mesh norms)
    if (c.use_graphs && !c.host_check && !c.cond_failed) {
        cudaGraphExec_t cexec = nullptr;
        if (get_cond_graph(h, R, precision, pcg, &cexec) == LBMG_OK)
            return solve_cond(h, cexec, rd, xin, xout, host_out, x, cnt, nrhs, R, tol, max_cycles, pcg, check,
                              precision, stats, s);
        c.cond_failed = true;   // no conditional graphs here: the host reads the norms each iteration
    }
    if (pcg && c.ninst > 1)
        return solve_pcg_batch(h, rd, xin, xout, host_out, x, cnt, nrhs, R, tol, max_cycles, precision, stats, s);
    cudaGraphExec_t exec = nullptr;
    if (c.use_graphs) LBMG_TRY(get_graph(h, R, precision, pcg, &exec));
    h->syncs = 0;
    LBMG_CK(cudaMemcpyAsync(h->h_flag, c.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    LBMG_CK(cudaEventRecord(c.ev0, s));
    launch_pack(rd, Fl.n, nrhs, R, c.bs, s, c.fperm);
    launch_pack(xin, Fl.n, nrhs, R, c.xs, s, c.fperm);
    launch_residual<double>(Fl, Fl.A64, c.bs, c.xs, c.rs, R, s);
    const bool pairs = pair_iterate(c, precision, pcg);
    if (pairs) launch_split(c.xs, c.xs_hi, c.xs_lo, (int64_t)Fl.n * R, s);
    if (pcg) {
        LBMG_CK(cudaMemsetAsync(c.pcg_z, 0, (size_t)Fl.n * R * sizeof(double), s));
        LBMG_CK(cudaMemsetAsync(c.pcg_p, 0, (size_t)Fl.n * R * sizeof(double), s));
        LBMG_CK(cudaMemsetAsync(c.pcg_s, 0, kPcgScalars * sizeof(double), s));
    }
    double nb[4] = {0, 0, 0, 0}, nr[4] = {0, 0, 0, 0}, r0[4] = {0, 0, 0, 0};
    int cycles = 0, status = LBMG_OK;
    float smooth_ms = 0.0f;
    bool conv = false;
    const bool learned = !pcg && c.learned_on;
    bool dropped = false;
    if (learned) {
        LBMG_CK(cudaMemsetAsync(&c.ctl->learned_off, 0, sizeof(int), s));
        if (!check) launch_norms(c.rs, Fl.n, R, c.norm_part, c.norm_out, s);   // the correction reads them
    }
    if (check) {
        launch_norms(c.bs, Fl.n, R, c.norm_part, c.norm_out, s);
        LBMG_TRY(read_norms(h, R, s, nb));
        launch_norms(c.rs, Fl.n, R, c.norm_part, c.norm_out, s);
        LBMG_TRY(read_norms(h, R, s, nr));
        if (*h->h_flag != 0) return LBMG_COARSE_FACTOR;
        auto rel = [&](int r) { return rel_residual(nr[r], nb[r]); };
        for (int r = 0; r < nrhs; r++) r0[r] = rel(r);
        for (;;) {
            conv = true;
            bool bad = false;
            for (int r = 0; r < nrhs; r++) {
                const double v = rel(r);
                if (!(v <= tol)) conv = false;
                if (!std::isfinite(v) || v > 1e6 * std::max(r0[r], 1e-300)) bad = true;
            }
            if (bad) { status = LBMG_DIVERGED; break; }
            if (conv || cycles >= max_cycles) break;
            double prev[4];
            for (int r = 0; r < nrhs; r++) prev[r] = rel(r);
            if (exec) LBMG_CK(cudaGraphLaunch(exec, s));
            else if (pcg) enqueue_pcg_iteration(c, R, precision, s);
            else enqueue_iteration(c, R, precision, s);
            LBMG_TRY(read_norms(h, R, s, nr));
            // acceptance test of the learned correction: a residual that grew drops it for good
            if (learned && !dropped)
                for (int r = 0; r < nrhs; r++)
                    if (rel(r) > prev[r]) dropped = true;
            if (dropped) LBMG_CK(cudaMemsetAsync(&c.ctl->learned_off, 1, sizeof(int), s));
            if (c.D > c.d0) {
                float a0 = 0, a1 = 0;
                if (cudaEventElapsedTime(&a0, c.ev_smooth[0], c.ev_smooth[1]) != cudaSuccess ||
                    cudaEventElapsedTime(&a1, c.ev_smooth[2], c.ev_smooth[3]) != cudaSuccess) {
                    cudaGetLastError();
                    a0 = a1 = 0.0f;
                }
                smooth_ms += a0 + a1;
            }
            cycles++;
        }
        if (!conv && status == LBMG_OK) status = LBMG_NOT_CONVERGED;
        if (stats) {
            stats->cycles = cycles;
            stats->converged = conv ? 1 : 0;
            for (int r = 0; r < 4; r++) {
                stats->rel_residual[r] = r < nrhs ? rel(r) : 0.0;
                stats->initial_residual[r] = r < nrhs ? r0[r] : 0.0;
            }
        }
    } else {
        for (int k = 0; k < max_cycles; k++) {
            if (exec) LBMG_CK(cudaGraphLaunch(exec, s));
            else if (pcg) enqueue_pcg_iteration(c, R, precision, s);
            else enqueue_iteration(c, R, precision, s);
        }
        cycles = max_cycles;
    }
    if (pairs) launch_join(c.xs_hi, c.xs_lo, c.xs, (int64_t)Fl.n * R, s);
    launch_unpack(c.xs, Fl.n, nrhs, R, xout, s, c.fperm);
    LBMG_CK(cudaEventRecord(c.ev1, s));
    LBMG_TRY(finish_output(x, xout, cnt, host_out, s, &h->syncs));
    if (stats) {
        LBMG_CK(cudaEventSynchronize(c.ev1));
        if (!host_out) h->syncs++;
        float ms = 0;
        cudaEventElapsedTime(&ms, c.ev0, c.ev1);
        stats->ms_total = ms;
        stats->ms_fine_smooth = smooth_ms;
        stats->host_syncs = h->syncs;
        stats->learned = learned ? 1 : 0;
        stats->learned_fallback = dropped ? 1 : 0;
        if (!check) stats->cycles = cycles;
    }
    return status;
}

int lbmg_cmcf_step(lbmg_handle h, const double *X, double delta, double *x, double tol, int max_cycles,
                   int precision, int solver, double *X_next, lbmg_stats *stats, void *stream) {
    if (!h || !X || !x || !X_next || !(delta > 0) || !std::isfinite(delta) || !(tol >= 0)) return LBMG_INVALID_ARG;
    if (solver != 0 && solver != 1) return LBMG_INVALID_ARG;
    Ctx &c = h->c;
    if (c.ninst != 1) return LBMG_INVALID_ARG;   // one mesh: one embedding
    if (!on_device(X) || !on_device(x) || !on_device(X_next)) {
        g_cuda_err = "lbmg_cmcf_step: X, x and X_next must be device pointers";
        return LBMG_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!c.cmcf_w) {
        LBMG_TRY(h->alloc(&c.cmcf_w, (size_t)std::max(c.nt, 1)));
        LBMG_TRY(h->alloc(&c.cmcf_rhs, 3 * (size_t)c.lev[c.D].n));
    }
    // M_t: the build-time mass matrix with every triangle weighted by its current area ratio
    launch_cmcf_weights(c, X, c.cmcf_w, s);
    LBMG_TRY(lbmg_assemble(h, delta, stream));
    // M_t u_t: the current positions, linear per triangle, integrated with the same weights
    launch_project_rhs(c, X, 3, c.cmcf_rhs, s);
    const int st = solve_impl(h, c.cmcf_rhs, x, 3, tol, max_cycles, precision, stats, stream, true, solver == 1);
    if (st != LBMG_OK && st != LBMG_NOT_CONVERGED) return st;
    launch_eval_vertices(c, x, 3, X_next, s);
    LBMG_TRY(check_launch());
    return st;
}

int lbmg_eigs(lbmg_handle h, int k, double tol, int max_iters, const double *X0, double *lambda, double *X,
              double *residuals, int *iters, void *stream) {
    if (!h || !X0 || !lambda || !X || !iters || !(tol > 0) || max_iters < 0) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    if (h->c.ninst != 1 || !on_device(X0) || !on_device(X)) {
        g_cuda_err = "lbmg_eigs: single meshes, device pointers X0 and X";
        return LBMG_INVALID_ARG;
    }
    std::string err;
    const int st = lobpcg(h->c, k, tol, max_iters, X0, lambda, X, residuals, iters, (cudaStream_t)stream, err);
    if (st != 0) g_cuda_err = err;
    switch (st) {
        case 0: return LBMG_OK;
        case 1: return LBMG_INVALID_ARG;
        case 2: return LBMG_CUDA_ERROR;
        case 3: return LBMG_DIVERGED;
        default: return LBMG_NOT_CONVERGED;
    }
}

int lbmg_solve_pcg(lbmg_handle h, const double *rhs, double *x, int nrhs, double tol, int max_iters, int precision,
                   lbmg_stats *stats, void *stream) {
    if (!(tol >= 0)) return LBMG_INVALID_ARG;
    return solve_impl(h, rhs, x, nrhs, tol, max_iters, precision, stats, stream, true, true);
}

int lbmg_solve(lbmg_handle h, const double *rhs, double *x, int nrhs, double tol, int max_cycles, int precision,
               lbmg_stats *stats, void *stream) {
    if (!(tol >= 0)) return LBMG_INVALID_ARG;
    return solve_impl(h, rhs, x, nrhs, tol, max_cycles, precision, stats, stream, true);
}

int lbmg_vcycles(lbmg_handle h, const double *rhs, double *x, int nrhs, int cycles, int precision, void *stream) {
    return solve_impl(h, rhs, x, nrhs, 0.0, cycles, precision, nullptr, stream, false);
}

int lbmg_residual(lbmg_handle h, int d, const double *rhs, const double *x, double *r, int nrhs, void *stream) {
    LBMG_TRY(check_level(h, d));
    if (!rhs || !x || !r || nrhs < 1 || nrhs > 4) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &L = h->c.lev[d];
    const int R = stride_for(nrhs);
    const size_t cnt = (size_t)L.n * nrhs;
    const double *bd, *xd;
    double *rd;
    bool host_out;
    LBMG_TRY(input_ptr(h, rhs, cnt, 0, s, &bd));
    launch_pack(bd, L.n, nrhs, R, L.b64, s);
    LBMG_TRY(input_ptr(h, x, cnt, 1, s, &xd));
    launch_pack(xd, L.n, nrhs, R, L.x64, s);
    launch_residual<double>(L, L.A64, L.b64, L.x64, L.r64, R, s);
    LBMG_TRY(output_ptr(h, r, cnt, 0, &rd, &host_out));
    launch_unpack(L.r64, L.n, nrhs, R, rd, s);
    return finish_output(r, rd, cnt, host_out, s);
}

int lbmg_residual_split(lbmg_handle h, int d, const double *rhs, const double *x, double *r, int nrhs,
                        void *stream) {
    LBMG_TRY(check_level(h, d));
    if (!rhs || !x || !r || nrhs < 1 || nrhs > 4) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    DevLevel &L = h->c.lev[d];
    if (!L.pk_v2) {
        g_cuda_err = "lbmg_residual_split: the level has no packed copy (the coarsest level)";
        return LBMG_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int R = stride_for(nrhs);
    const size_t cnt = (size_t)L.n * nrhs;
    const double *bd, *xd;
    double *rd;
    bool host_out;
    LBMG_TRY(input_ptr(h, rhs, cnt, 0, s, &bd));
    launch_pack(bd, L.n, nrhs, R, L.b64, s);
    LBMG_TRY(input_ptr(h, x, cnt, 1, s, &xd));
    launch_pack(xd, L.n, nrhs, R, L.x64, s);
    launch_split(L.x64, L.x32, L.r32, (int64_t)L.n * R, s);   // the level's FP32 vectors as scratch
    launch_packed_residual_split(L, L.b64, L.x32, L.r32, L.r64, R, s, nullptr);
    LBMG_TRY(output_ptr(h, r, cnt, 0, &rd, &host_out));
    launch_unpack(L.r64, L.n, nrhs, R, rd, s);
    return finish_output(r, rd, cnt, host_out, s);
}

int lbmg_smooth(lbmg_handle h, int d, const double *rhs, double *x, int nrhs, int sweeps, int precision, void *stream) {
    LBMG_TRY(check_level(h, d));
    if (!rhs || !x || nrhs < 1 || nrhs > 4 || sweeps < 0) return LBMG_INVALID_ARG;
    if (precision != LBMG_FP64 && precision != LBMG_MIXED) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &L = h->c.lev[d];
    const int R = stride_for(nrhs);
    const size_t cnt = (size_t)L.n * nrhs;
    const int64_t m = (int64_t)L.n * R;
    const double *bd, *xd;
    LBMG_TRY(input_ptr(h, rhs, cnt, 0, s, &bd));
    launch_pack(bd, L.n, nrhs, R, L.b64, s);
    LBMG_TRY(input_ptr(h, x, cnt, 1, s, &xd));
    launch_pack(xd, L.n, nrhs, R, L.x64, s);
    if (precision == LBMG_MIXED) {
        launch_to_float(L.b64, L.b32, m, s);
        launch_to_float(L.x64, L.x32, m, s);
        enqueue_smooth<float>(h->c, L, R, sweeps, true, s, nullptr);
        if (m) to_double_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(L.x32, L.x64, m);
    } else {
        enqueue_smooth<double>(h->c, L, R, sweeps, true, s, nullptr);
    }
    double *xo;
    bool host_out;
    LBMG_TRY(output_ptr(h, x, cnt, 1, &xo, &host_out));
    launch_unpack(L.x64, L.n, nrhs, R, xo, s);
    return finish_output(x, xo, cnt, host_out, s);
}

int lbmg_restrict(lbmg_handle h, int d, const double *r_fine, double *r_coarse, int nrhs, void *stream) {
    LBMG_TRY(check_level(h, d));
    if (d == h->c.d0 || !r_fine || !r_coarse || nrhs < 1 || nrhs > 4) return LBMG_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &Lf = h->c.lev[d], &Lc = h->c.lev[d - 1];
    const int R = stride_for(nrhs);
    const double *rf;
    LBMG_TRY(input_ptr(h, r_fine, (size_t)Lf.n * nrhs, 0, s, &rf));
    launch_pack(rf, Lf.n, nrhs, R, Lf.r64, s);
    launch_restrict<double>(Lc, Lf.r64, Lc.b64, R, s);
    double *out;
    bool host_out;
    LBMG_TRY(output_ptr(h, r_coarse, (size_t)Lc.n * nrhs, 1, &out, &host_out));
    launch_unpack(Lc.b64, Lc.n, nrhs, R, out, s);
    return finish_output(r_coarse, out, (size_t)Lc.n * nrhs, host_out, s);
}

int lbmg_prolong_add(lbmg_handle h, int d, const double *x_coarse, double *x_fine, int nrhs, void *stream) {
    LBMG_TRY(check_level(h, d));
    if (d == h->c.d0 || !x_coarse || !x_fine || nrhs < 1 || nrhs > 4) return LBMG_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &Lf = h->c.lev[d], &Lc = h->c.lev[d - 1];
    const int R = stride_for(nrhs);
    const double *xc, *xf;
    LBMG_TRY(input_ptr(h, x_coarse, (size_t)Lc.n * nrhs, 0, s, &xc));
    launch_pack(xc, Lc.n, nrhs, R, Lc.x64, s);
    LBMG_TRY(input_ptr(h, x_fine, (size_t)Lf.n * nrhs, 1, s, &xf));
    launch_pack(xf, Lf.n, nrhs, R, Lf.x64, s);
    launch_prolong_add<double>(Lf, Lc.x64, Lf.x64, R, s);
    double *out;
    bool host_out;
    LBMG_TRY(output_ptr(h, x_fine, (size_t)Lf.n * nrhs, 1, &out, &host_out));
    launch_unpack(Lf.x64, Lf.n, nrhs, R, out, s);
    return finish_output(x_fine, out, (size_t)Lf.n * nrhs, host_out, s);
}

int lbmg_launch_counts(lbmg_handle h, int precision, int *assemble, int *project_rhs, int *per_cycle,
                       int *solve_fixed) {
    if (!h) return LBMG_INVALID_ARG;
    const Ctx &c = h->c;
    const int levels = c.D - c.d0;
    if (assemble) *assemble = 2 + levels + (levels + 1) + 3;
    if (project_rhs) *project_rhs = 2;
    auto per_sweep = [&](const int *cs) {
        if (c.smoother == LBMG_JACOBI) return 2;
        int k = 0;
        for (int q = 0; q < 8; q++) k += cs[q + 1] > cs[q];
        return k;
    };
    int cyc = 0;
    if (c.gamma == 1 && !c.coarse_smooth) {
        const bool narrow = c.persist_dn >= c.d0 && c.smoother != LBMG_JACOBI && precision == LBMG_MIXED;
        const bool smem = c.narrow.dn >= c.d0 && c.smoother != LBMG_JACOBI && precision == LBMG_MIXED;
        const int bottom = smem ? c.narrow.dn : (narrow ? c.persist_dn : c.d0);
        cyc = 1;   // the one-block bottom cycle, or the coarse apply
        for (int d = bottom + 1; d <= c.D; d++) {   // sweeps, residual, restriction, prolongation
            const DevLevel &L = c.lev[d];
            const bool whole = precision == LBMG_MIXED && c.smoother != LBMG_JACOBI &&
                               L.shape[0][kShapeSmooth].tpb == kSweepShapeTpb && L.pk_map && c.sweep_bar;
            if (whole) cyc += (c.nu1 > 0) + (c.nu2 > 0);   // one cooperative launch per smoothing
            else {
                cyc += (c.nu1 + c.nu2) * per_sweep(L.cs);
                // below the finest level the restriction does colour 0 of the first sweep
                if (d < c.D && c.smoother != LBMG_JACOBI && c.nu1 > 0 && L.cs[1] > L.cs[0]) cyc -= 1;
            }
            cyc += 3 + (L.ncb > 0);
        }
    } else {
        // the general cycle: gamma visits of each coarser level
        long visit = c.coarse_smooth ? (long)(c.nu1 + c.nu2) * per_sweep(c.lev[c.d0].cs_all) : 1;
        for (int d = c.d0 + 1; d <= c.D; d++) visit = (long)(c.nu1 + c.nu2) * per_sweep(c.lev[d].cs) + 3 + c.gamma * visit;
        cyc = (int)std::min<long>(visit, 1 << 30);
    }
    cyc += (precision == LBMG_MIXED ? 2 : 1) + 1 + 2;   // conversion/update, FP64 residual, norms
    const bool persistent = c.persistent && c.persist_ok && c.smoother == LBMG_GS_COLOURED;
    // the persistent solve runs every cycle inside one launch: two packs, the solve, one unpack
    if (per_cycle) *per_cycle = persistent ? 0 : cyc;
    if (solve_fixed) *solve_fixed = persistent ? 4 : 2 + 1 + 2 + 2 + 1;
    return LBMG_OK;
}

int lbmg_autotune(lbmg_handle h, int nrhs, int precision, int reps, int *timed, void *stream) {
    if (!h || nrhs < 1 || nrhs > 4 || reps < 1 || reps > 64) return LBMG_INVALID_ARG;
    if (precision != LBMG_FP64 && precision != LBMG_MIXED) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    Ctx &c = h->c;
    const cudaError_t e = (cudaError_t)autotune(c, stride_for(nrhs), precision, reps, (cudaStream_t)stream, timed);
    if (c.graph.exec) { cudaGraphExecDestroy(c.graph.exec); c.graph.exec = nullptr; }
    if (e != cudaSuccess) {
        g_cuda_err = std::string("autotune: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return LBMG_CUDA_ERROR;
    }
    return LBMG_OK;
}

int lbmg_launch_shape(lbmg_handle h, int d, int precision, int *out) {
    LBMG_TRY(check_level(h, d));
    if (!out || (precision != LBMG_FP64 && precision != LBMG_MIXED)) return LBMG_INVALID_ARG;
    const DevLevel &L = h->c.lev[d];
    const int p = precision == LBMG_FP64;
    out[0] = L.shape[p][kShapeSmooth].tpr;
    out[1] = L.shape[p][kShapeSmooth].tpb;
    out[2] = L.shape[p][kShapeResidual].tpr;
    out[3] = L.shape[p][kShapeResidual].tpb;
    return LBMG_OK;
}

int lbmg_tuned_times(lbmg_handle h, int d, int precision, float *ms) {
    LBMG_TRY(check_level(h, d));
    if (!ms || (precision != LBMG_FP64 && precision != LBMG_MIXED)) return LBMG_INVALID_ARG;
    const DevLevel &L = h->c.lev[d];
    const int p = precision == LBMG_FP64;
    ms[0] = L.tuned_ms[p][kShapeSmooth];
    ms[1] = L.tuned_ms[p][kShapeResidual];
    return LBMG_OK;
}

int lbmg_set_launch_shape(lbmg_handle h, int d, int precision, int kind, int tpr, int tpb) {
    LBMG_TRY(check_level(h, d));
    if (precision != LBMG_FP64 && precision != LBMG_MIXED) return LBMG_INVALID_ARG;
    if (kind != 0 && kind != 1) return LBMG_INVALID_ARG;
    // tpb = 1024 with 4 threads per row: the whole-sweep cooperative kernel (FP32 sweeps only)
    const bool sweep = tpb == kSweepShapeTpb && tpr == 4 && kind == kShapeSmooth && precision == LBMG_MIXED;
    if ((tpr != 4 && tpr != 8 && tpr != 16) || tpb < 32 || (tpb > 512 && !sweep) || tpb % 32 != 0)
        return LBMG_INVALID_ARG;
    LaunchShape &sh = h->c.lev[d].shape[precision == LBMG_FP64][kind];
    sh.tpr = tpr;
    sh.tpb = tpb;
    h->c.lev[d].tuned_ms[precision == LBMG_FP64][kind] = 0.f;
    if (h->c.graph.exec) { cudaGraphExecDestroy(h->c.graph.exec); h->c.graph.exec = nullptr; }
    return LBMG_OK;
}

int lbmg_set_host_check(lbmg_handle h, int on) {
    if (!h || (on != 0 && on != 1)) return LBMG_INVALID_ARG;
    h->c.host_check = on;
    return LBMG_OK;
}

int lbmg_tune_cache_save(const char *path) {
    if (!path) return LBMG_INVALID_ARG;
    return tune_cache_save(path) == 0 ? LBMG_OK : LBMG_INVALID_ARG;
}

int lbmg_tune_cache_load(const char *path) {
    if (!path) return LBMG_INVALID_ARG;
    return tune_cache_load(path) == 0 ? LBMG_OK : LBMG_INVALID_ARG;
}

static int learned_ready(lbmg_handle h, cudaStream_t s) {
    if (!h) return LBMG_INVALID_ARG;
    if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
    if (h->c.ninst != 1) {
        g_cuda_err = "the learned correction needs a single-mesh handle";
        return LBMG_INVALID_ARG;
    }
    const int st = learned_setup(h->c, s);
    if (st == 1) return LBMG_INVALID_ARG;
    if (st) return LBMG_OUT_OF_MEMORY;
    return LBMG_OK;
}

int lbmg_learned_nparams(void) { return learned_nparams(); }

int lbmg_learned_params(lbmg_handle h, double *get, const double *set, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    LBMG_TRY(learned_ready(h, s));
    return learned_params(h->c, get, set, s) ? LBMG_CUDA_ERROR : LBMG_OK;
}

int lbmg_learned_state(lbmg_handle h, double *get, const double *set, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    LBMG_TRY(learned_ready(h, s));
    if (set && !(set[3 * (size_t)learned_nparams()] >= 0)) return LBMG_INVALID_ARG;
    return learned_state(h->c, get, set, s) ? LBMG_CUDA_ERROR : LBMG_OK;
}

int lbmg_learned_collect(lbmg_handle h, const double *rhs, int ns, int skip, int keep, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!rhs || ns < 1 || ns > 4 || skip < 0 || keep < 1) return LBMG_INVALID_ARG;
    LBMG_TRY(learned_ready(h, s));
    const double *rd;
    const size_t cnt = (size_t)h->c.lev[h->c.D].n * ns;
    if (!on_device(rhs) && cnt > h->io_cap) return LBMG_INVALID_ARG;
    LBMG_TRY(input_ptr(h, rhs, cnt, 0, s, &rd));
    return learned_collect(h->c, rd, ns, skip, keep, s) ? LBMG_CUDA_ERROR : LBMG_OK;
}

int lbmg_learned_loss_grad(lbmg_handle h, const double *r0, int ns, double *loss, double *grad, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!r0 || !loss || ns < 1 || ns > 4) return LBMG_INVALID_ARG;
    LBMG_TRY(learned_ready(h, s));
    const double *rd;
    LBMG_TRY(input_ptr(h, r0, (size_t)h->c.lev[h->c.D].n * ns, 0, s, &rd));
    return learned_loss_grad(h->c, rd, ns, loss, grad, s) ? LBMG_CUDA_ERROR : LBMG_OK;
}

int lbmg_learned_train(lbmg_handle h, int steps, double lr, const int *order, int batch, double *loss_hist,
                       void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (steps < 0 || !order || batch < 1 || batch > 8 || !(lr > 0)) return LBMG_INVALID_ARG;
    LBMG_TRY(learned_ready(h, s));
    const int st = learned_train(h->c, steps, lr, order, batch, loss_hist, s);
    return st == 1 ? LBMG_INVALID_ARG : (st ? LBMG_CUDA_ERROR : LBMG_OK);
}

int lbmg_learned_enable(lbmg_handle h, int on, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    LBMG_TRY(learned_ready(h, s));
    if (on && h->c.persistent) {
        g_cuda_err = "the learned correction runs on the graph and host-loop solves, not the persistent one";
        return LBMG_INVALID_ARG;
    }
    return learned_enable(h->c, on, s) ? LBMG_CUDA_ERROR : LBMG_OK;
}

int lbmg_learned_apply(lbmg_handle h, const double *r, int ns, int precision, double *omega, double *delta,
                       void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!r || !omega || !delta || ns < 1 || ns > 4) return LBMG_INVALID_ARG;
    if (precision != LBMG_FP64 && precision != LBMG_MIXED) return LBMG_INVALID_ARG;
    if (!on_device(r) || !on_device(omega) || !on_device(delta)) {
        g_cuda_err = "lbmg_learned_apply: r, omega and delta must be device pointers";
        return LBMG_INVALID_ARG;
    }
    LBMG_TRY(learned_ready(h, s));
    return learned_apply(h->c, r, ns, precision, omega, delta, s) ? LBMG_CUDA_ERROR : LBMG_OK;
}

int lbmg_get_dofs(lbmg_handle h, int d, int *corner, int *mintri) {
    LBMG_TRY(check_level(h, d));
    copy_dofs(h->c.host.lev[d], corner, mintri);
    return LBMG_OK;
}

int lbmg_get_matrix(lbmg_handle h, int d, int *rowptr, int *col, double *M, double *L) {
    LBMG_TRY(check_level(h, d));
    copy_pattern(h->c.host.lev[d], rowptr, col);
    if (M || L) {
        if (!h->c.assembled) return LBMG_NOT_ASSEMBLED;
        const DevLevel &dl = h->c.lev[d];
        if (M) LBMG_CK(cudaMemcpy(M, dl.M, dl.nnz * sizeof(double), cudaMemcpyDeviceToHost));
        if (L) LBMG_CK(cudaMemcpy(L, dl.L, dl.nnz * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return LBMG_OK;
}

int lbmg_get_prolongation(lbmg_handle h, int d, int *parents, double *weights) {
    LBMG_TRY(check_level(h, d));
    if (d == h->c.d0) return LBMG_INVALID_ARG;
    copy_prolongation(h->c.host.lev[d], parents, weights);
    return LBMG_OK;
}

int lbmg_host_build(const double *V, int nv, const int *F, int nt, int depth, const lbmg_options *opt,
                    lbmg_host_handle *out) {
    if (!out || !V || !F) return LBMG_INVALID_ARG;
    *out = nullptr;
    lbmg_options o;
    lbmg_default_options(&o);
    if (opt) o = *opt;
    LBMG_TRY(check_build_options(o));
    lbmg_host_ctx *h = new (std::nothrow) lbmg_host_ctx();
    if (!h) return LBMG_OUT_OF_MEMORY;
    const int st = build_single_host(V, nv, F, nt, depth, o, h->H);
    if (st != 0) {
        delete h;
        return st;
    }
    *out = h;
    return LBMG_OK;
}

int lbmg_host_build_batch(const double *const *V, const int *nv, const int *const *F, const int *nt,
                          const int *depth, int ninst, const lbmg_options *opt, lbmg_host_handle *out) {
    if (!out || !V || !nv || !F || !nt || !depth || ninst < 1) return LBMG_INVALID_ARG;
    *out = nullptr;
    lbmg_options o;
    lbmg_default_options(&o);
    if (opt) o = *opt;
    LBMG_TRY(check_batch_options(o));
    lbmg_host_ctx *h = new (std::nothrow) lbmg_host_ctx();
    if (!h) return LBMG_OUT_OF_MEMORY;
    const int st = build_batch_host(V, nv, F, nt, depth, ninst, o, h->H);
    if (st != 0) {
        delete h;
        return st;
    }
    *out = h;
    return LBMG_OK;
}

int lbmg_host_instances(lbmg_host_handle h, int *ninst, int *depth, int *min_depth) {
    if (!h) return LBMG_INVALID_ARG;
    if (ninst) *ninst = h->H.ninst;
    for (int i = 0; i < h->H.ninst; i++) {
        if (depth) depth[i] = h->H.inst_D[i];
        if (min_depth) min_depth[i] = h->H.inst_d0[i];
    }
    return LBMG_OK;
}

int lbmg_host_row_instances(lbmg_host_handle h, int d, int *inst) {
    if (!h || d < h->H.d0 || d > h->H.D) return LBMG_INVALID_ARG;
    const HostLevel &L = h->H.lev[d];
    if (inst) std::memcpy(inst, L.inst.data(), L.inst.size() * sizeof(int));
    return LBMG_OK;
}

void lbmg_host_destroy(lbmg_host_handle h) { delete h; }

int lbmg_host_levels(lbmg_host_handle h, int *min_depth, int *depth) {
    if (!h) return LBMG_INVALID_ARG;
    if (min_depth) *min_depth = h->H.d0;
    if (depth) *depth = h->H.D;
    return LBMG_OK;
}

int lbmg_host_level_info(lbmg_host_handle h, int d, long *ndof, long *nnz, long *nfrag) {
    if (!h || d < h->H.d0 || d > h->H.D) return LBMG_INVALID_ARG;
    const HostLevel &L = h->H.lev[d];
    if (ndof) *ndof = L.ndof;
    if (nnz) *nnz = L.rp.empty() ? 0 : (long)L.rp[L.ndof];
    if (nfrag) *nfrag = d == h->H.D ? h->H.nfrag : 0;
    return LBMG_OK;
}

int lbmg_host_get_dofs(lbmg_host_handle h, int d, int *corner, int *mintri) {
    if (!h || d < h->H.d0 || d > h->H.D) return LBMG_INVALID_ARG;
    copy_dofs(h->H.lev[d], corner, mintri);
    return LBMG_OK;
}

int lbmg_host_get_pattern(lbmg_host_handle h, int d, int *rowptr, int *col) {
    if (!h || d < h->H.d0 || d > h->H.D) return LBMG_INVALID_ARG;
    copy_pattern(h->H.lev[d], rowptr, col);
    return LBMG_OK;
}

int lbmg_host_get_prolongation(lbmg_host_handle h, int d, int *parents, double *weights) {
    if (!h || d <= h->H.d0 || d > h->H.D) return LBMG_INVALID_ARG;
    copy_prolongation(h->H.lev[d], parents, weights);
    return LBMG_OK;
}

}  // extern "C"
