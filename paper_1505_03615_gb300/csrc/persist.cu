// persist.cu -- the whole defect-correction solve (Chuang & Kazhdan, Section 4.3)
// in one cooperative kernel launch.
//
// Each V-cycle is a sequence of dependent phases (8 colours per Gauss-Seidel
// sweep, residual, restriction, prolongation on every level).  Launching each
// phase as its own kernel costs a launch gap per phase; here all blocks of a
// grid of one block per SM walk the phases together and meet at a grid barrier
// between them.  Levels with few rows ("narrow": the bottom of the hierarchy
// down to the dense coarse solve) run inside block 0 alone, separated by
// __syncthreads, while the other blocks wait at the next grid barrier.  The
// loop over cycles, the FP64 residual and its norms run in the same launch, so
// a whole solve is one launch and one read-back.
//
// Every wait is bounded: a barrier that does not complete within ~1 s sets the
// status word and every block returns.  Vectors written during the launch are
// read with L2-only loads (ld.global.cg) so that no SM uses a stale L1 line.
#include <vector>

#include "lbmg_internal.h"

namespace lbmg {

namespace {

constexpr int kG = 8;                 // threads per matrix row
constexpr unsigned long long kWaitNs = 1000000000ull;   // a barrier gives up after one second
constexpr unsigned long long kSpinCap = 1ull << 28;     // and in any case after this many polls

template <class T, int R>
__device__ __forceinline__ void ldcg_vec(const T *p, T (&v)[R]) {
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = __ldcg(p + r);
}
template <>
__device__ __forceinline__ void ldcg_vec<float, 4>(const float *p, float (&v)[4]) {
    const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void ldcg_vec<double, 2>(const double *p, double (&v)[2]) {
    const double2 q = __ldcg(reinterpret_cast<const double2 *>(p));
    v[0] = q.x; v[1] = q.y;
}
template <>
__device__ __forceinline__ void ldcg_vec<double, 4>(const double *p, double (&v)[4]) {
    const double2 q0 = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 q1 = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded grid barrier on a monotonic arrival counter bar[0] (zeroed before the
// launch): arrival k belongs to barrier k / expected, which completes when the
// counter reaches the next multiple of `expected` (gridDim.x, plus phantom
// participants when the bounded-wait path is being tested).  The arrival is a
// release, the polling an acquire, so the block's writes before the barrier
// are visible to every block after it.
__device__ bool grid_sync(unsigned *bar, int *status, unsigned expected) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
        const unsigned target = (old / expected + 1) * expected;
        const unsigned long long t0 = globaltimer();
        unsigned long long spins = 0;
        while ((int)(ld_acquire(bar) - target) < 0) {
            ++spins;
            if (((spins & 1023) == 0 && globaltimer() - t0 > kWaitNs) || spins > kSpinCap) {
                atomicExch(status, 1);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T, int R>
struct Lv {
    int n, ns, ncb;
    int cs[9];
    const int *cb;                  // this level's coarsest blocks: (level, mesh, first row, rows, inverse offset)
    const int *rp, *ci;
    const T *A, *dinv;
    const int *par;
    const int8_t *npl2;
    const int *crp;
    const uint32_t *cch;
    T *x, *b, *r;
};

struct Team { int tid, nthr; };

// row-group loop: every warp iterates the same number of times so that the
// group shuffles see all 32 lanes
template <class T, int R, class F>
__device__ __forceinline__ void for_rows(int r0, int r1, Team tm, F &&body) {
    const int g = tm.tid / kG, lane = tm.tid % kG, ng = tm.nthr / kG;
    const int warp_first = (tm.tid / 32) * (32 / kG);
    for (int base = r0 + warp_first; base < r1; base += ng) {
        const int row = base + (g - warp_first);
        body(row, row < r1, lane);
    }
}

template <class T, int R>
__device__ __forceinline__ void row_dot(const Lv<T, R> &L, int row, bool active, int lane, const T *x, T (&acc)[R]) {
#pragma unroll
    for (int q = 0; q < R; q++) acc[q] = T(0);
    if (active) {
        const int k1 = __ldg(L.rp + row + 1);
        for (int k = __ldg(L.rp + row) + lane; k < k1; k += kG) {
            const int j = __ldg(L.ci + k);
            const T a = __ldg(L.A + k);
            T v[R];
            ldcg_vec<T, R>(x + (size_t)j * R, v);
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] = fma(a, v[q], acc[q]);
        }
    }
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < R; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o, kG);
}

template <class T, int R>
__device__ void gs_colour(const Lv<T, R> &L, int c, Team tm) {
    const T *dv = L.dinv;
    for_rows<T, R>(L.cs[c], L.cs[c + 1], tm, [&](int row, bool active, int lane) {
        T acc[R];
        row_dot<T, R>(L, row, active, lane, L.x, acc);
        if (active && lane == 0) {
            const T d = __ldg(dv + row);
            T bv[R], xv[R];
            ldcg_vec<T, R>(L.b + (size_t)row * R, bv);
            ldcg_vec<T, R>(L.x + (size_t)row * R, xv);
#pragma unroll
            for (int q = 0; q < R; q++) L.x[(size_t)row * R + q] = xv[q] + (bv[q] - acc[q]) * d;
        }
    });
}

template <class T, int R>
__device__ void residual(const Lv<T, R> &L, Team tm) {
    for_rows<T, R>(0, L.ns, tm, [&](int row, bool active, int lane) {
        T acc[R];
        row_dot<T, R>(L, row, active, lane, L.x, acc);
        if (active && lane == 0) {
            T bv[R];
            ldcg_vec<T, R>(L.b + (size_t)row * R, bv);
#pragma unroll
            for (int q = 0; q < R; q++) L.r[(size_t)row * R + q] = bv[q] - acc[q];
        }
    });
}

// b_c = P^T r_f, x_c = 0
template <class T, int R>
__device__ void restrict_to(const Lv<T, R> &Lc, const T *rf, Team tm) {
    for (int J = tm.tid; J < Lc.n; J += tm.nthr) {
        T acc[R];
#pragma unroll
        for (int q = 0; q < R; q++) acc[q] = T(0);
        for (int k = __ldg(Lc.crp + J); k < __ldg(Lc.crp + J + 1); k++) {
            const uint32_t e = __ldg(Lc.cch + k);
            const T w = T(1) / T(1u << (e >> kPackShift));
            T v[R];
            ldcg_vec<T, R>(rf + (size_t)(e & kPackMask) * R, v);
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] = fma(w, v[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < R; q++) { Lc.b[(size_t)J * R + q] = acc[q]; Lc.x[(size_t)J * R + q] = T(0); }
    }
}

// x_f += P x_c
template <class T, int R>
__device__ void prolong_from(const Lv<T, R> &Lf, const T *xc, Team tm) {
    for (int i = tm.tid; i < Lf.ns; i += tm.nthr) {
        const int np = 1 << __ldg(Lf.npl2 + i);
        T acc[R], v[R], xv[R];
#pragma unroll
        for (int q = 0; q < R; q++) acc[q] = T(0);
        for (int p = 0; p < np; p++) {
            ldcg_vec<T, R>(xc + (size_t)__ldg(Lf.par + 8 * (size_t)i + p) * R, v);
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] += v[q];
        }
        ldcg_vec<T, R>(Lf.x + (size_t)i * R, xv);
        const T w = T(1) / T(np);
#pragma unroll
        for (int q = 0; q < R; q++) Lf.x[(size_t)i * R + q] = xv[q] + w * acc[q];
    }
}

// x = inv b on each coarsest block of a level; a team takes blocks first..first+count-1 by stride
template <class T, int R>
__device__ void coarse_apply(const Lv<T, R> &L, const T *inv, int first, int stride, Team tm) {
    const int warp = tm.tid >> 5, lane = tm.tid & 31, nw = tm.nthr >> 5;
    for (int k = first; k < L.ncb; k += stride) {
        const int *cb = L.cb + 5 * k;
        const int row0 = cb[2], n = cb[3];
        const T *M = inv + cb[4];
        for (int row = warp; row < n; row += nw) {
            T acc[R];
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] = T(0);
            for (int j = lane; j < n; j += 32) {
                const T a = __ldg(M + (size_t)row * n + j);
                T v[R];
                ldcg_vec<T, R>(L.b + (size_t)(row0 + j) * R, v);
#pragma unroll
                for (int q = 0; q < R; q++) acc[q] = fma(a, v[q], acc[q]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < R; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < R; q++) L.x[(size_t)(row0 + row) * R + q] = acc[q];
        }
    }
}

// The bottom of a V-cycle, levels dn..d0, inside one block: b at level dn is given and its x
// is zero (or dn is the coarsest level); on return x at dn holds the correction.
template <class T, int R>
__device__ void narrow_cycle(const Lv<T, R> *lev, int dn, int d0, int nu1, int nu2, const T *cinv, Team blk) {
    for (int d = dn; d >= d0; d--) {
        const Lv<T, R> &L = lev[d];
        if (L.ncb > 0) { coarse_apply<T, R>(L, cinv, 0, 1, blk); __syncthreads(); }
        if (d == d0) break;
        for (int s = 0; s < nu1; s++)
            for (int c = 0; c < 8; c++) { gs_colour<T, R>(L, c, blk); __syncthreads(); }
        residual<T, R>(L, blk);
        __syncthreads();
        restrict_to<T, R>(lev[d - 1], L.r, blk);
        __syncthreads();
    }
    for (int d = d0 + 1; d <= dn; d++) {
        const Lv<T, R> &L = lev[d];
        prolong_from<T, R>(L, lev[d - 1].x, blk);
        __syncthreads();
        for (int s = 0; s < nu2; s++)
            for (int c = 7; c >= 0; c--) { gs_colour<T, R>(L, c, blk); __syncthreads(); }
    }
}

template <class T, int R>
__global__ void __launch_bounds__(1024, 1) narrow_cycle_kernel(const void *lev, int dn, int d0, int nu1, int nu2,
                                                               const void *cinv) {
    narrow_cycle<T, R>(reinterpret_cast<const Lv<T, R> *>(lev), dn, d0, nu1, nu2, reinterpret_cast<const T *>(cinv),
                       Team{(int)threadIdx.x, (int)blockDim.x});
}

}  // namespace

struct PersistParams {
    int D, d0, dn, nu1, nu2, max_cycles, nrhs;
    double tol2;
    const void *lev;          // Lv<T,R>[kMaxDepth+1] in device memory
    const void *cinv;
    // finest FP64 state
    const int *rpF, *ciF;
    const double *A64F, *bs;
    double *xs, *rs;
    const int *items;         // norm work items (mesh, first row, end row)
    int nitems, ninst;
    double *part;             // [nitems][8]
    double *norm;             // [ninst][16]: ||r||^2, ||b||^2, initial ||r||^2, previous ||r||^2 (4 each)
    unsigned *bar;
    unsigned expected;        // arrivals that complete a barrier
    int *status;
    int *cycles;
    unsigned long long *smooth_ns;
};

template <class T, int R>
__global__ void __launch_bounds__(1024, 1) solve_persistent_kernel(PersistParams p) {
    const Lv<T, R> *lev = reinterpret_cast<const Lv<T, R> *>(p.lev);
    const Team grid{(int)(blockIdx.x * blockDim.x + threadIdx.x), (int)(gridDim.x * blockDim.x)};
    const Team blk{(int)threadIdx.x, (int)blockDim.x};
    const bool b0 = blockIdx.x == 0;
    unsigned long long t_smooth = 0;

    // per-mesh norms of the FP64 residual rs (and, the first time, of bs): one warp per
    // work item (a chunk of the rows of one mesh and colour), then block 0 adds the
    // items of each mesh in order, so the sums do not depend on timing
    auto norms = [&](bool with_b) -> bool {
        const int warp = grid.tid >> 5, lane = grid.tid & 31, nw = grid.nthr >> 5;
        for (int it = warp; it < p.nitems; it += nw) {
            const int r0 = __ldg(p.items + 3 * it + 1), r1 = __ldg(p.items + 3 * it + 2);
            double acc[8];
#pragma unroll
            for (int q = 0; q < 8; q++) acc[q] = 0.0;
            for (int i = r0 + lane; i < r1; i += 32)
#pragma unroll
                for (int q = 0; q < R; q++) {
                    const double rv = __ldcg(p.rs + (size_t)i * R + q);
                    acc[q] = fma(rv, rv, acc[q]);
                    if (with_b) { const double bv = p.bs[(size_t)i * R + q]; acc[4 + q] = fma(bv, bv, acc[4 + q]); }
                }
#pragma unroll
            for (int q = 0; q < 8; q++)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (lane < 8) {
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < 8; q++) if (q == lane) v = acc[q];
                p.part[8 * (size_t)it + lane] = v;
            }
        }
        if (!grid_sync(p.bar, p.status, p.expected)) return false;
        if (b0) {
            for (int k = threadIdx.x; k < p.ninst * 8; k += blockDim.x) {
                const int m = k >> 3, q = k & 7;
                if (q >= 4 && !with_b) continue;
                double s = 0.0;
                for (int it = 0; it < p.nitems; it++)
                    if (__ldg(p.items + 3 * it) == m) s += __ldcg(p.part + 8 * (size_t)it + q);
                if (q < 4) {
                    const double prev = p.norm[16 * m + q];
                    p.norm[16 * m + 12 + q] = prev;
                }
                p.norm[16 * m + q] = s;
            }
        }
        return grid_sync(p.bar, p.status, p.expected);
    };

    // r = b - A x at the finest level (FP64)
    auto fine_residual = [&]() {
        for_rows<double, R>(0, lev[p.D].n, grid, [&](int row, bool active, int lane) {
            double acc[R];
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] = 0.0;
            if (active) {
                const int k1 = __ldg(p.rpF + row + 1);
                for (int k = __ldg(p.rpF + row) + lane; k < k1; k += kG) {
                    const int j = __ldg(p.ciF + k);
                    const double a = __ldg(p.A64F + k);
                    double v[R];
                    ldcg_vec<double, R>(p.xs + (size_t)j * R, v);
#pragma unroll
                    for (int q = 0; q < R; q++) acc[q] = fma(a, v[q], acc[q]);
                }
            }
#pragma unroll
            for (int o = kG / 2; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < R; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o, kG);
            if (active && lane == 0)
#pragma unroll
                for (int q = 0; q < R; q++) p.rs[(size_t)row * R + q] = p.bs[(size_t)row * R + q] - acc[q];
        });
    };

    fine_residual();
    if (!grid_sync(p.bar, p.status, p.expected)) return;
    if (!norms(true)) return;
    if (b0)
        for (int k = threadIdx.x; k < p.ninst * 4; k += blockDim.x)
            p.norm[16 * (k >> 2) + 8 + (k & 3)] = __ldcg(p.norm + 16 * (k >> 2) + (k & 3));
    if (!grid_sync(p.bar, p.status, p.expected)) return;

    int cyc = 0;
    for (;; cyc++) {
        bool done = true, bad = false;
        for (int m = 0; m < p.ninst; m++)
            for (int q = 0; q < p.nrhs; q++) {
                const double r2 = __ldcg(p.norm + 16 * m + q), b2 = __ldcg(p.norm + 16 * m + 4 + q);
                // relative to ||b||; a zero right-hand side is judged by the absolute residual
                if (!(r2 <= p.tol2 * (b2 > 0.0 ? b2 : 1.0))) done = false;
                if (!(r2 <= 1e300) || r2 > 1e12 * __ldcg(p.norm + 16 * m + 8 + q) + 1e-300) bad = true;   // NaN, inf or growth by 1e6
            }
        if (bad) { if (b0 && threadIdx.x == 0) atomicExch(p.status, 2); break; }
        if (done || cyc >= p.max_cycles) break;
        // b_D = T(r), x_D = 0
        {
            const Lv<T, R> &F = lev[p.D];
            for (int q = grid.tid; q < F.n * R; q += grid.nthr) { F.b[q] = (T)__ldcg(p.rs + q); F.x[q] = T(0); }
        }
        if (!grid_sync(p.bar, p.status, p.expected)) return;
        // down the wide levels (all blocks); dn < d0 means there are no narrow levels
        const int dw = p.dn >= p.d0 ? p.dn + 1 : p.d0;
        for (int d = p.D; d >= dw; d--) {
            const Lv<T, R> &L = lev[d];
            if (L.ncb > 0) {
                coarse_apply<T, R>(L, reinterpret_cast<const T *>(p.cinv), blockIdx.x, gridDim.x, blk);
                if (!grid_sync(p.bar, p.status, p.expected)) return;
            }
            if (d == p.d0) break;
            const unsigned long long t0 = (d == p.D && b0 && threadIdx.x == 0) ? globaltimer() : 0;
            for (int s = 0; s < p.nu1; s++)
                for (int c = 0; c < 8; c++) {
                    if (L.cs[c + 1] == L.cs[c]) continue;
                    gs_colour<T, R>(L, c, grid);
                    if (!grid_sync(p.bar, p.status, p.expected)) return;
                }
            if (d == p.D && b0 && threadIdx.x == 0) t_smooth += globaltimer() - t0;
            residual<T, R>(L, grid);
            if (!grid_sync(p.bar, p.status, p.expected)) return;
            restrict_to<T, R>(lev[d - 1], L.r, grid);
            if (!grid_sync(p.bar, p.status, p.expected)) return;
        }
        // the narrow levels, block 0 alone
        if (p.dn >= p.d0) {
            if (b0) narrow_cycle<T, R>(lev, p.dn, p.d0, p.nu1, p.nu2, reinterpret_cast<const T *>(p.cinv), blk);
            if (!grid_sync(p.bar, p.status, p.expected)) return;
        }
        // up the wide levels
        for (int d = dw > p.d0 ? dw : p.d0 + 1; d <= p.D; d++) {
            const Lv<T, R> &L = lev[d];
            prolong_from<T, R>(L, lev[d - 1].x, grid);
            if (!grid_sync(p.bar, p.status, p.expected)) return;
            const unsigned long long t0 = (d == p.D && b0 && threadIdx.x == 0) ? globaltimer() : 0;
            for (int s = 0; s < p.nu2; s++)
                for (int c = 7; c >= 0; c--) {
                    if (L.cs[c + 1] == L.cs[c]) continue;
                    gs_colour<T, R>(L, c, grid);
                    if (!grid_sync(p.bar, p.status, p.expected)) return;
                }
            if (d == p.D && b0 && threadIdx.x == 0) t_smooth += globaltimer() - t0;
        }
        // x += e (FP64), r = b - A x, norms
        {
            const Lv<T, R> &F = lev[p.D];
            for (int q = grid.tid; q < F.n * R; q += grid.nthr) p.xs[q] = __ldcg(p.xs + q) + (double)__ldcg(F.x + q);
        }
        if (!grid_sync(p.bar, p.status, p.expected)) return;
        fine_residual();
        if (!grid_sync(p.bar, p.status, p.expected)) return;
        if (!norms(false)) return;
    }
    if (b0 && threadIdx.x == 0) {
        *p.cycles = cyc;
        *p.smooth_ns = t_smooth;
    }
}

// host side -------------------------------------------------------------------

template <class T, int R>
static int launch_persist_t(const PersistParams &prm, int blocks, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, solve_persistent_kernel<T, R>, prm);
    return e == cudaSuccess ? 0 : (int)e;
}

size_t persist_view_bytes() { return sizeof(Lv<double, 4>) * (kMaxDepth + 1); }

// fill the per-level view table for precision T and stride R on the host
template <class T, int R>
static void fill_views(const Ctx &c, std::vector<char> &buf) {
    buf.assign(sizeof(Lv<T, R>) * (kMaxDepth + 1), 0);
    Lv<T, R> *v = reinterpret_cast<Lv<T, R> *>(buf.data());
    for (int d = c.d0; d <= c.D; d++) {
        const DevLevel &L = c.lev[d];
        Lv<T, R> &o = v[d];
        o.n = L.n;
        o.ns = L.ns;
        o.ncb = L.ncb;
        o.cb = c.cblk + 5 * L.cb0;
        for (int q = 0; q < 9; q++) o.cs[q] = L.cs[q];
        o.rp = L.rp; o.ci = L.ci;
        if constexpr (sizeof(T) == 4) {
            o.A = (const T *)L.A32; o.dinv = (const T *)L.dinv32;
            o.x = (T *)L.x32; o.b = (T *)L.b32; o.r = (T *)L.r32;
        } else {
            o.A = (const T *)L.A64; o.dinv = (const T *)L.dinv64;
            o.x = (T *)L.x64; o.b = (T *)L.b64; o.r = (T *)L.r64;
        }
        o.par = L.par; o.npl2 = L.npl2; o.crp = L.crp; o.cch = L.cch;
    }
}

// one block per launch: the bottom levels of a V-cycle from level `top` (graph path)
void launch_narrow_cycle(const Ctx &c, int precision, int R, int top, cudaStream_t s) {
    const void *views = precision == 1 ? c.views32 : c.views64;
    const void *inv = precision == 1 ? (const void *)c.cinv32 : (const void *)c.cinv64;
    if (precision == 1) {
        if (R == 1) narrow_cycle_kernel<float, 1><<<1, 1024, 0, s>>>(views, top, c.d0, c.nu1, c.nu2, inv);
        else if (R == 2) narrow_cycle_kernel<float, 2><<<1, 1024, 0, s>>>(views, top, c.d0, c.nu1, c.nu2, inv);
        else narrow_cycle_kernel<float, 4><<<1, 1024, 0, s>>>(views, top, c.d0, c.nu1, c.nu2, inv);
    } else {
        if (R == 1) narrow_cycle_kernel<double, 1><<<1, 1024, 0, s>>>(views, top, c.d0, c.nu1, c.nu2, inv);
        else if (R == 2) narrow_cycle_kernel<double, 2><<<1, 1024, 0, s>>>(views, top, c.d0, c.nu1, c.nu2, inv);
        else narrow_cycle_kernel<double, 4><<<1, 1024, 0, s>>>(views, top, c.d0, c.nu1, c.nu2, inv);
    }
}

int narrow_views_setup(Ctx &c) {
    std::vector<char> buf;
    fill_views<float, 4>(c, buf);
    if (cudaMemcpy(c.views32, buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return 1;
    fill_views<double, 4>(c, buf);
    if (cudaMemcpy(c.views64, buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return 1;
    return 0;
}

int persist_setup(Ctx &c) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_persistent_kernel<float, 4>, 1024, 0) != cudaSuccess)
        return 1;
    if (per_sm < 1) return 1;
    int pd = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pd, solve_persistent_kernel<double, 4>, 1024, 0);
    if (pd < 1) return 1;
    c.persist_blocks = sms;   // one block per SM
    // narrow levels: the bottom range whose every level has at most persist_narrow rows
    // narrow levels: the bottom range whose every level has at most persist_narrow rows
    // (persist_dn = d0 - 1: none, the bottom level itself is handled by all blocks)
    c.persist_dn = c.d0 - 1;
    for (int d = c.d0; d <= c.D; d++) {
        if (c.lev[d].n <= c.persist_narrow) c.persist_dn = d; else break;
    }
    return 0;
}

int persist_solve(Ctx &c, int precision, int R, int nrhs, double tol, int max_cycles, cudaStream_t s) {
    std::vector<char> buf;
    const bool f32 = precision == 1;
    if (f32) {
        if (R == 1) fill_views<float, 1>(c, buf); else if (R == 2) fill_views<float, 2>(c, buf); else fill_views<float, 4>(c, buf);
    } else {
        if (R == 1) fill_views<double, 1>(c, buf); else if (R == 2) fill_views<double, 2>(c, buf); else fill_views<double, 4>(c, buf);
    }
    if (buf.size() > c.persist_view_bytes) return 1;
    cudaError_t e = cudaMemcpyAsync(c.persist_views, buf.data(), buf.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return (int)e;
    cudaMemsetAsync(c.persist_state, 0, 64, s);
    PersistParams prm;
    prm.D = c.D; prm.d0 = c.d0; prm.dn = c.persist_dn; prm.nu1 = c.nu1; prm.nu2 = c.nu2;
    prm.max_cycles = max_cycles; prm.nrhs = nrhs; prm.tol2 = tol * tol;
    prm.lev = c.persist_views;
    prm.cinv = f32 ? (const void *)c.cinv32 : (const void *)c.cinv64;
    prm.rpF = c.lev[c.D].rp; prm.ciF = c.lev[c.D].ci; prm.A64F = c.lev[c.D].A64;
    prm.bs = c.bs; prm.xs = c.xs; prm.rs = c.rs;
    prm.items = c.nitem;
    prm.nitems = c.nnitem;
    prm.ninst = c.ninst;
    prm.part = c.item_part;
    prm.norm = c.inst_norm;
    unsigned char *st = reinterpret_cast<unsigned char *>(c.persist_state);
    prm.bar = reinterpret_cast<unsigned *>(st);
    prm.expected = (unsigned)(c.persist_blocks + c.barrier_phantoms);
    prm.status = reinterpret_cast<int *>(st + 16);
    prm.cycles = reinterpret_cast<int *>(st + 20);
    prm.smooth_ns = reinterpret_cast<unsigned long long *>(st + 24);
    const int B = c.persist_blocks;
    if (f32) {
        if (R == 1) return launch_persist_t<float, 1>(prm, B, s);
        if (R == 2) return launch_persist_t<float, 2>(prm, B, s);
        return launch_persist_t<float, 4>(prm, B, s);
    }
    if (R == 1) return launch_persist_t<double, 1>(prm, B, s);
    if (R == 2) return launch_persist_t<double, 2>(prm, B, s);
    return launch_persist_t<double, 4>(prm, B, s);
}

}  // namespace lbmg
