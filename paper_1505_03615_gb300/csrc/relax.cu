// relax.cu -- multigrid kernels of the V-cycle (Chuang & Kazhdan, Sections 4.3
// and 5.2): coloured Gauss-Seidel and weighted-Jacobi relaxation, residual,
// restriction P^T r, prolongation x += P e, the coarsest-level dense solve, and
// small vector kernels.  Vectors are row-major [n][R], R in {1, 2, 4}.
//
// Rows of one colour (one corner parity class) never couple, because supports
// of equal-parity corners are disjoint and the components of one corner are
// disjoint, so a colour is relaxed in parallel with exact Gauss-Seidel updates.
// A group of G threads shares one matrix row.
#include <algorithm>

#include "lbmg_internal.h"

namespace lbmg {

template <class T, int R>
__device__ __forceinline__ void load_vec(const T *__restrict__ p, T (&v)[R]) {
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = p[r];
}
template <>
__device__ __forceinline__ void load_vec<float, 4>(const float *__restrict__ p, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void load_vec<double, 2>(const double *__restrict__ p, double (&v)[2]) {
    const double2 q = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = q.x; v[1] = q.y;
}
template <>
__device__ __forceinline__ void load_vec<double, 4>(const double *__restrict__ p, double (&v)[4]) {
    const double2 q0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 q1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// x may be written by other rows of the same launch only at rows of the same
// colour, which this row never reads, so plain (non-__ldg) loads are not needed
// for correctness; __ldg is avoided anyway for x because the GS kernel writes it.
template <class T, int R>
__device__ __forceinline__ void load_x(const T *p, T (&v)[R]) {
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = p[r];
}

// The static part of a matrix row (pattern and values) is loaded before the
// kernel waits for its predecessor: each of the G threads of a row keeps its first
// P entries in registers, so after the wait only the x gathers remain.
template <class T, int G>
struct RowPrefetch {
    static constexpr int P = 32 / G;
    int k = 0, k1 = 0;
    int j[P];
    T a[P];
    __device__ __forceinline__ void load(int row, bool active, int lane, const int *__restrict__ rp,
                                         const int *__restrict__ ci, const T *__restrict__ A) {
        if (active) { k = __ldg(rp + row) + lane; k1 = __ldg(rp + row + 1); }
#pragma unroll
        for (int q = 0; q < P; q++) {
            const int kk = k + q * G;
            if (kk < k1) { j[q] = __ldg(ci + kk); a[q] = __ldg(A + kk); }
            else { j[q] = -1; a[q] = T(0); }
        }
    }
    template <int R>
    __device__ __forceinline__ void dot(const int *__restrict__ ci, const T *__restrict__ A, const T *x,
                                        T (&acc)[R]) const {
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = T(0);
#pragma unroll
        for (int q = 0; q < P; q++) {
            if (j[q] >= 0) {
                T xv[R];
                load_x<T, R>(x + (size_t)j[q] * R, xv);
#pragma unroll
                for (int r = 0; r < R; r++) acc[r] = fma(a[q], xv[r], acc[r]);
            }
        }
        for (int kk = k + P * G; kk < k1; kk += G) {
            const int jj = __ldg(ci + kk);
            const T aa = __ldg(A + kk);
            T xv[R];
            load_x<T, R>(x + (size_t)jj * R, xv);
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] = fma(aa, xv[r], acc[r]);
        }
    }
};

template <class T, int R, int G>
__device__ __forceinline__ void group_sum(T (&acc)[R]) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o, G);
}

template <class T, int R, int G>
__global__ void __launch_bounds__(512) smooth_colour_kernel(int r0, int r1, const int *__restrict__ rp,
                                                            const int *__restrict__ ci, const T *__restrict__ A,
                                                            const T *__restrict__ dinv, const T *__restrict__ b, T *x) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = r0 + tid / G, lane = tid % G;
    const bool active = row < r1;
    RowPrefetch<T, G> pf;
    pf.load(row, active, lane, rp, ci, A);
    const T d = (active && lane == 0) ? __ldg(dinv + row) : T(0);
    grid_dep_wait();
    grid_dep_launch();
    T acc[R];
    pf.template dot<R>(ci, A, x, acc);
    group_sum<T, R, G>(acc);
    if (active && lane == 0) {
#pragma unroll
        for (int r = 0; r < R; r++) x[(size_t)row * R + r] += (b[(size_t)row * R + r] - acc[r]) * d;
    }
}

template <class T, int R, int G>
__global__ void __launch_bounds__(512) residual_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const T *__restrict__ A, const T *__restrict__ b,
                                                       const T *x, T *__restrict__ r) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = tid / G, lane = tid % G;
    const bool active = row < n;
    RowPrefetch<T, G> pf;
    pf.load(row, active, lane, rp, ci, A);
    grid_dep_wait();
    grid_dep_launch();
    T acc[R];
    pf.template dot<R>(ci, A, x, acc);
    group_sum<T, R, G>(acc);
    if (active && lane == 0) {
#pragma unroll
        for (int q = 0; q < R; q++) r[(size_t)row * R + q] = b[(size_t)row * R + q] - acc[q];
    }
}

// kernel instance for (R, threads per row); nullptr for an unsupported pair
template <class T>
using SmoothFn = void (*)(int, int, const int *, const int *, const T *, const T *, const T *, T *);
template <class T>
using ResidualFn = void (*)(int, const int *, const int *, const T *, const T *, const T *, T *);

template <class T, int R>
SmoothFn<T> smooth_fn(int tpr) {
    switch (tpr) {
        case 4: return smooth_colour_kernel<T, R, 4>;
        case 8: return smooth_colour_kernel<T, R, 8>;
        case 16: return smooth_colour_kernel<T, R, 16>;
        default: return nullptr;
    }
}
template <class T, int R>
ResidualFn<T> residual_fn(int tpr) {
    switch (tpr) {
        case 4: return residual_kernel<T, R, 4>;
        case 8: return residual_kernel<T, R, 8>;
        case 16: return residual_kernel<T, R, 16>;
        default: return nullptr;
    }
}

template <class T>
void launch_sweeps(const Ctx &c, const DevLevel &L, int sweeps, bool forward, const T *A, const T *dinv, const T *b,
                   T *x, int R, cudaStream_t s, Chain *ch, int skip) {
    if (sweeps <= 0) return;
    skip = std::max(0, std::min(skip, 8));
    const LaunchShape &sh = L.shape[sizeof(T) == 8][kShapeSmooth];
    if (sizeof(T) == 4 && sh.tpb == kSweepShapeTpb && 8 * sweeps <= 32 && c.sweep_bar && A == (const T *)L.A32) {
        int seq[32];
        for (int q = skip; q < 8 * sweeps; q++) seq[q - skip] = forward ? q % 8 : 7 - q % 8;
        const int blocks = sh.grid > 0 && sh.grid < c.sweep_blocks[R] ? sh.grid : c.sweep_blocks[R];
        if (ch) ch->cut();   // a cooperative launch takes no programmatic serialisation
        if (launch_packed_sweep(L, seq, 8 * sweeps - skip, (const float *)dinv, (const float *)b, (float *)x, R,
                                c.sweep_bar, c.narrow.status, blocks, s))
            return;
        cudaGetLastError();   // refused: the per-colour launches below
    }
    for (int sw = 0; sw < sweeps; sw++)
        for (int q = sw == 0 ? skip : 0; q < 8; q++) {
            const int colour = forward ? q : 7 - q;
            // the colour that follows on this level: the next of this sweep, or the first of the next sweep
            const int nq = q < 7 ? q + 1 : (sw + 1 < sweeps ? 0 : -1);
            const int next = nq < 0 ? -1 : (forward ? nq : 7 - nq);
            launch_smooth_colour<T>(L, colour, A, dinv, b, x, R, s, ch, next);
        }
}

template <class T>
void launch_smooth_colour(const DevLevel &L, int colour, const T *A, const T *dinv, const T *b, T *x, int R,
                          cudaStream_t s, Chain *ch, int next) {
    const int r0 = L.cs[colour], r1 = L.cs[colour + 1];
    if (r1 <= r0) return;
    const LaunchShape &sh = L.shape[sizeof(T) == 8][kShapeSmooth];
    // four threads per row: the packed copy of the matrix (one 256-byte load per warp and quad)
    const int tpb = sh.tpb == kSweepShapeTpb ? 256 : sh.tpb;   // one colour of a whole-sweep level
    if (sh.tpr == 4 && launch_packed_smooth<T>(L, colour, A, dinv, b, x, R, tpb, s, ch, next)) return;
    const unsigned blocks = (unsigned)(((int64_t)(r1 - r0) * sh.tpr + tpb - 1) / tpb);
    const SmoothFn<T> k = R == 1 ? smooth_fn<T, 1>(sh.tpr) : R == 2 ? smooth_fn<T, 2>(sh.tpr) : smooth_fn<T, 4>(sh.tpr);
    klaunch(k, blocks, (unsigned)tpb, 0, s, ch, r0, r1, L.rp, L.ci, A, dinv, b, x);
}

template <class T>
void launch_residual(const DevLevel &L, const T *A, const T *b, const T *x, T *r, int R, cudaStream_t s, int nrows,
                     Chain *ch) {
    const int n = nrows < 0 ? L.n : nrows;
    if (n == 0) return;
    const LaunchShape &sh = L.shape[sizeof(T) == 8][kShapeResidual];
    if (sh.tpr == 4 && launch_packed_residual<T>(L, A, b, x, r, R, n, sh.tpb, s, ch)) return;
    const unsigned blocks = (unsigned)(((int64_t)n * sh.tpr + sh.tpb - 1) / sh.tpb);
    const ResidualFn<T> k =
        R == 1 ? residual_fn<T, 1>(sh.tpr) : R == 2 ? residual_fn<T, 2>(sh.tpr) : residual_fn<T, 4>(sh.tpr);
    klaunch(k, blocks, (unsigned)sh.tpb, 0, s, ch, n, L.rp, L.ci, A, b, x, r);
}

template <class T>
__global__ void jacobi_update_kernel(int n, int R, const T *__restrict__ dinv, const T *__restrict__ r, T *x, T omega) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * R) return;
    x[q] += omega * dinv[q / R] * r[q];
}

template <class T>
void launch_jacobi_update(const DevLevel &L, const T *dinv, const T *r, T *x, T omega, int R, cudaStream_t s) {
    const int64_t m = (int64_t)L.ns * R;
    if (m == 0) return;
    jacobi_update_kernel<T><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(L.ns, R, dinv, r, x, omega);
}

// b_c[J] = sum over fine children i of J of r_f[i] / #parents(i); x_c[J] = 0 when x_c is given.
// The first kPreChildren entries of the static child list are loaded before the
// grid-dependency wait, so after it only the residual gathers remain, all in flight
// together.
constexpr int kPreChildren = 16;

template <class T, int R>
__global__ void restrict_kernel(int nc, const int *__restrict__ crp, const uint32_t *__restrict__ cch,
                                const T *__restrict__ rf, T *__restrict__ bc, T *__restrict__ xc,
                                const T *__restrict__ dinv, int c1) {
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = J < nc;
    int k0 = 0, k1 = 0;
    uint32_t e[kPreChildren];
    if (active) { k0 = __ldg(crp + J); k1 = __ldg(crp + J + 1); }
    // colour 0 (rows [0, c1)) of the first sweep, fused: its inverse diagonal
    const T d = (active && dinv && J < c1) ? __ldg(dinv + J) : T(0);
#pragma unroll
    for (int u = 0; u < kPreChildren; u++) e[u] = k0 + u < k1 ? __ldg(cch + k0 + u) : 0u;
    grid_dep_wait();
    grid_dep_launch();
    if (!active) return;
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = T(0);
    auto child = [&](uint32_t ek) {
        const T w = T(1) / T(1u << (ek >> kPackShift));
        T v[R];
        load_x<T, R>(rf + (size_t)(ek & kPackMask) * R, v);
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = fma(w, v[r], acc[r]);
    };
#pragma unroll
    for (int u = 0; u < kPreChildren; u++)
        if (k0 + u < k1) child(e[u]);
    for (int k = k0 + kPreChildren; k < k1; k++) child(__ldg(cch + k));
#pragma unroll
    for (int r = 0; r < R; r++) bc[(size_t)J * R + r] = acc[r];
    if (xc) {
        if (dinv && J < c1) {
            // the colour kernels' step x = x + (b - A x) / a_ii with x = 0 (so A x = +0): 0 + b d
#pragma unroll
            for (int r = 0; r < R; r++) xc[(size_t)J * R + r] = T(0) + (acc[r] - T(0)) * d;
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) xc[(size_t)J * R + r] = T(0);
        }
    }
}

template <class T>
void launch_restrict(const DevLevel &Lc, const T *rf, T *bc, int R, cudaStream_t s, T *xc, Chain *ch,
                     bool first_colour) {
    if (Lc.n == 0) return;
    const unsigned blocks = (unsigned)((Lc.n + 255) / 256);
    auto k = R == 1 ? restrict_kernel<T, 1> : R == 2 ? restrict_kernel<T, 2> : restrict_kernel<T, 4>;
    const T *dinv = first_colour && xc ? (sizeof(T) == 4 ? (const T *)Lc.dinv32 : (const T *)Lc.dinv64) : nullptr;
    klaunch(k, blocks, 256u, 0, s, ch, Lc.n, Lc.crp, Lc.cch, rf, bc, xc, dinv, dinv ? Lc.cs[1] : 0);
}

// x_f[i] += (sum of parent values) / #parents(i)
template <class T, int R>
__global__ void prolong_add_kernel(int nf, const int *__restrict__ par, const int8_t *__restrict__ npl2,
                                   const T *__restrict__ xc, T *__restrict__ xf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < nf;
    int np = 0, p[8];
    if (active) {
        np = 1 << __ldg(npl2 + i);
#pragma unroll
        for (int q = 0; q < 8; q++) p[q] = q < np ? __ldg(par + 8 * (size_t)i + q) : 0;
    }
    grid_dep_wait();
    grid_dep_launch();
    if (!active) return;
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = T(0);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if (q < np) {
            T v[R];
            load_x<T, R>(xc + (size_t)p[q] * R, v);
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] += v[r];
        }
    }
    const T w = T(1) / T(np);
#pragma unroll
    for (int r = 0; r < R; r++) xf[(size_t)i * R + r] += w * acc[r];
}

template <class T>
void launch_prolong_add(const DevLevel &Lf, const T *xc, T *xf, int R, cudaStream_t s, Chain *ch) {
    if (Lf.ns == 0) return;   // only smoothed rows have a coarser level
    const unsigned blocks = (unsigned)((Lf.ns + 255) / 256);
    auto k = R == 1 ? prolong_add_kernel<T, 1> : R == 2 ? prolong_add_kernel<T, 2> : prolong_add_kernel<T, 4>;
    klaunch(k, blocks, 256u, 0, s, ch, Lf.ns, Lf.par, Lf.npl2, xc, xf);
}

// x = inv * b on every coarsest block of a level (one block per mesh), one warp per row
template <class T, int R>
__global__ void coarse_apply_kernel(const int *__restrict__ cblk, const T *__restrict__ inv, const T *__restrict__ b,
                                    T *__restrict__ x) {
    const int *cb = cblk + 5 * blockIdx.x;
    const int row0 = cb[2], n = cb[3];
    const T *M = inv + cb[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    grid_dep_wait();
    grid_dep_launch();
    for (int row = warp; row < n; row += nw) {
        T acc[R];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = T(0);
        for (int j = lane; j < n; j += 32) {
            const T a = M[(size_t)row * n + j];
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] = fma(a, b[(size_t)(row0 + j) * R + r], acc[r]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < R; r++) x[(size_t)(row0 + row) * R + r] = acc[r];
        }
    }
}

template <class T>
void launch_coarse_apply(const Ctx &c, const DevLevel &L, const T *inv, const T *b, T *x, int R, cudaStream_t s,
                         Chain *ch) {
    if (L.ncb == 0) return;
    const int *cb = c.cblk + 5 * L.cb0;
    auto k = R == 1 ? coarse_apply_kernel<T, 1> : R == 2 ? coarse_apply_kernel<T, 2> : coarse_apply_kernel<T, 4>;
    klaunch(k, (unsigned)L.ncb, 256u, 0, s, ch, cb, inv, b, x);
}

// ---- coarsest-level dense FP64 Cholesky of A + eps Id, eps = 1e-12 mean diag ----
// dense copy of each coarsest block (rows and columns row0..row0+n-1 of its level)
__global__ void dense_from_csr_kernel(const int *__restrict__ cblk, const int *const *__restrict__ rps,
                                      const int *const *__restrict__ cis, const double *const *__restrict__ As,
                                      double *__restrict__ D) {
    const int *cb = cblk + 5 * blockIdx.y;
    const int lev = cb[0], row0 = cb[2], n = cb[3];
    double *Dk = D + cb[4];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int *rp = rps[lev], *ci = cis[lev];
    const double *A = As[lev];
    for (int j = 0; j < n; j++) Dk[(size_t)i * n + j] = 0.0;
    for (int k = rp[row0 + i]; k < rp[row0 + i + 1]; k++) {
        const int j = ci[k] - row0;
        if (j >= 0 && j < n) Dk[(size_t)i * n + j] = A[k];
    }
}

__global__ void __launch_bounds__(1024) cholesky_kernel(const int *__restrict__ cblk, double *D, int *flag) {
    __shared__ double s_val;
    const int *cb = cblk + 5 * blockIdx.x;
    const int n = cb[3];
    double *Dk = D + cb[4];
    const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    if (tid == 0) {
        double tr = 0.0;
        for (int i = 0; i < n; i++) tr += Dk[(size_t)i * n + i];
        s_val = 1e-12 * tr / (double)(n > 0 ? n : 1);
    }
    __syncthreads();
    const double eps = s_val;
    for (int i = tid; i < n; i += nthr) Dk[(size_t)i * n + i] += eps;
    for (int j = 0; j < n; j++) {
        __syncthreads();
        if (tid == 0) {
            double d = Dk[(size_t)j * n + j];
            if (!(d > 0.0)) { atomicExch(flag, 1); d = 1.0; }
            s_val = sqrt(d);
            Dk[(size_t)j * n + j] = s_val;
        }
        __syncthreads();
        const double piv = s_val;
        for (int i = j + 1 + tid; i < n; i += nthr) Dk[(size_t)i * n + j] /= piv;
        __syncthreads();
        for (int i = j + 1 + warp; i < n; i += nw) {
            const double lij = Dk[(size_t)i * n + j];
            for (int k = j + 1 + lane; k <= i; k += 32) Dk[(size_t)i * n + k] -= lij * Dk[(size_t)k * n + j];
        }
    }
}

// column c of (L L^T)^{-1} of every block: forward then backward substitution on e_c
__global__ void __launch_bounds__(256) cholesky_inverse_kernel(const int *__restrict__ cblk, const double *__restrict__ D,
                                                               double *__restrict__ inv64, float *__restrict__ inv32) {
    extern __shared__ double y[];
    const int *cb = cblk + 5 * blockIdx.y;
    const int n = cb[3];
    const int c = blockIdx.x;
    if (c >= n) return;
    const double *Lf = D + cb[4];
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < n; i += nthr) y[i] = (i == c) ? 1.0 : 0.0;
    for (int k = 0; k < n; k++) {
        __syncthreads();
        if (tid == 0) y[k] /= Lf[(size_t)k * n + k];
        __syncthreads();
        const double yk = y[k];
        for (int i = k + 1 + tid; i < n; i += nthr) y[i] -= Lf[(size_t)i * n + k] * yk;
    }
    for (int k = n - 1; k >= 0; k--) {
        __syncthreads();
        if (tid == 0) y[k] /= Lf[(size_t)k * n + k];
        __syncthreads();
        const double yk = y[k];
        for (int i = tid; i < k; i += nthr) y[i] -= Lf[(size_t)k * n + i] * yk;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nthr) {
        inv64[cb[4] + (size_t)i * n + c] = y[i];
        inv32[cb[4] + (size_t)i * n + c] = (float)y[i];
    }
}

void launch_coarse_factor(const Ctx &c, const int *const *rps, const int *const *cis, const double *const *As,
                          cudaStream_t s) {
    if (c.ncblk == 0) return;
    dense_from_csr_kernel<<<dim3((c.n0max + 127) / 128, c.ncblk), 128, 0, s>>>(c.cblk, rps, cis, As, c.cdense);
    cholesky_kernel<<<c.ncblk, 1024, 0, s>>>(c.cblk, c.cdense, c.flag);
    cholesky_inverse_kernel<<<dim3(c.n0max, c.ncblk), 256, c.n0max * sizeof(double), s>>>(c.cblk, c.cdense, c.cinv64,
                                                                                         c.cinv32);
}

// ---- per-right-hand-side sums of squares, two passes (deterministic) ----
template <int R>
__global__ void __launch_bounds__(256) norm_partial_kernel(const double *__restrict__ v, int n, double *__restrict__ part) {
    __shared__ double sh[256][R];
    grid_dep_wait();
    grid_dep_launch();
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int r = 0; r < R; r++) { const double x = v[(size_t)i * R + r]; acc[r] = fma(x, x, acc[r]); }
#pragma unroll
    for (int r = 0; r < R; r++) sh[threadIdx.x][r] = acc[r];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int r = 0; r < R; r++) sh[threadIdx.x][r] += sh[threadIdx.x + o][r];
        __syncthreads();
    }
    if (threadIdx.x < R) part[blockIdx.x * 4 + threadIdx.x] = sh[0][threadIdx.x];
}

__global__ void __launch_bounds__(256) norm_final_kernel(const double *__restrict__ part, int nblocks, int R,
                                                         double *__restrict__ out) {
    __shared__ double sh[256][4];
    grid_dep_wait();
    grid_dep_launch();
    for (int r = 0; r < 4; r++) sh[threadIdx.x][r] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int r = 0; r < R; r++) sh[threadIdx.x][r] += part[b * 4 + r];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int r = 0; r < 4; r++) sh[threadIdx.x][r] += sh[threadIdx.x + o][r];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = threadIdx.x < R ? sh[0][threadIdx.x] : 0.0;
}

// ---- conjugate gradients preconditioned by the V-cycle (per right-hand side lane) ----
// partial sums of a_i . b_i per lane over a grid-stride range
template <int R>
__global__ void __launch_bounds__(256) dot_partial_kernel(const double *__restrict__ a, const double *__restrict__ b,
                                                          int n, double *__restrict__ part) {
    __shared__ double sh[256][R];
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; r++) acc[r] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] = fma(a[(size_t)i * R + r], b[(size_t)i * R + r], acc[r]);
#pragma unroll
    for (int r = 0; r < R; r++) sh[threadIdx.x][r] = acc[r];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int r = 0; r < R; r++) sh[threadIdx.x][r] += sh[threadIdx.x + o][r];
        __syncthreads();
    }
    if (threadIdx.x < R) part[blockIdx.x * 4 + threadIdx.x] = sh[0][threadIdx.x];
}

// one scalar step of lane r on the reduced value v (scalars sc, see pcg_scalar_kernel)
// (done: the lane already meets its tolerance and takes no further steps)
__device__ __forceinline__ void pcg_scalar_step(double *sc, int r, double v, int mode, bool done = false) {
    double *rz = sc + kPcgRz, *s1 = sc + kPcgS1, *s2 = sc + kPcgS2, *al = sc + kPcgAlpha, *be = sc + kPcgBeta,
           *rz0 = sc + kPcgRz0;
    if (mode == 0) {
        s2[r] = v;
    } else if (mode == 1) {
        if (rz[r] == 0.0 && rz0[r] == 0.0) rz0[r] = v;   // the first step
        const bool live = !done && v > kPcgStop * rz0[r];   // false at rounding level, for 0 and NaN
        s1[r] = live ? v : 0.0;
        be[r] = (live && rz[r] > 0.0) ? (v - s2[r]) / rz[r] : 0.0;
        rz[r] = live ? v : 0.0;
    } else {
        const double pap = -v;
        al[r] = (pap > 0.0 && s1[r] > 0.0) ? s1[r] / pap : 0.0;
    }
}

// one block: reduce the partial sums to v[lane], then
//   mode 0: s2 = v                         (r . z of the previous preconditioned residual)
//   mode 1: s1 = v; beta = (s1 - s2) / rz, rz = s1  (Polak-Ribiere; 0 on the first step, rz = 0;
//           a lane at rounding level, v <= kPcgStop * its first v, keeps beta = alpha = 0)
//   mode 2: alpha = s1 / (p . A p), with v = p . q and q = -A p
__global__ void pcg_scalar_kernel(const double *__restrict__ part, int nblocks, int R, double *__restrict__ sc,
                                  int mode) {
    __shared__ double sh[256][4];
    for (int r = 0; r < 4; r++) sh[threadIdx.x][r] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int r = 0; r < R; r++) sh[threadIdx.x][r] += part[b * 4 + r];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int r = 0; r < 4; r++) sh[threadIdx.x][r] += sh[threadIdx.x + o][r];
        __syncthreads();
    }
    if (threadIdx.x >= R) return;
    const int r = threadIdx.x;
    const double v = sh[0][r];
    pcg_scalar_step(sc, r, v, mode);
}

// p = z + beta p
__global__ void pcg_direction_kernel(const double *__restrict__ z, double *__restrict__ p,
                                     const double *__restrict__ sc, int64_t m, int R) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < m) p[q] = fma(sc[kPcgBeta + (int)(q % R)], p[q], z[q]);
}

// x += alpha p; r += alpha q (q = -A p)
__global__ void pcg_update_kernel(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                  const double *__restrict__ qv, const double *__restrict__ sc, int64_t m, int R) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const double a = sc[kPcgAlpha + (int)(q % R)];
    x[q] = fma(a, p[q], x[q]);
    r[q] = fma(a, qv[q], r[q]);
}

// ---- the same for a batch: per-mesh dot products over work items (row ranges of one
// mesh and colour; the items of mesh m are [istart[m], istart[m + 1])) ----
// per item, per lane: a.b (components 0..3) and, when c is given, c.d (4..7)
template <int R>
__global__ void __launch_bounds__(256) item_dot2_kernel(const int *__restrict__ items, int nitems,
                                                        const double *__restrict__ a, const double *__restrict__ b,
                                                        const double *__restrict__ cv, const double *__restrict__ dv,
                                                        double *__restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (it >= nitems) return;
    const int r0 = items[3 * it + 1], r1 = items[3 * it + 2];
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] = 0.0;
    for (int i = r0 + lane; i < r1; i += 32)
#pragma unroll
        for (int q = 0; q < R; q++) {
            acc[q] = fma(a[(size_t)i * R + q], b[(size_t)i * R + q], acc[q]);
            if (cv) acc[4 + q] = fma(cv[(size_t)i * R + q], dv[(size_t)i * R + q], acc[4 + q]);
        }
#pragma unroll
    for (int q = 0; q < 8; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane < 8) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < 8; q++) if (q == lane) v = acc[q];
        part[8 * (size_t)it + lane] = v;
    }
}

// per mesh m and component q < 8: out[m * ostride + q] = sum of its items' partials (in item order)
__global__ void inst_sum_kernel(const int *__restrict__ istart, int ninst, const double *__restrict__ part,
                                double *__restrict__ out, int ostride) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ninst * 8) return;
    const int m = k >> 3, q = k & 7;
    double s = 0.0;
    for (int it = istart[m]; it < istart[m + 1]; it++) s += part[8 * (size_t)it + q];
    out[(size_t)m * ostride + q] = s;
}

// per mesh m and lane r: the conjugate-gradient scalar step of pcg_scalar_kernel on
// v = sum of the mesh's item partials (component r); scalars at sc + m * kPcgScalars
//   norms: [ninst][16] per-mesh squared norms of r (0..3) and b (4..7) after the last step;
//   tol: the solve's tolerance.  A mesh lane that meets it takes no further steps: the other
//   meshes keep iterating, and a converged lane's FP32-preconditioned recurrence would
//   otherwise run on rounding noise.
__global__ void inst_pcg_scalar_kernel(const int *__restrict__ istart, int ninst, int R,
                                       const double *__restrict__ part, double *__restrict__ sc, int mode,
                                       const double *__restrict__ norms, const double *__restrict__ tol) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ninst * 4) return;
    const int m = k >> 2, r = k & 3;
    if (r >= R) return;
    double v = 0.0;
    for (int it = istart[m]; it < istart[m + 1]; it++) v += part[8 * (size_t)it + r];
    const double t = *tol;
    const bool done = norms[16 * (size_t)m + r] <= t * t * norms[16 * (size_t)m + 4 + r];
    pcg_scalar_step(sc + (size_t)m * kPcgScalars, r, v, mode, done);
}

// p = z + beta_mesh p; x += alpha_mesh p, r += alpha_mesh q (q = -A p), the mesh of a row from row_inst
__global__ void inst_pcg_direction_kernel(const double *__restrict__ z, double *__restrict__ p,
                                          const double *__restrict__ sc, const int *__restrict__ row_inst,
                                          int64_t m, int R) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const double *s = sc + (size_t)row_inst[q / R] * kPcgScalars;
    p[q] = fma(s[kPcgBeta + (int)(q % R)], p[q], z[q]);
}
__global__ void inst_pcg_update_kernel(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                       const double *__restrict__ qv, const double *__restrict__ sc,
                                       const int *__restrict__ row_inst, int64_t m, int R) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= m) return;
    const double a = sc[(size_t)row_inst[q / R] * kPcgScalars + kPcgAlpha + (int)(q % R)];
    x[q] = fma(a, p[q], x[q]);
    r[q] = fma(a, qv[q], r[q]);
}

void launch_item_dot2(const int *items, int nitems, const double *a, const double *b, const double *c,
                      const double *d, int R, double *part, cudaStream_t s) {
    if (nitems == 0) return;
    const unsigned blocks = (unsigned)((nitems + 7) / 8);
    if (R == 1) item_dot2_kernel<1><<<blocks, 256, 0, s>>>(items, nitems, a, b, c, d, part);
    else if (R == 2) item_dot2_kernel<2><<<blocks, 256, 0, s>>>(items, nitems, a, b, c, d, part);
    else item_dot2_kernel<4><<<blocks, 256, 0, s>>>(items, nitems, a, b, c, d, part);
}
void launch_inst_sum(const int *istart, int ninst, const double *part, double *out, int ostride, cudaStream_t s) {
    inst_sum_kernel<<<(unsigned)((ninst * 8 + 255) / 256), 256, 0, s>>>(istart, ninst, part, out, ostride);
}
void launch_inst_pcg_scalar(const int *istart, int ninst, int R, const double *part, double *sc, int mode,
                            const double *norms, const double *tol, cudaStream_t s) {
    inst_pcg_scalar_kernel<<<(unsigned)((ninst * 4 + 255) / 256), 256, 0, s>>>(istart, ninst, R, part, sc, mode,
                                                                                norms, tol);
}
void launch_inst_pcg_direction(const double *z, double *p, const double *sc, const int *row_inst, int n, int R,
                               cudaStream_t s) {
    const int64_t m = (int64_t)n * R;
    if (m) inst_pcg_direction_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(z, p, sc, row_inst, m, R);
}
void launch_inst_pcg_update(double *x, double *r, const double *p, const double *q, const double *sc,
                            const int *row_inst, int n, int R, cudaStream_t s) {
    const int64_t m = (int64_t)n * R;
    if (m) inst_pcg_update_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(x, r, p, q, sc, row_inst, m, R);
}

void launch_pcg_dot(const double *a, const double *b, int n, int R, double *part, double *sc, int mode,
                    cudaStream_t s) {
    if (R == 1) dot_partial_kernel<1><<<kNormBlocks, 256, 0, s>>>(a, b, n, part);
    else if (R == 2) dot_partial_kernel<2><<<kNormBlocks, 256, 0, s>>>(a, b, n, part);
    else dot_partial_kernel<4><<<kNormBlocks, 256, 0, s>>>(a, b, n, part);
    pcg_scalar_kernel<<<1, 256, 0, s>>>(part, kNormBlocks, R, sc, mode);
}
void launch_pcg_direction(const double *z, double *p, const double *sc, int n, int R, cudaStream_t s) {
    const int64_t m = (int64_t)n * R;
    if (m) pcg_direction_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(z, p, sc, m, R);
}
void launch_pcg_update(double *x, double *r, const double *p, const double *q, const double *sc, int n, int R,
                       cudaStream_t s) {
    const int64_t m = (int64_t)n * R;
    if (m) pcg_update_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(x, r, p, q, sc, m, R);
}

void launch_norms(const double *v, int n, int R, double *part, double *out, cudaStream_t s, Chain *ch) {
    auto k = R == 1 ? norm_partial_kernel<1> : R == 2 ? norm_partial_kernel<2> : norm_partial_kernel<4>;
    klaunch(k, (unsigned)kNormBlocks, 256u, 0, s, ch, v, n, part);
    klaunch(norm_final_kernel, 1u, 256u, 0, s, ch, (const double *)part, (int)kNormBlocks, R, out);
}

// ---- layout and elementwise kernels ----
// user row u of [n][nrhs] <-> internal row perm[u] of [n][R] (perm = null: identity)
__global__ void pack_kernel(const double *__restrict__ u, int n, int nrhs, int R, const int *__restrict__ perm,
                            double *__restrict__ v) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * R) return;
    const int64_t i = q / R;
    const int r = (int)(q % R);
    const int64_t row = perm ? perm[i] : i;
    v[row * R + r] = r < nrhs ? u[i * nrhs + r] : 0.0;
}
__global__ void unpack_kernel(const double *__restrict__ v, int n, int nrhs, int R, const int *__restrict__ perm,
                              double *__restrict__ u) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * nrhs) return;
    const int64_t i = q / nrhs;
    const int r = (int)(q % nrhs);
    const int64_t row = perm ? perm[i] : i;
    u[q] = v[row * R + r];
}
__global__ void to_float_kernel(const double *__restrict__ a, float *__restrict__ b, int64_t n,
                                float *__restrict__ zero) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    grid_dep_wait();
    grid_dep_launch();
    if (q < n) {
        b[q] = (float)a[q];
        if (zero) zero[q] = 0.f;
    }
}
__global__ void add_float_kernel(double *__restrict__ x, const float *__restrict__ e, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    grid_dep_wait();
    grid_dep_launch();
    if (q < n) x[q] += (double)e[q];
}
__global__ void add_double_kernel(double *__restrict__ x, const double *__restrict__ e, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) x[q] += e[q];
}

void launch_pack(const double *user, int n, int nrhs, int R, double *v, cudaStream_t s, const int *perm) {
    const int64_t m = (int64_t)n * R;
    if (m) pack_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(user, n, nrhs, R, perm, v);
}
void launch_unpack(const double *v, int n, int nrhs, int R, double *user, cudaStream_t s, const int *perm) {
    const int64_t m = (int64_t)n * nrhs;
    if (m) unpack_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(v, n, nrhs, R, perm, user);
}
void launch_to_float(const double *a, float *b, int64_t n, cudaStream_t s, float *zero, Chain *ch) {
    if (n) klaunch(to_float_kernel, (unsigned)((n + 255) / 256), 256u, 0, s, ch, a, b, n, zero);
}
void launch_add_float(double *x, const float *e, int64_t n, cudaStream_t s, Chain *ch) {
    if (n) klaunch(add_float_kernel, (unsigned)((n + 255) / 256), 256u, 0, s, ch, x, e, n);
}
void launch_add_double(double *x, const double *e, int64_t n, cudaStream_t s) {
    if (n) add_double_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, e, n);
}

// explicit instantiations
#define LBMG_INST(T)                                                                                           \
    template void launch_sweeps<T>(const Ctx &, const DevLevel &, int, bool, const T *, const T *, const T *, T *, \
                                   int, cudaStream_t, Chain *, int);                                          \
    template void launch_smooth_colour<T>(const DevLevel &, int, const T *, const T *, const T *, T *, int,   \
                                          cudaStream_t, Chain *, int);                                         \
    template void launch_residual<T>(const DevLevel &, const T *, const T *, const T *, T *, int, cudaStream_t, int, \
                                     Chain *);                                                                 \
    template void launch_jacobi_update<T>(const DevLevel &, const T *, const T *, T *, T, int, cudaStream_t);   \
    template void launch_restrict<T>(const DevLevel &, const T *, T *, int, cudaStream_t, T *, Chain *, bool); \
    template void launch_prolong_add<T>(const DevLevel &, const T *, T *, int, cudaStream_t, Chain *);         \
    template void launch_coarse_apply<T>(const Ctx &, const DevLevel &, const T *, const T *, T *, int, cudaStream_t, \
                                         Chain *);
LBMG_INST(float)
LBMG_INST(double)

}  // namespace lbmg
