// learned.cu -- learned residual correction in front of each multigrid cycle.
//
// Not in the paper, whose solver iterates the plain cycle on the residual (Section 4.3;
// Gauss-Seidel smoothing, Section 5.2).  Before each cycle of that iteration the
// current residual r receives a per-node correction
//     delta_i = omega_i r_i / a_ii      (every right-hand-side lane)
// and the cycle starts from delta instead of zero, i.e. e = delta + V(r - A delta).
// omega_i = 1 + y_i / (1 + |y_i|) in (0, 2) comes from a 30 -> 64 (ReLU) -> 1 network
// of node i's features: 28 from its stencil (row coefficients over a_ii summed per
// neighbour-corner offset, the relative diagonal, the entry count), computed once per
// assembly, and 2 from the residual, computed before every cycle: the local
// minimal-residual step q_i = r_i.z_i / z_i.z_i with z = A D^-1 r, fed as q / (1 + |q|),
// and the residual-energy share e_i / (e_i + mean e) with e_i = r_i.r_i.  Both residual
// features are invariant under scaling of r, so delta is homogeneous of degree one.
//
// Training minimises log(||C (r - A delta)||^2 / ||r||^2) (C = I - A V: the residual
// reduction of one learned iteration) over residual samples from plain V-cycle histories; the
// gradient is the exact adjoint (C^T g = g - V A g, V symmetric), in FP64 with the
// solver's kernels.  The dense layer runs on the tensor cores (mma.sync BF16 x BF16 ->
// FP32) both in the solve and in training.  A solve drops the correction for good once
// an iteration with it leaves a larger residual than the iteration before (the device
// stopping test sets the flag the correction kernel reads).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lbmg.h"
#include "lbmg_internal.h"

namespace lbmg {

// exported by api.cu: one FP64 V-cycle on A_top e = b_top from e = 0 (lev[top].x64)
void enqueue_vcycle64_from(Ctx &c, int top, int R, cudaStream_t s);

namespace {

constexpr int kF = 32;        // feature columns of the tensor-core tile
constexpr int kFS = 28;       // stencil features (columns 0..27)
constexpr int kFU = 30;       // used: + 2 residual features (columns 28, 29); 30, 31 stay zero
constexpr int kH = 64;        // hidden units
constexpr int kNP = kF * kH + kH + kH + 1;   // FP32 parameters: W1 [32][64], b1, w2, b2
constexpr int kMaxBatch = 8;

// ---------------------------------------------------------------- stencil features
// (GB300's FP64 rate is a small fraction of its FP32 rate: the features, which the network
// reads in BF16, are computed in FP32 from FP64 matrix entries, with one FP64 division per row)
constexpr int kDiagParts = 256;

// per-block partial sums of the diagonal, grid-stride over the rows
__global__ void __launch_bounds__(256) diag_partial_kernel(int n, const int *__restrict__ rp,
                                                           const int *__restrict__ ci, const double *__restrict__ A,
                                                           double *__restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = rp[i], hi = rp[i + 1];
        const int end = hi;
        while (lo < hi) { int mid = (lo + hi) >> 1; if (ci[mid] < i) lo = mid + 1; else hi = mid; }
        s += (lo < end && ci[lo] == i) ? A[lo] : 0.0;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// columns 0..27 of X (BF16 [npad][32]); columns 28..31 are zeroed.  part: kDiagParts partial
// sums of the diagonal (their total / n is the mean diagonal)
__global__ void __launch_bounds__(128) features_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const double *__restrict__ A, const int *__restrict__ corner,
                                                       const double *__restrict__ part, __nv_bfloat16 *__restrict__ X) {
    __shared__ double s_mean;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < kDiagParts; b++) t += part[b];
        s_mean = t / (double)(n > 0 ? n : 1);
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[kF];
#pragma unroll
    for (int q = 0; q < kF; q++) f[q] = 0.f;
    const int k0 = rp[i], k1 = rp[i + 1];
    double diag = 0.0;
    for (int k = k0; k < k1; k++) if (ci[k] == i) diag = A[k];
    const float inv = (float)(1.0 / diag);
    const int cx = corner[3 * i], cy = corner[3 * i + 1], cz = corner[3 * i + 2];
    for (int k = k0; k < k1; k++) {
        const int j = ci[k];
        const int ox = corner[3 * j] - cx + 1, oy = corner[3 * j + 1] - cy + 1, oz = corner[3 * j + 2] - cz + 1;
        const int b = (ox * 3 + oy) * 3 + oz;
        const float v = (float)A[k] * inv;
        if (b >= 0 && b < 27) {
#pragma unroll
            for (int q = 0; q < 27; q++) if (q == b) f[q] += v;
        }
    }
    f[13] = (float)(diag / s_mean);
    f[27] = (float)(k1 - k0) / 27.f;
    __nv_bfloat16 *o = X + (size_t)i * kF;
#pragma unroll
    for (int q = 0; q < kF; q++) o[q] = __float2bfloat16_rn(f[q]);
}

// ---------------------------------------------------------------- residual features
// features 28, 29 of one row from its residual r and w = r - A D^-1 r (so z = r - w), R lanes;
// ebar: the mean over rows of r_i.r_i.  z is formed in the input precision, the rest in FP32
// after an exact power-of-two scaling of the row (its largest |r|, |z| into [1/2, 1)), so that
// tiny residuals neither underflow nor break the invariance under scaling of r.
template <class T, int R>
__device__ __forceinline__ void residual_features(const T *__restrict__ r, const T *__restrict__ w, float ebar,
                                                  float &f28, float &f29) {
    float rv[R], zv[R], m = 0.f;
#pragma unroll
    for (int q = 0; q < R; q++) {
        rv[q] = (float)r[q];
        zv[q] = (float)(r[q] - w[q]);
        m = fmaxf(m, fmaxf(fabsf(rv[q]), fabsf(zv[q])));
    }
    f28 = 0.f;
    f29 = 0.f;
    if (!(m > 0.f) || !(m <= 3.0e38f)) return;   // zero (or non-finite) residual row
    int k;
    frexpf(m, &k);
    const float sc = ldexpf(1.f, -k);
    float rz = 0.f, zz = 0.f, e = 0.f;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const float a = rv[q] * sc, z = zv[q] * sc;
        rz = fmaf(a, z, rz);
        zz = fmaf(z, z, zz);
        e = fmaf(a, a, e);
    }
    const float qv = zz > 0.f ? rz / zz : 0.f;
    f28 = qv / (1.f + fabsf(qv));
    f29 = ebar > 0.f ? e / (e + ldexpf(ebar, -2 * k)) : 0.f;
}

__device__ __forceinline__ float mean_energy(const double *__restrict__ nr, int R, int n) {
    double s = 0.0;
    for (int q = 0; q < R; q++) s += nr[q];
    return (float)s / (float)(n > 0 ? n : 1);
}

// training path: columns 28, 29 of X for a sample r ([n][4] FP64), w = r - A D^-1 r,
// nr: the sample's squared norms per lane
__global__ void rfeat_kernel(int n, const double *__restrict__ r, const double *__restrict__ w,
                             const double *__restrict__ nr, __nv_bfloat16 *__restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f28, f29;
    residual_features<double, 4>(r + 4 * (size_t)i, w + 4 * (size_t)i, mean_energy(nr, 4, n), f28, f29);
    X[(size_t)i * kF + 28] = __float2bfloat16_rn(f28);
    X[(size_t)i * kF + 29] = __float2bfloat16_rn(f29);
}

// ---------------------------------------------------------------- tensor-core MLP
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ float omega_of(float y) { return 1.f + y / (1.f + fabsf(y)); }

// A fragments (m16n8k16, row-major A) of the 16 feature rows at row0: ks = 0 covers
// columns 0..15, ks = 1 columns 16..31.  Lane (g, t) holds rows g and g + 8.
__device__ __forceinline__ void load_features(const __nv_bfloat16 *__restrict__ X, int row0, int g, int t,
                                              uint32_t (&a)[2][4]) {
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
        const __nv_bfloat16 *x0 = X + (size_t)(row0 + g) * kF + ks * 16 + 2 * t;
        const __nv_bfloat16 *x8 = X + (size_t)(row0 + g + 8) * kF + ks * 16 + 2 * t;
        a[ks][0] = *reinterpret_cast<const uint32_t *>(x0);
        a[ks][1] = *reinterpret_cast<const uint32_t *>(x8);
        a[ks][2] = *reinterpret_cast<const uint32_t *>(x0 + 8);
        a[ks][3] = *reinterpret_cast<const uint32_t *>(x8 + 8);
    }
}

// Z = X W1 + b1 (16 x 64 per warp, FP32 accumulators acc[n-tile][4]), then
// y = relu(Z) w2 + b2 for rows g (y0) and g + 8 (y8), summed over the four lanes of a row
// group so every lane of the group holds them.  sW: W1^T [64][32] BF16 in shared memory.
__device__ __forceinline__ void mlp_tile(const uint32_t (&a)[2][4], const __nv_bfloat16 *sW,
                                         const float *b1, const float *w2, float b2, int g, int t,
                                         float (&acc)[8][4], float &y0, float &y8) {
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int col = nt * 8 + 2 * t;
        acc[nt][0] = b1[col]; acc[nt][1] = b1[col + 1]; acc[nt][2] = b1[col]; acc[nt][3] = b1[col + 1];
    }
#pragma unroll
    for (int ks = 0; ks < 2; ks++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            uint32_t b[2];
            const __nv_bfloat16 *w = sW + (nt * 8 + g) * kF + ks * 16 + 2 * t;
            b[0] = *reinterpret_cast<const uint32_t *>(w);
            b[1] = *reinterpret_cast<const uint32_t *>(w + 8);
            mma_bf16(acc[nt], a[ks], b);
        }
    y0 = 0.f;
    y8 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int col = nt * 8 + 2 * t;
        y0 += fmaxf(acc[nt][0], 0.f) * w2[col] + fmaxf(acc[nt][1], 0.f) * w2[col + 1];
        y8 += fmaxf(acc[nt][2], 0.f) * w2[col] + fmaxf(acc[nt][3], 0.f) * w2[col + 1];
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y8 += __shfl_xor_sync(0xffffffffu, y8, 1);
    y8 += __shfl_xor_sync(0xffffffffu, y8, 2);
    y0 += b2;
    y8 += b2;
}

// training path forward: y (and Z for the backward pass) of every row; one warp per 16 rows,
// X has ceil(n/16)*16 rows
__global__ void __launch_bounds__(256) mlp_forward_kernel(int n, const __nv_bfloat16 *__restrict__ X,
                                                          const __nv_bfloat16 *__restrict__ W1T,
                                                          const float *__restrict__ prm, float *__restrict__ Z,
                                                          float *__restrict__ y) {
    __shared__ __align__(16) __nv_bfloat16 sW[kH * kF];
    for (int q = threadIdx.x; q < kH * kF; q += blockDim.x) sW[q] = W1T[q];
    __syncthreads();
    const float *b1 = prm + kF * kH, *w2 = b1 + kH, *b2 = w2 + kH;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int row0 = (blockIdx.x * (blockDim.x >> 5) + warp) * 16;
    if (row0 >= n) return;
    uint32_t a[2][4];
    load_features(X, row0, g, t, a);
    float acc[8][4], y0, y8;
    mlp_tile(a, sW, b1, w2, b2[0], g, t, acc, y0, y8);
    const int r_a = row0 + g, r_b = row0 + g + 8;
    if (Z) {
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const int col = nt * 8 + 2 * t;
            if (r_a < n) *reinterpret_cast<float2 *>(Z + (size_t)r_a * kH + col) = make_float2(acc[nt][0], acc[nt][1]);
            if (r_b < n) *reinterpret_cast<float2 *>(Z + (size_t)r_b * kH + col) = make_float2(acc[nt][2], acc[nt][3]);
        }
    }
    if (t == 0) {
        if (r_a < n) y[r_a] = y0;
        if (r_b < n) y[r_b] = y8;
    }
}

// ---------------------------------------------------------------- solve path
// b = r (to the cycle's precision), x = D^-1 r: the Jacobi start that the correction scales
template <class T, int R>
__global__ void lr_prep_kernel(int n, const double *__restrict__ r, const T *__restrict__ dinv, T *__restrict__ b,
                               T *__restrict__ x) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const T di = q < (int64_t)n * R ? dinv[q / R] : T(0);
    grid_dep_wait();
    grid_dep_launch();
    if (q >= (int64_t)n * R) return;
    const T v = (T)r[q];
    b[q] = v;
    x[q] = di * v;
}

// x_i *= omega_i with omega from the network; r: the residual (cycle precision), w = r - A x
// (x = D^-1 r on entry), nr: squared norms of r per lane.  One warp per 16 rows; the stencil
// features and the weights are loaded before the grid-dependency wait.  When *off is set (the
// solve dropped the correction) x is zeroed instead: the plain cycle.
template <class T, int R>
__global__ void __launch_bounds__(256) lr_solve_kernel(int n, const __nv_bfloat16 *__restrict__ X,
                                                       const __nv_bfloat16 *__restrict__ W1T,
                                                       const float *__restrict__ prm, const T *__restrict__ r,
                                                       const T *__restrict__ w, const double *__restrict__ nr,
                                                       const int *off, T *__restrict__ x, double *__restrict__ omega_out) {
    __shared__ __align__(16) __nv_bfloat16 sW[kH * kF];
    __shared__ float sP[2 * kH + 1];
    for (int q = threadIdx.x; q < kH * kF; q += blockDim.x) sW[q] = W1T[q];
    for (int q = threadIdx.x; q < 2 * kH + 1; q += blockDim.x) sP[q] = prm[kF * kH + q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int row0 = (blockIdx.x * (blockDim.x >> 5) + warp) * 16;
    __shared__ float s_ebar;
    uint32_t a[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
    if (row0 < n) load_features(X, row0, g, t, a);
    grid_dep_wait();
    grid_dep_launch();
    if (threadIdx.x == 0) s_ebar = mean_energy(nr, R, n);   // once per block (FP64 is scarce)
    __syncthreads();
    if (row0 >= n) return;
    const int ra = row0 + g, rb = row0 + g + 8;
    if (off && *(volatile const int *)off != 0) {
        if (t < R) {
            if (ra < n) x[(size_t)ra * R + t] = T(0);
            if (rb < n) x[(size_t)rb * R + t] = T(0);
        }
        if (omega_out && t == 0) {
            if (ra < n) omega_out[ra] = 0.0;
            if (rb < n) omega_out[rb] = 0.0;
        }
        return;
    }
    if (t == 2) {   // this lane's ks = 1 fragment holds columns 28, 29 of rows g and g + 8
        const float eb = s_ebar;
        float fa28 = 0.f, fa29 = 0.f, fb28 = 0.f, fb29 = 0.f;
        if (ra < n) residual_features<T, R>(r + (size_t)ra * R, w + (size_t)ra * R, eb, fa28, fa29);
        if (rb < n) residual_features<T, R>(r + (size_t)rb * R, w + (size_t)rb * R, eb, fb28, fb29);
        a[1][2] = pack2(__float2bfloat16_rn(fa28), __float2bfloat16_rn(fa29));
        a[1][3] = pack2(__float2bfloat16_rn(fb28), __float2bfloat16_rn(fb29));
    }
    float acc[8][4], y0, y8;
    mlp_tile(a, sW, sP, sP + kH, sP[2 * kH], g, t, acc, y0, y8);
    const float oa = omega_of(y0), ob = omega_of(y8);
    if (t < R) {
        if (ra < n) x[(size_t)ra * R + t] *= (T)oa;
        if (rb < n) x[(size_t)rb * R + t] *= (T)ob;
    }
    if (omega_out && t == 0) {
        if (ra < n) omega_out[ra] = oa;
        if (rb < n) omega_out[rb] = ob;
    }
}

// ---------------------------------------------------------------- training path (FP64, 4 lanes)
__global__ void scale_rows_kernel(int n, const double *__restrict__ dinv, const double *__restrict__ r,
                                  double *__restrict__ u) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < (int64_t)n * 4) u[q] = dinv[q >> 2] * r[q];
}

// omega = 1 + y / (1 + |y|); delta = omega u
__global__ void omega_delta_kernel(int n, const float *__restrict__ y, const double *__restrict__ u,
                                   double *__restrict__ omega, double *__restrict__ delta) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    const double om = (double)omega_of(y[q >> 2]);
    if ((q & 3) == 0) omega[q >> 2] = om;
    delta[q] = om * u[q];
}

// loss = log(||R1||^2 / ||R0||^2) from the per-lane squared norms (0 for a zero sample)
__global__ void loss_kernel(const double *__restrict__ nb, const double *__restrict__ nr, double *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int q = 0; q < 4; q++) { a += nr[q]; b += nb[q]; }
    *out = (a > 0.0 && b > 0.0) ? log(a / b) : 0.0;
}

// g = 2 R1 / ||R1||^2, the gradient of log ||R1||^2
__global__ void seed_kernel(int n, const double *__restrict__ R1, const double *__restrict__ nr,
                            double *__restrict__ g) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    const double a = nr[0] + nr[1] + nr[2] + nr[3];
    g[q] = a > 0.0 ? 2.0 * R1[q] / a : 0.0;
}

__global__ void axpy_kernel(int64_t m, double a, const double *__restrict__ x, double *__restrict__ y) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < m) y[q] += a * x[q];
}

// dL/domega_i = sum_q (dL/ddelta)_iq u_iq; dy = dL/domega / (1 + |y|)^2, times the batch weight
__global__ void dy_kernel(int n, const double *__restrict__ dD, const double *__restrict__ u,
                          const float *__restrict__ y, double weight, float *__restrict__ dy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int q = 0; q < 4; q++) s += dD[4 * (size_t)i + q] * u[4 * (size_t)i + q];
    const double a = 1.0 + fabs((double)y[i]);
    dy[i] = (float)(weight * s / (a * a));
}

__global__ void gather_samples_kernel(int n, const double *__restrict__ bank, int sel, double *__restrict__ out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < (int64_t)n * 4) out[q] = bank[(size_t)sel * n * 4 + q];
}

// columns c0..c0+lanes-1 of a user-ordered [n][ns] array into lanes of internal [n][4]
__global__ void pack_cols_kernel(const double *__restrict__ u, int n, int ns, int c0, int lanes,
                                 const int *__restrict__ fperm, double *__restrict__ out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    const int i = (int)(q >> 2), lane = (int)(q & 3);
    out[4 * (size_t)fperm[i] + lane] = lane < lanes ? u[(size_t)i * ns + c0 + lane] : 0.0;
}

// parameter gradients: dW1 = X^T dZ on the tensor cores, dZ = dy w2 (Z > 0); db1, dw2, db2 in FP32.
// One warp per 16-row chunk; per-block partial sums in `part` [gridDim][kNP].
__global__ void __launch_bounds__(256) mlp_backward_kernel(int n, const __nv_bfloat16 *__restrict__ X,
                                                           const float *__restrict__ Z, const float *__restrict__ dy,
                                                           const float *__restrict__ prm, float *__restrict__ part) {
    __shared__ __align__(16) __nv_bfloat16 sX[8][16][kF];
    __shared__ __align__(16) __nv_bfloat16 sD[8][16][kH];
    __shared__ float sAcc[kNP];
    const float *w2 = prm + kF * kH + kH;
    for (int q = threadIdx.x; q < kNP; q += blockDim.x) sAcc[q] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nchunks = (n + 15) / 16;
    float acc[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.f;
    float db1[2] = {0.f, 0.f}, dw2[2] = {0.f, 0.f}, db2 = 0.f;
    for (int ch = blockIdx.x * 8 + warp; ch < nchunks; ch += gridDim.x * 8) {
        const int row0 = ch * 16;
        // stage X rows and dZ rows of this chunk (zero beyond n)
        for (int q = lane; q < 16 * kF; q += 32) {
            const int rr = q / kF, cc = q % kF;
            sX[warp][rr][cc] = row0 + rr < n ? X[(size_t)(row0 + rr) * kF + cc] : __float2bfloat16_rn(0.f);
        }
        for (int q = lane; q < 16 * kH; q += 32) {
            const int rr = q / kH, cc = q % kH;
            float v = 0.f;
            if (row0 + rr < n) {
                const float z = Z[(size_t)(row0 + rr) * kH + cc];
                const float d = dy[row0 + rr];
                v = z > 0.f ? d * w2[cc] : 0.f;
            }
            sD[warp][rr][cc] = __float2bfloat16_rn(v);
        }
        __syncwarp();
        // column sums in FP32 straight from Z and dy (lane owns columns 2*lane, 2*lane+1)
        for (int rr = 0; rr < 16 && row0 + rr < n; rr++) {
            const float d = dy[row0 + rr];
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const int cc = 2 * lane + e;
                const float z = Z[(size_t)(row0 + rr) * kH + cc];
                if (z > 0.f) { db1[e] += d * w2[cc]; dw2[e] += z * d; }
            }
            if (lane == 0) db2 += d;
        }
        // dW1[m][n] += sum_k X[k][m] dZ[k][n]: A = X^T (m = feature, k = row), B = dZ (k = row, n = hidden)
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            uint32_t a[4];
            const int m0 = mt * 16 + g;
            a[0] = pack2(sX[warp][2 * t][m0], sX[warp][2 * t + 1][m0]);
            a[1] = pack2(sX[warp][2 * t][m0 + 8], sX[warp][2 * t + 1][m0 + 8]);
            a[2] = pack2(sX[warp][2 * t + 8][m0], sX[warp][2 * t + 9][m0]);
            a[3] = pack2(sX[warp][2 * t + 8][m0 + 8], sX[warp][2 * t + 9][m0 + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                uint32_t b[2];
                const int c0 = nt * 8 + g;
                b[0] = pack2(sD[warp][2 * t][c0], sD[warp][2 * t + 1][c0]);
                b[1] = pack2(sD[warp][2 * t + 8][c0], sD[warp][2 * t + 9][c0]);
                mma_bf16(acc[mt][nt], a, b);
            }
        }
        __syncwarp();
    }
    // reduce warps of the block into shared memory
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const int m = mt * 16 + g, col = nt * 8 + 2 * t;
            atomicAdd(&sAcc[m * kH + col], acc[mt][nt][0]);
            atomicAdd(&sAcc[m * kH + col + 1], acc[mt][nt][1]);
            atomicAdd(&sAcc[(m + 8) * kH + col], acc[mt][nt][2]);
            atomicAdd(&sAcc[(m + 8) * kH + col + 1], acc[mt][nt][3]);
        }
#pragma unroll
    for (int e = 0; e < 2; e++) {
        atomicAdd(&sAcc[kF * kH + 2 * lane + e], db1[e]);
        atomicAdd(&sAcc[kF * kH + kH + 2 * lane + e], dw2[e]);
    }
    if (lane == 0) atomicAdd(&sAcc[kNP - 1], db2);
    __syncthreads();
    for (int q = threadIdx.x; q < kNP; q += blockDim.x) part[(size_t)blockIdx.x * kNP + q] = sAcc[q];
}

// grad[q] (+)= sum over blocks of part, in a fixed order
__global__ void grad_reduce_kernel(int nblocks, const float *__restrict__ part, int accumulate,
                                   double *__restrict__ grad) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNP) return;
    double s = accumulate ? grad[q] : 0.0;
    for (int b = 0; b < nblocks; b++) s += (double)part[(size_t)b * kNP + q];
    grad[q] = s;
}

// Adam on FP32 master parameters (rows 30, 31 of W1 stay zero); refreshes the BF16 W1^T
__global__ void adam_kernel(float lr, float b1t, float b2t, const double *__restrict__ grad, float *__restrict__ prm,
                            float *__restrict__ m, float *__restrict__ v, __nv_bfloat16 *__restrict__ W1T) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNP) return;
    if (q < kF * kH && q / kH >= kFU) return;
    const float gq = (float)grad[q];
    const float mq = 0.9f * m[q] + 0.1f * gq, vq = 0.999f * v[q] + 0.001f * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float p = prm[q] - lr * (mq / b1t) / (sqrtf(vq / b2t) + 1e-8f);
    prm[q] = p;
    if (q < kF * kH) W1T[(q % kH) * kF + q / kH] = __float2bfloat16_rn(p);
}

__global__ void w1t_from_prm_kernel(const float *__restrict__ prm, __nv_bfloat16 *__restrict__ W1T) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kF * kH) return;
    W1T[(q % kH) * kF + q / kH] = __float2bfloat16_rn(q / kH < kFU ? prm[q] : 0.f);
}

template <class T>
cudaError_t lalloc(T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, (count ? count : 1) * sizeof(T));
    return e;
}

inline unsigned blocks_for(int64_t m) { return (unsigned)((m + 255) / 256); }

}  // namespace

// ---------------------------------------------------------------- host side

struct Learned {
    int n = 0, npad = 0, part_blocks = 152, adam_t = 0;
    // inference: features, weights, Adam moments
    __nv_bfloat16 *X = nullptr, *W1T = nullptr;
    float *prm = nullptr, *m = nullptr, *v = nullptr;
    double *omega64 = nullptr;
    double *diag_part = nullptr;
    int *corner = nullptr;
    // training (allocated by the first training call)
    bool train_ready = false;
    float *Z = nullptr, *y = nullptr, *dy = nullptr, *part = nullptr;
    double *grad = nullptr, *omega = nullptr, *nb = nullptr, *nr = nullptr, *nrm_part = nullptr;
    double *r0 = nullptr, *u = nullptr, *w = nullptr, *d = nullptr, *r1 = nullptr, *R1 = nullptr;
    double *g = nullptr, *tmp = nullptr, *zero4 = nullptr;
    double *loss_dev = nullptr;
    int loss_cap = 0;
    double *bank = nullptr;
    int bank_cap = 0, bank_n = 0;
};

void learned_free(Ctx &c) {
    Learned *L = c.learned;
    if (!L) return;
    void *ptrs[] = {L->X, L->W1T, L->prm, L->m, L->v, L->omega64, L->diag_part, L->corner, L->Z, L->y, L->dy, L->part,
                    L->grad, L->omega, L->nb, L->nr, L->nrm_part, L->r0, L->u, L->w, L->d, L->r1, L->R1, L->g,
                    L->tmp, L->zero4, L->loss_dev, L->bank};
    for (void *q : ptrs) if (q) cudaFree(q);
    delete L;
    c.learned = nullptr;
    c.learned_on = 0;
}

int learned_setup(Ctx &c, cudaStream_t s) {
    (void)s;
    if (c.learned) return 0;
    if (c.D == c.d0) return 1;   // the cycle needs a coarser level
    Learned *L = new Learned();
    c.learned = L;
    const DevLevel &F = c.lev[c.D];
    L->n = F.n;
    L->npad = (F.n + 15) / 16 * 16;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    ok(lalloc(&L->X, (size_t)L->npad * kF));
    ok(lalloc(&L->W1T, (size_t)kH * kF));
    ok(lalloc(&L->prm, kNP)); ok(lalloc(&L->m, kNP)); ok(lalloc(&L->v, kNP));
    ok(lalloc(&L->omega64, L->n)); ok(lalloc(&L->diag_part, kDiagParts)); ok(lalloc(&L->corner, 3 * (size_t)L->n));
    if (e == cudaSuccess)
        e = cudaMemcpy(L->corner, c.host.lev[c.D].corner.data(), 3 * sizeof(int) * (size_t)L->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { learned_free(c); return 2; }
    return 0;
}

static int train_setup(Ctx &c) {
    Learned *L = c.learned;
    if (L->train_ready) return 0;
    const size_t n = (size_t)L->n, n4 = 4 * n;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    ok(lalloc(&L->Z, n * kH)); ok(lalloc(&L->y, n)); ok(lalloc(&L->dy, n));
    ok(lalloc(&L->part, (size_t)L->part_blocks * kNP)); ok(lalloc(&L->grad, kNP)); ok(lalloc(&L->omega, n));
    ok(lalloc(&L->nb, 4)); ok(lalloc(&L->nr, 4)); ok(lalloc(&L->nrm_part, 4 * (size_t)kNormBlocks));
    ok(lalloc(&L->r0, n4)); ok(lalloc(&L->u, n4)); ok(lalloc(&L->w, n4)); ok(lalloc(&L->d, n4));
    ok(lalloc(&L->r1, n4)); ok(lalloc(&L->R1, n4)); ok(lalloc(&L->g, n4)); ok(lalloc(&L->tmp, n4));
    ok(lalloc(&L->zero4, n4));
    if (e != cudaSuccess) return 2;
    L->train_ready = true;
    return 0;
}

// stencil features of the current finest matrix (after each assembly)
static void learned_features(Ctx &c, cudaStream_t s) {
    Learned *L = c.learned;
    const DevLevel &F = c.lev[c.D];
    diag_partial_kernel<<<kDiagParts, 256, 0, s>>>(F.n, F.rp, F.ci, F.A64, L->diag_part);
    features_kernel<<<(F.n + 127) / 128, 128, 0, s>>>(F.n, F.rp, F.ci, F.A64, L->corner, L->diag_part, L->X);
}

int learned_params(Ctx &c, double *get, const double *set, cudaStream_t s) {
    Learned *L = c.learned;
    std::vector<float> h(kNP);
    if (set) {
        for (int q = 0; q < kNP; q++) h[q] = (float)set[q];
        for (int r = kFU; r < kF; r++) for (int j = 0; j < kH; j++) h[r * kH + j] = 0.f;
        if (cudaMemcpyAsync(L->prm, h.data(), sizeof(float) * kNP, cudaMemcpyHostToDevice, s) != cudaSuccess) return 2;
        cudaMemsetAsync(L->m, 0, sizeof(float) * kNP, s);
        cudaMemsetAsync(L->v, 0, sizeof(float) * kNP, s);
        L->adam_t = 0;
        w1t_from_prm_kernel<<<(kF * kH + 255) / 256, 256, 0, s>>>(L->prm, L->W1T);
        if (cudaStreamSynchronize(s) != cudaSuccess) return 2;   // h is a pageable source
    }
    if (get) {
        if (cudaMemcpyAsync(h.data(), L->prm, sizeof(float) * kNP, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 2;
        if (cudaStreamSynchronize(s) != cudaSuccess) return 2;
        for (int q = 0; q < kNP; q++) get[q] = h[q];
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// the whole optimiser state: parameters, Adam's two moments, its step count (3 kNP + 1)
int learned_state(Ctx &c, double *get, const double *set, cudaStream_t s) {
    Learned *L = c.learned;
    std::vector<float> h(3 * (size_t)kNP);
    float *dst[3] = {L->prm, L->m, L->v};
    if (set) {
        for (size_t q = 0; q < h.size(); q++) h[q] = (float)set[q];
        for (int k = 0; k < 3; k++)
            for (int r = kFU; r < kF; r++) for (int j = 0; j < kH; j++) h[(size_t)k * kNP + r * kH + j] = 0.f;
        for (int k = 0; k < 3; k++)
            if (cudaMemcpyAsync(dst[k], h.data() + (size_t)k * kNP, sizeof(float) * kNP, cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
                return 2;
        L->adam_t = (int)set[3 * kNP];
        w1t_from_prm_kernel<<<(kF * kH + 255) / 256, 256, 0, s>>>(L->prm, L->W1T);
        if (cudaStreamSynchronize(s) != cudaSuccess) return 2;
    }
    if (get) {
        for (int k = 0; k < 3; k++)
            if (cudaMemcpyAsync(h.data() + (size_t)k * kNP, dst[k], sizeof(float) * kNP, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
                return 2;
        if (cudaStreamSynchronize(s) != cudaSuccess) return 2;
        for (size_t q = 0; q < h.size(); q++) get[q] = h[q];
        get[3 * kNP] = L->adam_t;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// one residual sample R0 = L->r0 ([n][4], lanes beyond the sample's zero): loss into *loss_slot
// (device), and with need_grad its gradient, weighted, into L->grad (added when accumulate)
static void sample_pass(Ctx &c, bool need_grad, double weight, bool accumulate, double *loss_slot, cudaStream_t s) {
    Learned *L = c.learned;
    DevLevel &F = c.lev[c.D];
    const int n = F.n;
    const int64_t m4 = (int64_t)n * 4;
    const unsigned g4 = blocks_for(m4);
    // features of the sample: u = D^-1 R0, w = R0 - A u, columns 28, 29
    launch_norms(L->r0, n, 4, L->nrm_part, L->nb, s);
    scale_rows_kernel<<<g4, 256, 0, s>>>(n, F.dinv64, L->r0, L->u);
    launch_residual<double>(F, F.A64, L->r0, L->u, L->w, 4, s, -1);
    rfeat_kernel<<<blocks_for(n), 256, 0, s>>>(n, L->r0, L->w, L->nb, L->X);
    mlp_forward_kernel<<<(L->npad / 16 + 7) / 8, 256, 0, s>>>(n, L->X, L->W1T, L->prm, need_grad ? L->Z : nullptr, L->y);
    omega_delta_kernel<<<g4, 256, 0, s>>>(n, L->y, L->u, L->omega, L->d);
    // the learned iteration: r1 = R0 - A delta, R1 = r1 - A V r1
    launch_residual<double>(F, F.A64, L->r0, L->d, L->r1, 4, s, -1);
    cudaMemcpyAsync(F.b64, L->r1, sizeof(double) * m4, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(F.x64, 0, sizeof(double) * m4, s);
    enqueue_vcycle64_from(c, c.D, 4, s);
    launch_residual<double>(F, F.A64, L->r1, F.x64, L->R1, 4, s, -1);
    launch_norms(L->R1, n, 4, L->nrm_part, L->nr, s);
    loss_kernel<<<1, 32, 0, s>>>(L->nb, L->nr, loss_slot);
    if (!need_grad) return;
    // adjoint: g = 2 R1 / ||R1||^2; C^T g = g - V A g; dL/ddelta = -A C^T g
    seed_kernel<<<g4, 256, 0, s>>>(n, L->R1, L->nr, L->g);
    launch_residual<double>(F, F.A64, L->zero4, L->g, L->tmp, 4, s, -1);          // -A g
    cudaMemcpyAsync(F.b64, L->tmp, sizeof(double) * m4, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(F.x64, 0, sizeof(double) * m4, s);
    enqueue_vcycle64_from(c, c.D, 4, s);                                           // -V A g
    axpy_kernel<<<g4, 256, 0, s>>>(m4, 1.0, F.x64, L->g);                           // C^T g
    launch_residual<double>(F, F.A64, L->zero4, L->g, L->tmp, 4, s, -1);          // -A C^T g
    dy_kernel<<<blocks_for(n), 256, 0, s>>>(n, L->tmp, L->u, L->y, weight, L->dy);
    mlp_backward_kernel<<<L->part_blocks, 256, 0, s>>>(n, L->X, L->Z, L->dy, L->prm, L->part);
    grad_reduce_kernel<<<(kNP + 255) / 256, 256, 0, s>>>(L->part_blocks, L->part, accumulate ? 1 : 0, L->grad);
}

static int ensure_loss(Learned *L, int count) {
    if (count <= L->loss_cap) return 0;
    if (L->loss_dev) cudaFree(L->loss_dev);
    L->loss_dev = nullptr;
    L->loss_cap = 0;
    if (lalloc(&L->loss_dev, (size_t)count) != cudaSuccess) return 2;
    L->loss_cap = count;
    return 0;
}

int learned_loss_grad(Ctx &c, const double *r0_user, int ns, double *loss, double *grad, cudaStream_t s) {
    Learned *L = c.learned;
    if (train_setup(c) || ensure_loss(L, 1)) return 2;
    learned_features(c, s);
    launch_pack(r0_user, L->n, ns, 4, L->r0, s, c.fperm);
    sample_pass(c, grad != nullptr, 1.0, false, L->loss_dev, s);
    if (cudaMemcpyAsync(loss, L->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return 2;
    if (grad && cudaMemcpyAsync(grad, L->grad, sizeof(double) * kNP, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return 2;
    return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// residual histories of plain FP64 V-cycles from x = 0 on the columns of rhs ([n][ns] user
// order, device, ns <= 4): the residual block before cycles skip .. skip + keep - 1
int learned_collect(Ctx &c, const double *rhs_user, int ns, int skip, int keep, cudaStream_t s) {
    Learned *L = c.learned;
    if (train_setup(c)) return 2;
    DevLevel &F = c.lev[c.D];
    const int n = F.n;
    const size_t blk = 4 * (size_t)n;
    const int need = L->bank_n + keep;
    if (need > L->bank_cap) {
        double *nbk = nullptr;
        if (lalloc(&nbk, (size_t)need * blk) != cudaSuccess) return 2;
        if (L->bank) {
            cudaMemcpyAsync(nbk, L->bank, sizeof(double) * (size_t)L->bank_n * blk, cudaMemcpyDeviceToDevice, s);
            cudaStreamSynchronize(s);
            cudaFree(L->bank);
        }
        L->bank = nbk;
        L->bank_cap = need;
    }
    const int64_t m4 = (int64_t)blk;
    double *b = L->r1, *x = L->R1, *r = L->w;
    pack_cols_kernel<<<blocks_for(m4), 256, 0, s>>>(rhs_user, n, ns, 0, ns, c.fperm, b);
    cudaMemsetAsync(x, 0, sizeof(double) * m4, s);
    for (int k = 0; k < skip + keep; k++) {
        launch_residual<double>(F, F.A64, b, x, r, 4, s, -1);
        if (k >= skip)
            cudaMemcpyAsync(L->bank + (size_t)(L->bank_n + k - skip) * blk, r, sizeof(double) * m4,
                            cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(F.b64, r, sizeof(double) * m4, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(F.x64, 0, sizeof(double) * m4, s);
        enqueue_vcycle64_from(c, c.D, 4, s);
        launch_add_double(x, F.x64, m4, s);
    }
    L->bank_n += keep;
    return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// Adam steps over bank samples; order: host [steps][batch] sample indices; the step's
// gradient is the mean over its samples; loss_hist (host, may be null): mean loss per step
int learned_train(Ctx &c, int steps, double lr, const int *order, int batch, double *loss_hist, cudaStream_t s) {
    Learned *L = c.learned;
    if (batch < 1 || batch > kMaxBatch || steps < 0) return 1;
    for (size_t q = 0; q < (size_t)steps * batch; q++)
        if (order[q] < 0 || order[q] >= L->bank_n) return 1;
    if (train_setup(c) || ensure_loss(L, std::max(1, steps * batch))) return 2;
    const int n = L->n;
    learned_features(c, s);
    for (int it = 0; it < steps; it++) {
        for (int j = 0; j < batch; j++) {
            gather_samples_kernel<<<blocks_for((int64_t)n * 4), 256, 0, s>>>(n, L->bank, order[(size_t)it * batch + j],
                                                                            L->r0);
            sample_pass(c, true, 1.0 / batch, j > 0, L->loss_dev + (size_t)it * batch + j, s);
        }
        L->adam_t++;
        const float b1t = 1.f - powf(0.9f, (float)L->adam_t), b2t = 1.f - powf(0.999f, (float)L->adam_t);
        adam_kernel<<<(kNP + 255) / 256, 256, 0, s>>>((float)lr, b1t, b2t, L->grad, L->prm, L->m, L->v, L->W1T);
    }
    std::vector<double> lh((size_t)std::max(1, steps * batch));
    if (steps > 0 &&
        cudaMemcpyAsync(lh.data(), L->loss_dev, sizeof(double) * steps * batch, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return 2;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return 2;
    if (loss_hist)
        for (int it = 0; it < steps; it++) {
            double a = 0.0;
            for (int j = 0; j < batch; j++) a += lh[(size_t)it * batch + j];
            loss_hist[it] = a / batch;
        }
    return 0;
}

// on: the solves of this handle put the learned correction in front of every cycle (the
// stencil features are refreshed here and after every assembly)
int learned_enable(Ctx &c, int on, cudaStream_t s) {
    if (!on) { c.learned_on = 0; return 0; }
    learned_features(c, s);
    c.learned_on = 1;
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

void learned_refresh(Ctx &c, cudaStream_t s) {
    if (c.learned && c.learned_on) learned_features(c, s);
}

namespace {

template <class T> struct LV;
template <> struct LV<float> {
    static float *b(DevLevel &F) { return F.b32; }
    static float *x(DevLevel &F) { return F.x32; }
    static float *r(DevLevel &F) { return F.r32; }
    static const float *A(DevLevel &F) { return F.A32; }
    static const float *dinv(DevLevel &F) { return F.dinv32; }
};
template <> struct LV<double> {
    static double *b(DevLevel &F) { return F.b64; }
    static double *x(DevLevel &F) { return F.x64; }
    static double *r(DevLevel &F) { return F.r64; }
    static const double *A(DevLevel &F) { return F.A64; }
    static const double *dinv(DevLevel &F) { return F.dinv64; }
};

// b = r, x = omega D^-1 r at the finest level, from the FP64 residual rs ([n][R]) with
// squared norms nr; three launches of one dependent chain
template <class T, int R>
void enqueue_correction(Ctx &c, const double *rs, const double *nr, const int *off, double *omega_out,
                        cudaStream_t s, Chain *ch) {
    Learned *L = c.learned;
    DevLevel &F = c.lev[c.D];
    const int n = F.n;
    klaunch(lr_prep_kernel<T, R>, blocks_for((int64_t)n * R), 256u, 0, s, ch, n, rs, LV<T>::dinv(F), LV<T>::b(F),
            LV<T>::x(F));
    launch_residual<T>(F, LV<T>::A(F), LV<T>::b(F), LV<T>::x(F), LV<T>::r(F), R, s, -1, ch);
    klaunch(lr_solve_kernel<T, R>, (unsigned)((L->npad / 16 + 7) / 8), 256u, 0, s, ch, n,
            (const __nv_bfloat16 *)L->X, (const __nv_bfloat16 *)L->W1T, (const float *)L->prm,
            (const T *)LV<T>::b(F), (const T *)LV<T>::r(F), nr, off, LV<T>::x(F), omega_out);
}

template <class T>
void enqueue_correction_R(Ctx &c, int R, const double *rs, const double *nr, const int *off, double *omega_out,
                          cudaStream_t s, Chain *ch) {
    if (R == 1) enqueue_correction<T, 1>(c, rs, nr, off, omega_out, s, ch);
    else if (R == 2) enqueue_correction<T, 2>(c, rs, nr, off, omega_out, s, ch);
    else enqueue_correction<T, 4>(c, rs, nr, off, omega_out, s, ch);
}

// user-ordered outputs of learned_apply
template <class T>
__global__ void delta_to_user_kernel(int n, int ns, const T *__restrict__ x, const double *__restrict__ om,
                                     const int *__restrict__ fperm, double *__restrict__ delta,
                                     double *__restrict__ omega) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int i = fperm[u];
    for (int q = 0; q < ns; q++) delta[(size_t)u * ns + q] = (double)x[4 * (size_t)i + q];
    omega[u] = om[i];
}

}  // namespace

// the solve's correction in front of a cycle: b_T = r, x_T = omega D^-1 r (ctl->learned_off
// set: x_T = 0), reading the residual c.rs and its squared norms c.norm_out
void learned_enqueue(Ctx &c, int R, int precision, cudaStream_t s, Chain *ch) {
    const int *off = &c.ctl->learned_off;
    if (precision == LBMG_MIXED) enqueue_correction_R<float>(c, R, c.rs, c.norm_out, off, nullptr, s, ch);
    else enqueue_correction_R<double>(c, R, c.rs, c.norm_out, off, nullptr, s, ch);
}

// the correction of one residual r ([n][ns] user order, device, ns <= 4) by the solve's kernels:
// omega (host or device double[n]) and delta ([n][ns]), both user order, device
int learned_apply(Ctx &c, const double *r_user, int ns, int precision, double *omega_dev, double *delta_dev,
                  cudaStream_t s) {
    Learned *L = c.learned;
    if (train_setup(c)) return 2;
    const int n = L->n;
    learned_features(c, s);
    launch_pack(r_user, n, ns, 4, L->r0, s, c.fperm);
    launch_norms(L->r0, n, 4, L->nrm_part, L->nb, s);
    Chain ch;   // plain launches
    DevLevel &F = c.lev[c.D];
    if (precision == LBMG_MIXED) {
        enqueue_correction<float, 4>(c, L->r0, L->nb, nullptr, L->omega64, s, &ch);
        delta_to_user_kernel<float><<<blocks_for(n), 256, 0, s>>>(n, ns, F.x32, L->omega64, c.fperm, delta_dev, omega_dev);
    } else {
        enqueue_correction<double, 4>(c, L->r0, L->nb, nullptr, L->omega64, s, &ch);
        delta_to_user_kernel<double><<<blocks_for(n), 256, 0, s>>>(n, ns, F.x64, L->omega64, c.fperm, delta_dev, omega_dev);
    }
    return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int learned_nparams() { return kNP; }

}  // namespace lbmg
