// learned.cu -- learned relaxation weights for the finest-level Gauss-Seidel sweeps.
//
// Not in the paper, whose smoother is plain Gauss-Seidel (Sections 4.3, 5.2).  A
// 28 -> 64 (ReLU) -> 1 network maps each finest-level node's stencil (row
// coefficients over A_ii, summed per neighbour-corner offset, plus the relative
// diagonal and the entry count) to y; the node's sweep update is scaled by
// omega = 1.45 + 0.45 y / (1 + |y|), in (1, 1.9), which keeps the sweep
// convergent for SPD systems.  Training minimises the residual left by one
// V-cycle whose finest sweeps use those weights, over residuals taken from the
// histories of plain V-cycles; the gradient is the exact adjoint of the cycle
// (colour steps in reverse, and the symmetric coarse V-cycle for the coarse
// correction).  The dense layers run on the tensor cores (mma.sync BF16 x BF16
// -> FP32); the cycle and its adjoint run in FP64 with the solver's kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lbmg_internal.h"

namespace lbmg {

// exported by api.cu: one FP64 V-cycle on A_top e = b_top from e = 0 (lev[top].x64)
void enqueue_vcycle64_from(Ctx &c, int top, int R, cudaStream_t s);

namespace {

constexpr int kF = 32;        // feature columns (28 used)
constexpr int kH = 64;        // hidden units
constexpr int kNP = kF * kH + kH + kH + 1;   // FP32 parameters: W1 [32][64], b1, w2, b2

// ---------------------------------------------------------------- features
__global__ void mean_diag_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const double *__restrict__ A, double *__restrict__ out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int lo = rp[i], hi = rp[i + 1];
        while (lo < hi) { int mid = (lo + hi) >> 1; if (ci[mid] < i) lo = mid + 1; else hi = mid; }
        s += A[lo];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (double)(n > 0 ? n : 1);
}

__global__ void features_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                const double *__restrict__ A, const int *__restrict__ corner,
                                const double *__restrict__ mean_diag, __nv_bfloat16 *__restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[kF];
#pragma unroll
    for (int q = 0; q < kF; q++) f[q] = 0.f;
    double diag = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) if (ci[k] == i) diag = A[k];
    const int cx = corner[3 * i], cy = corner[3 * i + 1], cz = corner[3 * i + 2];
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        const int ox = corner[3 * j] - cx + 1, oy = corner[3 * j + 1] - cy + 1, oz = corner[3 * j + 2] - cz + 1;
        const int b = (ox * 3 + oy) * 3 + oz;
        if (b >= 0 && b < 27) {
#pragma unroll
            for (int q = 0; q < 27; q++) if (q == b) f[q] += (float)(A[k] / diag);
        }
    }
    f[13] = (float)(diag / *mean_diag);
    f[27] = (float)(rp[i + 1] - rp[i]) / 27.f;
    __nv_bfloat16 *o = X + (size_t)i * kF;
#pragma unroll
    for (int q = 0; q < kF; q++) o[q] = __float2bfloat16_rn(f[q]);
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

// Z = X W1 + b1 (FP32), y = relu(Z) w2 + b2; one warp per 16 rows.  X has ceil(n/16)*16 rows.
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
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int col = nt * 8 + 2 * t;
        acc[nt][0] = b1[col]; acc[nt][1] = b1[col + 1]; acc[nt][2] = b1[col]; acc[nt][3] = b1[col + 1];
    }
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
        uint32_t a[4];
        const __nv_bfloat16 *x0 = X + (size_t)(row0 + g) * kF + ks * 16 + 2 * t;
        const __nv_bfloat16 *x8 = X + (size_t)(row0 + g + 8) * kF + ks * 16 + 2 * t;
        a[0] = *reinterpret_cast<const uint32_t *>(x0);
        a[1] = *reinterpret_cast<const uint32_t *>(x8);
        a[2] = *reinterpret_cast<const uint32_t *>(x0 + 8);
        a[3] = *reinterpret_cast<const uint32_t *>(x8 + 8);
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            uint32_t b[2];
            const __nv_bfloat16 *w = sW + (nt * 8 + g) * kF + ks * 16 + 2 * t;
            b[0] = *reinterpret_cast<const uint32_t *>(w);
            b[1] = *reinterpret_cast<const uint32_t *>(w + 8);
            mma_bf16(acc[nt], a, b);
        }
    }
    float y0 = 0.f, y8 = 0.f;
    const int r_a = row0 + g, r_b = row0 + g + 8;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int col = nt * 8 + 2 * t;
        y0 += fmaxf(acc[nt][0], 0.f) * w2[col] + fmaxf(acc[nt][1], 0.f) * w2[col + 1];
        y8 += fmaxf(acc[nt][2], 0.f) * w2[col] + fmaxf(acc[nt][3], 0.f) * w2[col + 1];
        if (Z) {
            if (r_a < n) *reinterpret_cast<float2 *>(Z + (size_t)r_a * kH + col) = make_float2(acc[nt][0], acc[nt][1]);
            if (r_b < n) *reinterpret_cast<float2 *>(Z + (size_t)r_b * kH + col) = make_float2(acc[nt][2], acc[nt][3]);
        }
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y8 += __shfl_xor_sync(0xffffffffu, y8, 1);
    y8 += __shfl_xor_sync(0xffffffffu, y8, 2);
    if (t == 0) {
        if (r_a < n) y[r_a] = y0 + b2[0];
        if (r_b < n) y[r_b] = y8 + b2[0];
    }
}

// omega = 1.45 + 0.45 y / (1 + |y|); learned inverse diagonals omega / a_ii
__global__ void omega_kernel(int n, const float *__restrict__ y, const double *__restrict__ dinv64,
                             const float *__restrict__ dinv32, double *__restrict__ omega, double *__restrict__ dl64,
                             float *__restrict__ dl32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double yy = (double)y[i];
    const double om = 1.45 + 0.45 * yy / (1.0 + fabs(yy));
    omega[i] = om;
    if (dl64) dl64[i] = om * dinv64[i];
    // rows that relaxation skips (inverse diagonal 0) stay skipped
    if (dl32) dl32[i] = dinv32[i] != 0.f ? (float)(om * dinv64[i]) : 0.f;
}

// ---------------------------------------------------------------- V-cycle adjoint pieces
// delta = 0 except colour rows: omega r / a_ii   (vectors [n][4])
__global__ void colour_delta_kernel(int r0, int r1, int n, const double *__restrict__ omega,
                                    const double *__restrict__ dinv, const double *__restrict__ r,
                                    double *__restrict__ delta) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    const int i = (int)(q >> 2);
    delta[q] = (i >= r0 && i < r1) ? omega[i] * dinv[i] * r[q] : 0.0;
}

// rows of one colour: domega_i += -sum_q (A g)_iq r_iq / a_ii ; g_i -= omega_i/a_ii (A g)_i
// (nAg holds -(A g), from the residual kernel with a zero right-hand side)
__global__ void colour_adjoint_kernel(int r0, int r1, const double *__restrict__ omega,
                                      const double *__restrict__ dinv, const double *__restrict__ nAg,
                                      const double *__restrict__ r, double *__restrict__ g,
                                      double *__restrict__ domega) {
    const int i = r0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r1) return;
    double s = 0.0;
    for (int q = 0; q < 4; q++) {
        const double ag = -nAg[4 * (size_t)i + q];
        s += ag * r[4 * (size_t)i + q];
        g[4 * (size_t)i + q] -= omega[i] * dinv[i] * ag;
    }
    domega[i] -= s * dinv[i];
}

__global__ void axpy_kernel(int64_t m, double a, const double *__restrict__ x, double *__restrict__ y) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < m) y[q] += a * x[q];
}

// g = 2 w_q r (w_q per lane)
__global__ void seed_adjoint_kernel(int n, const double *__restrict__ r, const double *__restrict__ w,
                                    double *__restrict__ g) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    g[q] = 2.0 * w[q & 3] * r[q];
}

__global__ void gather_samples_kernel(int n, const double *__restrict__ bank, const int *__restrict__ sel, int ns,
                                      double *__restrict__ out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    const int i = (int)(q >> 2), lane = (int)(q & 3);
    out[q] = lane < ns ? bank[(size_t)sel[lane] * n + i] : 0.0;
}

// columns c0..c0+lanes-1 of a user-ordered [n][ns] array into lanes of internal [n][4]
__global__ void pack_cols_kernel(const double *__restrict__ u, int n, int ns, int c0, int lanes,
                                 const int *__restrict__ fperm, double *__restrict__ out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    const int i = (int)(q >> 2), lane = (int)(q & 3);
    out[4 * (size_t)fperm[i] + lane] = lane < lanes ? u[(size_t)i * ns + c0 + lane] : 0.0;
}

__global__ void store_sample_kernel(int n, int lane, const double *__restrict__ r, double *__restrict__ bank) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) bank[i] = r[4 * (size_t)i + lane];
}

// dy = domega * 0.45 / (1 + |y|)^2
__global__ void dy_kernel(int n, const double *__restrict__ domega, const float *__restrict__ y,
                          float *__restrict__ dy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = 1.0 + fabs((double)y[i]);
    dy[i] = (float)(domega[i] * 0.45 / (a * a));
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

// grad[q] = sum over blocks of part (fixed order)
__global__ void grad_reduce_kernel(int nblocks, const float *__restrict__ part, double *__restrict__ grad) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNP) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; b++) s += (double)part[(size_t)b * kNP + q];
    grad[q] = s;
}

// Adam on FP32 master parameters (rows 28..31 of W1 stay zero); refreshes the BF16 W1^T
__global__ void adam_kernel(float lr, float b1t, float b2t, const double *__restrict__ grad, float *__restrict__ prm,
                            float *__restrict__ m, float *__restrict__ v, __nv_bfloat16 *__restrict__ W1T) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNP) return;
    if (q < kF * kH && q / kH >= 28) return;
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
    W1T[(q % kH) * kF + q / kH] = __float2bfloat16_rn(q / kH < 28 ? prm[q] : 0.f);
}

}  // namespace


// ---------------------------------------------------------------- host side

namespace {

template <class T>
cudaError_t lalloc(T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
    if (e == cudaSuccess) cudaMemset(*p, 0, (count ? count : 1) * sizeof(T));
    return e;
}

}  // namespace

struct Learned {
    int n = 0, npad = 0, nsteps = 0, part_blocks = 0, adam_t = 0;
    __nv_bfloat16 *X = nullptr, *W1T = nullptr;
    float *prm = nullptr, *m = nullptr, *v = nullptr, *Z = nullptr, *y = nullptr, *dy = nullptr, *part = nullptr;
    double *mean = nullptr, *omega = nullptr, *domega = nullptr, *grad = nullptr, *wq = nullptr;
    double *snap = nullptr, *delta = nullptr, *g = nullptr, *tmp = nullptr, *w = nullptr, *zero4 = nullptr;
    double *nrm_part = nullptr, *nrm_out = nullptr;
    int *sel = nullptr, *corner = nullptr;
    double *bank = nullptr;
    int bank_cap = 0, bank_n = 0;
    double *dl64 = nullptr;
    float *dl32 = nullptr;
};

void learned_free(Ctx &c) {
    Learned *L = c.learned;
    if (!L) return;
    void *ptrs[] = {L->X, L->W1T, L->prm, L->m, L->v, L->Z, L->y, L->dy, L->part, L->mean, L->omega, L->domega,
                    L->grad, L->wq, L->snap, L->delta, L->g, L->tmp, L->w, L->zero4, L->nrm_part, L->nrm_out,
                    L->sel, L->corner, L->bank, L->dl64, L->dl32};
    for (void *q : ptrs) if (q) cudaFree(q);
    delete L;
    c.learned = nullptr;
}

int learned_setup(Ctx &c, cudaStream_t s) {
    if (c.learned) return 0;
    if (c.D == c.d0) return 1;   // needs a coarser level for the cycle
    Learned *L = new Learned();
    c.learned = L;
    const DevLevel &F = c.lev[c.D];
    L->n = F.n;
    L->npad = (F.n + 15) / 16 * 16;
    L->nsteps = 8 * (c.nu1 + c.nu2) + 1;
    L->part_blocks = 152;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    ok(lalloc(&L->X, (size_t)L->npad * kF));
    ok(lalloc(&L->W1T, (size_t)kH * kF));
    ok(lalloc(&L->prm, kNP)); ok(lalloc(&L->m, kNP)); ok(lalloc(&L->v, kNP));
    ok(lalloc(&L->Z, (size_t)L->n * kH)); ok(lalloc(&L->y, L->n)); ok(lalloc(&L->dy, L->n));
    ok(lalloc(&L->part, (size_t)L->part_blocks * kNP));
    ok(lalloc(&L->mean, 1)); ok(lalloc(&L->omega, L->n)); ok(lalloc(&L->domega, L->n));
    ok(lalloc(&L->grad, kNP)); ok(lalloc(&L->wq, 4));
    ok(lalloc(&L->snap, (size_t)(L->nsteps + 1) * L->n * 4));
    ok(lalloc(&L->delta, (size_t)L->n * 4)); ok(lalloc(&L->g, (size_t)L->n * 4)); ok(lalloc(&L->tmp, (size_t)L->n * 4));
    ok(lalloc(&L->w, (size_t)L->n * 4)); ok(lalloc(&L->zero4, (size_t)L->n * 4));
    ok(lalloc(&L->nrm_part, 4 * (size_t)kNormBlocks)); ok(lalloc(&L->nrm_out, 8));
    ok(lalloc(&L->sel, 4)); ok(lalloc(&L->corner, 3 * (size_t)L->n));
    ok(lalloc(&L->dl64, L->n)); ok(lalloc(&L->dl32, L->n));
    if (e != cudaSuccess) { learned_free(c); return 2; }
    cudaMemcpy(L->corner, c.host.lev[c.D].corner.data(), 3 * sizeof(int) * (size_t)L->n, cudaMemcpyHostToDevice);
    return 0;
}

// features of the current finest matrix (call after assembly)
static void learned_features(Ctx &c, cudaStream_t s) {
    Learned *L = c.learned;
    const DevLevel &F = c.lev[c.D];
    mean_diag_kernel<<<1, 1024, 0, s>>>(F.n, F.rp, F.ci, F.A64, L->mean);
    features_kernel<<<(F.n + 127) / 128, 128, 0, s>>>(F.n, F.rp, F.ci, F.A64, L->corner, L->mean, L->X);
}

static void learned_forward(Ctx &c, bool keepZ, cudaStream_t s) {
    Learned *L = c.learned;
    const int warps = L->npad / 16;
    mlp_forward_kernel<<<(warps + 7) / 8, 256, 0, s>>>(L->n, L->X, L->W1T, L->prm, keepZ ? L->Z : nullptr, L->y);
}

int learned_params(Ctx &c, double *get, const double *set, cudaStream_t s) {
    Learned *L = c.learned;
    std::vector<float> h(kNP);
    if (set) {
        for (int q = 0; q < kNP; q++) h[q] = (float)set[q];
        for (int r = 28; r < kF; r++) for (int j = 0; j < kH; j++) h[r * kH + j] = 0.f;
        if (cudaMemcpyAsync(L->prm, h.data(), sizeof(float) * kNP, cudaMemcpyHostToDevice, s) != cudaSuccess) return 2;
        cudaMemsetAsync(L->m, 0, sizeof(float) * kNP, s);
        cudaMemsetAsync(L->v, 0, sizeof(float) * kNP, s);
        L->adam_t = 0;
        w1t_from_prm_kernel<<<(kF * kH + 255) / 256, 256, 0, s>>>(L->prm, L->W1T);
    }
    if (get) {
        if (cudaMemcpyAsync(h.data(), L->prm, sizeof(float) * kNP, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 2;
        cudaStreamSynchronize(s);
        for (int q = 0; q < kNP; q++) get[q] = h[q];
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// loss (and gradient) of one V-cycle with learned finest sweeps on residual samples
// r0 = L->snap[0] ([n][4], lanes beyond ns zero)
static int learned_loss_grad_dev(Ctx &c, int ns, bool need_grad, double *loss, cudaStream_t s) {
    Learned *L = c.learned;
    DevLevel &F = c.lev[c.D], &Cc = c.lev[c.D - 1];
    const int n = F.n;
    const int64_t m4 = (int64_t)n * 4;
    const unsigned g4 = (unsigned)((m4 + 255) / 256);
    learned_forward(c, need_grad, s);
    omega_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, L->y, F.dinv64, F.dinv32, L->omega, nullptr, nullptr);
    // forward through the cycle
    int sidx = 0;
    auto snap = [&](int k) { return L->snap + (size_t)k * m4; };
    auto colour_step = [&](int col) {
        colour_delta_kernel<<<g4, 256, 0, s>>>(F.cs[col], F.cs[col + 1], n, L->omega, F.dinv64, snap(sidx), L->delta);
        launch_residual<double>(F, F.A64, snap(sidx), L->delta, snap(sidx + 1), 4, s, n);
        sidx++;
    };
    for (int q = 0; q < c.nu1; q++) for (int col = 0; col < 8; col++) colour_step(col);
    {
        launch_restrict<double>(Cc, snap(sidx), Cc.b64, 4, s);
        cudaMemsetAsync(Cc.x64, 0, sizeof(double) * 4 * (size_t)Cc.n, s);
        enqueue_vcycle64_from(c, c.D - 1, 4, s);
        cudaMemsetAsync(L->w, 0, sizeof(double) * m4, s);
        launch_prolong_add<double>(F, Cc.x64, L->w, 4, s);
        launch_residual<double>(F, F.A64, snap(sidx), L->w, snap(sidx + 1), 4, s, n);
        sidx++;
    }
    for (int q = 0; q < c.nu2; q++) for (int col = 7; col >= 0; col--) colour_step(col);
    // loss weights 1 / (ns ||r0||^2) and loss
    double nb[4], nr[4], w[4] = {0, 0, 0, 0};
    launch_norms(snap(0), n, 4, L->nrm_part, L->nrm_out, s);
    cudaMemcpyAsync(nb, L->nrm_out, sizeof nb, cudaMemcpyDeviceToHost, s);
    launch_norms(snap(sidx), n, 4, L->nrm_part, L->nrm_out, s);
    cudaMemcpyAsync(nr, L->nrm_out, sizeof nr, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return 2;
    double lsum = 0.0;
    for (int q = 0; q < ns; q++) { w[q] = nb[q] > 0 ? 1.0 / (ns * nb[q]) : 0.0; lsum += w[q] * nr[q]; }
    *loss = lsum;
    if (!need_grad) return 0;
    // adjoint
    cudaMemcpyAsync(L->wq, w, sizeof w, cudaMemcpyHostToDevice, s);
    seed_adjoint_kernel<<<g4, 256, 0, s>>>(n, snap(sidx), L->wq, L->g);
    cudaMemsetAsync(L->domega, 0, sizeof(double) * n, s);
    auto colour_adj = [&](int col) {
        sidx--;
        launch_residual<double>(F, F.A64, L->zero4, L->g, L->tmp, 4, s, n);          // tmp = -A g
        const int r0 = F.cs[col], r1 = F.cs[col + 1];
        if (r1 > r0)
            colour_adjoint_kernel<<<(r1 - r0 + 255) / 256, 256, 0, s>>>(r0, r1, L->omega, F.dinv64, L->tmp, snap(sidx),
                                                                       L->g, L->domega);
    };
    for (int q = 0; q < c.nu2; q++) for (int col = 0; col < 8; col++) colour_adj(col);
    {
        sidx--;
        launch_residual<double>(F, F.A64, L->zero4, L->g, L->tmp, 4, s, n);          // -A g
        launch_restrict<double>(Cc, L->tmp, Cc.b64, 4, s);                           // -P^T A g
        cudaMemsetAsync(Cc.x64, 0, sizeof(double) * 4 * (size_t)Cc.n, s);
        enqueue_vcycle64_from(c, c.D - 1, 4, s);                                     // -V P^T A g
        cudaMemsetAsync(L->w, 0, sizeof(double) * m4, s);
        launch_prolong_add<double>(F, Cc.x64, L->w, 4, s);                           // -P V P^T A g
        axpy_kernel<<<g4, 256, 0, s>>>(m4, 1.0, L->w, L->g);
    }
    for (int q = 0; q < c.nu1; q++) for (int col = 7; col >= 0; col--) colour_adj(col);
    dy_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, L->domega, L->y, L->dy);
    mlp_backward_kernel<<<L->part_blocks, 256, 0, s>>>(n, L->X, L->Z, L->dy, L->prm, L->part);
    grad_reduce_kernel<<<(kNP + 255) / 256, 256, 0, s>>>(L->part_blocks, L->part, L->grad);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int learned_loss_grad(Ctx &c, const double *r0_user, int ns, double *loss, double *grad, cudaStream_t s) {
    Learned *L = c.learned;
    learned_features(c, s);
    launch_pack(r0_user, c.lev[c.D].n, ns, 4, L->snap, s, c.fperm);
    int st = learned_loss_grad_dev(c, ns, grad != nullptr, loss, s);
    if (st) return st;
    if (grad) {
        cudaMemcpyAsync(grad, L->grad, sizeof(double) * kNP, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return 2;
    }
    return 0;
}

// residual histories of plain FP64 V-cycles: rhs columns [n][ns] (user order, device)
int learned_collect(Ctx &c, const double *rhs_user, int ns, int skip, int keep, cudaStream_t s) {
    Learned *L = c.learned;
    DevLevel &F = c.lev[c.D];
    const int n = F.n;
    const int need = L->bank_n + ns * keep;
    if (need > L->bank_cap) {
        double *nb = nullptr;
        if (lalloc(&nb, (size_t)need * n) != cudaSuccess) return 2;
        if (L->bank) { cudaMemcpyAsync(nb, L->bank, sizeof(double) * (size_t)L->bank_n * n, cudaMemcpyDeviceToDevice, s); cudaStreamSynchronize(s); cudaFree(L->bank); }
        L->bank = nb;
        L->bank_cap = need;
    }
    for (int c0 = 0; c0 < ns; c0 += 4) {
        const int lanes = std::min(4, ns - c0);
        double *b = L->tmp, *x = L->w, *r = L->delta;
        pack_cols_kernel<<<(unsigned)(((int64_t)n * 4 + 255) / 256), 256, 0, s>>>(rhs_user, n, ns, c0, lanes, c.fperm, b);
        cudaMemsetAsync(x, 0, sizeof(double) * 4 * (size_t)n, s);
        for (int k = 0; k < skip + keep; k++) {
            launch_residual<double>(F, F.A64, b, x, r, 4, s, n);
            if (k >= skip)
                for (int q = 0; q < lanes; q++)
                    store_sample_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, q, r, L->bank + (size_t)(L->bank_n + q * keep + (k - skip)) * n);
            cudaMemcpyAsync(F.b64, r, sizeof(double) * 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
            cudaMemsetAsync(F.x64, 0, sizeof(double) * 4 * (size_t)n, s);
            enqueue_vcycle64_from(c, c.D, 4, s);
            launch_add_double(x, F.x64, (int64_t)n * 4, s);
        }
        L->bank_n += lanes * keep;
    }
    return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// Adam steps over bank samples; order: host [steps][batch] sample indices, batch <= 4
int learned_train(Ctx &c, int steps, double lr, const int *order, int batch, double *loss_hist, cudaStream_t s) {
    Learned *L = c.learned;
    const int n = c.lev[c.D].n;
    if (batch < 1 || batch > 4 || L->bank_n == 0) return 1;
    learned_features(c, s);
    for (int it = 0; it < steps; it++) {
        int sel[4] = {0, 0, 0, 0};
        for (int q = 0; q < batch; q++) {
            sel[q] = order[(size_t)it * batch + q];
            if (sel[q] < 0 || sel[q] >= L->bank_n) return 1;
        }
        cudaMemcpyAsync(L->sel, sel, sizeof sel, cudaMemcpyHostToDevice, s);
        gather_samples_kernel<<<(unsigned)(((int64_t)n * 4 + 255) / 256), 256, 0, s>>>(n, L->bank, L->sel, batch, L->snap);
        double loss = 0;
        int st = learned_loss_grad_dev(c, batch, true, &loss, s);
        if (st) return st;
        if (loss_hist) loss_hist[it] = loss;
        L->adam_t++;
        const float b1t = 1.f - powf(0.9f, (float)L->adam_t), b2t = 1.f - powf(0.999f, (float)L->adam_t);
        adam_kernel<<<(kNP + 255) / 256, 256, 0, s>>>((float)lr, b1t, b2t, L->grad, L->prm, L->m, L->v, L->W1T);
    }
    return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// omega for the current matrix; the solve then scales its finest sweeps by it
int learned_enable(Ctx &c, int on, cudaStream_t s) {
    Learned *L = c.learned;
    if (!on) { c.learned_on = 0; return 0; }
    DevLevel &F = c.lev[c.D];
    learned_features(c, s);
    learned_forward(c, false, s);
    omega_kernel<<<(F.n + 255) / 256, 256, 0, s>>>(F.n, L->y, F.dinv64, F.dinv32, L->omega, L->dl64, L->dl32);
    c.learned_dinv64 = L->dl64;
    c.learned_dinv32 = L->dl32;
    c.learned_on = 1;
    return cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int learned_omega(Ctx &c, double *omega_user) {
    Learned *L = c.learned;
    const int n = c.lev[c.D].n;
    std::vector<double> om(n);
    if (cudaMemcpy(om.data(), L->omega, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
    for (int u = 0; u < n; u++) omega_user[u] = om[c.host.fperm[u]];
    return 0;
}

int learned_nparams() { return kNP; }

}  // namespace lbmg
