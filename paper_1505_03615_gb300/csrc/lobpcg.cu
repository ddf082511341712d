// lobpcg.cu -- the smallest eigenpairs of L x = lambda M x on the finest level (the spectral
// analysis of Section 5.1), by the locally optimal block preconditioned conjugate gradient
// method, preconditioned by one FP64 V-cycle of the assembled A = M + t L.
//
// Each iteration works on the basis U = [X W P] of the current eigenvector block X, its
// preconditioned residuals W = V(L X - M X Lambda) and the previous search directions P,
// and replaces X and P by the Rayleigh-Ritz combinations of U:
//   - on the device: the products L U and M U (CSR, FP64), the V-cycles of the residuals
//     (four columns per cycle), the Gram matrices U^T L U and U^T M U (two-pass sums), and
//     the combinations of U, L U and M U with the Ritz coefficients;
//   - on the host: the small Rayleigh-Ritz problem (at most 48 x 48): the columns are scaled
//     to unit M-norm, directions of the M-Gram matrix below 1e-13 of its largest eigenvalue
//     are dropped (W and P become nearly dependent as the iteration converges), and the
//     reduced symmetric problem is solved by cyclic Jacobi rotations.
// The host reads the Gram matrices and the residual norms once per iteration.
// Blocks are stored column by column ([columns][n]) in the device dof order.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lbmg_internal.h"

namespace lbmg {

// exported by api.cu: one FP64 V-cycle on A_top e = b_top from e = 0 (lev[top].x64)
void enqueue_vcycle64_from(Ctx &c, int top, int R, cudaStream_t s);

namespace {

constexpr int kMaxK = 16;
constexpr int kMaxM = 3 * kMaxK;
constexpr int kGramBlocks = 256;

__global__ void spmv_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ a, const double *__restrict__ x, double *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) s = fma(a[k], x[ci[k]], s);
    y[i] = s;
}

// part[blk][a][b] = sum over this block's rows i of U[a][i] V[b][i]  (a < ma, b < mb <= kMaxM):
// tiles of 32 rows of every column go through shared memory, each thread owns a few (a, b) pairs
constexpr int kTile = 32;
constexpr int kPairsPerThread = (kMaxM * kMaxM + 255) / 256;
__global__ void __launch_bounds__(256) gram_partial_kernel(int n, int ma, int mb, const double *__restrict__ U,
                                                           const double *__restrict__ V, double *__restrict__ part) {
    __shared__ double su[kMaxM][kTile], sv[kMaxM][kTile];
    const int rows = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * rows, i1 = min(n, i0 + rows);
    double acc[kPairsPerThread];
#pragma unroll
    for (int q = 0; q < kPairsPerThread; q++) acc[q] = 0.0;
    for (int t0 = i0; t0 < i1; t0 += kTile) {
        for (int e = threadIdx.x; e < kMaxM * kTile; e += blockDim.x) {
            const int a = e / kTile, r = e % kTile, i = t0 + r;
            su[a][r] = (a < ma && i < i1) ? U[(size_t)a * n + i] : 0.0;
            sv[a][r] = (a < mb && i < i1) ? V[(size_t)a * n + i] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPairsPerThread; q++) {
            const int pr = threadIdx.x + q * blockDim.x;
            if (pr < ma * mb) {
                const int a = pr / mb, b = pr % mb;
                double s = acc[q];
#pragma unroll 8
                for (int r = 0; r < kTile; r++) s = fma(su[a][r], sv[b][r], s);
                acc[q] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kPairsPerThread; q++) {
        const int pr = threadIdx.x + q * blockDim.x;
        if (pr < ma * mb) part[(size_t)blockIdx.x * ma * mb + pr] = acc[q];
    }
}

__global__ void gram_final_kernel(int nblocks, int mm, const double *__restrict__ part, double *__restrict__ out) {
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= mm) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; b++) s += part[(size_t)b * mm + pr];
    out[pr] = s;
}

// Out[j][i] = sum_{a < m} U[a + a0][i] Y[a][j]  (Y: m x k, row-major), j < k
__global__ void combine_kernel(int n, int m, int k, int a0, const double *__restrict__ U, const double *__restrict__ Y,
                               double *__restrict__ Out) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * k) return;
    const int j = (int)(q / n), i = (int)(q % n);
    double s = 0.0;
    for (int a = 0; a < m; a++) s = fma(U[(size_t)(a + a0) * n + i], Y[a * k + j], s);
    Out[(size_t)j * n + i] = s;
}

// R[j] = LX[j] - lambda_j MX[j]
__global__ void residual_block_kernel(int n, int k, const double *__restrict__ LX, const double *__restrict__ MX,
                                      const double *__restrict__ lam, double *__restrict__ R) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * k) return;
    const int j = (int)(q / n);
    R[q] = LX[q] - lam[j] * MX[q];
}

// four columns [4][n] <-> interleaved [n][4] (missing columns zero)
__global__ void interleave4_kernel(int n, int nc, const double *__restrict__ cols, double *__restrict__ v) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * 4) return;
    const int i = (int)(q >> 2), c = (int)(q & 3);
    v[q] = c < nc ? cols[(size_t)c * n + i] : 0.0;
}
__global__ void deinterleave4_kernel(int n, int nc, const double *__restrict__ v, double *__restrict__ cols) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * nc) return;
    const int c = (int)(q / n), i = (int)(q % n);
    cols[q] = v[(size_t)i * 4 + c];
}

// user [n][k] (user order) <-> columns [k][n] (device order): row perm[u] of the device order
__global__ void user_to_cols_kernel(int n, int k, const double *__restrict__ u, const int *__restrict__ perm,
                                    double *__restrict__ cols) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * k) return;
    const int r = (int)(q / k), j = (int)(q % k);
    cols[(size_t)j * n + perm[r]] = u[q];
}
__global__ void cols_to_user_kernel(int n, int k, const double *__restrict__ cols, const int *__restrict__ perm,
                                    double *__restrict__ u) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * k) return;
    const int r = (int)(q / k), j = (int)(q % k);
    u[q] = cols[(size_t)j * n + perm[r]];
}

inline unsigned nb(int64_t m) { return (unsigned)((m + 255) / 256); }

// cyclic Jacobi eigen-decomposition of the symmetric r x r matrix S (row-major, overwritten):
// eigenvalues in w (ascending), eigenvectors in the columns of Q (row-major r x r)
void jacobi_eig(int r, std::vector<double> &S, std::vector<double> &w, std::vector<double> &Q) {
    Q.assign((size_t)r * r, 0.0);
    for (int i = 0; i < r; i++) Q[(size_t)i * r + i] = 1.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < r; i++)
            for (int j = 0; j < r; j++) {
                const double v = S[(size_t)i * r + j] * S[(size_t)i * r + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < r; p++)
            for (int q = p + 1; q < r; q++) {
                const double apq = S[(size_t)p * r + q];
                if (apq == 0.0) continue;
                const double app = S[(size_t)p * r + p], aqq = S[(size_t)q * r + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < r; k++) {   // columns p, q of S
                    const double skp = S[(size_t)k * r + p], skq = S[(size_t)k * r + q];
                    S[(size_t)k * r + p] = c * skp - s * skq;
                    S[(size_t)k * r + q] = s * skp + c * skq;
                }
                for (int k = 0; k < r; k++) {   // rows p, q
                    const double spk = S[(size_t)p * r + k], sqk = S[(size_t)q * r + k];
                    S[(size_t)p * r + k] = c * spk - s * sqk;
                    S[(size_t)q * r + k] = s * spk + c * sqk;
                }
                for (int k = 0; k < r; k++) {
                    const double qkp = Q[(size_t)k * r + p], qkq = Q[(size_t)k * r + q];
                    Q[(size_t)k * r + p] = c * qkp - s * qkq;
                    Q[(size_t)k * r + q] = s * qkp + c * qkq;
                }
            }
    }
    std::vector<int> order(r);
    for (int i = 0; i < r; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return S[(size_t)a * r + a] < S[(size_t)b * r + b]; });
    w.resize(r);
    std::vector<double> Qs((size_t)r * r);
    for (int j = 0; j < r; j++) {
        w[j] = S[(size_t)order[j] * r + order[j]];
        for (int i = 0; i < r; i++) Qs[(size_t)i * r + j] = Q[(size_t)i * r + order[j]];
    }
    Q.swap(Qs);
}

// Rayleigh-Ritz on the m-column basis with Gram matrices GL = U^T L U, GM = U^T M U (row-major):
// Y (m x k, row-major) and the Ritz values theta (k); false if fewer than k directions survive
bool rayleigh_ritz(int m, int k, const std::vector<double> &GL, const std::vector<double> &GM, std::vector<double> &Y,
                   std::vector<double> &theta) {
    std::vector<double> d(m);
    for (int a = 0; a < m; a++) d[a] = GM[(size_t)a * m + a] > 0 ? 1.0 / std::sqrt(GM[(size_t)a * m + a]) : 0.0;
    std::vector<double> S((size_t)m * m), B((size_t)m * m);
    for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++) {
            B[(size_t)a * m + b] = d[a] * d[b] * 0.5 * (GM[(size_t)a * m + b] + GM[(size_t)b * m + a]);
            S[(size_t)a * m + b] = d[a] * d[b] * 0.5 * (GL[(size_t)a * m + b] + GL[(size_t)b * m + a]);
        }
    std::vector<double> mu, Q;
    jacobi_eig(m, B, mu, Q);
    const double mmax = mu.empty() ? 0.0 : mu.back();
    std::vector<int> keep;
    for (int j = 0; j < m; j++)
        if (mu[j] > 1e-13 * mmax) keep.push_back(j);
    const int r = (int)keep.size();
    if (r < k) return false;
    // T = Q_keep diag(mu^-1/2): the scaled basis becomes M-orthonormal
    std::vector<double> T((size_t)m * r);
    for (int a = 0; a < m; a++)
        for (int j = 0; j < r; j++) T[(size_t)a * r + j] = Q[(size_t)a * m + keep[j]] / std::sqrt(mu[keep[j]]);
    std::vector<double> ST((size_t)m * r, 0.0), Red((size_t)r * r, 0.0);
    for (int a = 0; a < m; a++)
        for (int j = 0; j < r; j++) {
            double s = 0.0;
            for (int b = 0; b < m; b++) s += S[(size_t)a * m + b] * T[(size_t)b * r + j];
            ST[(size_t)a * r + j] = s;
        }
    for (int i = 0; i < r; i++)
        for (int j = 0; j < r; j++) {
            double s = 0.0;
            for (int a = 0; a < m; a++) s += T[(size_t)a * r + i] * ST[(size_t)a * r + j];
            Red[(size_t)i * r + j] = s;
        }
    std::vector<double> th, Z;
    jacobi_eig(r, Red, th, Z);
    Y.assign((size_t)m * k, 0.0);
    theta.assign(th.begin(), th.begin() + k);
    for (int a = 0; a < m; a++)
        for (int j = 0; j < k; j++) {
            double s = 0.0;
            for (int q = 0; q < r; q++) s += T[(size_t)a * r + q] * Z[(size_t)q * r + j];
            Y[(size_t)a * k + j] = d[a] * s;   // back to the unscaled columns
        }
    return true;
}

struct Lobpcg {
    int n = 0;
    double *U = nullptr, *LU = nullptr, *MU = nullptr;   // [3k][n]: X, W, P blocks
    double *T1 = nullptr, *T2 = nullptr, *T3 = nullptr;  // [3k][n] new X/P blocks of U, LU, MU
    double *part = nullptr, *G = nullptr, *Yd = nullptr, *lam = nullptr;
    std::vector<void *> mem;
    ~Lobpcg() {
        for (void *p : mem) cudaFree(p);
    }
    cudaError_t alloc(double **p, size_t count) {
        cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(double));
        if (e == cudaSuccess) mem.push_back(*p);
        return e;
    }
};

}  // namespace

int lobpcg(Ctx &c, int k, double tol, int max_iters, const double *X_user, double *lambda, double *X_out, double *res,
           int *iters, cudaStream_t s, std::string &err) {
    const DevLevel &F = c.lev[c.D];
    const int n = F.n;
    if (k < 1 || k > kMaxK || n < 3 * k) { err = "lbmg_eigs: 1 <= k <= 16 and 3k <= functions"; return 1; }
    Lobpcg w;
    w.n = n;
    const size_t blk = (size_t)3 * k * n;
    cudaError_t e = cudaSuccess;
    for (double **p : {&w.U, &w.LU, &w.MU, &w.T1, &w.T2, &w.T3})
        if (e == cudaSuccess) e = w.alloc(p, blk);
    if (e == cudaSuccess) e = w.alloc(&w.part, (size_t)kGramBlocks * kMaxM * kMaxM * 2);
    if (e == cudaSuccess) e = w.alloc(&w.G, (size_t)kMaxM * kMaxM * 2 + 2 * kMaxK);
    if (e == cudaSuccess) e = w.alloc(&w.Yd, (size_t)kMaxM * kMaxK * 2);
    if (e == cudaSuccess) e = w.alloc(&w.lam, kMaxK);
    if (e != cudaSuccess) { err = std::string("lbmg_eigs: cudaMalloc: ") + cudaGetErrorString(e); return 2; }
    auto col = [&](double *B, int j) { return B + (size_t)j * n; };
    auto apply = [&](double *B, int j0, int cnt) {   // L and M of columns j0.. of U
        for (int j = j0; j < j0 + cnt; j++) {
            spmv_kernel<<<nb(n), 256, 0, s>>>(n, F.rp, F.ci, F.L, col(w.U, j), col(w.LU, j));
            spmv_kernel<<<nb(n), 256, 0, s>>>(n, F.rp, F.ci, F.M, col(w.U, j), col(w.MU, j));
        }
    };
    auto gram = [&](int ma, const double *A, int mb, const double *B, double *out) {
        gram_partial_kernel<<<kGramBlocks, 256, 0, s>>>(n, ma, mb, A, B, w.part);
        gram_final_kernel<<<nb(ma * mb), 256, 0, s>>>(kGramBlocks, ma * mb, w.part, out);
    };
    // start: the user's block, M-orthonormalised by a Rayleigh-Ritz step on itself
    user_to_cols_kernel<<<nb((int64_t)n * k), 256, 0, s>>>(n, k, X_user, c.fperm, w.U);
    apply(w.U, 0, k);
    std::vector<double> GL, GM, Y, theta, lam_h(k, 0.0), rn(k, 0.0);
    int m = k, it = 0;
    bool have_p = false, conv = false;
    for (;; it++) {
        // Gram matrices of the current basis (X, or X W P) and the host's Rayleigh-Ritz step
        std::vector<double> host((size_t)2 * m * m);
        gram(m, w.U, m, w.LU, w.G);
        gram(m, w.U, m, w.MU, w.G + (size_t)m * m);
        if ((e = cudaMemcpyAsync(host.data(), w.G, host.size() * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            err = std::string("lbmg_eigs: ") + cudaGetErrorString(e);
            return 2;
        }
        GL.assign(host.begin(), host.begin() + (size_t)m * m);
        GM.assign(host.begin() + (size_t)m * m, host.end());
        if (!rayleigh_ritz(m, k, GL, GM, Y, theta)) {
            if (have_p) {   // the basis lost rank: drop the search directions and retry
                m = 2 * k;
                have_p = false;
                it--;
                continue;
            }
            err = "lbmg_eigs: the block lost rank";
            return 3;
        }
        for (int j = 0; j < k; j++) lam_h[j] = theta[j];
        // X = U Y (with L X, M X), P = [W P] Y_{W,P}: combinations written to T, then moved into U
        if ((e = cudaMemcpyAsync(w.Yd, Y.data(), Y.size() * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(w.lam, lam_h.data(), k * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
            err = std::string("lbmg_eigs: ") + cudaGetErrorString(e);
            return 2;
        }
        const unsigned g = nb((int64_t)n * k);
        combine_kernel<<<g, 256, 0, s>>>(n, m, k, 0, w.U, w.Yd, w.T1);
        combine_kernel<<<g, 256, 0, s>>>(n, m, k, 0, w.LU, w.Yd, w.T2);
        combine_kernel<<<g, 256, 0, s>>>(n, m, k, 0, w.MU, w.Yd, w.T3);
        if (m > k) {   // the new search directions: the W (and P) part of the combination
            combine_kernel<<<g, 256, 0, s>>>(n, m - k, k, k, w.U, w.Yd + (size_t)k * k, w.T1 + (size_t)k * n);
            combine_kernel<<<g, 256, 0, s>>>(n, m - k, k, k, w.LU, w.Yd + (size_t)k * k, w.T2 + (size_t)k * n);
            combine_kernel<<<g, 256, 0, s>>>(n, m - k, k, k, w.MU, w.Yd + (size_t)k * k, w.T3 + (size_t)k * n);
        }
        const size_t xs = (size_t)k * n * sizeof(double);
        // U = [X_new, W (next), P_new]: X into block 0, P into block 2
        cudaMemcpyAsync(w.U, w.T1, xs, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(w.LU, w.T2, xs, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(w.MU, w.T3, xs, cudaMemcpyDeviceToDevice, s);
        if (m > k) {
            cudaMemcpyAsync(w.U + (size_t)2 * k * n, w.T1 + (size_t)k * n, xs, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(w.LU + (size_t)2 * k * n, w.T2 + (size_t)k * n, xs, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(w.MU + (size_t)2 * k * n, w.T3 + (size_t)k * n, xs, cudaMemcpyDeviceToDevice, s);
            have_p = true;
        }
        // residuals R = L X - M X Lambda into the W block, with their norms and those of M X
        residual_block_kernel<<<g, 256, 0, s>>>(n, k, w.LU, w.MU, w.lam, w.U + (size_t)k * n);
        std::vector<double> nrm((size_t)4 * k * k);
        gram(k, w.U + (size_t)k * n, k, w.U + (size_t)k * n, w.G);
        gram(k, w.MU, k, w.MU, w.G + (size_t)k * k);
        if ((e = cudaMemcpyAsync(nrm.data(), w.G, (size_t)2 * k * k * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            err = std::string("lbmg_eigs: ") + cudaGetErrorString(e);
            return 2;
        }
        conv = true;
        for (int j = 0; j < k; j++) {
            const double r2 = nrm[(size_t)j * k + j], mx2 = nrm[(size_t)k * k + (size_t)j * k + j];
            rn[j] = mx2 > 0 ? std::sqrt(r2 / mx2) : INFINITY;
            if (!(rn[j] <= tol)) conv = false;
        }
        if (conv || it >= max_iters) break;
        // W = V(R): one FP64 V-cycle of A = M + t L per column, four columns per cycle
        DevLevel &Fw = c.lev[c.D];
        for (int j0 = 0; j0 < k; j0 += 4) {
            const int nc = std::min(4, k - j0);
            interleave4_kernel<<<nb((int64_t)n * 4), 256, 0, s>>>(n, nc, w.U + (size_t)(k + j0) * n, Fw.b64);
            cudaMemsetAsync(Fw.x64, 0, (size_t)n * 4 * sizeof(double), s);
            enqueue_vcycle64_from(c, c.D, 4, s);
            deinterleave4_kernel<<<nb((int64_t)n * nc), 256, 0, s>>>(n, nc, Fw.x64, w.U + (size_t)(k + j0) * n);
        }
        apply(w.U, k, k);
        m = have_p ? 3 * k : 2 * k;
    }
    cols_to_user_kernel<<<nb((int64_t)n * k), 256, 0, s>>>(n, k, w.U, c.fperm, X_out);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        err = std::string("lbmg_eigs: ") + cudaGetErrorString(e);
        return 2;
    }
    for (int j = 0; j < k; j++) {
        lambda[j] = lam_h[j];
        if (res) res[j] = rn[j];
    }
    *iters = it;
    return conv ? 0 : 4;
}

}  // namespace lbmg
