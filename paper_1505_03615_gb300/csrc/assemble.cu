// assemble.cu -- Galerkin matrices and right-hand sides of the split B-spline
// hierarchy (Chuang & Kazhdan, Eq. 2 and Sections 5.1-5.3).
//
// Finest level: one thread per fragment (a triangle piece inside one voxel)
// integrates the 27 moments int u^i v^j w^k dA (i,j,k <= 2, local voxel
// coordinates) with a collapsed Gauss-Legendre rule on each sub-triangle of the
// piece's fan (exact to degree 6).  Every product of two trilinear hats, and of
// their tangential gradients, is a combination of those moments, so the 36 + 36
// local entries follow from a separable contraction of the moments, one axis at a
// time, pruned to the 90 integrals the entries use.  GB300 runs FP64 at a small
// fraction of its FP32 rate, so this kernel is bound by the number of FP64
// instructions: a thread per fragment needs no cross-lane reduction and no idle
// lanes, and fragments are taken in order of vertex count so that a warp's
// threads run the same number of sub-triangles.  A second kernel sums each
// stored entry's contributions through a precomputed list (no atomics).  Coarser
// levels are the Galerkin products P^T A P of Eq. 4's prolongation, summed the
// same way.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lbmg_internal.h"

namespace lbmg {

__constant__ double c_glx[kNQ], c_glw[kNQ];
// the collapsed rule on the reference triangle {xi, eta >= 0, xi + eta <= 1}:
// point q = (xi, eta) and weight, kNQ * kNQ points
__constant__ double c_qxi[kNQ * kNQ], c_qeta[kNQ * kNQ], c_qw[kNQ * kNQ];
// per-axis factor types over (1, t, t^2):
// 0: 1, 1: 1-t, 2: t, 3: (1-t)^2, 4: t(1-t), 5: t^2
__constant__ double c_type[6][3] = {{1, 0, 0}, {1, -1, 0}, {0, 1, 0}, {1, -2, 1}, {0, 1, -1}, {0, 0, 1}};

static bool g_gl_ready = false;

// Gauss-Legendre rule on [0,1] by the Golub-Welsch method: the nodes on [-1,1] are the eigenvalues
// of the symmetric tridiagonal Jacobi matrix of the Legendre three-term recurrence (zero diagonal,
// off-diagonal k / sqrt(4k^2 - 1)), each weight is twice the squared first component of the unit
// eigenvector; the eigenproblem is solved by cyclic Jacobi rotations (n is a handful).  Nodes
// ascending.
static void gauss_legendre01(int n, double *x, double *w) {
    std::vector<double> A((size_t)n * n, 0.0), V((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    for (int k = 1; k < n; k++) {
        const double b = k / std::sqrt(4.0 * k * k - 1.0);
        A[(size_t)(k - 1) * n + k] = A[(size_t)k * n + k - 1] = b;
    }
    for (int sweep = 0; sweep < 64; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off < 1e-60) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                // the rotation in the (p, q) plane that zeroes A_pq: A <- J^T A J, V <- V J
                const double th = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; i++) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    for (int i = 0; i < n; i++) {
        const int e = ord[i];
        x[i] = 0.5 * (A[(size_t)e * n + e] + 1.0);
        w[i] = V[e] * V[e];   // 2 v_0^2 on [-1, 1], halved on [0, 1]
    }
}

static void ensure_gl() {
    if (g_gl_ready) return;
    double x[kNQ], w[kNQ];
    gauss_legendre01(kNQ, x, w);
    cudaMemcpyToSymbol(c_glx, x, sizeof x);
    cudaMemcpyToSymbol(c_glw, w, sizeof w);
    double qx[kNQ * kNQ], qe[kNQ * kNQ], qw[kNQ * kNQ];
    for (int a = 0; a < kNQ; a++)
        for (int b = 0; b < kNQ; b++) {
            qx[a * kNQ + b] = x[a];
            qe[a * kNQ + b] = x[b] * (1.0 - x[a]);
            qw[a * kNQ + b] = w[a] * w[b] * (1.0 - x[a]);
        }
    cudaMemcpyToSymbol(c_qxi, qx, sizeof qx);
    cudaMemcpyToSymbol(c_qeta, qe, sizeof qe);
    cudaMemcpyToSymbol(c_qw, qw, sizeof qw);
    g_gl_ready = true;
}

// Integral of the per-axis factor type ty (the table c_type) from the integrals
// (m0, m1, m2) of 1, t, t^2 along that axis.  ty is a compile-time constant at
// every call, so only the needed differences are formed, and identical ones are
// shared between calls.
__device__ __forceinline__ double ftype(int ty, double m0, double m1, double m2) {
    switch (ty) {
        case 0: return m0;                        // 1
        case 1: return m0 - m1;                   // 1 - t
        case 2: return m1;                        // t
        case 3: return fma(-2.0, m1, m0) + m2;    // (1 - t)^2
        case 4: return m1 - m2;                   // t (1 - t)
        default: return m2;                       // t^2
    }
}

// G(a, b, c) = integral of type_a(u) type_b(v) type_c(w) from the moments m[i][j][k]
__device__ __forceinline__ double gz(const double (&m)[27], int i, int j, int c) {
    return ftype(c, m[i * 9 + j * 3], m[i * 9 + j * 3 + 1], m[i * 9 + j * 3 + 2]);
}
__device__ __forceinline__ double gy(const double (&m)[27], int i, int b, int c) {
    return ftype(b, gz(m, i, 0, c), gz(m, i, 1, c), gz(m, i, 2, c));
}
__device__ __forceinline__ double G3(const double (&m)[27], int a, int b, int c) {
    return ftype(a, gy(m, 0, b, c), gy(m, 1, b, c), gy(m, 2, b, c));
}

constexpr int kMomThreads = 128;

// One thread per fragment (taken in the order forder).  Writes the 27 moments and
// the 36 (M, L) local pair entries, pairs (a, b), a <= b, in upper-triangular order.
constexpr int kStagePerFrag = 36;   // local (M, L) pairs a <= b of the 8 corner functions of a piece

__global__ void __launch_bounds__(kMomThreads)
fragment_moments_kernel(int nfrag, const int *__restrict__ forder, const double *__restrict__ poly,
                        const int *__restrict__ pstart, const int *__restrict__ ftri,
                        const double *__restrict__ tnormal, double *__restrict__ moments, double *__restrict__ stage) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nfrag) return;
    const int f = __ldg(forder + t);
    const int p0 = __ldg(pstart + f), np = __ldg(pstart + f + 1) - p0;
    const double *P = poly + 3 * (size_t)p0;
    const double *nrm = tnormal + 3 * (size_t)__ldg(ftri + f);
    const double n0 = __ldg(nrm), n1 = __ldg(nrm + 1), n2 = __ldg(nrm + 2);
    const double a0 = __ldg(P), a1 = __ldg(P + 1), a2 = __ldg(P + 2);
    double m[27];
#pragma unroll
    for (int q = 0; q < 27; q++) m[q] = 0.0;
    double b0 = __ldg(P + 3), b1 = __ldg(P + 4), b2 = __ldg(P + 5);
    for (int sub = 2; sub < np; sub++) {
        const double c0 = __ldg(P + 3 * sub), c1 = __ldg(P + 3 * sub + 1), c2 = __ldg(P + 3 * sub + 2);
        const double e10 = b0 - a0, e11 = b1 - a1, e12 = b2 - a2;
        const double e20 = c0 - a0, e21 = c1 - a1, e22 = c2 - a2;
        // twice the sub-triangle's area: the piece lies in its triangle's plane,
        // so the edge cross product is parallel to the unit normal
        const double jac = fabs(fma(fma(e11, e22, -e12 * e21), n0,
                                    fma(fma(e12, e20, -e10 * e22), n1, fma(e10, e21, -e11 * e20) * n2)));
#pragma unroll
        for (int q = 0; q < kNQ * kNQ; q++) {
            const double xi = c_qxi[q], eta = c_qeta[q];
            const double u = fma(eta, e20, fma(xi, e10, a0));
            const double v = fma(eta, e21, fma(xi, e11, a1));
            const double z = fma(eta, e22, fma(xi, e12, a2));
            const double w = c_qw[q] * jac;
            const double wu = w * u;
            const double pu[3] = {w, wu, wu * u};
            const double v2 = v * v, z2 = z * z;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const double s[3] = {pu[i], pu[i] * v, pu[i] * v2};
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    m[i * 9 + j * 3] += s[j];
                    m[i * 9 + j * 3 + 1] = fma(s[j], z, m[i * 9 + j * 3 + 1]);
                    m[i * 9 + j * 3 + 2] = fma(s[j], z2, m[i * 9 + j * 3 + 2]);
                }
            }
        }
        b0 = c0; b1 = c1; b2 = c2;
    }
    double *mo = moments + 27 * (size_t)f;
#pragma unroll
    for (int q = 0; q < 27; q++) mo[q] = m[q];
    // tangential projector I - n n^T
    const double nv[3] = {n0, n1, n2};
    double2 *st = reinterpret_cast<double2 *>(stage) + kStagePerFrag * (size_t)f;
    int p = 0;
#pragma unroll
    for (int a = 0; a < 8; a++) {
#pragma unroll
        for (int b = a; b < 8; b++) {
            const int ab[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
            const int bb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
            int pt[3];
#pragma unroll
            for (int k = 0; k < 3; k++) pt[k] = 3 + ab[k] + bb[k];     // phi_a phi_b along axis k
            const double Mab = G3(m, pt[0], pt[1], pt[2]);   // in finest-unit area: fine_gather scales it
            double Lab = 0.0;
#pragma unroll
            for (int pp = 0; pp < 3; pp++)
#pragma unroll
                for (int qq = 0; qq < 3; qq++) {
                    const double Q = (pp == qq ? 1.0 : 0.0) - nv[pp] * nv[qq];
                    int ty[3];
                    double sgn;
                    if (pp == qq) {
                        // d_p phi_a d_p phi_b: constant along p, products along the others
                        sgn = (ab[pp] ? 1.0 : -1.0) * (bb[pp] ? 1.0 : -1.0);
#pragma unroll
                        for (int k = 0; k < 3; k++) ty[k] = k == pp ? 0 : pt[k];
                    } else {
                        // d_p phi_a d_q phi_b: phi_b along p, phi_a along q
                        sgn = (ab[pp] ? 1.0 : -1.0) * (bb[qq] ? 1.0 : -1.0);
#pragma unroll
                        for (int k = 0; k < 3; k++) ty[k] = k == pp ? 1 + bb[k] : (k == qq ? 1 + ab[k] : pt[k]);
                    }
                    Lab = fma(Q * sgn, G3(m, ty[0], ty[1], ty[2]), Lab);
                }
            st[p] = make_double2(Mab, Lab);
            p++;
        }
    }
}

void launch_fragment_moments(const Ctx &c, cudaStream_t s) {
    ensure_gl();
    if (c.nfrag == 0) return;
    const int blocks = (c.nfrag + kMomThreads - 1) / kMomThreads;
    fragment_moments_kernel<<<blocks, kMomThreads, 0, s>>>(c.nfrag, c.forder, c.poly, c.pstart, c.ftri, c.tnormal,
                                                           c.moments, c.stage);
}

// finest level: sum the local-pair contributions of every stored entry
__global__ void fine_gather_kernel(int64_t nnz, const int64_t *__restrict__ arp, const uint32_t *__restrict__ aidx,
                                   const double2 *__restrict__ stage, const double *__restrict__ fscale, double t,
                                   double *__restrict__ M, double *__restrict__ L, double *__restrict__ A64,
                                   float *__restrict__ A32) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    double m = 0.0, l = 0.0;
    const int64_t k1 = arp[s + 1];
    int64_t k = arp[s];
    // eight list entries, then their eight values, in flight together; the sum keeps its order
    for (; k + 8 <= k1; k += 8) {
        uint32_t ix[8];
#pragma unroll
        for (int u = 0; u < 8; u++) ix[u] = __ldg(aidx + k + u);
        double2 v[8];
        double w[8];
#pragma unroll
        for (int u = 0; u < 8; u++) { v[u] = __ldg(stage + ix[u]); w[u] = __ldg(fscale + ix[u] / kStagePerFrag); }
#pragma unroll
        for (int u = 0; u < 8; u++) { m = fma(v[u].x, w[u], m); l += v[u].y; }
    }
    for (; k < k1; k++) {
        const uint32_t ix = aidx[k];
        const double2 v = __ldg(stage + ix);
        m = fma(v.x, __ldg(fscale + ix / kStagePerFrag), m);
        l += v.y;
    }
    M[s] = m;
    L[s] = l;
    const double a = m + t * l;
    A64[s] = a;
    A32[s] = (float)a;
}

void launch_fine_gather(const Ctx &c, double t, cudaStream_t s) {
    const DevLevel &L = c.lev[c.D];
    const int threads = 256;
    fine_gather_kernel<<<(unsigned)((L.nnz + threads - 1) / threads), threads, 0, s>>>(
        L.nnz, c.arp, c.aidx, reinterpret_cast<const double2 *>(c.stage), c.frag_scale, t, L.M, L.L, L.A64, L.A32);
}

// coarse level: (P^T A P)_ab = sum over listed fine entries of 2^-e A_il
__global__ void galerkin_kernel(int64_t nnz, const int64_t *__restrict__ grp, const uint32_t *__restrict__ gidx,
                                const double *__restrict__ Mf, const double *__restrict__ Lf, double t,
                                double *__restrict__ M, double *__restrict__ L, double *__restrict__ A64,
                                float *__restrict__ A32) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    double m = 0.0, l = 0.0;
    const int64_t k1 = grp[s + 1];
    int64_t k = grp[s];
    // eight list entries, then their sixteen values, in flight together; the sum keeps its order
    for (; k + 8 <= k1; k += 8) {
        uint32_t e[8];
#pragma unroll
        for (int u = 0; u < 8; u++) e[u] = __ldg(gidx + k + u);
        double mv[8], lv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) { mv[u] = __ldg(Mf + (e[u] & kGalMask)); lv[u] = __ldg(Lf + (e[u] & kGalMask)); }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const double w = ldexp(1.0, -(int)(e[u] >> kGalShift));
            m = fma(w, mv[u], m);
            l = fma(w, lv[u], l);
        }
    }
    for (; k < k1; k++) {
        const uint32_t e = __ldg(gidx + k);
        const uint32_t idx = e & kGalMask;
        const double w = ldexp(1.0, -(int)(e >> kGalShift));
        m = fma(w, __ldg(Mf + idx), m);
        l = fma(w, __ldg(Lf + idx), l);
    }
    M[s] = m;
    L[s] = l;
    const double a = m + t * l;
    A64[s] = a;
    A32[s] = (float)a;
}

void launch_galerkin(const Ctx &c, int dc, double t, cudaStream_t s) {
    const DevLevel &Lc = c.lev[dc], &Lf = c.lev[dc + 1];
    const int threads = 256;
    galerkin_kernel<<<(unsigned)((Lc.nnz + threads - 1) / threads), threads, 0, s>>>(
        Lc.nnz, Lc.grp, Lc.gidx, Lf.M, Lf.L, t, Lc.M, Lc.L, Lc.A64, Lc.A32);
}

// Relaxation skips rows whose diagonal is below this fraction of the level's mean
// diagonal (or not positive).  Such functions meet the mesh in slivers where the hat
// and its tangential gradient nearly vanish: their diagonals (1e-27 to 1e-40 of the mean,
// depending on the rounding of the quadrature) lie below the rounding error of the moment
// contraction that produced them (so they can even come out negative), down to FP32's range
// (1/a_ii overflows), and they carry no measurable mass or stiffness.  Their coefficients stay at zero correction; the residual
// still includes their rows.
constexpr double kDiagFloor = 1e-20;
constexpr int kDiagBlocks = 256;

// per-block partial sums of the diagonal A_ii
__global__ void __launch_bounds__(256) diag_sum_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const double *__restrict__ A64, double *__restrict__ part) {
    __shared__ double sh[256];
    double sum = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int end = rp[i + 1];
        int lo = rp[i], hi = end;
        while (lo < hi) { int mid = (lo + hi) >> 1; if (ci[mid] < i) lo = mid + 1; else hi = mid; }
        sum += (lo < end && ci[lo] == i) ? A64[lo] : 0.0;
    }
    sh[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// FP64 and FP32 inverse diagonals, 0 for rows below the floor
__global__ void __launch_bounds__(256) inverse_diag_kernel(int n, const int *__restrict__ rp,
                                                           const int *__restrict__ ci, const double *__restrict__ A64,
                                                           const double *__restrict__ part, int nparts,
                                                           double *__restrict__ d64, float *__restrict__ d32) {
    __shared__ double s_thr;
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int b = 0; b < nparts; b++) sum += part[b];
        s_thr = kDiagFloor * (sum / (double)n);
    }
    __syncthreads();
    const double thr = s_thr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int end = rp[i + 1];
        int lo = rp[i], hi = end;
        while (lo < hi) { int mid = (lo + hi) >> 1; if (ci[mid] < i) lo = mid + 1; else hi = mid; }
        const double a = (lo < end && ci[lo] == i) ? A64[lo] : 0.0;
        const double inv = (a > 0.0 && a >= thr) ? 1.0 / a : 0.0;
        d64[i] = inv;
        d32[i] = (float)inv;
    }
}

void launch_inverse_diag(const DevLevel &L, double *part, cudaStream_t s) {
    if (L.n == 0) return;
    const int blocks = std::min(kDiagBlocks, (L.n + 255) / 256);
    diag_sum_kernel<<<blocks, 256, 0, s>>>(L.n, L.rp, L.ci, L.A64, part);
    inverse_diag_kernel<<<std::min(1024, (L.n + 255) / 256), 256, 0, s>>>(L.n, L.rp, L.ci, L.A64, part, blocks,
                                                                         L.dinv64, L.dinv32);
}

// right-hand side: int f b_a over each fragment from its moments, f affine on the triangle
__global__ void fragment_rhs_kernel(int nfrag, int nrhs, const double *__restrict__ moments,
                                    const int *__restrict__ ftri, const int *__restrict__ fvox,
                                    const int *__restrict__ F, const double *__restrict__ Vg,
                                    const double *__restrict__ fv, const double *__restrict__ fscale,
                                    double *__restrict__ out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfrag) return;
    const int t = ftri[f];
    const int ia = F[3 * t], ib = F[3 * t + 1], ic = F[3 * t + 2];
    const double *A = Vg + 3 * (size_t)ia, *B = Vg + 3 * (size_t)ib, *C = Vg + 3 * (size_t)ic;
    double e1[3], e2[3], lo[3];
    for (int k = 0; k < 3; k++) { e1[k] = B[k] - A[k]; e2[k] = C[k] - A[k]; lo[k] = (double)fvox[3 * f + k] - A[k]; }
    const double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const double det = g11 * g22 - g12 * g12;
    double m[27];
#pragma unroll
    for (int q = 0; q < 27; q++) m[q] = __ldg(moments + 27 * (size_t)f + q);
    // per corner a: int b_a and int u_k b_a (types 1 + bit: phi along an axis, 4 + bit: t phi)
    double Ib[8], Iu[8][3];
#pragma unroll
    for (int a = 0; a < 8; a++) {
        const int b0 = a & 1, b1 = (a >> 1) & 1, b2 = (a >> 2) & 1;
        Ib[a] = G3(m, 1 + b0, 1 + b1, 1 + b2);
        Iu[a][0] = G3(m, 4 + b0, 1 + b1, 1 + b2);
        Iu[a][1] = G3(m, 1 + b0, 4 + b1, 1 + b2);
        Iu[a][2] = G3(m, 1 + b0, 1 + b1, 4 + b2);
    }
    const double idet = 1.0 / det, fs = fscale[f];
    for (int r = 0; r < nrhs; r++) {
        const double fa = fv[(size_t)ia * nrhs + r], fb = fv[(size_t)ib * nrhs + r], fc = fv[(size_t)ic * nrhs + r];
        const double d1 = fb - fa, d2 = fc - fa;
        const double al = (g22 * d1 - g12 * d2) * idet, be = (g11 * d2 - g12 * d1) * idet;
        double g[3];
        for (int k = 0; k < 3; k++) g[k] = al * e1[k] + be * e2[k];     // tangential gradient of f
        const double beta0 = fa + g[0] * lo[0] + g[1] * lo[1] + g[2] * lo[2];
        for (int a = 0; a < 8; a++) {
            const double v = beta0 * Ib[a] + g[0] * Iu[a][0] + g[1] * Iu[a][1] + g[2] * Iu[a][2];
            out[(8 * (size_t)f + a) * 4 + r] = v * fs;
        }
    }
}

__global__ void rhs_gather_kernel(int n, int nrhs, const int64_t *__restrict__ rrp, const uint32_t *__restrict__ ridx,
                                  const double *__restrict__ stage, const int *__restrict__ fiperm,
                                  double *__restrict__ rhs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc[4] = {0, 0, 0, 0};
    for (int64_t k = rrp[i]; k < rrp[i + 1]; k++) {
        const double *v = stage + 4 * (size_t)ridx[k];
        for (int r = 0; r < 4; r++) acc[r] += v[r];
    }
    const size_t u = (size_t)fiperm[i];
    for (int r = 0; r < nrhs; r++) rhs[u * nrhs + r] = acc[r];
}

void launch_project_rhs(const Ctx &c, const double *fv, int nrhs, double *rhs_out, cudaStream_t s) {
    fragment_rhs_kernel<<<(c.nfrag + 127) / 128, 128, 0, s>>>(c.nfrag, nrhs, c.moments, c.ftri, c.fvox, c.F, c.Vg, fv,
                                                               c.frag_scale, c.stage_rhs);
    const int n = c.lev[c.D].n;
    rhs_gather_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, nrhs, c.rrp, c.ridx, c.stage_rhs, c.fiperm, rhs_out);
}

__global__ void eval_vertices_kernel(int nv, int nrhs, const int *__restrict__ vdof, const double *__restrict__ vw,
                                     const double *__restrict__ x, double *__restrict__ u) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double acc[4] = {0, 0, 0, 0};
    for (int a = 0; a < 8; a++) {
        const int d = vdof[8 * (size_t)v + a];
        if (d < 0) continue;
        const double w = vw[8 * (size_t)v + a];
        for (int r = 0; r < nrhs; r++) acc[r] = fma(w, x[(size_t)d * nrhs + r], acc[r]);
    }
    for (int r = 0; r < nrhs; r++) u[(size_t)v * nrhs + r] = acc[r];
}

void launch_eval_vertices(const Ctx &c, const double *x, int nrhs, double *u, cudaStream_t s) {
    eval_vertices_kernel<<<(c.nv + 255) / 256, 256, 0, s>>>(c.nv, nrhs, c.vdof, c.vw, x, u);
}

}  // namespace lbmg
