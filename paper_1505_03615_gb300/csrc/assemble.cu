// assemble.cu -- Galerkin matrices and right-hand sides of the split B-spline
// hierarchy (Chuang & Kazhdan, Eq. 2 and Sections 5.1-5.3).
//
// Finest level: one warp per fragment (a triangle piece inside one voxel)
// integrates the 27 moments int u^i v^j w^k dA (i,j,k <= 2, local voxel
// coordinates) with a collapsed Gauss-Legendre rule on each sub-triangle of the
// piece's fan (exact to degree 6).  Every product of two trilinear hats, and of
// their tangential gradients, is a combination of those moments, so the 36 + 36
// local entries follow from a separable 3-stage contraction.  A second kernel
// sums each stored entry's contributions through a precomputed list (no
// atomics).  Coarser levels are the Galerkin products P^T A P of Eq. 4's
// prolongation, summed the same way.
#include "lbmg_internal.h"

namespace lbmg {

__constant__ double c_glx[kNQ], c_glw[kNQ];
// per-axis factor types over (1, t, t^2):
// 0: 1, 1: 1-t, 2: t, 3: (1-t)^2, 4: t(1-t), 5: t^2
__constant__ double c_type[6][3] = {{1, 0, 0}, {1, -1, 0}, {0, 1, 0}, {1, -2, 1}, {0, 1, -1}, {0, 0, 1}};

static bool g_gl_ready = false;

// Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n
static void gauss_legendre01(int n, double *x, double *w) {
    for (int i = 0; i < n; i++) {
        double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
        double pn = 0, dpn = 1;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; k++) { double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0); p0 = p1; p1 = p2; }
            pn = p1;
            dpn = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = pn / dpn;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 1; k < n; k++) { double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0); p0 = p1; p1 = p2; }
        dpn = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = 0.5 * (z + 1.0);
        w[i] = 1.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

static void ensure_gl() {
    if (g_gl_ready) return;
    double x[kNQ], w[kNQ];
    gauss_legendre01(kNQ, x, w);
    cudaMemcpyToSymbol(c_glx, x, sizeof x);
    cudaMemcpyToSymbol(c_glw, w, sizeof w);
    g_gl_ready = true;
}

constexpr int kWarpsPerBlock = 8;

// One warp per fragment.  Writes the 27 moments and the 36 (M, L) local pair entries.
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
fragment_moments_kernel(int nfrag, const double *__restrict__ poly, const int *__restrict__ pstart,
                        const int *__restrict__ ftri, const double *__restrict__ tnormal,
                        const double *__restrict__ fscale, double *__restrict__ moments, double *__restrict__ stage) {
    __shared__ double sh[kWarpsPerBlock][27 + 54 + 108 + 216];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int f = blockIdx.x * kWarpsPerBlock + warp;
    if (f >= nfrag) return;
    double *sm = sh[warp], *h1 = sm + 27, *h2 = h1 + 54, *G = h2 + 108;
    const int p0 = pstart[f], np = pstart[f + 1] - p0;
    const double *P = poly + 3 * (size_t)p0;
    const int npts = (np - 2) * kNQ * kNQ;
    double m[27];
#pragma unroll
    for (int q = 0; q < 27; q++) m[q] = 0.0;
    for (int q = lane; q < npts; q += 32) {
        const int sub = q / (kNQ * kNQ), qa = (q / kNQ) % kNQ, qb = q % kNQ;
        const double *A = P, *B = P + 3 * (sub + 1), *C = P + 3 * (sub + 2);
        double e1[3], e2[3];
#pragma unroll
        for (int k = 0; k < 3; k++) { e1[k] = B[k] - A[k]; e2[k] = C[k] - A[k]; }
        double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
        double jac = sqrt(cx * cx + cy * cy + cz * cz);
        double xa = c_glx[qa];
        double xi = xa, eta = c_glx[qb] * (1.0 - xa);
        double w = c_glw[qa] * c_glw[qb] * (1.0 - xa) * jac;
        double u = A[0] + xi * e1[0] + eta * e2[0];
        double v = A[1] + xi * e1[1] + eta * e2[1];
        double z = A[2] + xi * e1[2] + eta * e2[2];
        double pu[3] = {w, w * u, w * u * u}, pv[3] = {1.0, v, v * v}, pz[3] = {1.0, z, z * z};
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                double uv = pu[i] * pv[j];
#pragma unroll
                for (int k = 0; k < 3; k++) m[i * 9 + j * 3 + k] = fma(uv, pz[k], m[i * 9 + j * 3 + k]);
            }
    }
#pragma unroll
    for (int q = 0; q < 27; q++) {
        double v = m[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        m[q] = v;
    }
    if (lane < 27) {
        double mv = 0;
#pragma unroll
        for (int q = 0; q < 27; q++) if (q == lane) mv = m[q];
        sm[lane] = mv;
        moments[27 * (size_t)f + lane] = mv;
    }
    __syncwarp();
    // contraction along z: h1[(i*3+j)*6+tz]
    for (int q = lane; q < 54; q += 32) {
        const int ij = q / 6, tz = q % 6;
        h1[q] = c_type[tz][0] * sm[ij * 3] + c_type[tz][1] * sm[ij * 3 + 1] + c_type[tz][2] * sm[ij * 3 + 2];
    }
    __syncwarp();
    // along y: h2[(i*6+ty)*6+tz]
    for (int q = lane; q < 108; q += 32) {
        const int i = q / 36, ty = (q / 6) % 6, tz = q % 6;
        h2[q] = c_type[ty][0] * h1[(i * 3 + 0) * 6 + tz] + c_type[ty][1] * h1[(i * 3 + 1) * 6 + tz] +
                c_type[ty][2] * h1[(i * 3 + 2) * 6 + tz];
    }
    __syncwarp();
    // along x: G[(tx*6+ty)*6+tz]
    for (int q = lane; q < 216; q += 32) {
        const int tx = q / 36, yz = q % 36;
        G[q] = c_type[tx][0] * h2[0 * 36 + yz] + c_type[tx][1] * h2[1 * 36 + yz] + c_type[tx][2] * h2[2 * 36 + yz];
    }
    __syncwarp();
    const double *n = tnormal + 3 * (size_t)ftri[f];
    const double nn[3] = {n[0], n[1], n[2]};
    for (int p = lane; p < 36; p += 32) {
        // pair (a, b), a <= b, in upper-triangular order
        int a = 0, rem = p;
        while (rem >= 8 - a) { rem -= 8 - a; a++; }
        const int b = a + rem;
        int ab[3], bb[3];
#pragma unroll
        for (int k = 0; k < 3; k++) { ab[k] = (a >> k) & 1; bb[k] = (b >> k) & 1; }
        auto Pt = [&](int k) { return 3 + ab[k] + bb[k]; };           // phi_a phi_b along axis k
        auto gidx = [](int tx, int ty, int tz) { return (tx * 6 + ty) * 6 + tz; };
        const double Mab = G[gidx(Pt(0), Pt(1), Pt(2))];
        double Lab = 0.0;
#pragma unroll
        for (int pp = 0; pp < 3; pp++)
#pragma unroll
            for (int qq = 0; qq < 3; qq++) {
                const double Q = (pp == qq ? 1.0 : 0.0) - nn[pp] * nn[qq];
                int t[3];
                double sgn;
                if (pp == qq) {
                    sgn = (ab[pp] ? 1.0 : -1.0) * (bb[pp] ? 1.0 : -1.0);
#pragma unroll
                    for (int k = 0; k < 3; k++) t[k] = (k == pp) ? 0 : Pt(k);
                } else {
                    sgn = (ab[pp] ? 1.0 : -1.0) * (bb[qq] ? 1.0 : -1.0);
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        t[k] = (k == pp) ? 1 + bb[k] : (k == qq) ? 1 + ab[k] : Pt(k);
                }
                Lab = fma(Q * sgn, G[gidx(t[0], t[1], t[2])], Lab);
            }
        stage[2 * (36 * (size_t)f + p)] = Mab * fscale[f];
        stage[2 * (36 * (size_t)f + p) + 1] = Lab;
    }
}

void launch_fragment_moments(const Ctx &c, cudaStream_t s) {
    ensure_gl();
    const int blocks = (c.nfrag + kWarpsPerBlock - 1) / kWarpsPerBlock;
    fragment_moments_kernel<<<blocks, 32 * kWarpsPerBlock, 0, s>>>(
        c.nfrag, c.poly, c.pstart, c.ftri, c.tnormal, c.frag_scale, c.moments, c.stage);
}

// finest level: sum the local-pair contributions of every stored entry
__global__ void fine_gather_kernel(int64_t nnz, const int64_t *__restrict__ arp, const uint32_t *__restrict__ aidx,
                                   const double2 *__restrict__ stage, double t, double *__restrict__ M,
                                   double *__restrict__ L, double *__restrict__ A64, float *__restrict__ A32) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    double m = 0.0, l = 0.0;
    for (int64_t k = arp[s]; k < arp[s + 1]; k++) {
        const double2 v = stage[aidx[k]];
        m += v.x;
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
        L.nnz, c.arp, c.aidx, reinterpret_cast<const double2 *>(c.stage), t, L.M, L.L, L.A64, L.A32);
}

// coarse level: (P^T A P)_ab = sum over listed fine entries of 2^-e A_il
__global__ void galerkin_kernel(int64_t nnz, const int64_t *__restrict__ grp, const uint32_t *__restrict__ gidx,
                                const double *__restrict__ Mf, const double *__restrict__ Lf, double t,
                                double *__restrict__ M, double *__restrict__ L, double *__restrict__ A64,
                                float *__restrict__ A32) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    double m = 0.0, l = 0.0;
    for (int64_t k = grp[s]; k < grp[s + 1]; k++) {
        const uint32_t e = gidx[k];
        const uint32_t idx = e & kPackMask;
        const double w = ldexp(1.0, -(int)(e >> kPackShift));
        m = fma(w, Mf[idx], m);
        l = fma(w, Lf[idx], l);
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

__global__ void inverse_diag_kernel(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                    const double *__restrict__ A64, double *__restrict__ d64, float *__restrict__ d32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int end = rp[i + 1];
    int lo = rp[i], hi = end;
    while (lo < hi) { int mid = (lo + hi) >> 1; if (ci[mid] < i) lo = mid + 1; else hi = mid; }
    const double inv = (lo < end && ci[lo] == i) ? 1.0 / A64[lo] : 0.0;
    d64[i] = inv;
    d32[i] = (float)inv;
}

void launch_inverse_diag(const DevLevel &L, cudaStream_t s) {
    inverse_diag_kernel<<<(L.n + 255) / 256, 256, 0, s>>>(L.n, L.rp, L.ci, L.A64, L.dinv64, L.dinv32);
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
    const double *m = moments + 27 * (size_t)f;
    // per corner: int b_a and int u_k b_a
    double Ib[8], Iu[8][3];
    for (int a = 0; a < 8; a++) {
        const int bits[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
        int ts[3], tu[3];
        for (int k = 0; k < 3; k++) { ts[k] = 1 + bits[k]; tu[k] = 4 + bits[k]; }   // phi and t*phi
        for (int which = 0; which < 4; which++) {
            int ty[3] = {ts[0], ts[1], ts[2]};
            if (which > 0) ty[which - 1] = tu[which - 1];
            double acc = 0.0;
            for (int i = 0; i < 3; i++) {
                const double ci = c_type[ty[0]][i];
                if (ci == 0.0) continue;
                for (int j = 0; j < 3; j++) {
                    const double cj = c_type[ty[1]][j];
                    if (cj == 0.0) continue;
                    for (int k = 0; k < 3; k++) {
                        const double ck = c_type[ty[2]][k];
                        if (ck == 0.0) continue;
                        acc = fma(ci * cj * ck, m[i * 9 + j * 3 + k], acc);
                    }
                }
            }
            if (which == 0) Ib[a] = acc; else Iu[a][which - 1] = acc;
        }
    }
    for (int r = 0; r < nrhs; r++) {
        const double fa = fv[(size_t)ia * nrhs + r], fb = fv[(size_t)ib * nrhs + r], fc = fv[(size_t)ic * nrhs + r];
        const double d1 = fb - fa, d2 = fc - fa;
        const double al = (g22 * d1 - g12 * d2) / det, be = (g11 * d2 - g12 * d1) / det;
        double g[3];
        for (int k = 0; k < 3; k++) g[k] = al * e1[k] + be * e2[k];     // tangential gradient of f
        const double beta0 = fa + g[0] * lo[0] + g[1] * lo[1] + g[2] * lo[2];
        for (int a = 0; a < 8; a++) {
            const double v = beta0 * Ib[a] + g[0] * Iu[a][0] + g[1] * Iu[a][1] + g[2] * Iu[a][2];
            out[(8 * (size_t)f + a) * 4 + r] = v * fscale[f];
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
