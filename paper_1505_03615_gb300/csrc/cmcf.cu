// cmcf.cu -- the metric of one conformalized mean-curvature-flow step (Section 5.3) on
// the device.
//
// A step solves (M_t + delta L_0) u_{t+1} = M_t u_t on the build-time function space.
// The surface has moved by an affine map per triangle, so the area element of triangle T
// at time t is its build-time one times w_T = A_t(T) / A_0(T); M_t is the build-time mass
// matrix with every fragment of T weighted by w_T, and L_0 stays as built.  The assembly
// and projection kernels already multiply each fragment's mass and right-hand-side
// contributions (not its stiffness) by a per-fragment scale, the physical area of one
// finest-grid unit of area (sigma^2); a step sets that scale to sigma^2 w_T from the
// current vertex positions.
#include "lbmg_internal.h"

namespace lbmg {

namespace {

__device__ __forceinline__ double tri_area2(const double *P, int a, int b, int c) {
    const double e1[3] = {P[3 * b] - P[3 * a], P[3 * b + 1] - P[3 * a + 1], P[3 * b + 2] - P[3 * a + 2]};
    const double e2[3] = {P[3 * c] - P[3 * a], P[3 * c + 1] - P[3 * a + 1], P[3 * c + 2] - P[3 * a + 2]};
    const double n0 = e1[1] * e2[2] - e1[2] * e2[1];
    const double n1 = e1[2] * e2[0] - e1[0] * e2[2];
    const double n2 = e1[0] * e2[1] - e1[1] * e2[0];
    return sqrt(n0 * n0 + n1 * n1 + n2 * n2);   // twice the area
}

// w_T = area of T at the positions X (world units) / its build-time area (grid units x sigma^2);
// a triangle of zero build-time area gets 0 (it has no fragments)
__global__ void cmcf_weight_kernel(int nt, const int *__restrict__ F, const double *__restrict__ Vg,
                                   const double *__restrict__ X, double sigma2, double *__restrict__ w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int a = F[3 * t], b = F[3 * t + 1], c = F[3 * t + 2];
    const double a0 = tri_area2(Vg, a, b, c) * sigma2;
    w[t] = a0 > 0.0 ? tri_area2(X, a, b, c) / a0 : 0.0;
}

__global__ void cmcf_frag_scale_kernel(int nfrag, const int *__restrict__ ftri, const double *__restrict__ w,
                                       double sigma2, double *__restrict__ scale) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfrag) return;
    scale[f] = sigma2 * w[ftri[f]];
}

}  // namespace

void launch_cmcf_weights(const Ctx &c, const double *X, double *tri_w, cudaStream_t s) {
    const double sigma2 = c.host.sigma * c.host.sigma;
    if (c.nt > 0) cmcf_weight_kernel<<<(c.nt + 255) / 256, 256, 0, s>>>(c.nt, c.F, c.Vg, X, sigma2, tri_w);
    if (c.nfrag > 0)
        cmcf_frag_scale_kernel<<<(c.nfrag + 255) / 256, 256, 0, s>>>(c.nfrag, c.ftri, tri_w, sigma2, c.frag_scale);
}

}  // namespace lbmg
