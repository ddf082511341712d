// clip.cu -- the finest-level pieces of the mesh on the GPU (row a1 of the hierarchy build).
//
// A piece is the part of one triangle inside one finest voxel (Section 3.2, Definition 2;
// the split space of Section 4.2 is built from these pieces).  One thread per triangle runs
// the host builder's sweep: the triangle is cut by the planes x = i + 1 into slabs, each slab
// by y = j + 1, each of those by z = k + 1, and a cell is kept when its area exceeds
// kFragTau.  A first pass counts the pieces and vertices of every triangle, the host turns
// the counts into offsets, and a second pass writes the pieces there.  The arithmetic is the
// host's (the same plane intersections, in the same order); polygon vertices agree with the
// host's up to FMA contraction, i.e. to a few units of the last place.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hier.h"

namespace lbmg {

namespace {

constexpr int kClipMaxV = 12;   // a triangle clipped by a box has at most 9 vertices

struct CPoly {
    double v[kClipMaxV][3];
    int n;
};

// the part of `in` below (lo) and above (hi) the plane x[axis] = c; false if a result would
// exceed kClipMaxV vertices
__device__ bool clip_split(const CPoly &in, int axis, double c, CPoly &lo, CPoly &hi) {
    lo.n = 0;
    hi.n = 0;
    for (int i = 0; i < in.n; i++) {
        const double *a = in.v[i], *b = in.v[(i + 1) % in.n];
        const double da = a[axis] - c, db = b[axis] - c;
        if (da <= 0) {
            if (lo.n >= kClipMaxV) return false;
            for (int k = 0; k < 3; k++) lo.v[lo.n][k] = a[k];
            lo.n++;
        }
        if (da >= 0) {
            if (hi.n >= kClipMaxV) return false;
            for (int k = 0; k < 3; k++) hi.v[hi.n][k] = a[k];
            hi.n++;
        }
        if ((da < 0 && db > 0) || (da > 0 && db < 0)) {
            if (lo.n >= kClipMaxV || hi.n >= kClipMaxV) return false;
            const double t = (c - a[axis]) / (b[axis] - a[axis]);
            double p[3];
            for (int k = 0; k < 3; k++) p[k] = a[k] + t * (b[k] - a[k]);
            p[axis] = c;
            for (int k = 0; k < 3; k++) { lo.v[lo.n][k] = p[k]; hi.v[hi.n][k] = p[k]; }
            lo.n++;
            hi.n++;
        }
    }
    return true;
}

__device__ double clip_area(const CPoly &p) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int i = 1; i + 1 < p.n; i++) {
        double e1[3], e2[3];
        for (int k = 0; k < 3; k++) { e1[k] = p.v[i][k] - p.v[0][k]; e2[k] = p.v[i + 1][k] - p.v[0][k]; }
        s0 += e1[1] * e2[2] - e1[2] * e2[1];
        s1 += e1[2] * e2[0] - e1[0] * e2[2];
        s2 += e1[0] * e2[1] - e1[1] * e2[0];
    }
    return 0.5 * sqrt(s0 * s0 + s1 * s1 + s2 * s2);
}

__device__ void clip_range(const CPoly &p, int axis, int N, int &lo, int &hi) {
    double mn = p.v[0][axis], mx = mn;
    for (int i = 1; i < p.n; i++) { mn = fmin(mn, p.v[i][axis]); mx = fmax(mx, p.v[i][axis]); }
    lo = max(0, (int)floor(mn));
    hi = min(N - 1, (int)floor(mx));
}

// kWrite = false: cnt[t] pieces and vcnt[t] vertices of triangle t.  kWrite = true: piece
// q = foff[t] + (its rank) gets ftri, fvox[3], fnv (vertex count) and its vertices, voxel-local,
// at fpoly + 3 * (voff[t] + vertices before it), never beyond the counts of the first pass.
template <bool kWrite>
__global__ void clip_kernel(int nt, const double *__restrict__ Vg, const int *__restrict__ F, int N,
                            int *__restrict__ cnt, int *__restrict__ vcnt, const long long *__restrict__ foff,
                            const long long *__restrict__ voff, int *__restrict__ ftri, int *__restrict__ fvox,
                            int *__restrict__ fnv, double *__restrict__ fpoly, int *__restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    CPoly rest, slabx, rest2, slaby, rest3, cell, below, above;
    rest.n = 3;
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 3; a++) rest.v[k][a] = Vg[3 * (size_t)F[3 * t + k] + a];
    int nf = 0, nvx = 0;
    long long fq = kWrite ? foff[t] : 0, vq = kWrite ? voff[t] : 0;
    bool ok = true;
    int x0, x1;
    clip_range(rest, 0, N, x0, x1);
    for (int ix = x0; ix <= x1 && rest.n >= 3 && ok; ix++) {
        if (ix < x1) { ok = clip_split(rest, 0, (double)(ix + 1), below, above); slabx = below; rest = above; }
        else slabx = rest;
        if (!ok || slabx.n < 3) continue;
        int y0, y1;
        clip_range(slabx, 1, N, y0, y1);
        rest2 = slabx;
        for (int iy = y0; iy <= y1 && rest2.n >= 3 && ok; iy++) {
            if (iy < y1) { ok = clip_split(rest2, 1, (double)(iy + 1), below, above); slaby = below; rest2 = above; }
            else slaby = rest2;
            if (!ok || slaby.n < 3) continue;
            int z0, z1;
            clip_range(slaby, 2, N, z0, z1);
            rest3 = slaby;
            for (int iz = z0; iz <= z1 && rest3.n >= 3 && ok; iz++) {
                if (iz < z1) { ok = clip_split(rest3, 2, (double)(iz + 1), below, above); cell = below; rest3 = above; }
                else cell = rest3;
                if (!ok || cell.n < 3) continue;
                if (!(clip_area(cell) > kFragTau)) continue;
                // the write pass reproduces the count pass; stay inside this triangle's slots regardless
                if (kWrite && (nf >= cnt[t] || nvx + cell.n > vcnt[t])) { ok = false; continue; }
                if (kWrite) {
                    ftri[fq] = t;
                    fvox[3 * fq] = ix;
                    fvox[3 * fq + 1] = iy;
                    fvox[3 * fq + 2] = iz;
                    fnv[fq] = cell.n;
                    for (int q = 0; q < cell.n; q++) {
                        fpoly[3 * (vq + q)] = cell.v[q][0] - (double)ix;
                        fpoly[3 * (vq + q) + 1] = cell.v[q][1] - (double)iy;
                        fpoly[3 * (vq + q) + 2] = cell.v[q][2] - (double)iz;
                    }
                    fq++;
                    vq += cell.n;
                }
                nf++;
                nvx += cell.n;
            }
        }
    }
    if (!ok) atomicExch(status, 1);
    if (!kWrite) {
        cnt[t] = nf;
        vcnt[t] = nvx;
    } else if (nf != cnt[t] || nvx != vcnt[t]) {
        atomicExch(status, 1);
    }
}

template <class T>
cudaError_t dalloc(T **p, size_t count) { return cudaMalloc((void **)p, (count ? count : 1) * sizeof(T)); }

}  // namespace

int gpu_cut_triangles(const HostHierarchy &H, int N, std::vector<FragOut> &out, std::string &err) {
    const int nt = H.nt;
    out.clear();
    if (nt == 0) return 0;
    double *Vg = nullptr, *fpoly = nullptr;
    int *F = nullptr, *cnt = nullptr, *vcnt = nullptr, *ftri = nullptr, *fvox = nullptr, *fnv = nullptr, *status = nullptr;
    long long *foff = nullptr, *voff = nullptr;
    std::vector<void *> owned;
    auto fail = [&](const char *what, cudaError_t e) {
        err = std::string("GPU clipping: ") + what + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        for (void *q : owned) cudaFree(q);
        return e == cudaErrorMemoryAllocation ? 3 : 7;   // LBMG_OUT_OF_MEMORY, LBMG_CUDA_ERROR
    };
    cudaError_t e;
    if ((e = dalloc(&Vg, H.Vg.size())) != cudaSuccess) return fail("allocation", e);
    owned.push_back(Vg);
    if ((e = dalloc(&F, H.F.size())) != cudaSuccess) return fail("allocation", e);
    owned.push_back(F);
    if ((e = dalloc(&cnt, nt)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(cnt);
    if ((e = dalloc(&vcnt, nt)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(vcnt);
    if ((e = dalloc(&status, 1)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(status);
    if ((e = cudaMemcpy(Vg, H.Vg.data(), H.Vg.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail("copy", e);
    if ((e = cudaMemcpy(F, H.F.data(), H.F.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail("copy", e);
    if ((e = cudaMemset(status, 0, sizeof(int))) != cudaSuccess) return fail("memset", e);
    const int threads = 128, blocks = (nt + threads - 1) / threads;
    clip_kernel<false><<<blocks, threads>>>(nt, Vg, F, N, cnt, vcnt, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                            status);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail("count pass", e);
    std::vector<int> hc(nt), hv(nt);
    cudaMemcpy(hc.data(), cnt, nt * sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(hv.data(), vcnt, nt * sizeof(int), cudaMemcpyDeviceToHost);
    std::vector<long long> fo(nt), vo(nt);
    long long nf = 0, nvx = 0;
    for (int t = 0; t < nt; t++) { fo[t] = nf; vo[t] = nvx; nf += hc[t]; nvx += hv[t]; }
    if ((e = dalloc(&foff, nt)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(foff);
    if ((e = dalloc(&voff, nt)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(voff);
    if ((e = dalloc(&ftri, nf)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(ftri);
    if ((e = dalloc(&fvox, 3 * nf)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(fvox);
    if ((e = dalloc(&fnv, nf)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(fnv);
    if ((e = dalloc(&fpoly, 3 * nvx)) != cudaSuccess) return fail("allocation", e);
    owned.push_back(fpoly);
    cudaMemcpy(foff, fo.data(), nt * sizeof(long long), cudaMemcpyHostToDevice);
    cudaMemcpy(voff, vo.data(), nt * sizeof(long long), cudaMemcpyHostToDevice);
    clip_kernel<true><<<blocks, threads>>>(nt, Vg, F, N, cnt, vcnt, foff, voff, ftri, fvox, fnv, fpoly, status);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail("write pass", e);
    int hs = 0;
    cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost);
    std::vector<int> htri(nf), hvox(3 * nf), hnv(nf);
    std::vector<double> hpoly(3 * nvx);
    cudaMemcpy(htri.data(), ftri, nf * sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(hvox.data(), fvox, 3 * nf * sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(hnv.data(), fnv, nf * sizeof(int), cudaMemcpyDeviceToHost);
    e = cudaMemcpy(hpoly.data(), fpoly, 3 * nvx * sizeof(double), cudaMemcpyDeviceToHost);
    for (void *q : owned) cudaFree(q);
    owned.clear();
    if (e != cudaSuccess) return fail("copy back", e);
    if (hs != 0) {
        err = "GPU clipping: a piece exceeded the kernel's vertex capacity";
        return 7;
    }
    out.resize(nf);
    std::vector<long long> vq(nf + 1, 0);   // first polygon vertex of each piece
    for (long long q = 0; q < nf; q++) vq[q + 1] = vq[q] + hnv[q];
#pragma omp parallel for schedule(static)
    for (long long q = 0; q < nf; q++) {
        FragOut &f = out[q];
        f.key = 0;
        f.tri = htri[q];
        for (int a = 0; a < 3; a++) f.vox[a] = hvox[3 * q + a];
        f.poly.assign(hpoly.begin() + 3 * vq[q], hpoly.begin() + 3 * vq[q + 1]);
    }
    return 0;
}

}  // namespace lbmg
