// hier.cpp -- host construction of the split B-spline hierarchy (Chuang & Kazhdan,
// Sections 3.2, 4.1-4.3) in the layout the CUDA kernels consume.
//
// Finest level: every triangle is cut into voxel pieces by sweeping the grid
// planes axis by axis.  Coarser levels reuse those pieces: a triangle meets a
// coarse voxel exactly when it has a piece in one of its fine sub-voxels.  For
// each corner the triangles meeting its support are joined through shared mesh
// edges that meet the open support cube, or shared vertices inside it; each
// resulting component is one function b_k^i.  Dofs are ordered by corner
// parity colour, then Morton key, then smallest triangle, so that one colour is
// a contiguous range of rows with no couplings inside it.
#include "hier.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <memory>
#include <numeric>
#include <stdexcept>

#ifdef _OPENMP
#include <omp.h>
#include <parallel/algorithm>
#define LBMG_SORT __gnu_parallel::sort
#else
#define LBMG_SORT std::sort
#endif

namespace lbmg {
namespace {

struct Pt { double v[3]; };
using Poly = std::vector<Pt>;

// split polygon by the plane x[axis] = c into the part below and the part above
void split_poly(const Poly &in, int axis, double c, Poly &lo, Poly &hi) {
    lo.clear(); hi.clear();
    const size_t n = in.size();
    for (size_t i = 0; i < n; i++) {
        const Pt &a = in[i], &b = in[(i + 1) % n];
        double da = a.v[axis] - c, db = b.v[axis] - c;
        if (da <= 0) lo.push_back(a);
        if (da >= 0) hi.push_back(a);
        if ((da < 0 && db > 0) || (da > 0 && db < 0)) {
            double t = (c - a.v[axis]) / (b.v[axis] - a.v[axis]);
            Pt p;
            for (int k = 0; k < 3; k++) p.v[k] = a.v[k] + t * (b.v[k] - a.v[k]);
            p.v[axis] = c;
            lo.push_back(p);
            hi.push_back(p);
        }
    }
}

double poly_area(const Poly &p) {
    double s[3] = {0, 0, 0};
    for (size_t i = 1; i + 1 < p.size(); i++) {
        double e1[3], e2[3];
        for (int k = 0; k < 3; k++) { e1[k] = p[i].v[k] - p[0].v[k]; e2[k] = p[i + 1].v[k] - p[0].v[k]; }
        s[0] += e1[1] * e2[2] - e1[2] * e2[1];
        s[1] += e1[2] * e2[0] - e1[0] * e2[2];
        s[2] += e1[0] * e2[1] - e1[1] * e2[0];
    }
    return 0.5 * std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
}

// cut triangle t into finest-voxel pieces by sweeping planes along x, then y, then z
void cut_triangle(const HostHierarchy &H, int t, int N, std::vector<FragOut> &out) {
    Poly tri(3);
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 3; a++) tri[k].v[a] = H.Vg[3 * (size_t)H.F[3 * t + k] + a];
    auto range = [&](const Poly &p, int axis, int &lo, int &hi) {
        double mn = p[0].v[axis], mx = mn;
        for (auto &q : p) { mn = std::min(mn, q.v[axis]); mx = std::max(mx, q.v[axis]); }
        lo = std::max(0, (int)std::floor(mn));
        hi = std::min(N - 1, (int)std::floor(mx));
    };
    Poly below, above, rest, rest2, rest3;
    int x0, x1;
    range(tri, 0, x0, x1);
    rest = tri;
    for (int ix = x0; ix <= x1 && rest.size() >= 3; ix++) {
        Poly slabx;
        if (ix < x1) { split_poly(rest, 0, (double)(ix + 1), below, above); slabx = below; rest = above; }
        else slabx = rest;
        if (slabx.size() < 3) continue;
        int y0, y1;
        range(slabx, 1, y0, y1);
        rest2 = slabx;
        for (int iy = y0; iy <= y1 && rest2.size() >= 3; iy++) {
            Poly slaby;
            if (iy < y1) { split_poly(rest2, 1, (double)(iy + 1), below, above); slaby = below; rest2 = above; }
            else slaby = rest2;
            if (slaby.size() < 3) continue;
            int z0, z1;
            range(slaby, 2, z0, z1);
            rest3 = slaby;
            for (int iz = z0; iz <= z1 && rest3.size() >= 3; iz++) {
                Poly cell;
                if (iz < z1) { split_poly(rest3, 2, (double)(iz + 1), below, above); cell = below; rest3 = above; }
                else cell = rest3;
                if (cell.size() < 3) continue;
                if (!(poly_area(cell) > kFragTau)) continue;
                FragOut f;
                f.tri = t;
                f.vox[0] = ix; f.vox[1] = iy; f.vox[2] = iz;
                f.key = morton(ix, iy, iz);
                f.poly.resize(cell.size() * 3);
                for (size_t q = 0; q < cell.size(); q++)
                    for (int a = 0; a < 3; a++) f.poly[3 * q + a] = cell[q].v[a] - (double)f.vox[a];
                out.push_back(std::move(f));
            }
        }
    }
}

// does the closed segment [a,b] meet the open box (lo,hi)^3 ?
bool segment_hits_open_box(const double *a, const double *b, const double *lo, const double *hi) {
    double tmin = -INFINITY, tmax = INFINITY;
    for (int k = 0; k < 3; k++) {
        const double d = b[k] - a[k];
        if (d == 0.0) {
            if (!(a[k] > lo[k] && a[k] < hi[k])) return false;
            continue;
        }
        double t1 = (lo[k] - a[k]) / d, t2 = (hi[k] - a[k]) / d;
        if (t2 < t1) std::swap(t1, t2);
        tmin = std::max(tmin, t1);
        tmax = std::min(tmax, t2);
    }
    return tmin < tmax && tmin < 1.0 && tmax > 0.0;
}

bool point_in_open_box(const double *p, const double *lo, const double *hi) {
    return p[0] > lo[0] && p[0] < hi[0] && p[1] > lo[1] && p[1] < hi[1] && p[2] > lo[2] && p[2] < hi[2];
}

using KT = CornerTri;
inline bool kt_less(const KT &a, const KT &b) { return a.key < b.key || (a.key == b.key && a.tri < b.tri); }

// CSR lists of the positions i of bucket[i], each bucket's positions ascending: a sort of
// the keys bucket * 2^32 + i (fewer than 2^32 entries)
void bucket_positions(int64_t nb, const std::vector<int32_t> &bucket, std::vector<int64_t> &ptr,
                      std::vector<uint32_t> &out) {
    const size_t m = bucket.size();
    if (m > (size_t)UINT32_MAX) throw std::length_error("list too long for 32-bit positions");
    std::vector<uint64_t> key(m);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < m; i++) key[i] = (uint64_t)(uint32_t)bucket[i] << 32 | (uint64_t)i;
    LBMG_SORT(key.begin(), key.end());
    out.resize(m);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < m; i++) out[i] = (uint32_t)key[i];
    ptr.assign(nb + 1, 0);
    for (size_t i = 0; i < m; i++) ptr[(key[i] >> 32) + 1]++;
    for (int64_t i = 0; i < nb; i++) ptr[i + 1] += ptr[i];
}

// (bucket, value) pairs into CSR, the values of one bucket in input order
template <class V>
void bucket_csr(int64_t nb, const std::vector<int32_t> &bucket, const std::vector<V> &val,
                std::vector<int64_t> &ptr, std::vector<V> &out) {
    std::vector<uint32_t> pos;
    bucket_positions(nb, bucket, ptr, pos);
    out.resize(pos.size());
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < pos.size(); i++) out[i] = val[pos[i]];
}

int lookup_dof(const HostLevel &L, uint64_t key, int tri) {
    const KT probe{key, tri};
    size_t lo = 0, hi = L.ct.size();
    while (lo < hi) {
        size_t mid = (lo + hi) / 2;
        if (kt_less(L.ct[mid], probe)) lo = mid + 1; else hi = mid;
    }
    if (lo < L.ct.size() && L.ct[lo].key == key && L.ct[lo].tri == tri) return L.ct_dof[lo];
    return -1;
}

// split basis of one level from its (voxel, triangle) cells
void build_level_basis(HostHierarchy &H, HostLevel &L, const std::vector<KT> &cells,
                       const std::vector<int32_t> &adj_ptr, const std::vector<int32_t> &adj,
                       const std::vector<int32_t> &vt_ptr, const std::vector<int32_t> &vt, const GpuBasis *gb) {
    const int shift = H.D - L.d;
    const double s = (double)(1 << shift);
    // (corner, triangle) pairs
    std::vector<KT> ct;
    // a corner of depth d has coordinates up to 2^d, so its Morton key has 3 (d + 1) bits; when
    // key and triangle fit one 64-bit word, the pairs are sorted as such words (same order)
    int tbits = 1;
    while (tbits < 31 && (1LL << tbits) < (int64_t)H.nt) tbits++;
    std::vector<uint64_t> gw;   // the GPU's sorted unique words (gb only)
    const bool on_gpu = gb != nullptr && 3 * (L.d + 1) + tbits <= 64;
    if (on_gpu) {
        std::string err;
        if (!gpu_corner_pairs(cells, tbits, 3 * (L.d + 1), gw, err)) throw BuildCudaError(err);
        ct.resize(gw.size());
        const uint64_t tmask = (1ULL << tbits) - 1;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)gw.size(); i++) ct[i] = KT{gw[i] >> tbits, (int32_t)(gw[i] & tmask)};
    } else if (3 * (L.d + 1) + tbits <= 64) {
        std::vector<uint64_t> w(cells.size() * 8);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)cells.size(); i++) {
            uint32_t vx = compact3(cells[i].key), vy = compact3(cells[i].key >> 1), vz = compact3(cells[i].key >> 2);
            for (int a = 0; a < 8; a++)
                w[8 * i + a] = morton(vx + (a & 1), vy + ((a >> 1) & 1), vz + ((a >> 2) & 1)) << tbits |
                               (uint64_t)(uint32_t)cells[i].tri;
        }
        LBMG_SORT(w.begin(), w.end());
        w.erase(std::unique(w.begin(), w.end()), w.end());
        ct.resize(w.size());
        const uint64_t tmask = (1ULL << tbits) - 1;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)w.size(); i++) ct[i] = KT{w[i] >> tbits, (int32_t)(w[i] & tmask)};
    } else {
        ct.resize(cells.size() * 8);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)cells.size(); i++) {
            uint32_t vx = compact3(cells[i].key), vy = compact3(cells[i].key >> 1), vz = compact3(cells[i].key >> 2);
            for (int a = 0; a < 8; a++)
                ct[8 * i + a] = KT{morton(vx + (a & 1), vy + ((a >> 1) & 1), vz + ((a >> 2) & 1)), cells[i].tri};
        }
        LBMG_SORT(ct.begin(), ct.end(), kt_less);
        ct.erase(std::unique(ct.begin(), ct.end(), [](const KT &a, const KT &b) { return a.key == b.key && a.tri == b.tri; }), ct.end());
    }
    const size_t m = ct.size();
    // corner groups
    std::vector<int64_t> gstart;
    for (size_t i = 0; i < m; i++) if (i == 0 || ct[i].key != ct[i - 1].key) gstart.push_back((int64_t)i);
    gstart.push_back((int64_t)m);
    const int64_t ng = (int64_t)gstart.size() - 1;
    std::vector<int32_t> comp(m);          // component label inside the corner, ordered by min triangle
    std::vector<int32_t> ncomp(ng);
    // Corners are taken largest first, one at a time: on coarse levels a few corners hold
    // most of the mesh each, and they must not queue behind one another on one thread.
    // With the GPU labelling the host takes only the runs the GPU leaves (ncomp < 0).
    std::vector<int64_t> order;
    if (on_gpu) {
        std::string err;
        if (!gpu_run_components(gb, gw, gstart, tbits, H.split, s, comp, ncomp, err)) throw BuildCudaError(err);
        for (int64_t g = 0; g < ng; g++) if (ncomp[g] < 0) order.push_back(g);
    } else {
        order.resize(ng);
        std::iota(order.begin(), order.end(), (int64_t)0);
    }
    std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        const int64_t sx = gstart[x + 1] - gstart[x], sy = gstart[y + 1] - gstart[y];
        return sx > sy || (sx == sy && x < y);
    });
#pragma omp parallel
    {
        std::vector<int32_t> par, lab;
        // position of each triangle within the current corner's list, -1 when absent
        std::vector<int32_t> slot_of(H.nt, -1);
#pragma omp for schedule(dynamic, 1)
        for (int64_t o = 0; o < (int64_t)order.size(); o++) {
            const int64_t g = order[o];
            const int64_t b = gstart[g], e = gstart[g + 1];
            const int n = (int)(e - b);
            par.resize(n);
            lab.assign(n, -1);
            std::iota(par.begin(), par.end(), 0);
            for (int i = 0; i < n; i++) slot_of[ct[b + i].tri] = i;
            auto find = [&](int x) { while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; } return x; };
            auto unite = [&](int x, int y) { x = find(x); y = find(y); if (x != y) { if (x < y) par[y] = x; else par[x] = y; } };
            auto local = [&](int tri) -> int { return slot_of[tri]; };
            if (H.split) {
                uint64_t key = ct[b].key;
                double c[3] = {(double)compact3(key), (double)compact3(key >> 1), (double)compact3(key >> 2)};
                double lo[3], hi[3];
                for (int a = 0; a < 3; a++) { lo[a] = (c[a] - 1.0) * s; hi[a] = (c[a] + 1.0) * s; }
                for (int i = 0; i < n; i++) {
                    const int t = ct[b + i].tri;
                    for (int e3 = 0; e3 < 3; e3++) {
                        const int va = H.F[3 * t + e3], vb = H.F[3 * t + (e3 + 1) % 3];
                        bool tested = false, hit = false;
                        for (int q = adj_ptr[3 * t + e3]; q < adj_ptr[3 * t + e3 + 1]; q++) {
                            int j = local(adj[q]);
                            if (j < 0) continue;
                            if (!tested) {
                                hit = segment_hits_open_box(&H.Vg[3 * (size_t)va], &H.Vg[3 * (size_t)vb], lo, hi);
                                tested = true;
                            }
                            if (hit) unite(i, j);
                        }
                    }
                    for (int e3 = 0; e3 < 3; e3++) {
                        const int v = H.F[3 * t + e3];
                        if (!point_in_open_box(&H.Vg[3 * (size_t)v], lo, hi)) continue;
                        for (int q = vt_ptr[v]; q < vt_ptr[v + 1]; q++) {
                            int j = local(vt[q]);
                            if (j >= 0) unite(i, j);
                        }
                    }
                }
            } else {
                for (int i = 0; i < n; i++) par[i] = 0;
            }
            int nc = 0;
            for (int i = 0; i < n; i++) {
                int r = find(i);
                if (lab[r] < 0) lab[r] = nc++;
                comp[b + i] = lab[r];
            }
            ncomp[g] = nc;
            for (int i = 0; i < n; i++) slot_of[ct[b + i].tri] = -1;
        }
    }
    // dofs: one per (corner, component); order by colour, Morton key, smallest triangle
    struct DofRec { int colour; uint64_t key; int32_t mintri; int64_t group; int32_t comp; };
    std::vector<int64_t> gbase(ng + 1, 0);
    for (int64_t g = 0; g < ng; g++) gbase[g + 1] = gbase[g] + ncomp[g];
    std::vector<DofRec> dofs(gbase[ng]);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < ng; g++) {
        const int64_t b = gstart[g];
        const uint64_t key = ct[b].key;
        const int colour = (compact3(key) & 1) | ((compact3(key >> 1) & 1) << 1) | ((compact3(key >> 2) & 1) << 2);
        // labels number the components in the order of their first (smallest) triangle, so the first
        // occurrences of labels 0, 1, 2, ... come in that order along the run
        int next = 0;
        for (int64_t i = b; i < gstart[g + 1] && next < ncomp[g]; i++)
            if (comp[i] == next) {
                dofs[gbase[g] + next] = DofRec{colour, key, ct[i].tri, g, next};
                next++;
            }
    }
    LBMG_SORT(dofs.begin(), dofs.end(), [](const DofRec &a, const DofRec &b) {
        if (a.colour != b.colour) return a.colour < b.colour;
        if (a.key != b.key) return a.key < b.key;
        return a.mintri < b.mintri;
    });
    L.ndof = (int)dofs.size();
    L.corner.resize(3 * (size_t)L.ndof);
    L.mintri.resize(L.ndof);
    for (int c = 0; c <= 8; c++) L.colour_start[c] = 0;
    std::vector<int32_t> dof_id(gbase[ng]);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < L.ndof; i++) {
        const DofRec &r = dofs[i];
        L.corner[3 * i] = (int)compact3(r.key);
        L.corner[3 * i + 1] = (int)compact3(r.key >> 1);
        L.corner[3 * i + 2] = (int)compact3(r.key >> 2);
        L.mintri[i] = r.mintri;
        dof_id[gbase[r.group] + r.comp] = i;
    }
    for (int i = 0; i < L.ndof; i++) L.colour_start[dofs[i].colour + 1]++;
    for (int c = 0; c < 8; c++) L.colour_start[c + 1] += L.colour_start[c];
    L.ct_dof.resize(m);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < ng; g++)
        for (int64_t i = gstart[g]; i < gstart[g + 1]; i++) L.ct_dof[i] = dof_id[gbase[g] + comp[i]];
    L.ct = std::move(ct);
}

// Sparsity pattern of n rows over ncols columns and the contribution list of every stored
// entry, built row by row.  emit(i, f) calls f(col, value) for each contribution to row i,
// in list order; row i stores the distinct cols, sorted, and the list of stored entry
// (i, col) holds the values of the contributions to it in the order they were emitted.
// Each thread keeps dense per-column marks, so a contribution costs O(1).
template <class Emit>
void rows_with_lists(int n, int ncols, const Emit &emit, HostLevel &L, std::vector<int64_t> &lptr,
                     std::vector<uint32_t> &lidx) {
    std::vector<int32_t> cnt(n);
#pragma omp parallel
    {
        std::vector<int32_t> seen(ncols, -1);
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; i++) {
            int32_t m = 0;
            emit(i, [&](int32_t c, uint32_t) { if (seen[c] != i) { seen[c] = i; m++; } });
            cnt[i] = m;
        }
    }
    int64_t total = 0;
    for (int i = 0; i < n; i++) total += cnt[i];
    if (total > (int64_t)INT32_MAX) throw std::length_error("level has too many stored entries for 32-bit rows");
    L.rp.assign(n + 1, 0);
    for (int i = 0; i < n; i++) L.rp[i + 1] = L.rp[i] + cnt[i];
    const int64_t nnz = L.rp[n];
    L.ci.resize(nnz);
    std::vector<int64_t> pos(nnz + 1, 0);   // contributions per stored entry, then list starts
#pragma omp parallel
    {
        std::vector<int32_t> seen(ncols, -1), slot(ncols);
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; i++) {
            int32_t *row = L.ci.data() + L.rp[i];
            int m = 0;
            emit(i, [&](int32_t c, uint32_t) { if (seen[c] != i) { seen[c] = i; row[m++] = c; } });
            std::sort(row, row + m);
            for (int q = 0; q < m; q++) slot[row[q]] = L.rp[i] + q;
            emit(i, [&](int32_t c, uint32_t) { pos[slot[c] + 1]++; });
        }
    }
    for (int64_t k = 0; k < nnz; k++) pos[k + 1] += pos[k];
    lptr = pos;
    lidx.resize(pos[nnz]);
    // each row fills only its own entries' lists
#pragma omp parallel
    {
        std::vector<int32_t> slot(ncols);
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; i++) {
            for (int32_t k = L.rp[i]; k < L.rp[i + 1]; k++) slot[L.ci[k]] = k;
            emit(i, [&](int32_t c, uint32_t v) { lidx[pos[slot[c]]++] = v; });
        }
    }
}

}  // namespace

int build_host_hierarchy(const double *V, int nv, const int *F, int nt, int depth, int min_depth,
                         int coarse_max, int split, int threads, HostHierarchy &H, std::string &err,
                         bool fail_alloc, bool gpu_clip) {
    if (!V || !F || nv < 3 || nt < 1 || depth < 1 || depth > kMaxDepth) { err = "bad mesh size or depth"; return 1; }
    for (int64_t i = 0; i < 3 * (int64_t)nt; i++)
        if (F[i] < 0 || F[i] >= nv) { err = "triangle index out of range"; return 1; }
    for (int64_t i = 0; i < 3 * (int64_t)nv; i++)
        if (!std::isfinite(V[i])) { err = "non-finite vertex coordinate"; return 1; }
    if (min_depth > depth) { err = "min_depth > depth"; return 1; }
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    H = HostHierarchy();
    H.D = depth; H.nv = nv; H.nt = nt; H.split = split ? 1 : 0;
    const int N = 1 << depth;
    // embedding: bounding box centred in a cube of side 1.1 x largest extent, finest-grid units
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < nv; i++)
        for (int a = 0; a < 3; a++) { mn[a] = std::min(mn[a], V[3 * i + a]); mx[a] = std::max(mx[a], V[3 * i + a]); }
    double ext = 0;
    for (int a = 0; a < 3; a++) { H.center[a] = 0.5 * (mn[a] + mx[a]); ext = std::max(ext, mx[a] - mn[a]); }
    if (!(ext > 0)) { err = "mesh has zero extent"; return 2; }
    H.S = 1.1 * ext;
    H.sigma = H.S / (double)N;
    H.Vg.resize(3 * (size_t)nv);
    for (int i = 0; i < nv; i++)
        for (int a = 0; a < 3; a++) H.Vg[3 * i + a] = (V[3 * i + a] - H.center[a]) / H.S * (double)N + 0.5 * (double)N;
    H.F.assign(F, F + 3 * (size_t)nt);
    H.tri_normal.resize(3 * (size_t)nt);
    for (int t = 0; t < nt; t++) {
        const double *A = &H.Vg[3 * (size_t)F[3 * t]], *B = &H.Vg[3 * (size_t)F[3 * t + 1]], *C = &H.Vg[3 * (size_t)F[3 * t + 2]];
        double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int a = 0; a < 3; a++) H.tri_normal[3 * t + a] = l > 0 ? n[a] / l : 0.0;
    }
    // mesh adjacency: triangles across each triangle edge, triangles around each vertex
    std::vector<int32_t> adj_ptr(3 * (size_t)nt + 1, 0), adj;
    {
        struct E { uint64_t key; int32_t slot; };
        std::vector<E> es(3 * (size_t)nt);
        for (int t = 0; t < nt; t++)
            for (int e = 0; e < 3; e++) {
                uint64_t a = (uint32_t)F[3 * t + e], b = (uint32_t)F[3 * t + (e + 1) % 3];
                es[3 * t + e] = E{a < b ? (a << 32 | b) : (b << 32 | a), 3 * t + e};
            }
        LBMG_SORT(es.begin(), es.end(), [](const E &x, const E &y) { return x.key < y.key || (x.key == y.key && x.slot < y.slot); });
        std::vector<int32_t> cnt(3 * (size_t)nt, 0);
        for (size_t i = 0; i < es.size();) {
            size_t j = i;
            while (j < es.size() && es[j].key == es[i].key) j++;
            for (size_t a = i; a < j; a++) cnt[es[a].slot] = (int32_t)(j - i - 1);
            i = j;
        }
        for (size_t i = 0; i < cnt.size(); i++) adj_ptr[i + 1] = adj_ptr[i] + cnt[i];
        adj.resize(adj_ptr.back());
        std::vector<int32_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
        for (size_t i = 0; i < es.size();) {
            size_t j = i;
            while (j < es.size() && es[j].key == es[i].key) j++;
            for (size_t a = i; a < j; a++)
                for (size_t b = i; b < j; b++)
                    if (a != b) adj[fill[es[a].slot]++] = es[b].slot / 3;
            i = j;
        }
    }
    std::vector<int32_t> vt_ptr(nv + 1, 0), vt(3 * (size_t)nt);
    for (int64_t i = 0; i < 3 * (int64_t)nt; i++) vt_ptr[F[i] + 1]++;
    for (int i = 0; i < nv; i++) vt_ptr[i + 1] += vt_ptr[i];
    {
        std::vector<int32_t> fill(vt_ptr.begin(), vt_ptr.end() - 1);
        for (int t = 0; t < nt; t++)
            for (int e = 0; e < 3; e++) vt[fill[F[3 * t + e]]++] = t;
    }

    // the mesh on the device for the GPU labelling of row a2 (with gpu_clip)
    std::unique_ptr<GpuBasis, void (*)(GpuBasis *)> gbase(nullptr, gpu_basis_free);
    if (gpu_clip) {
        gbase.reset(gpu_basis_setup(H, adj_ptr, adj, vt_ptr, vt, err));
        if (!gbase) return 7;   // LBMG_CUDA_ERROR
    }
    // finest fragments
    std::vector<FragOut> frags;
    if (gpu_clip) {
        const int st = gpu_cut_triangles(H, N, frags, err);
        if (st) return st;
#pragma omp parallel for schedule(static)
        for (long q = 0; q < (long)frags.size(); q++) frags[q].key = morton(frags[q].vox[0], frags[q].vox[1], frags[q].vox[2]);
    } else {
#ifdef _OPENMP
        int nth = omp_get_max_threads();
#else
        int nth = 1;
#endif
        std::vector<std::vector<FragOut>> part(nth);
#pragma omp parallel
        {
#ifdef _OPENMP
            int me = omp_get_thread_num();
#else
            int me = 0;
#endif
#pragma omp for schedule(dynamic, 512)
            for (int t = 0; t < nt; t++) cut_triangle(H, t, N, part[me]);
        }
        size_t total = 0;
        for (auto &p : part) total += p.size();
        frags.reserve(total);
        for (auto &p : part) for (auto &f : p) frags.push_back(std::move(f));
    }
    if (frags.empty()) { err = "no triangle piece of positive area"; return 2; }
    if (fail_alloc) throw std::bad_alloc();
    LBMG_SORT(frags.begin(), frags.end(), [](const FragOut &a, const FragOut &b) {
        return a.key < b.key || (a.key == b.key && a.tri < b.tri);
    });
    H.nfrag = (int)frags.size();
    H.frag_tri.resize(H.nfrag);
    H.frag_vox.resize(3 * (size_t)H.nfrag);
    H.frag_pstart.resize(H.nfrag + 1);
    H.frag_pstart[0] = 0;
    for (int f = 0; f < H.nfrag; f++) H.frag_pstart[f + 1] = H.frag_pstart[f] + (int32_t)(frags[f].poly.size() / 3);
    H.frag_poly.resize(3 * (size_t)H.frag_pstart[H.nfrag]);
#pragma omp parallel for schedule(static)
    for (int f = 0; f < H.nfrag; f++) {
        H.frag_tri[f] = frags[f].tri;
        for (int a = 0; a < 3; a++) H.frag_vox[3 * f + a] = frags[f].vox[a];
        std::copy(frags[f].poly.begin(), frags[f].poly.end(), H.frag_poly.begin() + 3 * (size_t)H.frag_pstart[f]);
    }

    // levels from the finest down
    H.lev.assign(depth + 1, HostLevel());
    std::vector<KT> cells(H.nfrag);
#pragma omp parallel for schedule(static)
    for (int f = 0; f < H.nfrag; f++) {
        cells[f] = KT{frags[f].key, frags[f].tri};
        std::vector<double>().swap(frags[f].poly);   // the pieces' polygons are freed by all threads
    }
    frags.clear();
    frags.shrink_to_fit();
    cells.erase(std::unique(cells.begin(), cells.end(), [](const KT &a, const KT &b) { return a.key == b.key && a.tri == b.tri; }), cells.end());
    int d = depth;
    for (;;) {
        HostLevel &L = H.lev[d];
        L.d = d;
        build_level_basis(H, L, cells, adj_ptr, adj, vt_ptr, vt, gbase.get());
        if (min_depth >= 0) { if (d <= min_depth) break; }
        else if (L.ndof <= coarse_max) break;
        if (d == 0) break;
        // coarse cells: (voxel >> 1, triangle), Morton key >> 3
        for (auto &c : cells) c.key >>= 3;
        LBMG_SORT(cells.begin(), cells.end(), kt_less);
        cells.erase(std::unique(cells.begin(), cells.end(), [](const KT &a, const KT &b) { return a.key == b.key && a.tri == b.tri; }), cells.end());
        d--;
    }
    H.d0 = d;

    // finest fragments -> dofs of their 8 corners
    HostLevel &LF = H.lev[depth];
    H.frag_dof.resize(8 * (size_t)H.nfrag);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int f = 0; f < H.nfrag; f++)
        for (int a = 0; a < 8; a++) {
            uint64_t key = morton(H.frag_vox[3 * f] + (a & 1), H.frag_vox[3 * f + 1] + ((a >> 1) & 1), H.frag_vox[3 * f + 2] + ((a >> 2) & 1));
            int dof = lookup_dof(LF, key, H.frag_tri[f]);
            if (dof < 0) bad++;
            H.frag_dof[8 * (size_t)f + a] = dof;
        }
    if (bad) { err = "internal: fragment corner without a function"; return 1; }

    // finest right-hand-side lists: per dof, fragment * 8 + corner of its incidences, fragments ascending
    bucket_positions(LF.ndof, H.frag_dof, H.rrp, H.ridx);
    // finest pattern and assembly contribution lists: row i couples with every corner dof of
    // the fragments incident to it; stored entry (i, j) lists 36 f + pair(a, b) for each such
    // fragment f with corner a at i and corner b at j (the 8 corners of a fragment are 8
    // different dofs, so each fragment contributes once), fragments ascending
    rows_with_lists(LF.ndof, LF.ndof, [&](int i, auto &&f) {
        for (int64_t q = H.rrp[i]; q < H.rrp[i + 1]; q++) {
            const size_t fr = H.ridx[q] >> 3;
            const int a = (int)(H.ridx[q] & 7u);
            for (int b = 0; b < 8; b++) f(H.frag_dof[8 * fr + b], (uint32_t)(36 * fr + pair_index(a, b)));
        }
    }, LF, H.arp, H.aidx);

    // prolongation, restriction lists and Galerkin contributions, finest to coarsest
    for (int df = depth; df > H.d0; df--) {
        HostLevel &Lf = H.lev[df], &Lc = H.lev[df - 1];
        Lf.par.assign(8 * (size_t)Lf.ndof, -1);
        Lf.npar_log2.assign(Lf.ndof, 0);
        int missing = 0;
#pragma omp parallel for schedule(static) reduction(+ : missing)
        for (int i = 0; i < Lf.ndof; i++) {
            const int *k = &Lf.corner[3 * (size_t)i];
            int cand[3][2], cnt[3];
            for (int a = 0; a < 3; a++) {
                if ((k[a] & 1) == 0) { cand[a][0] = k[a] >> 1; cnt[a] = 1; }
                else { cand[a][0] = (k[a] - 1) >> 1; cand[a][1] = (k[a] + 1) >> 1; cnt[a] = 2; }
            }
            int m = 0;
            for (int x = 0; x < cnt[0]; x++)
                for (int y = 0; y < cnt[1]; y++)
                    for (int z = 0; z < cnt[2]; z++) {
                        int p = lookup_dof(Lc, morton(cand[0][x], cand[1][y], cand[2][z]), Lf.mintri[i]);
                        if (p < 0) missing++;
                        Lf.par[8 * (size_t)i + m++] = p;
                    }
            std::sort(Lf.par.begin() + 8 * (size_t)i, Lf.par.begin() + 8 * (size_t)i + m);
            Lf.npar_log2[i] = (int8_t)((cnt[0] - 1) + (cnt[1] - 1) + (cnt[2] - 1));
        }
        if (missing) { err = "internal: fine function without parent component"; return 1; }
        // restriction: children of each coarse dof
        {
            std::vector<int32_t> b;
            std::vector<uint32_t> v;
            for (int i = 0; i < Lf.ndof; i++)
                for (int q = 0; q < (1 << Lf.npar_log2[i]); q++) {
                    b.push_back(Lf.par[8 * (size_t)i + q]);
                    v.push_back((uint32_t)i | ((uint32_t)Lf.npar_log2[i] << kPackShift));
                }
            std::vector<int64_t> ptr;
            bucket_csr(Lc.ndof, b, v, ptr, Lc.cch);
            Lc.crp.assign(ptr.begin(), ptr.end());
        }
        // coarse pattern and Galerkin contributions: (P^T A P)_ab = sum_{i,l} A_il / (np_i np_l),
        // coarse row a from its children i (ascending), their stored entries k = (i, l)
        // (ascending) and the parents b of l; an (i, k) pair reaches a given (a, b) at most once
        // since the parents of a function are distinct
        if ((int64_t)Lf.rp[Lf.ndof] > (int64_t)kGalMask) { err = "level too large for packed Galerkin lists"; return 1; }
        rows_with_lists(Lc.ndof, Lc.ndof, [&](int a, auto &&f) {
            for (int32_t q = Lc.crp[a]; q < Lc.crp[a + 1]; q++) {
                const int i = (int)(Lc.cch[q] & kPackMask);
                for (int32_t k = Lf.rp[i]; k < Lf.rp[i + 1]; k++) {
                    const int l = Lf.ci[k];
                    const uint32_t e = (uint32_t)(Lf.npar_log2[i] + Lf.npar_log2[l]);
                    for (int pb = 0; pb < (1 << Lf.npar_log2[l]); pb++)
                        f(Lf.par[8 * (size_t)l + pb], (uint32_t)k | (e << kGalShift));
                }
            }
        }, Lc, Lc.grp, Lc.gidx);
    }

    // vertex evaluation at the finest level
    H.vdof.assign(8 * (size_t)nv, -1);
    H.vw.assign(8 * (size_t)nv, 0.0);
#pragma omp parallel for schedule(static)
    for (int v = 0; v < nv; v++) {
        if (vt_ptr[v] == vt_ptr[v + 1]) continue;
        const int t = vt[vt_ptr[v]];
        const double *p = &H.Vg[3 * (size_t)v];
        int vox[3];
        for (int a = 0; a < 3; a++) vox[a] = std::min(N - 1, std::max(0, (int)std::floor(p[a])));
        for (int a = 0; a < 8; a++) {
            int c[3] = {vox[0] + (a & 1), vox[1] + ((a >> 1) & 1), vox[2] + ((a >> 2) & 1)};
            double w = 1.0;
            for (int k = 0; k < 3; k++) w *= std::max(0.0, 1.0 - std::fabs(p[k] - (double)c[k]));
            if (!(w > 0)) continue;
            int dof = lookup_dof(LF, morton(c[0], c[1], c[2]), t);
            if (dof < 0) continue;
            H.vdof[8 * (size_t)v + a] = dof;
            H.vw[8 * (size_t)v + a] = w;
        }
    }
    return 0;
}

}  // namespace lbmg
