// basis.cu -- the split labelling of the hierarchy build (row a2) on the GPU.
//
// Per level, every (corner, triangle) pair of the level's cells (the 8 corners of each cell
// a triangle meets, Section 4.2) is formed, sorted and made unique; each corner's run of
// triangles is then split into the connected components of the corner's support on the
// mesh (the functions b_k^i of Section 4.2): two triangles of the run are joined through a
// shared edge that meets the open support cube, or a shared vertex inside it.  Runs of at
// most kSmallRun triangles are labelled one thread per run; longer runs (the coarse levels'), one
// thread per pair with a shared lock-free union-find.  Labels number a run's components in the order
// of their smallest triangle, so they do not depend on the order of the unions.  The box
// tests are divisions and comparisons only, exactly as on the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hier.h"

namespace lbmg {

namespace {

constexpr int kRT = 256, kRI = 16, kRTile = kRT * kRI;   // radix tile: 256 threads x 16 keys
constexpr int kDigits = 16;                               // 4-bit digits
// a run's parents and labels in 8 bits each in the thread's local memory: positions and labels 0..254,
// 255 marks "no label yet"
constexpr int kSmallRun = 255;

// the (corner, triangle) words of cell i: morton(corner) << tbits | tri
__global__ void pairs_kernel(long long ncell, const uint64_t *__restrict__ ckey, const int *__restrict__ ctri,
                             int tbits, uint64_t *__restrict__ w) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    const uint64_t k = ckey[i];
    const uint32_t vx = compact3(k), vy = compact3(k >> 1), vz = compact3(k >> 2);
    for (int a = 0; a < 8; a++)
        w[8 * i + a] = morton(vx + (a & 1), vy + ((a >> 1) & 1), vz + ((a >> 2) & 1)) << tbits |
                       (uint64_t)(uint32_t)ctri[i];
}

// per-thread digit counts of the 16 keys a thread owns, and their exclusive prefix over the
// block's threads in hist[digit][thread]; block totals in tot[digit]
__device__ void tile_counts(const uint64_t *__restrict__ in, long long n, int shift, unsigned (*hist)[kRT],
                            unsigned *tot) {
    const long long base = (long long)blockIdx.x * kRTile + (long long)threadIdx.x * kRI;
    unsigned c[kDigits];
#pragma unroll
    for (int d = 0; d < kDigits; d++) c[d] = 0;
    for (int q = 0; q < kRI; q++) {
        const long long i = base + q;
        if (i < n) c[(in[i] >> shift) & 15]++;
    }
#pragma unroll
    for (int d = 0; d < kDigits; d++) hist[d][threadIdx.x] = c[d];
    __syncthreads();
    if (threadIdx.x < kDigits) {
        unsigned run = 0;
        for (int t = 0; t < kRT; t++) {
            const unsigned v = hist[threadIdx.x][t];
            hist[threadIdx.x][t] = run;
            run += v;
        }
        tot[threadIdx.x] = run;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kRT) radix_count_kernel(const uint64_t *__restrict__ in, long long n, int shift,
                                                          unsigned *__restrict__ bcount, int nb) {
    __shared__ unsigned hist[kDigits][kRT];
    __shared__ unsigned tot[kDigits];
    tile_counts(in, n, shift, hist, tot);
    if (threadIdx.x < kDigits) bcount[(size_t)threadIdx.x * nb + blockIdx.x] = tot[threadIdx.x];
}

// exclusive scan, in place, of the digit-major block counts (kDigits * nb entries): one block
__global__ void radix_scan_kernel(unsigned *__restrict__ bcount, long long total) {
    __shared__ unsigned long long part[1024];
    const long long per = (total + blockDim.x - 1) / blockDim.x;
    const long long b = threadIdx.x * per, e = min(total, b + per);
    unsigned long long s = 0;
    for (long long i = b; i < e; i++) s += bcount[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int t = 0; t < (int)blockDim.x; t++) { const unsigned long long v = part[t]; part[t] = run; run += v; }
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (long long i = b; i < e; i++) { const unsigned v = bcount[i]; bcount[i] = (unsigned)run; run += v; }
}

// stable scatter: a key goes to its digit's offset for this block, plus the keys of that digit
// in earlier threads of the block, plus those earlier in its own thread
__global__ void __launch_bounds__(kRT) radix_scatter_kernel(const uint64_t *__restrict__ in,
                                                            uint64_t *__restrict__ out, long long n, int shift,
                                                            const unsigned *__restrict__ boff, int nb) {
    __shared__ unsigned hist[kDigits][kRT];
    __shared__ unsigned tot[kDigits];
    tile_counts(in, n, shift, hist, tot);
    unsigned pos[kDigits];
#pragma unroll
    for (int d = 0; d < kDigits; d++) pos[d] = boff[(size_t)d * nb + blockIdx.x] + hist[d][threadIdx.x];
    const long long base = (long long)blockIdx.x * kRTile + (long long)threadIdx.x * kRI;
    for (int q = 0; q < kRI; q++) {
        const long long i = base + q;
        if (i < n) {
            const uint64_t v = in[i];
            const int d = (int)((v >> shift) & 15);
            unsigned p = 0;
#pragma unroll
            for (int dd = 0; dd < kDigits; dd++)
                if (dd == d) p = pos[dd]++;
            out[p] = v;
        }
    }
}

// flags of first occurrences (unique words) and their exclusive prefix, in tiles
__global__ void first_flags_kernel(const uint64_t *__restrict__ w, long long n, unsigned *__restrict__ f) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) f[i] = (i == 0 || w[i] != w[i - 1]) ? 1u : 0u;
}

// block sums of f over tiles of kRTile
__global__ void tile_sum_kernel(const unsigned *__restrict__ f, long long n, unsigned *__restrict__ sums) {
    __shared__ unsigned sh[kRT];
    const long long base = (long long)blockIdx.x * kRTile;
    unsigned s = 0;
    for (int q = threadIdx.x; q < kRTile; q += kRT) {
        const long long i = base + q;
        if (i < n) s += f[i];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kRT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}

// compaction: tile offset (scanned sums) + the flags before i inside the tile, one thread
// per tile row of 16 consecutive entries
__global__ void __launch_bounds__(kRT) compact_kernel(const uint64_t *__restrict__ w, const unsigned *__restrict__ f,
                                                      long long n, const unsigned *__restrict__ toff,
                                                      uint64_t *__restrict__ out) {
    __shared__ unsigned sh[kRT];
    const long long base = (long long)blockIdx.x * kRTile + (long long)threadIdx.x * kRI;
    unsigned c = 0;
    for (int q = 0; q < kRI; q++) if (base + q < n) c += f[base + q];
    sh[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int t = 0; t < kRT; t++) { const unsigned v = sh[t]; sh[t] = run; run += v; }
    }
    __syncthreads();
    unsigned p = toff[blockIdx.x] + sh[threadIdx.x];
    for (int q = 0; q < kRI; q++) {
        const long long i = base + q;
        if (i < n && f[i]) out[p++] = w[i];
    }
}

__device__ bool seg_hits_open_box(const double *a, const double *b, const double *lo, const double *hi) {
    double tmin = -INFINITY, tmax = INFINITY;
    for (int k = 0; k < 3; k++) {
        const double d = b[k] - a[k];
        if (d == 0.0) {
            if (!(a[k] > lo[k] && a[k] < hi[k])) return false;
            continue;
        }
        double t1 = (lo[k] - a[k]) / d, t2 = (hi[k] - a[k]) / d;
        if (t2 < t1) { const double tt = t1; t1 = t2; t2 = tt; }
        tmin = fmax(tmin, t1);
        tmax = fmin(tmax, t2);
    }
    return tmin < tmax && tmin < 1.0 && tmax > 0.0;
}

__device__ bool pt_in_open_box(const double *p, const double *lo, const double *hi) {
    return p[0] > lo[0] && p[0] < hi[0] && p[1] > lo[1] && p[1] < hi[1] && p[2] > lo[2] && p[2] < hi[2];
}

// run g = ct[gs[g] .. gs[g+1]) of one corner (triangles ascending): its component label per
// entry and the run's component count; runs longer than kSmallRun get ncomp = -1 (labelled below)
__global__ void small_runs_kernel(long long ng, const long long *__restrict__ gs, const uint64_t *__restrict__ ct,
                                  int tbits, int split, double s, const int *__restrict__ F,
                                  const double *__restrict__ Vg, const int *__restrict__ adj_ptr,
                                  const int *__restrict__ adj, const int *__restrict__ vt_ptr,
                                  const int *__restrict__ vt, int *__restrict__ comp, int *__restrict__ ncomp) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const long long b = gs[g];
    const int n = (int)(gs[g + 1] - b);
    if (n > kSmallRun) { ncomp[g] = -1; return; }
    const uint64_t tmask = (1ULL << tbits) - 1;
    // parents and labels of the run's positions (at most kSmallRun of them)
    uint8_t par[kSmallRun], lab[kSmallRun];
    for (int i = 0; i < n; i++) { par[i] = (uint8_t)i; lab[i] = 0xff; }
    auto tri = [&](int i) { return (int)(ct[b + i] & tmask); };
    auto local = [&](int t) -> int {   // position of triangle t in the run (triangles ascending), -1 if absent
        int lo = 0, hi = n;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (tri(mid) < t) lo = mid + 1; else hi = mid; }
        return (lo < n && tri(lo) == t) ? lo : -1;
    };
    auto find = [&](int x) { while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; } return x; };
    auto unite = [&](int x, int y) {
        x = find(x); y = find(y);
        if (x != y) { if (x < y) par[y] = (uint8_t)x; else par[x] = (uint8_t)y; }
    };
    if (split) {
        const uint64_t key = ct[b] >> tbits;
        const double c[3] = {(double)compact3(key), (double)compact3(key >> 1), (double)compact3(key >> 2)};
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) { lo[a] = (c[a] - 1.0) * s; hi[a] = (c[a] + 1.0) * s; }
        for (int i = 0; i < n; i++) {
            const int t = tri(i);
            for (int e3 = 0; e3 < 3; e3++) {
                const int va = F[3 * t + e3], vb = F[3 * t + (e3 + 1) % 3];
                bool tested = false, hit = false;
                for (int q = adj_ptr[3 * t + e3]; q < adj_ptr[3 * t + e3 + 1]; q++) {
                    const int j = local(adj[q]);
                    if (j < 0) continue;
                    if (!tested) {
                        hit = seg_hits_open_box(Vg + 3 * (size_t)va, Vg + 3 * (size_t)vb, lo, hi);
                        tested = true;
                    }
                    if (hit) unite(i, j);
                }
            }
            for (int e3 = 0; e3 < 3; e3++) {
                const int v = F[3 * t + e3];
                if (!pt_in_open_box(Vg + 3 * (size_t)v, lo, hi)) continue;
                for (int q = vt_ptr[v]; q < vt_ptr[v + 1]; q++) {
                    const int j = local(vt[q]);
                    if (j >= 0) unite(i, j);
                }
            }
        }
    } else {
        for (int i = 0; i < n; i++) par[i] = 0;
    }
    int nc = 0;
    for (int i = 0; i < n; i++) {
        const int r = find(i);
        if (lab[r] == 0xff) lab[r] = (uint8_t)nc++;
        comp[b + i] = lab[r];
    }
    ncomp[g] = nc;
}

// ---- runs longer than kSmallRun: one thread per (corner, triangle) pair, a shared union-find ----
// Every pair of a long run joins its edge and vertex neighbours in the run, as the thread-per-run
// kernel does, into one parent array over all pairs.  Unions hook the larger root under the smaller
// (compare-and-swap on a root), finds halve paths with plain stores of ancestors; parents only ever
// decrease, so the forest stays acyclic, and every component's root is its smallest position, which
// makes the labels (roots ranked in order) those of the sequential labelling.  Loops are bounded: on
// a bound the status word is set and the host reports a failure.

__device__ int uf_find(int *par, int x, int *status) {
    volatile int *vp = par;
    for (int it = 0; it < (1 << 26); it++) {
        const int p = vp[x];
        if (p == x) return x;
        const int gp = vp[p];
        if (gp != p) vp[x] = gp;
        x = gp;
    }
    atomicExch(status, 1);
    return x;
}

__device__ void uf_union(int *par, int a, int b, int *status) {
    for (int it = 0; it < (1 << 20); it++) {
        a = uf_find(par, a, status);
        b = uf_find(par, b, status);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        if (atomicCAS(par + a, a, b) == a) return;
    }
    atomicExch(status, 1);
}

// run of each pair (-1 when its run was labelled by the thread-per-run kernel); parents initialised
__global__ void long_init_kernel(long long m, long long ng, const long long *__restrict__ gs,
                                 const int *__restrict__ ncomp, int *__restrict__ rid, int *__restrict__ par) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    long long lo = 0, hi = ng;   // the run g with gs[g] <= i < gs[g + 1]
    while (hi - lo > 1) { const long long mid = (lo + hi) >> 1; if (gs[mid] <= i) lo = mid; else hi = mid; }
    rid[i] = ncomp[lo] < 0 ? (int)lo : -1;
    par[i] = (int)i;
}

__global__ void long_union_kernel(long long m, const long long *__restrict__ gs, const uint64_t *__restrict__ ct,
                                  const int *__restrict__ rid, int tbits, int split, double s,
                                  const int *__restrict__ F, const double *__restrict__ Vg,
                                  const int *__restrict__ adj_ptr, const int *__restrict__ adj,
                                  const int *__restrict__ vt_ptr, const int *__restrict__ vt, int *par, int *status) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int g = rid[i];
    if (g < 0) return;
    const long long b = gs[g], e = gs[g + 1];
    if (!split) { uf_union(par, (int)i, (int)b, status); return; }
    const uint64_t tmask = (1ULL << tbits) - 1;
    auto local = [&](int t) -> long long {   // position of triangle t in the run, -1 if absent
        long long lo = b, hi = e;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if ((int)(ct[mid] & tmask) < t) lo = mid + 1; else hi = mid;
        }
        return (lo < e && (int)(ct[lo] & tmask) == t) ? lo : -1;
    };
    const uint64_t key = ct[i] >> tbits;
    const int t = (int)(ct[i] & tmask);
    const double c[3] = {(double)compact3(key), (double)compact3(key >> 1), (double)compact3(key >> 2)};
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) { lo[a] = (c[a] - 1.0) * s; hi[a] = (c[a] + 1.0) * s; }
    for (int e3 = 0; e3 < 3; e3++) {
        const int va = F[3 * t + e3], vb = F[3 * t + (e3 + 1) % 3];
        bool tested = false, hit = false;
        for (int q = adj_ptr[3 * t + e3]; q < adj_ptr[3 * t + e3 + 1]; q++) {
            const long long j = local(adj[q]);
            if (j < 0) continue;
            if (!tested) {
                hit = seg_hits_open_box(Vg + 3 * (size_t)va, Vg + 3 * (size_t)vb, lo, hi);
                tested = true;
            }
            if (hit) uf_union(par, (int)i, (int)j, status);
        }
    }
    for (int e3 = 0; e3 < 3; e3++) {
        const int v = F[3 * t + e3];
        if (!pt_in_open_box(Vg + 3 * (size_t)v, lo, hi)) continue;
        for (int q = vt_ptr[v]; q < vt_ptr[v + 1]; q++) {
            const long long j = local(vt[q]);
            if (j >= 0) uf_union(par, (int)i, (int)j, status);
        }
    }
}

// the flags of the roots of long runs (the forest no longer changes, only paths are halved)
__global__ void long_root_kernel(long long m, const int *__restrict__ rid, int *par, unsigned *__restrict__ flag,
                                 int *status) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    if (rid[i] < 0) { flag[i] = 0u; return; }
    flag[i] = uf_find(par, (int)i, status) == (int)i ? 1u : 0u;
}

// exclusive prefix of the flags: tile offset (scanned tile sums) + the flags before i in the tile
__global__ void __launch_bounds__(kRT) rank_kernel(const unsigned *__restrict__ f, long long n,
                                                   const unsigned *__restrict__ toff, unsigned *__restrict__ rank) {
    __shared__ unsigned sh[kRT];
    const long long base = (long long)blockIdx.x * kRTile + (long long)threadIdx.x * kRI;
    unsigned c = 0;
    for (int q = 0; q < kRI; q++) if (base + q < n) c += f[base + q];
    sh[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int t = 0; t < kRT; t++) { const unsigned v = sh[t]; sh[t] = run; run += v; }
    }
    __syncthreads();
    unsigned p = toff[blockIdx.x] + sh[threadIdx.x];
    for (int q = 0; q < kRI; q++) {
        const long long i = base + q;
        if (i < n) { rank[i] = p; p += f[i]; }
    }
}

// labels of the long runs' pairs (their root's rank within the run) and the runs' component counts;
// the root comes from a find, since concurrent path halving may leave a pair's parent an ancestor below it
__global__ void long_label_kernel(long long m, const long long *__restrict__ gs, const int *__restrict__ rid,
                                  int *par, const unsigned *__restrict__ rank, int *__restrict__ comp, int *status) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int g = rid[i];
    if (g < 0) return;
    comp[i] = (int)(rank[uf_find(par, (int)i, status)] - rank[gs[g]]);
}

__global__ void long_count_kernel(long long ng, long long m, const long long *__restrict__ gs,
                                  const unsigned *__restrict__ rank, unsigned total, int *__restrict__ ncomp) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ng || ncomp[g] >= 0) return;
    const unsigned end = gs[g + 1] < m ? rank[gs[g + 1]] : total;
    ncomp[g] = (int)(end - rank[gs[g]]);
}

template <class T>
cudaError_t balloc(T **p, size_t count) { return cudaMalloc((void **)p, (count ? count : 1) * sizeof(T)); }

}  // namespace

// ---------------------------------------------------------------- host side

struct GpuBasis {
    int *F = nullptr, *adj_ptr = nullptr, *adj = nullptr, *vt_ptr = nullptr, *vt = nullptr;
    double *Vg = nullptr;
};

void gpu_basis_free(GpuBasis *G) {
    if (!G) return;
    void *ptrs[] = {G->F, G->adj_ptr, G->adj, G->vt_ptr, G->vt, G->Vg};
    for (void *q : ptrs) if (q) cudaFree(q);
    delete G;
}

GpuBasis *gpu_basis_setup(const HostHierarchy &H, const std::vector<int32_t> &adj_ptr,
                          const std::vector<int32_t> &adj, const std::vector<int32_t> &vt_ptr,
                          const std::vector<int32_t> &vt, std::string &err) {
    GpuBasis *G = new GpuBasis();
    cudaError_t e = cudaSuccess;
    auto up = [&](auto **dst, const auto &v) {
        if (e != cudaSuccess) return;
        e = balloc(dst, v.size());
        if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice);
    };
    up(&G->F, H.F);
    up(&G->Vg, H.Vg);
    up(&G->adj_ptr, adj_ptr);
    up(&G->adj, adj);
    up(&G->vt_ptr, vt_ptr);
    up(&G->vt, vt);
    if (e != cudaSuccess) {
        err = std::string("GPU labelling: ") + cudaGetErrorString(e);
        cudaGetLastError();
        gpu_basis_free(G);
        return nullptr;
    }
    return G;
}

// sorted unique (corner, triangle) words of the cells; false on a CUDA failure (err set)
bool gpu_corner_pairs(const std::vector<CornerTri> &cells, int tbits, int key_bits, std::vector<uint64_t> &words,
                      std::string &err) {
    const long long nc = (long long)cells.size(), n = 8 * nc;
    uint64_t *ckey = nullptr, *w = nullptr, *w2 = nullptr;
    int *ctri = nullptr;
    unsigned *bc = nullptr, *flags = nullptr, *sums = nullptr;
    std::vector<void *> owned;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    const int nb = (int)((n + kRTile - 1) / kRTile);
    chk(balloc(&ckey, nc)); owned.push_back(ckey);
    chk(balloc(&ctri, nc)); owned.push_back(ctri);
    chk(balloc(&w, n)); owned.push_back(w);
    chk(balloc(&w2, n)); owned.push_back(w2);
    chk(balloc(&bc, (size_t)kDigits * nb)); owned.push_back(bc);
    chk(balloc(&flags, n)); owned.push_back(flags);
    chk(balloc(&sums, nb)); owned.push_back(sums);
    if (e == cudaSuccess) {
        std::vector<uint64_t> hk(nc);
        std::vector<int> ht(nc);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < nc; i++) { hk[i] = cells[i].key; ht[i] = cells[i].tri; }
        chk(cudaMemcpy(ckey, hk.data(), nc * sizeof(uint64_t), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(ctri, ht.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
    }
    long long m = 0;
    if (e == cudaSuccess && n > 0) {
        pairs_kernel<<<(unsigned)((nc + 255) / 256), 256>>>(nc, ckey, ctri, tbits, w);
        const int bits = key_bits + tbits;
        for (int shift = 0; shift < bits; shift += 4) {
            radix_count_kernel<<<nb, kRT>>>(w, n, shift, bc, nb);
            radix_scan_kernel<<<1, 1024>>>(bc, (long long)kDigits * nb);
            radix_scatter_kernel<<<nb, kRT>>>(w, w2, n, shift, bc, nb);
            std::swap(w, w2);
        }
        first_flags_kernel<<<(unsigned)((n + 255) / 256), 256>>>(w, n, flags);
        tile_sum_kernel<<<nb, kRT>>>(flags, n, sums);
        chk(cudaDeviceSynchronize());
        std::vector<unsigned> hs(nb);
        chk(cudaMemcpy(hs.data(), sums, nb * sizeof(unsigned), cudaMemcpyDeviceToHost));
        std::vector<unsigned> toff(nb);
        for (int q = 0; q < nb; q++) { toff[q] = (unsigned)m; m += hs[q]; }
        chk(cudaMemcpy(bc, toff.data(), nb * sizeof(unsigned), cudaMemcpyHostToDevice));
        compact_kernel<<<nb, kRT>>>(w, flags, n, bc, w2);
        chk(cudaDeviceSynchronize());
        words.resize(m);
        chk(cudaMemcpy(words.data(), w2, m * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    }
    for (void *q : owned) if (q) cudaFree(q);
    if (e != cudaSuccess) {
        err = std::string("GPU corner pairs: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return false;
    }
    return true;
}

// component labels of the runs gstart[g] .. gstart[g+1] of the sorted words (ncomp[g] = -1: a
// run left to the host, only when the pairs do not fit 31-bit positions); false on a CUDA failure
bool gpu_run_components(const GpuBasis *G, const std::vector<uint64_t> &words, const std::vector<int64_t> &gstart,
                        int tbits, int split, double s, std::vector<int32_t> &comp, std::vector<int32_t> &ncomp,
                        std::string &err) {
    const long long m = (long long)words.size(), ng = (long long)gstart.size() - 1;
    uint64_t *ct = nullptr;
    long long *gs = nullptr;
    int *dcomp = nullptr, *dn = nullptr;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    chk(balloc(&ct, m));
    chk(balloc(&gs, ng + 1));
    chk(balloc(&dcomp, m));
    chk(balloc(&dn, ng));
    if (e == cudaSuccess) {
        chk(cudaMemcpy(ct, words.data(), m * sizeof(uint64_t), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(gs, gstart.data(), (ng + 1) * sizeof(long long), cudaMemcpyHostToDevice));
        chk(cudaMemset(dcomp, 0, m * sizeof(int)));
    }
    int *rid = nullptr, *par = nullptr, *status = nullptr;
    unsigned *flag = nullptr, *rank = nullptr, *tsum = nullptr;
    int hstatus = 0;
    if (e == cudaSuccess && ng > 0) {
        small_runs_kernel<<<(unsigned)((ng + 127) / 128), 128>>>(ng, gs, ct, tbits, split, s, G->F, G->Vg, G->adj_ptr,
                                                                 G->adj, G->vt_ptr, G->vt, dcomp, dn);
        chk(cudaDeviceSynchronize());
        ncomp.resize(ng);
        chk(cudaMemcpy(ncomp.data(), dn, ng * sizeof(int), cudaMemcpyDeviceToHost));
        bool any_long = false;
        for (long long g = 0; g < ng && e == cudaSuccess; g++) if (ncomp[g] < 0) { any_long = true; break; }
        if (any_long && e == cudaSuccess && m < (long long)INT32_MAX) {
            const int nb = (int)((m + kRTile - 1) / kRTile);
            chk(balloc(&rid, m));
            chk(balloc(&par, m));
            chk(balloc(&flag, m));
            chk(balloc(&rank, m));
            chk(balloc(&tsum, nb));
            chk(balloc(&status, 1));
            if (e == cudaSuccess) chk(cudaMemset(status, 0, sizeof(int)));
            if (e == cudaSuccess) {
                const unsigned bm = (unsigned)((m + 255) / 256);
                long_init_kernel<<<bm, 256>>>(m, ng, gs, dn, rid, par);
                long_union_kernel<<<bm, 256>>>(m, gs, ct, rid, tbits, split, s, G->F, G->Vg, G->adj_ptr, G->adj,
                                               G->vt_ptr, G->vt, par, status);
                long_root_kernel<<<bm, 256>>>(m, rid, par, flag, status);
                tile_sum_kernel<<<nb, kRT>>>(flag, m, tsum);
                chk(cudaDeviceSynchronize());
                std::vector<unsigned> hs(nb), toff(nb);
                chk(cudaMemcpy(hs.data(), tsum, nb * sizeof(unsigned), cudaMemcpyDeviceToHost));
                unsigned total = 0;
                for (int q = 0; q < nb; q++) { toff[q] = total; total += hs[q]; }
                chk(cudaMemcpy(tsum, toff.data(), nb * sizeof(unsigned), cudaMemcpyHostToDevice));
                if (e == cudaSuccess) {
                    rank_kernel<<<nb, kRT>>>(flag, m, tsum, rank);
                    long_label_kernel<<<bm, 256>>>(m, gs, rid, par, rank, dcomp, status);
                    long_count_kernel<<<(unsigned)((ng + 255) / 256), 256>>>(ng, m, gs, rank, total, dn);
                    chk(cudaDeviceSynchronize());
                    chk(cudaMemcpy(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost));
                    chk(cudaMemcpy(ncomp.data(), dn, ng * sizeof(int), cudaMemcpyDeviceToHost));
                }
            }
        }
        comp.resize(m);
        chk(cudaMemcpy(comp.data(), dcomp, m * sizeof(int), cudaMemcpyDeviceToHost));
    }
    void *ptrs[] = {ct, gs, dcomp, dn, rid, par, flag, rank, tsum, status};
    for (void *q : ptrs) if (q) cudaFree(q);
    if (e != cudaSuccess) {
        err = std::string("GPU labelling: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return false;
    }
    if (hstatus != 0) {
        err = "GPU labelling: a union-find loop reached its bound";
        return false;
    }
    return true;
}

}  // namespace lbmg
