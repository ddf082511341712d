// packed.cu -- packed storage of a level's matrix for the row kernels of the V-cycle
// (coloured Gauss-Seidel colour sweep and residual, Sections 4.3 and 5.2).
//
// On large levels these kernels stream the matrix from HBM.  With four threads per
// row, two things limit plain CSR: a warp's load touches the scattered 16-byte pieces
// of eight rows, and a warp spends many instructions per non-zero on row bounds.  The
// packed copy removes both:
//
//  - The rows of each colour are grouped by their number of quads Q = ceil(len / 4);
//    within one Q, rows keep the level's order (Morton order of their corners, which
//    keeps the x gathers of neighbouring rows close).  Every 8 consecutive rows of one
//    (colour, Q) class form a group, handled by one warp with four lanes per row.
//  - A group stores 32 Q entries: quad q of slot s at base + 32 q + 4 s, so lane
//    4 s + l reads its row's entry 4 q + l at base + 32 q + lane -- one aligned
//    256-byte load per warp and quad, no index arithmetic.  Entries beyond a row's
//    length, and the slots of a class's last group that have no row, are pads
//    (column -1), about 5% of the entries on the seeded meshes.
//  - Per group: (base, Q) and the 8 rows of its slots (-1 for none).
//  - FP32 entries are (column, value bits) pairs, one 8-byte load each; FP64 entries
//    keep columns and values in two arrays with the same order.
// A row's sum runs over the same entries as in CSR, in another order (four lanes,
// each in its own order, then a shuffle reduction).
#include <algorithm>

#include "lbmg_internal.h"

namespace lbmg {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPkPrefetch = 8;   // quads per lane held in registers before the grid-dependency wait
constexpr int kMaxSweepColours = 32;

template <class T> struct PkMat;
template <> struct PkMat<float> {
    const int2 *e;
    __device__ __forceinline__ void get(int64_t k, int &j, float &a) const {
        const int2 v = __ldg(e + k);
        j = v.x;
        a = __int_as_float(v.y);
    }
};
template <> struct PkMat<double> {
    const int *col;
    const double *val;
    __device__ __forceinline__ void get(int64_t k, int &j, double &a) const {
        j = __ldg(col + k);
        a = __ldg(val + k);
    }
};

template <class T, int R>
__device__ __forceinline__ void load_row(const T *p, T (&v)[R]) {
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = p[r];
}
template <>
__device__ __forceinline__ void load_row<float, 4>(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void load_row<double, 2>(const double *p, double (&v)[2]) {
    const double2 q = *reinterpret_cast<const double2 *>(p);
    v[0] = q.x; v[1] = q.y;
}
template <>
__device__ __forceinline__ void load_row<double, 4>(const double *p, double (&v)[4]) {
    const double2 q0 = reinterpret_cast<const double2 *>(p)[0];
    const double2 q1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// One warp per group.  kGs: Gauss-Seidel update x += (b - A x) / A_ii (rows of one
// colour, which never couple); otherwise r = b - A x.  Before the grid-dependency wait
// a warp loads its group, its entries and (kGs) the inverse diagonal; after it, the
// row's own b and x and the x gathers go out together.  x is read with plain loads: a
// colour launch writes x only at rows of its own colour, which it never gathers.
template <class T, int R, bool kGs>
__global__ void __launch_bounds__(512) pk_row_kernel(int g0, int g1, const int2 *__restrict__ gq,
                                                     const int *__restrict__ rows, PkMat<T> m,
                                                     const T *__restrict__ dinv, const T *__restrict__ b, T *x,
                                                     T *__restrict__ r, const char *__restrict__ pf, int64_t pf_bytes,
                                                     int pf_chunk, const PkRuns runs) {
    // the next colour's entries into L2 (static data, so before the grid-dependency wait):
    // one bulk prefetch of a 256-byte-aligned slice per block
    if (pf && threadIdx.x == 0) {
        const int64_t off = (int64_t)blockIdx.x * pf_chunk;
        if (off < pf_bytes) {
            const unsigned len = (unsigned)(pf_bytes - off < pf_chunk ? pf_bytes - off : pf_chunk);
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pf + off), "r"(len) : "memory");
        }
    }
    const int lane = threadIdx.x & 31;
    const int g = g0 + (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (g >= g1) return;   // whole warps only (blockDim is a multiple of 32)
    // the group's position: from the colour's runs (no load; unrolled over constant indices, so the
    // table stays in the parameter bank), else from its header
    int64_t base;
    int Q;
    if (runs.n > 0) {
        int rg = runs.g[0], rb = runs.b[0], rq = runs.q[0];
#pragma unroll
        for (int t = 1; t < kPkRuns; t++) {
            const bool in = t < runs.n && g >= runs.g[t];
            rg = in ? runs.g[t] : rg;
            rb = in ? runs.b[t] : rb;
            rq = in ? runs.q[t] : rq;
        }
        base = ((int64_t)rb + (int64_t)(g - rg) * rq) * 32;
        Q = rq;
    } else {
        const int2 hd = __ldg(gq + g);
        base = (int64_t)(unsigned)hd.x * 32;
        Q = hd.y;
    }
    const int row = __ldg(rows + 8 * (size_t)g + (lane >> 2));
    const bool lead = row >= 0 && (lane & 3) == 0;
    int j[kPkPrefetch];
    T a[kPkPrefetch];
#pragma unroll
    for (int q = 0; q < kPkPrefetch; q++) {
        j[q] = -1;
        a[q] = T(0);
        if (q < Q) m.get(base + 32 * q + lane, j[q], a[q]);
    }
    T d = T(0);
    if (kGs && lead) d = __ldg(dinv + row);
    grid_dep_wait();
    grid_dep_launch();
    T bv[R], xo[R];
    if (lead) {
        load_row<T, R>(b + (size_t)row * R, bv);
        if (kGs) load_row<T, R>(x + (size_t)row * R, xo);
    }
    T acc[R];
#pragma unroll
    for (int c = 0; c < R; c++) acc[c] = T(0);
#pragma unroll
    for (int q = 0; q < kPkPrefetch; q++) {
        if (j[q] >= 0) {
            T xv[R];
            load_row<T, R>(x + (size_t)j[q] * R, xv);
#pragma unroll
            for (int c = 0; c < R; c++) acc[c] = fma(a[q], xv[c], acc[c]);
        }
    }
    for (int q = kPkPrefetch; q < Q; q++) {   // rows of more than 32 entries
        int jj;
        T aa;
        m.get(base + 32 * q + lane, jj, aa);
        if (jj >= 0) {
            T xv[R];
            load_row<T, R>(x + (size_t)jj * R, xv);
#pragma unroll
            for (int c = 0; c < R; c++) acc[c] = fma(aa, xv[c], acc[c]);
        }
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < R; c++) acc[c] += __shfl_xor_sync(kFull, acc[c], o, 4);
    if (lead) {
        if (kGs) {
#pragma unroll
            for (int c = 0; c < R; c++) x[(size_t)row * R + c] = xo[c] + (bv[c] - acc[c]) * d;
        } else {
#pragma unroll
            for (int c = 0; c < R; c++) r[(size_t)row * R + c] = bv[c] - acc[c];
        }
    }
}

__global__ void pk_fill_kernel(int64_t total, const int *__restrict__ map, const int *__restrict__ col,
                               const float *__restrict__ A32, const double *__restrict__ A64, int2 *__restrict__ e32,
                               double *__restrict__ v64, float2 *__restrict__ v2) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= total) return;
    const int src = __ldg(map + k);
    e32[k] = make_int2(__ldg(col + k), src >= 0 ? __float_as_int(__ldg(A32 + src)) : 0);
    const double a = src >= 0 ? __ldg(A64 + src) : 0.0;
    v64[k] = a;
    const float hi = (float)a;
    v2[k] = make_float2(hi, (float)(a - (double)hi));
}

// ---- the mixed solve's outer residual in pairs of FP32 ----
// GB300 executes FP64 at a small fraction of its FP32 rate, so an FP64 residual over the
// finest level is bound by FP64 arithmetic, not by memory.  Here each FP64 value is a pair
// of FP32 numbers (hi + lo) and every product and sum is carried as such a pair:
//   a x = ah xh + (ah xl + al xh + e),  e = fma(ah, xh, -ah xh) the exact rounding error,
// and the running sum (s, c) absorbs each term by Knuth's two-sum.  The dropped al xl and the
// FP32 rounding of the small terms leave about 2^-44 relative to sum |a x|; b - (s + c) is
// formed in FP64.  Same traversal as pk_row_kernel (one warp per 8-row group).
// (the _rn intrinsics keep the compiler from fusing these into FMAs, which would break the
// error-free transformations)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int R>
__device__ __forceinline__ void ld_pair_row(const float *h, const float *l, float (&vh)[R], float (&vl)[R]) {
#pragma unroll
    for (int c = 0; c < R; c++) { vh[c] = h[c]; vl[c] = l[c]; }
}
template <>
__device__ __forceinline__ void ld_pair_row<4>(const float *h, const float *l, float (&vh)[4], float (&vl)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(h), b = *reinterpret_cast<const float4 *>(l);
    vh[0] = a.x; vh[1] = a.y; vh[2] = a.z; vh[3] = a.w;
    vl[0] = b.x; vl[1] = b.y; vl[2] = b.z; vl[3] = b.w;
}

template <int R>
__global__ void __launch_bounds__(256) pk_split_residual_kernel(int g1, const int2 *__restrict__ gq,
                                                                const int *__restrict__ rows,
                                                                const int *__restrict__ col,
                                                                const float2 *__restrict__ v2,
                                                                const double *__restrict__ b,
                                                                const float *__restrict__ xh,
                                                                const float *__restrict__ xl,
                                                                double *__restrict__ r) {
    const int lane = threadIdx.x & 31;
    const int g = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (g >= g1) return;   // whole warps only
    const int2 hd = __ldg(gq + g);
    const int64_t base = (int64_t)(unsigned)hd.x * 32;
    const int Q = hd.y;
    const int row = __ldg(rows + 8 * (size_t)g + (lane >> 2));
    int j[kPkPrefetch];
    float2 a[kPkPrefetch];
#pragma unroll
    for (int q = 0; q < kPkPrefetch; q++) {
        j[q] = -1;
        a[q] = make_float2(0.f, 0.f);
        if (q < Q) {
            j[q] = __ldg(col + base + 32 * q + lane);
            a[q] = __ldg(v2 + base + 32 * q + lane);
        }
    }
    grid_dep_wait();
    grid_dep_launch();
    float sh[R], sl[R];
#pragma unroll
    for (int c = 0; c < R; c++) { sh[c] = 0.f; sl[c] = 0.f; }
    auto term = [&](int jj, float2 aa) {
        float vh[R], vl[R];
        ld_pair_row<R>(xh + (size_t)jj * R, xl + (size_t)jj * R, vh, vl);
#pragma unroll
        for (int c = 0; c < R; c++) {
            const float p = __fmul_rn(aa.x, vh[c]);
            const float t = fmaf(aa.x, vl[c], fmaf(aa.y, vh[c], fmaf(aa.x, vh[c], -p)));
            float s2, e2;
            two_sum(sh[c], p, s2, e2);
            sh[c] = s2;
            sl[c] += e2 + t;
        }
    };
#pragma unroll
    for (int q = 0; q < kPkPrefetch; q++)
        if (j[q] >= 0) term(j[q], a[q]);
    for (int q = kPkPrefetch; q < Q; q++) {   // rows of more than 32 entries
        const int jj = __ldg(col + base + 32 * q + lane);
        if (jj >= 0) term(jj, __ldg(v2 + base + 32 * q + lane));
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < R; c++) {
            const float oh = __shfl_xor_sync(kFull, sh[c], o, 4), ol = __shfl_xor_sync(kFull, sl[c], o, 4);
            float s2, e2;
            two_sum(sh[c], oh, s2, e2);
            sh[c] = s2;
            sl[c] += ol + e2;
        }
    // every lane of the row holds the sums: lane l forms component l in FP64, so a warp issues
    // R FP64 instructions per step instead of 4 R (the FP64 pipe counts warp instructions)
    const int l = lane & 3;
    if (row >= 0 && l < R) {
        float h = sh[0], lo = sl[0];
#pragma unroll
        for (int c = 1; c < R; c++)
            if (l == c) { h = sh[c]; lo = sl[c]; }
        r[(size_t)row * R + l] = b[(size_t)row * R + l] - ((double)h + (double)lo);
    }
}

// x += e on the FP32 pair (xh, xl): two-sum, then renormalise so that |xl| <= ulp(xh) / 2
__global__ void add_pair_kernel(const float *__restrict__ e, float *__restrict__ xh, float *__restrict__ xl,
                                int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    grid_dep_wait();
    grid_dep_launch();
    if (q >= n) return;
    float s, err;
    two_sum(xh[q], e[q], s, err);
    const float t = __fadd_rn(xl[q], err);
    const float h = __fadd_rn(s, t);                   // fast two-sum (|s| >= |t| after a two-sum)
    xh[q] = h;
    xl[q] = __fsub_rn(t, __fsub_rn(h, s));
}

// x = xh + xl in FP64
__global__ void join_kernel(const float *__restrict__ xh, const float *__restrict__ xl, double *__restrict__ x,
                            int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < n) x[q] = (double)xh[q] + (double)xl[q];
}

__global__ void split_kernel(const double *__restrict__ x, float *__restrict__ xh, float *__restrict__ xl, int64_t n) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double v = x[q];
    const float h = (float)v;
    xh[q] = h;
    xl[q] = (float)(v - (double)h);
}

template <class T> PkMat<T> pk_mat(const DevLevel &L);
template <> PkMat<float> pk_mat<float>(const DevLevel &L) { return PkMat<float>{L.pk_e32}; }
template <> PkMat<double> pk_mat<double>(const DevLevel &L) { return PkMat<double>{L.pk_col, L.pk_v64}; }
template <class T> const T *level_A(const DevLevel &L);
template <> const float *level_A<float>(const DevLevel &L) { return L.A32; }
template <> const double *level_A<double>(const DevLevel &L) { return L.A64; }

// pf, pf_bytes: a byte range to prefetch into L2 (null: none), split over the blocks in
// 256-byte-aligned slices
template <class T, bool kGs>
void launch_rows(const DevLevel &L, int g0, int g1, const T *dinv, const T *b, T *x, T *r, int R, int tpb,
                 cudaStream_t s, Chain *ch, const char *pf = nullptr, int64_t pf_bytes = 0,
                 const PkRuns &runs = PkRuns()) {
    if (g1 <= g0) return;
    tpb = std::max(32, std::min(512, tpb / 32 * 32));
    const unsigned blocks = (unsigned)(((int64_t)(g1 - g0) * 32 + tpb - 1) / tpb);
    int chunk = 0;
    if (pf && pf_bytes > 0) {
        const int64_t per = (pf_bytes + blocks - 1) / blocks;
        chunk = (int)std::min<int64_t>((per + 255) / 256 * 256, 1 << 20);
        if ((int64_t)chunk * blocks < pf_bytes) pf = nullptr;   // slices would not cover it: skip
    } else {
        pf = nullptr;
    }
    auto k = R == 1 ? pk_row_kernel<T, 1, kGs> : R == 2 ? pk_row_kernel<T, 2, kGs> : pk_row_kernel<T, 4, kGs>;
    klaunch(k, blocks, (unsigned)tpb, 0, s, ch, g0, g1, (const int2 *)L.pk_gq, (const int *)L.pk_rows, pk_mat<T>(L),
            dinv, b, x, r, pf, pf ? pf_bytes : (int64_t)0, chunk, runs);
}

// ---- the finest level's whole sweep (all its colour steps) in one cooperative launch ----
// The colour launches of a sweep are serialised: each waits for the previous one to drain
// and fills the GPU again.  Here one block per SM walks the colour sequence and the blocks
// meet at a grid barrier between colours; before the barrier every warp loads the header
// and entries of its first group of the next colour, so that after it only the x gathers
// remain.  x is read with L2-only loads (another SM may have written it in the previous
// colour).  The barrier is bounded: after about a second it sets *status and every block
// returns.
struct SweepArgs {
    const int2 *gq;
    const int *rows;
    const int2 *e;
    const float *dinv, *b;
    float *x;
    int gs[9];
    int seq[kMaxSweepColours];
    int nseq;
    unsigned *bar;   // arrival counter, zero at launch
    int *status;
};

__device__ __forceinline__ unsigned sweep_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long sweep_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// barrier k completes when the counter reaches (k + 1) * gridDim.x; false after a timeout
__device__ bool sweep_sync(unsigned *bar, int *status, unsigned target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        const unsigned long long t0 = sweep_timer();
        unsigned long long spins = 0;
        while (sweep_ld_acquire(bar) < target) {
            ++spins;
            if (((spins & 1023) == 0 && sweep_timer() - t0 > 1000000000ull) || spins > (1ull << 28)) {
                atomicExch(status, 1);
                ok = 0;
                break;
            }
            if (*(volatile int *)status != 0) { ok = 0; break; }   // another block gave up
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int R>
__device__ __forceinline__ void ldcg_row(const float *p, float (&v)[R]) {
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = __ldcg(p + r);
}
template <>
__device__ __forceinline__ void ldcg_row<4>(const float *p, float (&v)[4]) {
    const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

// the static part of one group: header, this lane's row and its first kPkPrefetch quads
struct GroupRegs {
    int64_t base;
    int Q, row;
    float d;
    int j[kPkPrefetch];
    float a[kPkPrefetch];
};

__device__ __forceinline__ void load_group(const SweepArgs &p, int g, int lane, GroupRegs &G) {
    const int2 hd = __ldg(p.gq + g);
    G.base = (int64_t)(unsigned)hd.x * 32;
    G.Q = hd.y;
    G.row = __ldg(p.rows + 8 * (size_t)g + (lane >> 2));
    G.d = (G.row >= 0 && (lane & 3) == 0) ? __ldg(p.dinv + G.row) : 0.f;
#pragma unroll
    for (int q = 0; q < kPkPrefetch; q++) {
        G.j[q] = -1;
        G.a[q] = 0.f;
        if (q < G.Q) {
            const int2 v = __ldg(p.e + G.base + 32 * q + lane);
            G.j[q] = v.x;
            G.a[q] = __int_as_float(v.y);
        }
    }
}

template <int R>
__device__ __forceinline__ void relax_group(const SweepArgs &p, int lane, const GroupRegs &G) {
    const bool lead = G.row >= 0 && (lane & 3) == 0;
    float bv[R], xo[R], acc[R];
    if (lead) {
#pragma unroll
        for (int c = 0; c < R; c++) bv[c] = __ldg(p.b + (size_t)G.row * R + c);
        ldcg_row<R>(p.x + (size_t)G.row * R, xo);
    }
#pragma unroll
    for (int c = 0; c < R; c++) acc[c] = 0.f;
#pragma unroll
    for (int q = 0; q < kPkPrefetch; q++) {
        if (G.j[q] >= 0) {
            float xv[R];
            ldcg_row<R>(p.x + (size_t)G.j[q] * R, xv);
#pragma unroll
            for (int c = 0; c < R; c++) acc[c] = fmaf(G.a[q], xv[c], acc[c]);
        }
    }
    for (int q = kPkPrefetch; q < G.Q; q++) {   // rows of more than 32 entries
        const int2 v = __ldg(p.e + G.base + 32 * q + lane);
        if (v.x >= 0) {
            float xv[R];
            ldcg_row<R>(p.x + (size_t)v.x * R, xv);
#pragma unroll
            for (int c = 0; c < R; c++) acc[c] = fmaf(__int_as_float(v.y), xv[c], acc[c]);
        }
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < R; c++) acc[c] += __shfl_xor_sync(kFull, acc[c], o, 4);
    if (lead) {
#pragma unroll
        for (int c = 0; c < R; c++) p.x[(size_t)G.row * R + c] = xo[c] + (bv[c] - acc[c]) * G.d;
    }
}

template <int R>
__global__ void __launch_bounds__(1024, 1) pk_sweep_kernel(SweepArgs p) {
    const int lane = threadIdx.x & 31;
    const int wid = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    GroupRegs G;
    {
        const int c = p.seq[0];
        if (p.gs[c] + wid < p.gs[c + 1]) load_group(p, p.gs[c] + wid, lane, G);
    }
    for (int si = 0; si < p.nseq; si++) {
        const int c = p.seq[si];
        for (int g = p.gs[c] + wid; g < p.gs[c + 1]; g += nw) {
            if (g != p.gs[c] + wid) load_group(p, g, lane, G);
            relax_group<R>(p, lane, G);
        }
        if (si + 1 < p.nseq) {
            const int cn = p.seq[si + 1];
            if (p.gs[cn] + wid < p.gs[cn + 1]) load_group(p, p.gs[cn] + wid, lane, G);
            if (!sweep_sync(p.bar, p.status, (unsigned)(si + 1) * gridDim.x)) return;
        }
    }
}

}  // namespace

bool packed_layout(const HostLevel &hl, std::vector<int32_t> &gq, std::vector<int32_t> &rows,
                   std::vector<int32_t> &map, std::vector<int32_t> &col, int gs[10], int64_t *total) {
    const int n = hl.ndof;
    int rs[10];
    for (int c = 0; c <= 8; c++) rs[c] = hl.colour_start[c];
    rs[9] = n;
    auto quads = [&](int i) { return (int)((hl.rp[i + 1] - hl.rp[i] + 3) / 4); };
    gq.clear();
    rows.clear();
    int64_t base = 0;   // in units of 32 entries
    std::vector<int> order;
    for (int c = 0; c < 9; c++) {
        gs[c] = (int)(gq.size() / 2);
        // rows of the range by quad count, each count in the level's order (a stable counting sort)
        const int r0 = rs[c], r1 = rs[c + 1];
        int qmax = 0;
        for (int i = r0; i < r1; i++) qmax = std::max(qmax, quads(i));
        std::vector<int> cnt(qmax + 2, 0);
        for (int i = r0; i < r1; i++) cnt[quads(i) + 1]++;
        for (int q = 0; q <= qmax; q++) cnt[q + 1] += cnt[q];
        order.assign(r1 - r0, 0);
        for (int i = r0; i < r1; i++) order[cnt[quads(i)]++] = i;
        for (size_t a = 0; a < order.size();) {
            const int q = quads(order[a]);
            size_t e = a;
            while (e < order.size() && e < a + 8 && quads(order[e]) == q) e++;
            gq.push_back((int32_t)base);
            gq.push_back(q);
            for (size_t s = a; s < a + 8; s++) rows.push_back(s < e ? order[s] : -1);
            base += q;
            a = e;
        }
    }
    gs[9] = (int)(gq.size() / 2);
    if (base * 32 >= ((int64_t)1 << 31)) return false;   // 32-bit entry positions in the value map
    *total = base * 32;
    map.assign((size_t)*total, -1);
    col.assign((size_t)*total, -1);
    const int ng = gs[9];
#pragma omp parallel for schedule(dynamic, 1024)
    for (int g = 0; g < ng; g++) {
        const int64_t b0 = (int64_t)gq[2 * g] * 32;
        const int q = gq[2 * g + 1];
        for (int s = 0; s < 8; s++) {
            const int row = rows[8 * (size_t)g + s];
            if (row < 0) continue;
            const int64_t k0 = hl.rp[row], len = hl.rp[row + 1] - k0;
            for (int qq = 0; qq < q; qq++)
                for (int l = 0; l < 4; l++) {
                    const int k = 4 * qq + l;
                    if (k >= len) continue;
                    const int64_t pos = b0 + 32 * qq + 4 * s + l;
                    map[pos] = (int32_t)(k0 + k);
                    col[pos] = hl.ci[k0 + k];
                }
        }
    }
    return true;
}

void launch_packed_fill(const DevLevel &L, cudaStream_t s) {
    if (!L.pk_map || L.pk_total == 0) return;
    pk_fill_kernel<<<(unsigned)((L.pk_total + 255) / 256), 256, 0, s>>>(L.pk_total, L.pk_map, L.pk_col, L.A32, L.A64,
                                                                        L.pk_e32, L.pk_v64, L.pk_v2);
}

bool launch_packed_residual_split(const DevLevel &L, const double *b, const float *xh, const float *xl, double *r,
                                  int R, cudaStream_t s, Chain *ch) {
    if (!L.pk_map || !L.pk_v2) return false;
    const int g1 = L.pk_gs[9];
    if (g1 <= 0) return true;
    const unsigned blocks = (unsigned)(((int64_t)g1 * 32 + 255) / 256);
    auto k = R == 1 ? pk_split_residual_kernel<1> : R == 2 ? pk_split_residual_kernel<2> : pk_split_residual_kernel<4>;
    klaunch(k, blocks, 256u, 0, s, ch, g1, (const int2 *)L.pk_gq, (const int *)L.pk_rows, (const int *)L.pk_col,
            (const float2 *)L.pk_v2, b, xh, xl, r);
    return true;
}

void launch_add_pair(const float *e, float *xh, float *xl, int64_t n, cudaStream_t s, Chain *ch) {
    if (n) klaunch(add_pair_kernel, (unsigned)((n + 255) / 256), 256u, 0, s, ch, e, xh, xl, n);
}

void launch_join(const float *xh, const float *xl, double *x, int64_t n, cudaStream_t s) {
    if (n) join_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xh, xl, x, n);
}

void launch_split(const double *x, float *xh, float *xl, int64_t n, cudaStream_t s) {
    if (n) split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, xh, xl, n);
}

template <class T>
bool launch_packed_smooth(const DevLevel &L, int colour, const T *A, const T *dinv, const T *b, T *x, int R, int tpb,
                          cudaStream_t s, Chain *ch, int next) {
    if (!L.pk_map || A != level_A<T>(L)) return false;
    const char *pf = nullptr;
    int64_t pf_bytes = 0;
    if (sizeof(T) == 4 && next >= 0 && next < 8) {   // FP32 entries: (column, value) pairs
        pf = reinterpret_cast<const char *>(L.pk_e32 + L.pk_es[next]);
        pf_bytes = (L.pk_es[next + 1] - L.pk_es[next]) * (int64_t)sizeof(int2);
    }
    launch_rows<T, true>(L, L.pk_gs[colour], L.pk_gs[colour + 1], dinv, b, x, nullptr, R, tpb, s, ch, pf, pf_bytes,
                         L.pk_runs[colour]);
    return true;
}

template <class T>
bool launch_packed_residual(const DevLevel &L, const T *A, const T *b, const T *x, T *r, int R, int nrows, int tpb,
                            cudaStream_t s, Chain *ch) {
    if (!L.pk_map || A != level_A<T>(L)) return false;
    // the group ranges end exactly at the smoothed rows (ns) and at all rows (n)
    int g1;
    if (nrows == L.n) g1 = L.pk_gs[9];
    else if (nrows == L.ns) g1 = L.pk_gs[8];
    else return false;
    launch_rows<T, false>(L, 0, g1, (const T *)nullptr, b, const_cast<T *>(x), r, R, tpb, s, ch);
    return true;
}

// the whole sweep sequence `seq` (colours, in order) of level L in one cooperative launch;
// false when the level has no packed copy or the launch is refused
bool launch_packed_sweep(const DevLevel &L, const int *seq, int nseq, const float *dinv, const float *b, float *x,
                         int R, unsigned *bar, int *status, int blocks, cudaStream_t s) {
    if (!L.pk_map || nseq < 1 || nseq > kMaxSweepColours || blocks < 1) return false;
    SweepArgs p;
    p.gq = (const int2 *)L.pk_gq;
    p.rows = L.pk_rows;
    p.e = L.pk_e32;
    p.dinv = dinv;
    p.b = b;
    p.x = x;
    for (int q = 0; q < 9; q++) p.gs[q] = L.pk_gs[q];
    for (int q = 0; q < kMaxSweepColours; q++) p.seq[q] = q < nseq ? seq[q] : 0;
    p.nseq = nseq;
    p.bar = bar;
    p.status = status;
    if (cudaMemsetAsync(bar, 0, sizeof(unsigned), s) != cudaSuccess) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(1024);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (R == 1) e = cudaLaunchKernelEx(&cfg, pk_sweep_kernel<1>, p);
    else if (R == 2) e = cudaLaunchKernelEx(&cfg, pk_sweep_kernel<2>, p);
    else e = cudaLaunchKernelEx(&cfg, pk_sweep_kernel<4>, p);
    return e == cudaSuccess;
}

// resident blocks of the sweep kernel (1024 threads) per SM times the SMs: the largest grid a
// cooperative launch accepts
int packed_sweep_blocks(int R) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cudaError_t e = R == 1   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pk_sweep_kernel<1>, 1024, 0)
                    : R == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pk_sweep_kernel<2>, 1024, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pk_sweep_kernel<4>, 1024, 0);
    if (e != cudaSuccess) return 0;
    return per * sms;
}

template bool launch_packed_smooth<float>(const DevLevel &, int, const float *, const float *, const float *, float *,
                                          int, int, cudaStream_t, Chain *, int);
template bool launch_packed_smooth<double>(const DevLevel &, int, const double *, const double *, const double *,
                                           double *, int, int, cudaStream_t, Chain *, int);
template bool launch_packed_residual<float>(const DevLevel &, const float *, const float *, const float *, float *,
                                            int, int, int, cudaStream_t, Chain *);
template bool launch_packed_residual<double>(const DevLevel &, const double *, const double *, const double *,
                                             double *, int, int, int, cudaStream_t, Chain *);

}  // namespace lbmg
