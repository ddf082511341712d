// narrow.cu -- the bottom of the V-cycle (Chuang & Kazhdan, Section 4.3) inside
// one block, out of shared memory.
//
// The coarsest levels are tiny, so each of their ~35 phases per cycle (eight
// colours per Gauss-Seidel sweep, residual, restriction, prolongation) is pure
// latency: as separate launches each costs a launch gap, and even inside one
// block each phase waits on three dependent memory loads.  Here the static data
// of those levels (16-bit row pointers, column indices, children, and parents
// behind per-row offsets, FP32 values and inverse diagonals) are packed once into a
// compact blob, sized with x and b per level and one residual buffer shared by the
// levels to the block's opt-in shared memory; every
// cycle one block pulls the blob into shared memory with TMA bulk copies (issued
// before the kernel waits for its predecessor, so the copy overlaps the previous
// kernel), runs the bottom V-cycle there with block barriers between phases, and
// writes the correction of its top level back.  Four threads share a row, which
// keeps each phase short: a phase is a chain of dependent shared-memory loads.
// Only the dense coarse inverse and the top level's right-hand side and
// correction touch global memory.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lbmg_internal.h"

namespace lbmg {

namespace {

constexpr int kGN = 4;   // threads per matrix row
constexpr unsigned long long kCopyWaitNs = 1000000000ull;   // the blob copy is given up after one second
constexpr int kCopyChunk = 32768;                            // bytes per bulk copy instruction

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// wait for phase `parity` of the barrier, at most `limit` ns; false when it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, unsigned long long limit) {
    const unsigned long long t0 = now_ns();
    while (!mbar_try_wait(mbar, parity))
        if (now_ns() - t0 > limit) return false;
    return true;
}

template <int R>
__device__ __forceinline__ void sld(const float *p, float (&v)[R]) {
#pragma unroll
    for (int q = 0; q < R; q++) v[q] = p[q];
}
template <>
__device__ __forceinline__ void sld<4>(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

template <int R>
__device__ __forceinline__ void sst(float *p, const float (&v)[R]) {
#pragma unroll
    for (int q = 0; q < R; q++) p[q] = v[q];
}
template <>
__device__ __forceinline__ void sst<4>(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

struct SLev {
    const uint16_t *rp, *ci, *par, *crp, *cch;
    const float *A, *dinv;
    const uint16_t *pof;
    float *x, *b, *r;
};

__device__ SLev slev(const NarrowLevel &h, unsigned char *sm) {
    SLev s;
    s.rp = reinterpret_cast<const uint16_t *>(sm + h.o_rp);
    s.ci = reinterpret_cast<const uint16_t *>(sm + h.o_ci);
    s.A = reinterpret_cast<const float *>(sm + h.o_A);
    s.dinv = reinterpret_cast<const float *>(sm + h.o_dinv);
    s.par = h.o_par >= 0 ? reinterpret_cast<const uint16_t *>(sm + h.o_par) : nullptr;
    s.pof = h.o_pof >= 0 ? reinterpret_cast<const uint16_t *>(sm + h.o_pof) : nullptr;
    s.crp = h.o_crp >= 0 ? reinterpret_cast<const uint16_t *>(sm + h.o_crp) : nullptr;
    s.cch = h.o_cch >= 0 ? reinterpret_cast<const uint16_t *>(sm + h.o_cch) : nullptr;
    s.x = reinterpret_cast<float *>(sm + h.o_x);
    s.b = reinterpret_cast<float *>(sm + h.o_b);
    s.r = reinterpret_cast<float *>(sm + h.o_r);
    return s;
}

// row loop with 8-thread groups; every warp runs the same number of iterations
template <int R, class F>
__device__ __forceinline__ void row_groups(int r0, int r1, F &&body) {
    const int tid = threadIdx.x, g = tid / kGN, lane = tid % kGN, ng = blockDim.x / kGN;
    const int warp_first = (tid / 32) * (32 / kGN);
    for (int base = r0 + warp_first; base < r1; base += ng) {
        const int row = base + (g - warp_first);
        body(row, row < r1, lane);
    }
}

// A row's first kGN * kUnroll entries are taken in one predicated, fully unrolled
// step, so their loads are in flight together (a row has about 14 entries, fewer
// than one unrolled block of a runtime-count loop); longer rows finish in a loop.
constexpr int kUnroll = 4;

template <int R>
__device__ __forceinline__ void sdot(const SLev &L, int row, bool active, int lane, float (&acc)[R]) {
#pragma unroll
    for (int q = 0; q < R; q++) acc[q] = 0.f;
    if (active) {
        const int k0 = L.rp[row] + lane, k1 = L.rp[row + 1];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int k = k0 + u * kGN;
            if (k < k1) {
                const float a = L.A[k];
                float v[R];
                sld<R>(L.x + (size_t)L.ci[k] * R, v);
#pragma unroll
                for (int q = 0; q < R; q++) acc[q] = fmaf(a, v[q], acc[q]);
            }
        }
        for (int k = k0 + kUnroll * kGN; k < k1; k += kGN) {
            const float a = L.A[k];
            float v[R];
            sld<R>(L.x + (size_t)L.ci[k] * R, v);
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] = fmaf(a, v[q], acc[q]);
        }
    }
#pragma unroll
    for (int o = kGN / 2; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < R; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o, kGN);
}

// one Gauss-Seidel row update: the row's own inverse diagonal, right-hand side and
// value are loaded before its dot product, so only the update waits for the sum
template <int R>
__device__ __forceinline__ void gs_row(const SLev &L, int row, bool active, int lane) {
    const bool own = active && lane == 0;
    float xo[R], bo[R], dv = 0.f;
    if (own) {
        dv = L.dinv[row];
        sld<R>(L.b + (size_t)row * R, bo);
        sld<R>(L.x + (size_t)row * R, xo);
    }
    float acc[R];
    sdot<R>(L, row, active, lane, acc);
    if (own) {
#pragma unroll
        for (int q = 0; q < R; q++) xo[q] = fmaf(bo[q] - acc[q], dv, xo[q]);
        sst<R>(L.x + (size_t)row * R, xo);
    }
}

template <int R>
__global__ void __launch_bounds__(1024, 1) narrow_smem_kernel(const unsigned char *__restrict__ blob, int blob_bytes,
                                                              int vec_bytes, const NarrowParams pin,
                                                              const float *__restrict__ cinv, const int *__restrict__ cblk,
                                                              const float *__restrict__ b_top, float *__restrict__ x_top,
                                                              int *__restrict__ status, int extra_tx) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) unsigned long long mbar;
    // the level table, read by every phase, from shared memory rather than from
    // dynamically indexed kernel parameters
    __shared__ NarrowParams p;
    for (int q = threadIdx.x; q < (int)(sizeof(NarrowParams) / sizeof(int)); q += blockDim.x)
        reinterpret_cast<int *>(&p)[q] = reinterpret_cast<const int *>(&pin)[q];
    __shared__ int s_ok;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (threadIdx.x == 0) {
        // the blob is static during a solve: its copy starts before this kernel
        // waits for its predecessor
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // extra_tx > 0 only when a test injects bytes that never arrive
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(blob_bytes + extra_tx)
                     : "memory");
        for (int off = 0; off < blob_bytes; off += kCopyChunk) {
            const int bytes = min(kCopyChunk, blob_bytes - off);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    (uint32_t)__cvta_generic_to_shared(sm + off)),
                "l"(blob + off), "r"(bytes), "r"(mb)
                : "memory");
        }
    }
    for (int q = threadIdx.x; q < vec_bytes / 16; q += blockDim.x)
        reinterpret_cast<uint4 *>(sm + blob_bytes)[q] = make_uint4(0, 0, 0, 0);
    // b_top comes from the kernel before this one
    grid_dep_wait();
    grid_dep_launch();
    if (threadIdx.x == 0) {
        int ok = mbar_wait_bounded(mb, 0, kCopyWaitNs) ? 1 : 0;
        if (!ok) {
            // report, then give the copies in flight one more bounded wait before leaving
            atomicExch(status, 1);
            mbar_wait_bounded(mb, 0, kCopyWaitNs);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    // every thread observes the completed phase, which makes the copied bytes visible to it
    mbar_wait_bounded(mb, 0, kCopyWaitNs);
    const NarrowLevel &T = p.lev[p.dn - p.d0];
    {
        float *b = reinterpret_cast<float *>(sm + T.o_b);
        for (int q = threadIdx.x; q < T.n * R; q += blockDim.x) b[q] = b_top[q];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int d = p.dn; d >= p.d0; d--) {
        const NarrowLevel &H = p.lev[d - p.d0];
        const SLev L = slev(H, sm);
        // dense coarse blocks of this level: x = inv b
        for (int k = 0; k < H.ncb; k++) {
            const int *cb = cblk + 5 * (H.cb0 + k);
            const int row0 = cb[2], n = cb[3];
            const float *M = cinv + cb[4];
            // four rows per warp at a time, so that a warp keeps 4 x 4 loads of the inverse in flight
            for (int rb = warp; rb < n; rb += 4 * nw) {
                float acc[4][R];
#pragma unroll
                for (int u = 0; u < 4; u++)
#pragma unroll
                    for (int q = 0; q < R; q++) acc[u][q] = 0.f;
#pragma unroll 2
                for (int j = wl; j < n; j += 32) {
                    float v[R];
                    sld<R>(L.b + (size_t)(row0 + j) * R, v);
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int row = rb + u * nw;
                        if (row < n) {
                            const float a = __ldg(M + (size_t)row * n + j);
#pragma unroll
                            for (int q = 0; q < R; q++) acc[u][q] = fmaf(a, v[q], acc[u][q]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int q = 0; q < R; q++) acc[u][q] += __shfl_xor_sync(0xffffffffu, acc[u][q], o);
                    const int row = rb + u * nw;
                    if (wl == 0 && row < n) sst<R>(L.x + (size_t)(row0 + row) * R, acc[u]);
                }
            }
        }
        __syncthreads();
        if (d == p.d0) break;
        for (int s = 0; s < p.nu1; s++)
            for (int c = 0; c < 8; c++) {
                row_groups<R>(H.cs[c], H.cs[c + 1],
                              [&](int row, bool active, int lane) { gs_row<R>(L, row, active, lane); });
                __syncthreads();
            }
        row_groups<R>(0, H.ns, [&](int row, bool active, int lane) {
            float acc[R];
            sdot<R>(L, row, active, lane, acc);
            if (active && lane == 0)
#pragma unroll
                for (int q = 0; q < R; q++) L.r[(size_t)row * R + q] = L.b[(size_t)row * R + q] - acc[q];
        });
        __syncthreads();
        const NarrowLevel &HC = p.lev[d - 1 - p.d0];
        const SLev C = slev(HC, sm);
        for (int J = threadIdx.x; J < HC.n; J += blockDim.x) {
            float acc[R];
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] = 0.f;
            const int k0 = C.crp[J], k1 = C.crp[J + 1];
            auto child = [&](int k) {
                const uint16_t e = C.cch[k];
                const float w = 1.f / (float)(1u << (e >> 14));
                float v[R];
                sld<R>(L.r + (size_t)(e & 0x3fff) * R, v);
#pragma unroll
                for (int q = 0; q < R; q++) acc[q] = fmaf(w, v[q], acc[q]);
            };
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (k0 + u < k1) child(k0 + u);
            for (int k = k0 + 8; k < k1; k++) child(k);
#pragma unroll
            for (int q = 0; q < R; q++) { C.b[(size_t)J * R + q] = acc[q]; C.x[(size_t)J * R + q] = 0.f; }
        }
        __syncthreads();
    }
    for (int d = p.d0 + 1; d <= p.dn; d++) {
        const NarrowLevel &H = p.lev[d - p.d0];
        const SLev L = slev(H, sm), C = slev(p.lev[d - 1 - p.d0], sm);
        for (int i = threadIdx.x; i < H.ns; i += blockDim.x) {
            const int k0 = L.pof[i], np = L.pof[i + 1] - k0;
            float acc[R], v[R];
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] = 0.f;
#pragma unroll
            for (int q2 = 0; q2 < 8; q2++) {
                if (q2 < np) {
                    sld<R>(C.x + (size_t)L.par[k0 + q2] * R, v);
#pragma unroll
                    for (int q = 0; q < R; q++) acc[q] += v[q];
                }
            }
            const float w = 1.f / (float)np;
#pragma unroll
            for (int q = 0; q < R; q++) L.x[(size_t)i * R + q] += w * acc[q];
        }
        __syncthreads();
        for (int s = 0; s < p.nu2; s++)
            for (int c = 7; c >= 0; c--) {
                row_groups<R>(H.cs[c], H.cs[c + 1],
                              [&](int row, bool active, int lane) { gs_row<R>(L, row, active, lane); });
                __syncthreads();
            }
    }
    {
        const float *x = reinterpret_cast<const float *>(sm + T.o_x);
        for (int q = threadIdx.x; q < T.n * R; q += blockDim.x) x_top[q] = x[q];
    }
}

}  // namespace

// Pick the bottom levels that fit in shared memory and pack their static data.
// Returns 0 and leaves c.narrow.dn = d0 - 1 when no level fits.
int narrow_smem_setup(Ctx &c, size_t smem_budget) {
    NarrowParams &p = c.narrow.p;
    c.narrow.dn = c.d0 - 1;
    const HostHierarchy &H = c.host;
    auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    size_t best_blob = 0, best_vec = 0;
    int best_dn = c.d0 - 1;
    for (int dn = c.d0; dn <= c.D && dn - c.d0 < kMaxNarrow; dn++) {
        size_t blob = 0, vec = 0, rmax = 0;
        bool ok = true;
        for (int d = c.d0; d <= dn && ok; d++) {
            const HostLevel &L = H.lev[d];
            const size_t nnz = L.rp.empty() ? 0 : (size_t)L.rp[L.ndof];
            if (nnz >= 65535 || L.ndof >= 16384) { ok = false; break; }
            blob += align16(2 * (L.ndof + 1)) + align16(2 * nnz) + align16(4 * nnz) + align16(4 * (size_t)L.ndof);
            if (d > c.d0) {
                size_t np = 0;
                for (int i = 0; i < L.ndof; i++) np += (size_t)1 << L.npar_log2[i];
                if (np >= 65535) ok = false;
                blob += align16(2 * (L.ndof + 1)) + align16(2 * np);
            }
            if (d < dn) blob += align16(2 * (L.ndof + 1)) + align16(2 * L.cch.size());
            if (d < dn && L.cch.size() >= 65535) ok = false;
            vec += 2 * align16(16 * (size_t)L.ndof);   // x, b with room for 4 lanes
            rmax = std::max(rmax, align16(16 * (size_t)L.ndof));
        }
        vec += rmax;   // one residual buffer for all levels
        if (!ok || blob + vec > smem_budget) break;
        best_dn = dn; best_blob = blob; best_vec = vec;
    }
    if (best_dn < c.d0) return 0;
    // pack
    std::vector<unsigned char> buf(best_blob, 0);
    size_t off = 0, voff = best_blob;
    auto put = [&](const void *src, size_t bytes) {
        const size_t o = off;
        if (bytes) std::memcpy(buf.data() + o, src, bytes);
        off += align16(bytes);
        return (int)o;
    };
    p.d0 = c.d0; p.dn = best_dn; p.nu1 = c.nu1; p.nu2 = c.nu2;
    for (int d = c.d0; d <= best_dn; d++) {
        const HostLevel &L = H.lev[d];
        NarrowLevel &o = p.lev[d - c.d0];
        o = NarrowLevel();
        o.n = L.ndof; o.ns = L.ns;
        for (int q = 0; q < 9; q++) o.cs[q] = L.colour_start[q];
        o.cb0 = c.lev[d].cb0; o.ncb = c.lev[d].ncb;
        const size_t nnz = (size_t)L.rp[L.ndof];
        std::vector<uint16_t> rp16(L.ndof + 1), ci16(nnz);
        for (int i = 0; i <= L.ndof; i++) rp16[i] = (uint16_t)L.rp[i];
        for (size_t k = 0; k < nnz; k++) ci16[k] = (uint16_t)L.ci[k];
        o.o_rp = put(rp16.data(), 2 * rp16.size());
        o.o_ci = put(ci16.data(), 2 * nnz);
        o.o_A = (int)off; off += align16(4 * nnz);            // values: refreshed after every assembly
        o.o_dinv = (int)off; off += align16(4 * (size_t)L.ndof);
        o.nnz = (int)nnz;
        o.o_par = o.o_pof = o.o_crp = o.o_cch = -1;
        if (d > c.d0) {
            // the first 1 << npar_log2 of a row's 8 parent slots are its parents
            std::vector<uint16_t> pof16(L.ndof + 1), par16;
            for (int i = 0; i < L.ndof; i++) {
                pof16[i] = (uint16_t)par16.size();
                for (int q = 0; q < (1 << L.npar_log2[i]); q++) {
                    if (L.par[8 * (size_t)i + q] < 0) return 1;
                    par16.push_back((uint16_t)L.par[8 * (size_t)i + q]);
                }
            }
            pof16[L.ndof] = (uint16_t)par16.size();
            o.o_pof = put(pof16.data(), 2 * pof16.size());
            o.o_par = put(par16.data(), 2 * par16.size());
        }
        if (d < best_dn) {
            std::vector<uint16_t> crp16(L.ndof + 1), cch16(L.cch.size());
            for (int i = 0; i <= L.ndof; i++) crp16[i] = (uint16_t)L.crp[i];
            for (size_t k = 0; k < L.cch.size(); k++) {
                const uint32_t e = L.cch[k];
                cch16[k] = (uint16_t)((e & kPackMask) | ((e >> kPackShift) << 14));
            }
            o.o_crp = put(crp16.data(), 2 * crp16.size());
            o.o_cch = put(cch16.data(), 2 * cch16.size());
        }
        o.o_x = (int)voff; voff += align16(16 * (size_t)L.ndof);
        o.o_b = (int)voff; voff += align16(16 * (size_t)L.ndof);
    }
    for (int d = c.d0; d <= best_dn; d++) p.lev[d - c.d0].o_r = (int)voff;   // the shared residual buffer
    if (off != best_blob) return 1;
    if (cudaMalloc((void **)&c.narrow.blob, best_blob) != cudaSuccess) { cudaGetLastError(); c.narrow.blob = nullptr; return 1; }

    if (cudaMemcpy(c.narrow.blob, buf.data(), best_blob, cudaMemcpyHostToDevice) != cudaSuccess) return 1;
    c.narrow.blob_bytes = (int)best_blob;
    c.narrow.vec_bytes = (int)best_vec;
    // the limit is a property of the kernel, shared by every handle of the process: only ever raised,
    // so that a handle set up later with a smaller bottom does not lower it below this one's
    for (auto *k : {(const void *)narrow_smem_kernel<1>, (const void *)narrow_smem_kernel<2>, (const void *)narrow_smem_kernel<4>}) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 1;
        if (fa.maxDynamicSharedSizeBytes < (int)(best_blob + best_vec) &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(best_blob + best_vec)) != cudaSuccess)
            return 1;
    }
    c.narrow.dn = best_dn;
    return 0;
}

size_t narrow_smem_budget() {
    // the opt-in limit per block, less the kernel's static shared memory (its level table)
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, narrow_smem_kernel<4>) != cudaSuccess || optin <= (int)fa.sharedSizeBytes) {
        cudaGetLastError();
        return 200 * 1024;
    }
    return (size_t)optin - fa.sharedSizeBytes;
}

// copy the current FP32 values and inverse diagonals of the narrow levels into the blob
void narrow_smem_refresh(const Ctx &c, cudaStream_t s) {
    if (c.narrow.dn < c.d0) return;
    for (int d = c.d0; d <= c.narrow.dn; d++) {
        const NarrowLevel &o = c.narrow.p.lev[d - c.d0];
        cudaMemcpyAsync(c.narrow.blob + o.o_A, c.lev[d].A32, 4 * (size_t)o.nnz, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(c.narrow.blob + o.o_dinv, c.lev[d].dinv32, 4 * (size_t)o.n, cudaMemcpyDeviceToDevice, s);
    }
}

void launch_narrow_smem(const Ctx &c, int R, cudaStream_t s, Chain *ch) {
    const DevLevel &T = c.lev[c.narrow.dn];
    const int smem = c.narrow.blob_bytes + c.narrow.vec_bytes;
    auto k = R == 1 ? narrow_smem_kernel<1> : R == 2 ? narrow_smem_kernel<2> : narrow_smem_kernel<4>;
    klaunch(k, 1u, 1024u, (size_t)smem, s, ch, (const unsigned char *)c.narrow.blob, c.narrow.blob_bytes,
            c.narrow.vec_bytes, c.narrow.p, (const float *)c.cinv32, (const int *)c.cblk, (const float *)T.b32,
            T.x32, c.narrow.status, c.copy_phantoms);
}

}  // namespace lbmg
