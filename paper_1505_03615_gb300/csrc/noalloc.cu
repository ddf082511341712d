// noalloc.cu -- residual norms ||rhs - A_d x||_2 per right-hand side without any
// allocation by the call.
//
// Some callers cannot allocate device memory while they run: a time-critical
// loop cannot afford cudaMalloc's implicit device synchronisation or an
// out-of-memory failure halfway through a step, and a plug-in hosted by an
// application that owns the device memory budget may not grow it.  This entry
// point serves them: the two-pass reduction's partial sums (the only scratch it
// needs) live in one file-scope device array, which every GPU that loads the
// library keeps until the process exits; the caller passes inputs and output.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbmg.h"
#include "lbmg_internal.h"

namespace lbmg {
int noalloc_level(lbmg_handle h, int d, const DevLevel **out);
void noalloc_set_error(const std::string &msg);
}  // namespace lbmg

namespace {

constexpr int kBlocks = 512;                      // partial sums per right-hand side
constexpr int kThreads = 256;
constexpr int kScratchDoubles = kBlocks * 4;       // 16 KiB: 512 blocks x up to 4 right-hand sides

// Shared by every call on this device; a call overwrites all of it before reading.
static __device__ __align__(256) double g_partial[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// r = rhs - A x row by row (8 threads per row), squares summed per block
template <int R>
__global__ void __launch_bounds__(kThreads) residual_partial_kernel(int n, const int *__restrict__ rp,
                                                                    const int *__restrict__ ci,
                                                                    const double *__restrict__ A,
                                                                    const double *__restrict__ rhs,
                                                                    const double *__restrict__ x, int nrhs,
                                                                    double *__restrict__ partial) {
    __shared__ double sh[kThreads / 8][4];
    const int lane = threadIdx.x & 7;
    double sq[R];
#pragma unroll
    for (int q = 0; q < R; q++) sq[q] = 0.0;
    const int groups = gridDim.x * (kThreads / 8);
    const int g0 = blockIdx.x * (kThreads / 8) + (threadIdx.x >> 3);
    // every group of a warp runs the same number of iterations
    const int warp_base = blockIdx.x * (kThreads / 8) + ((threadIdx.x >> 5) << 2);
    for (int base = warp_base; base < n; base += groups) {
        const int row = base + (g0 - warp_base);
        double acc[R];
#pragma unroll
        for (int q = 0; q < R; q++) acc[q] = 0.0;
        if (row < n)
            for (int k = rp[row] + lane; k < rp[row + 1]; k += 8) {
                const double a = A[k];
                const int j = ci[k];
#pragma unroll
                for (int q = 0; q < R; q++)
                    if (q < nrhs) acc[q] = fma(a, x[(size_t)j * nrhs + q], acc[q]);
            }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < R; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o, 8);
        if (row < n && lane == 0)
#pragma unroll
            for (int q = 0; q < R; q++)
                if (q < nrhs) {
                    const double r = rhs[(size_t)row * nrhs + q] - acc[q];
                    sq[q] = fma(r, r, sq[q]);
                }
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; q++) sh[threadIdx.x >> 3][q] = q < R ? sq[q] : 0.0;
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 8; w++) s += sh[w][threadIdx.x];
        partial[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

__global__ void finish_kernel(const double *__restrict__ partial, int nblocks, int nrhs, double *__restrict__ out) {
    __shared__ double sh[kThreads][4];
    for (int q = 0; q < 4; q++) sh[threadIdx.x][q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int q = 0; q < 4; q++) sh[threadIdx.x][q] += partial[b * 4 + q];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 4; q++) sh[threadIdx.x][q] += sh[threadIdx.x + o][q];
        __syncthreads();
    }
    if (threadIdx.x < nrhs) out[threadIdx.x] = sqrt(sh[0][threadIdx.x]);
}

// device (or managed) memory of the current device: the kernels run there, with the handle's
// level arrays, so a buffer on another GPU is refused rather than read across devices
bool on_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeManaged || a.device == dev;
}

// device address of g_partial on the current device, looked up once per device
int scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { lbmg::noalloc_set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return LBMG_CUDA_ERROR; }
    if (dev < 0 || dev >= kMaxDevices) { lbmg::noalloc_set_error("device ordinal beyond the supported range"); return LBMG_INVALID_ARG; }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partial);
        if (e != cudaSuccess || !p) {
            lbmg::noalloc_set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return LBMG_CUDA_ERROR;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return LBMG_OK;
}

}  // namespace

extern "C" int lbmg_residual_norms_noalloc(lbmg_handle h, int d, const double *rhs, const double *x, int nrhs,
                                           double *norms, void *stream) {
    const lbmg::DevLevel *L = nullptr;
    const int lst = lbmg::noalloc_level(h, d, &L);
    if (lst != LBMG_OK) return lst;
    if (!rhs || !x || !norms) {
        lbmg::noalloc_set_error("lbmg_residual_norms_noalloc: null rhs, x or norms");
        return LBMG_INVALID_ARG;
    }
    if (!on_device_ptr(rhs) || !on_device_ptr(x) || !on_device_ptr(norms)) {
        lbmg::noalloc_set_error("lbmg_residual_norms_noalloc: rhs, x and norms must be device memory of the current "
                                "device");
        return LBMG_INVALID_ARG;
    }
    if (nrhs < 1 || nrhs > 4) {
        lbmg::noalloc_set_error("lbmg_residual_norms_noalloc: nrhs must be 1..4 (scratch holds 512 x 4 partial sums)");
        return LBMG_INVALID_ARG;
    }
    double *scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st != LBMG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = kBlocks;   // fixed: every call writes all kBlocks x 4 partial sums
    if (nrhs == 1) residual_partial_kernel<1><<<blocks, kThreads, 0, s>>>(L->n, L->rp, L->ci, L->A64, rhs, x, nrhs, scratch);
    else if (nrhs == 2) residual_partial_kernel<2><<<blocks, kThreads, 0, s>>>(L->n, L->rp, L->ci, L->A64, rhs, x, nrhs, scratch);
    else residual_partial_kernel<4><<<blocks, kThreads, 0, s>>>(L->n, L->rp, L->ci, L->A64, rhs, x, nrhs, scratch);
    finish_kernel<<<1, kThreads, 0, s>>>(scratch, blocks, nrhs, norms);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbmg::noalloc_set_error(std::string("lbmg_residual_norms_noalloc launch: ") + cudaGetErrorString(e));
        return LBMG_CUDA_ERROR;
    }
    return LBMG_OK;
}
