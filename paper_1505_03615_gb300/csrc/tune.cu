// tune.cu -- launch-shape autotuner for the row-parallel kernels of the V-cycle
// (the coloured Gauss-Seidel sweep of Sections 4.3 and 5.2 and the residual).
//
// How many threads share a matrix row and how many threads form a block decide
// how well a level's rows fill the 152 SMs and how long the shuffle reduction of
// a row is; the best pair depends on the level's row count and row length.  For
// each level and kernel the tuner captures a graph of the kernel exactly as the
// V-cycle launches it (a chain of dependent launches, `reps` sweeps), replays it,
// and keeps the fastest shape.  Results go into a process-wide cache keyed by
// (device name, precision, kernel, lanes, rows, non-zeros), which can be saved to
// and loaded from a text file.
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "lbmg_internal.h"

namespace lbmg {

namespace {

using Key = std::tuple<std::string, int, int, int, int64_t, int64_t>;   // device, fp64, kind, R, rows, nnz
std::map<Key, LaunchShape> g_cache;
std::mutex g_mu;

constexpr int kTpr[3] = {4, 8, 16};
constexpr int kTpb[3] = {128, 256, 512};

std::string device_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    std::string s = p.name;
    for (char &ch : s)
        if (ch == ' ' || ch == '\t') ch = '_';
    return s;
}

template <class T> struct V;
template <> struct V<float> {
    static const float *A(const DevLevel &L) { return L.A32; }
    static const float *dinv(const DevLevel &L) { return L.dinv32; }
    static float *x(DevLevel &L) { return L.x32; }
    static float *b(DevLevel &L) { return L.b32; }
    static float *r(DevLevel &L) { return L.r32; }
};
template <> struct V<double> {
    static const double *A(const DevLevel &L) { return L.A64; }
    static const double *dinv(const DevLevel &L) { return L.dinv64; }
    static double *x(DevLevel &L) { return L.x64; }
    static double *b(DevLevel &L) { return L.b64; }
    static double *r(DevLevel &L) { return L.r64; }
};

// device time of one sweep (8 colours) or one residual with the level's current shape
template <class T>
cudaError_t time_kernel(Ctx &c, DevLevel &L, int kind, int R, int reps, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    cudaStream_t cs = c.capture_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    Chain ch;
    ch.on = c.pdl != 0;   // the capture stream is an ordinary stream
    for (int q = 0; q < reps; q++) {
        if (kind == kShapeSmooth) {
            launch_sweeps<T>(c, L, 1, true, V<T>::A(L), V<T>::dinv(L), V<T>::b(L), V<T>::x(L), R, cs, &ch);
        } else {
            launch_residual<T>(L, V<T>::A(L), V<T>::b(L), V<T>::x(L), V<T>::r(L), R, cs, L.ns, &ch);
        }
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) return e;
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    constexpr int kReplays = 3;
    e = cudaGraphLaunch(x, cs);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
    for (int q = 0; q < kReplays && e == cudaSuccess; q++) e = cudaGraphLaunch(x, cs);
    if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaGraphExecDestroy(x);
    *ms /= (float)(kReplays * reps);
    return e;
}

template <class T>
cudaError_t tune_levels(Ctx &c, int R, int reps, int *timed) {
    const std::string dev = device_name();
    const int fp64 = sizeof(T) == 8;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int d = c.d0 + 1; d <= c.D && e == cudaSuccess; d++) {
        DevLevel &L = c.lev[d];
        if (L.ns == 0) continue;
        const size_t bytes = (size_t)L.n * 4 * sizeof(T);
        e = cudaMemsetAsync(V<T>::x(L), 0, bytes, c.capture_stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(V<T>::b(L), 0, bytes, c.capture_stream);
        for (int kind = 0; kind < 2 && e == cudaSuccess; kind++) {
            const Key key{dev, fp64, kind, R, (int64_t)L.ns, L.nnz};
            {
                std::lock_guard<std::mutex> lk(g_mu);
                auto it = g_cache.find(key);
                if (it != g_cache.end()) {
                    L.shape[fp64][kind] = it->second;
                    L.tuned_ms[fp64][kind] = 0.f;
                    continue;
                }
            }
            LaunchShape best = LaunchShape(), dflt = LaunchShape();
            float best_ms = 0.f, dflt_ms = 0.f;
            bool have = false;
            for (int a = 0; a < 3 && e == cudaSuccess; a++)
                for (int b = 0; b < 3 && e == cudaSuccess; b++) {
                    LaunchShape sh;
                    sh.tpr = kTpr[a];
                    sh.tpb = kTpb[b];
                    L.shape[fp64][kind] = sh;
                    float ms = 0.f;
                    e = time_kernel<T>(c, L, kind, R, reps, e0, e1, &ms);
                    if (e != cudaSuccess) break;
                    if (sh.tpr == dflt.tpr && sh.tpb == dflt.tpb) dflt_ms = ms;
                    if (!have || ms < best_ms) { best = sh; best_ms = ms; have = true; }
                }
            if (e != cudaSuccess) { L.shape[fp64][kind] = dflt; break; }
            // keep the default unless another shape is clearly faster (timing noise)
            if (dflt_ms > 0.f && best_ms > 0.98f * dflt_ms) { best = dflt; best_ms = dflt_ms; }
            // FP32 sweeps of a level with a packed copy: the whole-sweep cooperative kernel, kept when it
            // beats the colour launches by 2% (a refused launch or capture just leaves it out)
            // (grids of all SMs down to an eighth of them: on small levels fewer blocks make the grid
            // barrier between colours cheaper)
            if (kind == kShapeSmooth && !fp64 && L.pk_map && c.sweep_bar && c.sweep_blocks[R] > 0) {
                for (int div = 1; div <= 8; div *= 2) {
                    LaunchShape sw;
                    sw.tpr = 4;
                    sw.tpb = kSweepShapeTpb;
                    sw.grid = div == 1 ? 0 : std::max(1, c.sweep_blocks[R] / div);
                    L.shape[fp64][kind] = sw;
                    float ms = 0.f;
                    const cudaError_t es = time_kernel<T>(c, L, kind, R, reps, e0, e1, &ms);
                    if (es == cudaSuccess && ms > 0.f && ms < 0.98f * best_ms) { best = sw; best_ms = ms; }
                    if (es != cudaSuccess) {
                        cudaGetLastError();
                        cudaStreamSynchronize(c.capture_stream);
                        break;
                    }
                }
            }
            L.shape[fp64][kind] = best;
            L.tuned_ms[fp64][kind] = best_ms;
            {
                std::lock_guard<std::mutex> lk(g_mu);
                g_cache[key] = best;
            }
            if (timed) (*timed)++;
        }
        // the level vectors are scratch of the cycle: leave them zero
        if (e == cudaSuccess) e = cudaMemsetAsync(V<T>::x(L), 0, bytes, c.capture_stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(V<T>::r(L), 0, bytes, c.capture_stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.capture_stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

int autotune(Ctx &c, int R, int precision, int reps, cudaStream_t s, int *timed) {
    if (timed) *timed = 0;
    // the tuner runs on the handle's capture stream, after the caller's work
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.capture_stream, ev, 0);
    if (ev) cudaEventDestroy(ev);
    if (e == cudaSuccess) e = precision == 0 ? tune_levels<double>(c, R, reps, timed) : tune_levels<float>(c, R, reps, timed);
    return (int)e;
}

int tune_cache_save(const char *path) {
    FILE *f = std::fopen(path, "w");
    if (!f) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    std::fprintf(f, "# device fp64 kind lanes rows nnz threads_per_row threads_per_block [sweep_grid]\n");
    for (const auto &kv : g_cache) {
        const Key &k = kv.first;
        std::fprintf(f, "%s %d %d %d %lld %lld %d %d %d\n", std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k),
                     std::get<3>(k), (long long)std::get<4>(k), (long long)std::get<5>(k), kv.second.tpr,
                     kv.second.tpb, kv.second.grid);
    }
    return std::fclose(f) == 0 ? 0 : 1;
}

int tune_cache_load(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return 1;
    char line[512], name[256];
    int bad = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int fp64, kind, R, tpr, tpb, grid = 0;
        long long n, nnz;
        const int got = std::sscanf(line, "%255s %d %d %d %lld %lld %d %d %d", name, &fp64, &kind, &R, &n, &nnz, &tpr,
                                    &tpb, &grid);
        if ((got != 8 && got != 9) || grid < 0 ||
            (fp64 != 0 && fp64 != 1) || (kind != 0 && kind != 1) || (tpr != 4 && tpr != 8 && tpr != 16) ||
            tpb < 32 || (tpb > 512 && !(tpb == kSweepShapeTpb && tpr == 4 && kind == kShapeSmooth)) || tpb % 32 != 0) {
            bad = 1;
            continue;
        }
        LaunchShape sh;
        sh.tpr = tpr;
        sh.tpb = tpb;
        sh.grid = tpb == kSweepShapeTpb ? grid : 0;
        g_cache[Key{std::string(name), fp64, kind, R, (int64_t)n, (int64_t)nnz}] = sh;
    }
    std::fclose(f);
    return bad;
}

}  // namespace lbmg
