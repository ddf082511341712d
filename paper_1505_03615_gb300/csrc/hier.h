// hier.h -- host-side hierarchy of connectivity-split trilinear B-spline spaces
// (Chuang & Kazhdan, Sections 3.2 and 4), in the layout the CUDA kernels use.
#pragma once
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

namespace lbmg {

constexpr int kMaxDepth = 12;
constexpr double kFragTau = 1e-12;   // pieces of at most this area (finest voxel faces) are ignored
constexpr int kPackShift = 28;       // packed list entry: index | (log2 weight denominator << 28)
constexpr uint32_t kPackMask = (1u << kPackShift) - 1u;
// Galerkin list entry: fine stored-entry index | (log2 weight denominator << 29); the
// exponent is at most 6 (three bits), so the index may reach 2^29 - 1
constexpr int kGalShift = 29;
constexpr uint32_t kGalMask = (1u << kGalShift) - 1u;

// one finest piece of a triangle: its voxel's Morton key, the triangle, the voxel and the
// polygon's vertices in voxel-local coordinates (x, y, z per vertex)
struct FragOut { uint64_t key; int tri; int vox[3]; std::vector<double> poly; };

// Morton keys of grid cells and corners (21 bits per axis), for host and device code alike
#ifdef __CUDACC__
#define LBMG_HD __host__ __device__
#else
#define LBMG_HD
#endif
LBMG_HD inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}
LBMG_HD inline uint64_t morton(int x, int y, int z) {
    return spread3((uint32_t)x) | (spread3((uint32_t)y) << 1) | (spread3((uint32_t)z) << 2);
}
LBMG_HD inline uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ULL;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ULL;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00fULL;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffULL;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffULL;
    x = (x ^ (x >> 32)) & 0x1fffff;
    return (uint32_t)x;
}



struct CornerTri {
    uint64_t key;   // Morton key of a grid corner
    int32_t tri;    // a triangle meeting that corner's support
};

struct HostLevel {
    int d = 0;
    int ndof = 0;
    int ns = 0;                         // rows [0, ns) are smoothed; [ns, ndof) are coarsest-level rows
    int colour_start[9] = {0};          // smoothed rows sorted by corner parity colour 0..7
    int colour_all[9] = {0};            // colour ranges of all rows, kept on a single mesh's coarsest
                                        // level (whose rows are not smoothed unless it is relaxed)
    std::vector<int32_t> coarse;        // coarsest-level blocks: (instance, first row, rows) triples
    std::vector<int32_t> inst;          // [ndof] instance of each row
    std::vector<int32_t> corner;        // [ndof*3] grid corner index at depth d
    std::vector<int32_t> mintri;        // [ndof] smallest triangle of the component
    // (corner Morton key, triangle) pairs, sorted by key then triangle, and the dof of each
    std::vector<CornerTri> ct;
    std::vector<int32_t> ct_dof;
    // sparsity pattern of A_d, columns sorted per row
    std::vector<int32_t> rp, ci;
    // prolongation into this level from depth d-1: parents [ndof*8] (-1 pad), log2 #parents
    std::vector<int32_t> par;
    std::vector<int8_t> npar_log2;
    // as a coarse level: children of each dof, entries fine_dof | (log2 #parents << 28)
    std::vector<int32_t> crp;
    std::vector<uint32_t> cch;
    // as a coarse level: Galerkin contributions per stored entry,
    // entries fine_nnz | ((log2 np_i + log2 np_l) << 28)
    std::vector<int64_t> grp;
    std::vector<uint32_t> gidx;
};

struct HostHierarchy {
    int D = 0, d0 = 0, nv = 0, nt = 0, split = 1;
    int ninst = 1;                                    // meshes in this hierarchy (a batch when > 1)
    // per instance: finest depth, coarsest depth, vertex/triangle/user-row offsets and counts,
    // physical length per finest grid unit, cube side and centre
    std::vector<int32_t> inst_D, inst_d0, inst_voff, inst_toff, inst_uoff, inst_nfine;
    std::vector<double> inst_sigma, inst_S, inst_center;
    std::vector<double> frag_scale;                   // [nfrag] physical area per finest-unit area
    std::vector<int32_t> fperm;                       // user finest index -> row of the finest level
    std::vector<int32_t> seg;                         // finest rows of (colour, instance): [8*ninst][2]
    double S = 0, center[3] = {0, 0, 0}, sigma = 0;   // cube side, centre, physical length per finest unit
    std::vector<double> Vg;                           // vertices in finest-grid units
    std::vector<int32_t> F;
    std::vector<double> tri_normal;                   // unit normals [nt*3]
    std::vector<HostLevel> lev;                       // indexed by depth
    // finest-level fragments, sorted by voxel Morton key then triangle
    int nfrag = 0;
    std::vector<int32_t> frag_tri, frag_vox;          // vox [nfrag*3]
    std::vector<int32_t> frag_pstart;                 // [nfrag+1] into frag_poly (vertices)
    std::vector<double> frag_poly;                    // polygon vertices in voxel-local coordinates [0,1]^3
    std::vector<int32_t> frag_dof;                    // [nfrag*8] dof of each voxel corner (bit a = axis)
    // finest assembly: per stored entry, list of fragment*36 + local pair
    std::vector<int64_t> arp;
    std::vector<uint32_t> aidx;
    // finest right-hand side: per dof, list of fragment*8 + corner
    std::vector<int64_t> rrp;
    std::vector<uint32_t> ridx;
    // vertex evaluation at the finest level: [nv*8] dof (-1 none) and hat value
    std::vector<int32_t> vdof;
    std::vector<double> vw;
};

// Local index of the unordered corner pair (a, b), a <= b, in the 36 upper-triangular pairs.
inline int pair_index(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    return a * 8 - a * (a - 1) / 2 + (b - a);
}

// Concatenate separately built hierarchies into one batch: level depth D - k of
// the batch holds level inst_D - k of every instance that has it.  Smoothed rows
// are ordered by (colour, instance, own order); rows of instances whose coarsest
// level this is follow, instance by instance.  A batch of one keeps the layout.
int combine_batch(std::vector<HostHierarchy> &parts, HostHierarchy &B, std::string &err);

// Returns 0 on success, else an lbmg status code with a message in err.
// fail_alloc (tests): throw std::bad_alloc once the triangles are cut, as an exhausted host
// allocation would.
int build_host_hierarchy(const double *V, int nv, const int *F, int nt, int depth, int min_depth,
                         int coarse_max, int split, int threads, HostHierarchy &H, std::string &err,
                         bool fail_alloc = false, bool gpu_clip = false);

// Row a1 on the GPU (clip.cu): the finest pieces of every triangle of H (H.Vg, H.F, N = 2^depth
// voxels per axis), cut by the same sweep of axis planes as the host builder and kept when their
// area exceeds kFragTau; out gets them unsorted with key = 0.  Returns 0, or an lbmg status
// with a message in err (no device, a failed allocation, or a piece with more vertices than the
// kernel holds, which a triangle clipped by a box cannot have).
int gpu_cut_triangles(const HostHierarchy &H, int N, std::vector<FragOut> &out, std::string &err);

// Row a2 on the GPU (basis.cu): the mesh arrays on the device, the sorted unique (corner,
// triangle) words of a level's cells (morton(corner) << tbits | tri, key_bits bits of corner
// key), and the component labels of the runs of one corner in those words (runs of up to 255
// triangles one thread per run, longer ones one thread per pair with a shared union-find; ncomp =
// -1, labelled by the host, only when a level's pairs exceed 31-bit positions).  A CUDA failure
// throws BuildCudaError.
struct BuildCudaError : std::runtime_error {
    explicit BuildCudaError(const std::string &m) : std::runtime_error(m) {}
};
struct GpuBasis;
GpuBasis *gpu_basis_setup(const HostHierarchy &H, const std::vector<int32_t> &adj_ptr, const std::vector<int32_t> &adj,
                          const std::vector<int32_t> &vt_ptr, const std::vector<int32_t> &vt, std::string &err);
void gpu_basis_free(GpuBasis *G);
bool gpu_corner_pairs(const std::vector<CornerTri> &cells, int tbits, int key_bits, std::vector<uint64_t> &words,
                      std::string &err);
bool gpu_run_components(const GpuBasis *G, const std::vector<uint64_t> &words, const std::vector<int64_t> &gstart,
                        int tbits, int split, double s, std::vector<int32_t> &comp, std::vector<int32_t> &ncomp,
                        std::string &err);

}  // namespace lbmg
