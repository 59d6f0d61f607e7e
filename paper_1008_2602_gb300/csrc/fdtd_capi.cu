// fdtd_capi.cu -- the C-ABI of libfdtd.so (declared in include/fdtd.h).
//
// Host side of the CUDA path: validates the problem, precomputes what the
// kernels read (per-edge permittivity -> <=256-entry coefficient table +
// uint8 id per node, Eq. 5 grading -> 1D UPML factors per axis, Eq. 7 time
// step, slab decomposition of the UPML), owns device memory, captures chunks
// of steps into CUDA graphs and batches boards into one launch per phase.
#include <nvtx3/nvToolsExt.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <climits>
#include <memory>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "../../include/fdtd.h"
#include "fdtd_internal.h"

using namespace fdtd;

namespace {

const double kC0 = 299792458.0;
const double kMu0 = 4.0e-7 * 3.14159265358979323846;
const double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
const double kEta0 = kMu0 * kC0;

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return FDTD_ECUDA;
}

#define CK(call)                                           \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

int elem_size(int prec) { return prec == FDTD_FP32 ? 4 : 2; }

}  // namespace

int fdtd::set_error(int code, const char *msg)
{
    g_err = msg ? msg : "";
    return code;
}

struct fdtd_batch;

struct fdtd_ctx {
    // problem
    fdtd_grid g{};
    fdtd_boundary bnd{};
    std::vector<double> eps;
    std::vector<fdtd_box> boxes;
    std::vector<uint8_t> mask;
    int prec = FDTD_FP32;
    int device = 0;             // CUDA device the context's memory lives on
    double dt = 0.0;
    // host mirror of the device descriptor
    Board h{};
    Board *d = nullptr;
    std::vector<void *> allocs;
    std::vector<Source> src;
    std::vector<Probe> probe;
    std::vector<float4> ctab;
    int n_combo = 0;
    long long device_bytes = 0;
    bool started = false;       // first step queued: sources/probes/scale frozen
    bool own_stream = false;
    cudaStream_t stream = nullptr;
    cudaStream_t cur = nullptr; // stream work is queued on (batch stream while batched)
    long long host_step = 0;
    fdtd_batch *batch = nullptr;
    // single-board plan and graph
    fdtd_tuning tune{62, 8, 10, 16, 1, 38};
    bool plan_dirty = true;
    Plan plan{};
    long long *plan_buf = nullptr;   // device [0]=board ptr, then prefixes
    size_t plan_cap = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    cudaGraphExec_t graph2 = nullptr;   // pairs of steps (depth 2)
    int graph2_chunk = 0;
    size_t fbytes = 0;                  // bytes of one field component
    double *energy_buf = nullptr;    // partials + 2 outputs
    int energy_n = 0;
    int grid_cap = 0;
    std::vector<cudaEvent_t> events; // fdtd_step_profiled
    size_t zaux_n[2] = {0, 0};       // elements per fused-region z-UPML auxiliary array
    long long zplanes[2] = {0, 0};   // planes of the two z-UPML boxes
    CUtensorMap *tm_dev = nullptr;   // kNumMaps descriptors in device memory
};

struct fdtd_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<fdtd_ctx *> members;
    std::vector<long long> remaining;
    fdtd_tuning tune{62, 8, 10, 16, 1, 38};
    bool dirty = true;
    Plan plan{};
    long long *plan_buf = nullptr;
    size_t plan_cap = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    int prec = -1;
    int grid_cap = 0;
};

namespace {

int device_grid_cap()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1024;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 1024;
    return sms * 8;
}

template <typename P>
int dalloc(fdtd_ctx *c, P **out, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FDTD_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    c->allocs.push_back(p);
    c->device_bytes += (long long)bytes;
    *out = (P *)p;
    return FDTD_OK;
}

// Eq. 5 grading and the D/B recurrence factors at position x (cells) of an
// axis with N cells, UPML depths dlo / dhi, cell size d.
Coef upml_coef(double x, int N, int dlo, int dhi, double d, double m, double R0, double kmax, double dt)
{
    double rho = 0.0;
    int depth = 0;
    if (dlo > 0 && x < dlo) {
        rho = (dlo - x) / dlo;
        depth = dlo;
    } else if (dhi > 0 && x > N - dhi) {
        rho = (x - (N - dhi)) / dhi;
        depth = dhi;
    }
    double sigma = 0.0, kappa = 1.0;
    if (depth > 0) {
        const double smax = -(m + 1.0) * std::log(R0) / (2.0 * kEta0 * depth * d);
        const double r = std::pow(rho, m);
        sigma = smax * r;
        kappa = 1.0 + (kmax - 1.0) * r;
    }
    const double q = sigma * dt / (2.0 * kEps0);
    Coef c;
    c.b1 = (float)((kappa - q) / (kappa + q));
    c.g = (float)(1.0 / (kappa + q));
    c.ap = (float)(kappa + q);
    c.am = (float)(kappa - q);
    return c;
}

bool trivial(const Coef &c) { return c.b1 == 1.0f && c.g == 1.0f && c.ap == 1.0f && c.am == 1.0f; }

struct Axes {
    std::vector<Coef> cw[3][2];   // [axis][int/half][0..N]
};

void build_axes(const fdtd_grid &g, const fdtd_boundary &bnd, double dt, Axes &A)
{
    const int N[3] = {g.nx, g.ny, g.nz};
    const double D[3] = {g.dx, g.dy, g.dz};
    for (int w = 0; w < 3; ++w) {
        const int dlo = bnd.depth[2 * w], dhi = bnd.depth[2 * w + 1];
        A.cw[w][0].resize(N[w] + 1);
        A.cw[w][1].resize(N[w] + 1);
        for (int i = 0; i <= N[w]; ++i) {
            A.cw[w][0][i] = upml_coef((double)i, N[w], dlo, dhi, D[w], bnd.m, bnd.R0, bnd.kappa_max, dt);
            A.cw[w][1][i] = i < N[w] ? upml_coef(i + 0.5, N[w], dlo, dhi, D[w], bnd.m, bnd.R0, bnd.kappa_max, dt)
                                     : Coef{1.0f, 1.0f, 1.0f, 1.0f};
        }
    }
}
void build_axes(const fdtd_ctx *c, Axes &A) { build_axes(c->g, c->bnd, c->dt, A); }

double grid_dt(const fdtd_grid &g)
{
    return g.dt > 0 ? g.dt : g.courant / (kC0 * std::sqrt(1.0 / (g.dx * g.dx) + 1.0 / (g.dy * g.dy) + 1.0 / (g.dz * g.dz)));
}

// Fused region and slab boxes of a board (host only): sets the region's
// bounds, the slab boxes with their thread blocks, the z-UPML box planes and
// pitch in h, and which of the six auxiliaries each box keeps in aux.
// Returns false if the boxes exceed kMaxSlab.
bool layout_board(const fdtd_grid &g, const fdtd_boundary &bnd, const Axes &A, Board &h, bool aux[kMaxSlab][6],
                  long long zplanes[2])
{
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    // fused region F = [ix0,ix1) x [iy0,iy1) x [zlo,nz) and the slabs around it.
    // Under a z-UPML the bottom wall is PEC: its plane k = 0 holds the H~x, H~y
    // and E_z samples half a cell up (its tangential E is PEC, and H~z there
    // sees only the curl of that zero E), so the z-UPML launch works it as
    // its first plane (zlo = 0).  Otherwise k = 0 stays a slab plane.
    h.ix0 = std::max(bnd.depth[0], 1); h.ix1 = nx - bnd.depth[1];
    h.iy0 = std::max(bnd.depth[2], 1); h.iy1 = ny - bnd.depth[3];
    h.iz0 = std::max(bnd.depth[4], 1); h.iz1 = nz - bnd.depth[5];
    h.zlo = bnd.depth[4] > 0 ? 0 : 1;
    // The fused region's x bounds are rounded inward to whole 32-byte sectors
    // of a field row (8 FP32 or 16 FP16 nodes); the extra columns are plain
    // nodes that the slab kernels update.  Then no sector is written partly by
    // a slab launch and partly by a fused launch, which would leave it
    // partially written in L2 between the two launches.  A slab row costs
    // about the same at 12 and at 16 nodes (its price is the number of separate
    // row segments a warp touches, not their length).
    {
        const int xa = h.prec == kFP16 ? 16 : 8;
        const int ax0 = (h.ix0 + xa - 1) / xa * xa, ax1 = h.ix1 / xa * xa;
        if (ax1 - ax0 >= xa) { h.ix0 = ax0; h.ix1 = ax1; }
    }
    std::vector<std::array<int, 6>> boxes;
    const bool fused = h.ix1 > h.ix0 && h.iy1 > h.iy0 && nz >= 2;
    if (!fused) {
        h.ix0 = h.ix1 = h.iy0 = h.iy1 = 0;
        h.iz0 = 1; h.iz1 = nz; h.zlo = 1;
        boxes.push_back({0, nx + 1, 0, ny + 1, 0, nz + 1});
    } else {
        // The slabs are split where the set of graded axes changes, so that each
        // box carries only the auxiliaries its own nodes need: faces graded
        // along one axis keep two, edges and corners six.  Per axis the node
        // ranges are low UPML, middle and high UPML; the z ranges of the
        // outer boxes include the wall plane k = 0.
        // A high wall plane (i = nx, j = ny or k = nz) behind a PEC wall holds
        // no unknown: its tangential E edges are PEC, the normal H on it sees
        // the curl of those zero edges, and the other samples do not exist.
        // Everything there stays zero, so those planes are left out of the
        // boxes (their zeros are still read as neighbours).  The low wall
        // planes keep the H and E samples half a cell inside.
        const int xe = bnd.wall[1] == FDTD_WALL_PEC ? nx : nx + 1;
        const int ye = bnd.wall[3] == FDTD_WALL_PEC ? ny : ny + 1;
        const int ze = bnd.wall[5] == FDTD_WALL_PEC ? nz : nz + 1;
        const int xs[4] = {0, h.ix0, h.ix1, xe}, ys[4] = {0, h.iy0, h.iy1, ye};
        const int zs[4] = {0, h.iz0, std::max(h.iz1, h.iz0), ze};
        for (int zb = 0; zb < 3; zb += 2) {
            // z-UPML layers with the wall plane: y strips cut where the x
            // grading starts (each piece then keeps only the auxiliaries of
            // its own graded axes: on a sub-board whose y face is a cut, not
            // a UPML, the middle is a plain z face), then x strips
            for (int yb = 0; yb < 3; yb += 2)
                for (int xb = 0; xb < 3; ++xb) boxes.push_back({xs[xb], xs[xb + 1], ys[yb], ys[yb + 1], zs[zb], zs[zb + 1]});
            for (int xb = 0; xb < 3; xb += 2) boxes.push_back({xs[xb], xs[xb + 1], h.iy0, h.iy1, zs[zb], zs[zb + 1]});
            // the wall plane of the interior columns, unless the fused z-UPML
            // launch works it (zlo = 0) or it is a PEC high plane
            const int kw = zb == 0 ? 0 : nz;
            if (kw < ze && !(kw == 0 && h.zlo == 0)) boxes.push_back({h.ix0, h.ix1, h.iy0, h.iy1, kw, kw + 1});
        }
        // planes between the z-UPML layers: y faces, x faces, the four corner columns
        for (int yb = 0; yb < 3; yb += 2) boxes.push_back({h.ix0, h.ix1, ys[yb], ys[yb + 1], zs[1], zs[2]});
        for (int xb = 0; xb < 3; xb += 2) boxes.push_back({xs[xb], xs[xb + 1], h.iy0, h.iy1, zs[1], zs[2]});
        for (int yb = 0; yb < 3; yb += 2)
            for (int xb = 0; xb < 3; xb += 2) boxes.push_back({xs[xb], xs[xb + 1], ys[yb], ys[yb + 1], zs[1], zs[2]});
    }
    if ((int)boxes.size() > kMaxSlab) return false;
    h.n_slab = 0;
    int blocks = 0;
    for (const auto &bx : boxes) {
        if (bx[1] <= bx[0] || bx[3] <= bx[2] || bx[5] <= bx[4]) continue;
        Slab &sl = h.slab[h.n_slab];
        sl.i0 = bx[0]; sl.i1 = bx[1]; sl.j0 = bx[2]; sl.j1 = bx[3]; sl.k0 = bx[4]; sl.k1 = bx[5];
        sl.ni = sl.i1 - sl.i0; sl.nj = sl.j1 - sl.j0;
        sl.n = (long long)sl.ni * sl.nj * (sl.k1 - sl.k0);
        sl.block0 = blocks;
        // threads: (i, j) columns marching z, or (i, k) columns marching y for a single plane
        const long long cols = sl.k1 - sl.k0 == 1 ? (long long)sl.ni * ((sl.nj + kSlabKz - 1) / kSlabKz)
                                                  : (long long)sl.ni * sl.nj * ((sl.k1 - sl.k0 + kSlabKz - 1) / kSlabKz);
        blocks += (int)((cols + kSlabThreads - 1) / kSlabThreads);
        const int lo[3] = {sl.i0, sl.j0, sl.k0}, hi[3] = {sl.i1, sl.j1, sl.k1};
        auto any_nontrivial = [&](int axis, int half, bool need_b1g, bool need_apam) {
            for (int t = lo[axis]; t < hi[axis]; ++t) {
                const Coef &cf = A.cw[axis][half][t];
                if (need_b1g && (cf.b1 != 1.0f || cf.g != 1.0f)) return true;
                if (need_apam && (cf.ap != 1.0f || cf.am != 1.0f)) return true;
            }
            return false;
        };
        for (int comp = 0; comp < 6; ++comp) {
            const int w = comp % 3, w1 = (w + 1) % 3, w2 = (w + 2) % 3;
            const bool is_h = comp >= 3;
            // E: D recurrence along w1, E recurrence along w2 (integer), D->E along w (half)
            // H: B recurrence along w1, H recurrence along w2 (half),    B->H along w (integer)
            // An auxiliary is needed where D->E (B->H) is graded or both
            // recurrences are; otherwise the lossy form holds exactly (also
            // with FP16 field storage, whose 11-bit mantissa keeps the
            // per-step UPML decay applied to the stored value within the
            // storage mode's error target).
            const int rec = is_h ? 1 : 0;
            aux[h.n_slab][comp] = any_nontrivial(w, is_h ? 0 : 1, false, true) ||
                                  (any_nontrivial(w1, rec, true, false) && any_nontrivial(w2, rec, true, false));
            sl.aux[comp] = nullptr;
        }
        ++h.n_slab;
    }
    h.slab_blocks = blocks;
    // z-UPML boxes of the fused region: lower planes [zlo, iz0), upper [iz1, nz)
    h.zpitch = fused ? ((h.ix1 - h.ix0) + 7) & ~7 : 0;
    for (int bx = 0; bx < 2; ++bx) {
        const long long planes = bx == 0 ? (long long)h.iz0 - h.zlo : (long long)nz - h.iz1;
        zplanes[bx] = fused && planes > 0 ? planes : 0;
    }
    return true;
}

// Band boxes of the two-step pass: the one-node outer layer of the interior
// region I whose second step needs the slab kernels' intermediate state.  H+E
// boxes (high x face, high y face) first, then E-only boxes (low x face, low y
// face, bottom plane); disjoint, blocks numbered after the slab blocks.
void layout_band(Board &h)
{
    h.n_band = h.n_band_h = 0;
    h.band_blocks = h.band_h_blocks = 0;
    if (h.ix1 - h.ix0 < 3 || h.iy1 - h.iy0 < 3 || h.iz1 - h.iz0 < 3) return;
    const int ix0 = h.ix0, ix1 = h.ix1, iy0 = h.iy0, iy1 = h.iy1, iz0 = h.iz0, iz1 = h.iz1;
    const int boxes[5][6] = {{ix1 - 1, ix1, iy0, iy1, iz0, iz1},
                             {ix0, ix1 - 1, iy1 - 1, iy1, iz0, iz1},
                             {ix0, ix0 + 1, iy0, iy1 - 1, iz0, iz1},
                             {ix0 + 1, ix1 - 1, iy0, iy0 + 1, iz0, iz1},
                             {ix0 + 1, ix1 - 1, iy0 + 1, iy1 - 1, iz0, iz0 + 1}};
    if (h.n_slab + 5 > kMaxSlab) return;
    int blocks = h.slab_blocks;
    for (int b = 0; b < 5; ++b) {
        Slab &sl = h.slab[h.n_slab + b];
        sl.i0 = boxes[b][0]; sl.i1 = boxes[b][1]; sl.j0 = boxes[b][2]; sl.j1 = boxes[b][3];
        sl.k0 = boxes[b][4]; sl.k1 = boxes[b][5];
        sl.ni = sl.i1 - sl.i0; sl.nj = sl.j1 - sl.j0;
        sl.n = (long long)sl.ni * sl.nj * (sl.k1 - sl.k0);
        sl.block0 = blocks;
        for (int a = 0; a < 6; ++a) sl.aux[a] = nullptr;
        const long long cols = sl.k1 - sl.k0 == 1 ? (long long)sl.ni * ((sl.nj + kSlabKz - 1) / kSlabKz)
                                                  : (long long)sl.ni * sl.nj * ((sl.k1 - sl.k0 + kSlabKz - 1) / kSlabKz);
        blocks += (int)((cols + kSlabThreads - 1) / kSlabThreads);
        if (b == 1) h.band_h_blocks = blocks - h.slab_blocks;
    }
    h.band_blocks = blocks - h.slab_blocks;
    h.n_band = 5;
    h.n_band_h = 2;
}

// Per-node coefficient ids: ce = 1/eps_r(edge) for the three edges starting at
// the node (mean over the existing cells sharing the edge), 0 on PEC edges and
// on edges that do not exist.  Returns the table (<= 65536 rows) and the
// pitched id volume; the caller stores ids as uint8 when the table has at most
// 256 rows.
// Node coefficient ids of a geometry.  Plane-local ids are assigned in
// parallel over planes and merged into one table; the ids go to `cid`
// (uint16) or, when the table has at most kMaxCombo rows, to `c8`.  The
// buffers are one process-wide scratch, grown on demand and reused under its
// lock, so that their pages are first touched once per process rather than
// once per geometry.
struct NodeIds {
    uint16_t *cid = nullptr;   // [n], also the plane-local ids before the merge
    uint8_t *c8 = nullptr;     // [n], valid when `wide` is false
    bool wide = true;
    size_t n = 0;
};
struct IdScratch {
    std::mutex lock;
    std::unique_ptr<uint16_t[]> cid;
    std::unique_ptr<uint8_t[]> c8;
    size_t cap = 0;
    bool pinned = false;          // registered with CUDA (page-locked) for the uploads
    void reserve(size_t n)
    {
        if (n <= cap) return;
        unpin();
        cid.reset(new uint16_t[n]);
        c8.reset(new uint8_t[n]);
        cap = n;
    }
    // Page-lock the buffers once, so that uploads of the ids are asynchronous
    // DMA copies from pinned memory (host-only callers never need it; if the
    // registration fails the copies still work from pageable memory).
    void pin()
    {
        if (pinned || !cap) return;
        const bool a = cudaHostRegister(cid.get(), cap * sizeof(uint16_t), cudaHostRegisterDefault) == cudaSuccess;
        const bool b = cudaHostRegister(c8.get(), cap, cudaHostRegisterDefault) == cudaSuccess;
        if (!(a && b)) {
            if (a) cudaHostUnregister(cid.get());
            if (b) cudaHostUnregister(c8.get());
            cudaGetLastError();
            return;
        }
        pinned = true;
    }
    void unpin()
    {
        if (!pinned) return;
        cudaHostUnregister(cid.get());
        cudaHostUnregister(c8.get());
        cudaGetLastError();
        pinned = false;
    }
};
// Never destroyed: its buffers may be page-locked, and the CUDA runtime may
// already be shut down when static destructors run.
IdScratch &id_scratch()
{
    static IdScratch *s = new IdScratch;
    return *s;
}

int build_combo(const fdtd_ctx *c, const uint8_t *mat, NodeIds &ids, std::vector<float4> &table)
{
    const int nx = c->g.nx, ny = c->g.ny, nz = c->g.nz;
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    const int pitch = c->h.pitch;
    const long long ncell = (long long)nx * ny * nz;
    const int neps = (int)c->eps.size();
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long long t = 0; t < ncell; ++t) bad |= mat[t] >= neps;
    if (bad) return fail(FDTD_EINVAL, "material id out of range of eps_r");
    // PEC edge bits per node: 1 = x edge, 2 = y edge, 4 = z edge
    const size_t nnode = (size_t)NX * NY * NZ;
    std::unique_ptr<uint8_t[]> pec(new uint8_t[nnode]);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; ++k) std::memset(pec.get() + (size_t)k * NY * NX, 0, (size_t)NY * NX);
    // rows of one box are disjoint, so a box is marked in parallel over its rows
    auto mark_box = [&](int i0, int i1, int j0, int j1, int k0, int k1, bool par) {
        const int ka = std::max(k0, 0), kb = std::min(k1, nz), ja = std::max(j0, 0), jb = std::min(j1, ny);
        const int rows = (kb - ka + 1) * (jb - ja + 1);
#pragma omp parallel for schedule(static) if (par && rows > 64)
        for (int r = 0; r < rows; ++r) {
            const int k = ka + r / (jb - ja + 1), j = ja + r % (jb - ja + 1);
            for (int i = std::max(i0, 0); i <= std::min(i1, nx); ++i) {
                uint8_t bits = 0;
                if (i < i1 && i < nx) bits |= 1;
                if (j < j1 && j < ny) bits |= 2;
                if (k < k1 && k < nz) bits |= 4;
                pec[((size_t)k * NY + j) * NX + i] |= bits;
            }
        }
    };
    for (const fdtd_box &b : c->boxes) mark_box(b.i0, b.i1, b.j0, b.j1, b.k0, b.k1, true);
    if (!c->mask.empty())
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    if (c->mask[((size_t)k * ny + j) * nx + i]) mark_box(i, i + 1, j, j + 1, k, k + 1, false);
    const int *wall = c->bnd.wall;

    ids.n = (size_t)pitch * NY * NZ;
    uint16_t *const cid = ids.cid;   // caller-provided, ids.n entries
    std::vector<std::vector<float4>> plane_tab(NZ);
    std::vector<int> overflow(NZ, 0);
    std::vector<std::unordered_map<uint64_t, uint32_t>> plane_map(NZ);
    auto eps_cell = [&](int i, int j, int k) { return c->eps[mat[((size_t)k * ny + j) * nx + i]]; };
    const size_t sx = (size_t)nx, sxy = (size_t)nx * ny;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < NZ; ++k) {
        std::vector<float4> &tab = plane_tab[k];
        std::unordered_map<uint64_t, uint32_t> &map = plane_map[k];
        float4 last = make_float4(-1, -1, -1, 0);
        uint16_t last_id = 0;
        uint8_t last_pb = 0;
        // 1/mean(eps) of an edge from its n adjacent cells' sum s; neighbouring
        // edges mostly repeat (n, s), so the last quotient per direction is kept
        double qs[3] = {-1.0, -1.0, -1.0};
        int qn[3] = {0, 0, 0};
        float qv[3] = {0.f, 0.f, 0.f};
        auto quot = [&](int d, int n, double sum) {
            if (sum != qs[d] || n != qn[d]) {
                qs[d] = sum;
                qn[d] = n;
                qv[d] = (float)(n / sum);
            }
            return qv[d];
        };
        for (int j = 0; j < NY; ++j) {
            for (int i = NX; i < pitch; ++i) cid[((size_t)k * NY + j) * pitch + i] = 0;   // row padding
            // Away from the outer walls a node's triple is a function of its
            // eight cells' materials and its PEC bits alone: a node repeating
            // the previous node's (cells, bits) key takes the previous id.
            const bool inner_row = j >= 1 && j < ny && k >= 1 && k < nz;
            const uint8_t *m00 = inner_row ? mat + (size_t)(k - 1) * sxy + (size_t)(j - 1) * sx : nullptr;
            bool key_ok = false;
            uint64_t last_cells = 0;
            for (int i = 0; i < NX; ++i) {
                const uint8_t pb = pec[((size_t)k * NY + j) * NX + i];
                uint64_t cells = 0;
                const bool keyed = inner_row && i >= 1 && i < nx;
                if (keyed) {
                    // cells (i-1..i, j-1..j, k-1..k)
                    const uint8_t *q = m00 + (i - 1);
                    cells = (uint64_t)q[0] | (uint64_t)q[1] << 8 | (uint64_t)q[sx] << 16 | (uint64_t)q[sx + 1] << 24 |
                          (uint64_t)q[sxy] << 32 | (uint64_t)q[sxy + 1] << 40 | (uint64_t)q[sxy + sx] << 48 |
                          (uint64_t)q[sxy + sx + 1] << 56;
                    if (key_ok && cells == last_cells && pb == last_pb) {
                        cid[((size_t)k * NY + j) * pitch + i] = last_id;
                        continue;
                    }
                }
                key_ok = keyed;
                last_cells = cells;
                last_pb = pb;
                const bool wx = (i == 0 && wall[0] == FDTD_WALL_PEC) || (i == nx && wall[1] == FDTD_WALL_PEC);
                const bool wy = (j == 0 && wall[2] == FDTD_WALL_PEC) || (j == ny && wall[3] == FDTD_WALL_PEC);
                const bool wz = (k == 0 && wall[4] == FDTD_WALL_PEC) || (k == nz && wall[5] == FDTD_WALL_PEC);
                float ce[3] = {0.f, 0.f, 0.f};
                if (i < nx && !(pb & 1) && !wy && !wz) {
                    double s = 0; int n = 0;
                    for (int b = k - 1; b <= k; ++b)
                        for (int a = j - 1; a <= j; ++a)
                            if (a >= 0 && a < ny && b >= 0 && b < nz) { s += eps_cell(i, a, b); ++n; }
                    ce[0] = quot(0, n, s);
                }
                if (j < ny && !(pb & 2) && !wx && !wz) {
                    double s = 0; int n = 0;
                    for (int b = k - 1; b <= k; ++b)
                        for (int a = i - 1; a <= i; ++a)
                            if (a >= 0 && a < nx && b >= 0 && b < nz) { s += eps_cell(a, j, b); ++n; }
                    ce[1] = quot(1, n, s);
                }
                if (k < nz && !(pb & 4) && !wx && !wy) {
                    double s = 0; int n = 0;
                    for (int b = j - 1; b <= j; ++b)
                        for (int a = i - 1; a <= i; ++a)
                            if (a >= 0 && a < nx && b >= 0 && b < ny) { s += eps_cell(a, b, k); ++n; }
                    ce[2] = quot(2, n, s);
                }
                const float4 v = make_float4(ce[0], ce[1], ce[2], 0.f);
                uint16_t id;
                if (v.x == last.x && v.y == last.y && v.z == last.z) {
                    id = last_id;
                } else {
                    uint32_t bx, by, bz;
                    std::memcpy(&bx, &v.x, 4); std::memcpy(&by, &v.y, 4); std::memcpy(&bz, &v.z, 4);
                    // 64-bit key of the triple: exact when the plane's table stays small,
                    // collisions are resolved by comparing the stored row
                    const uint64_t key = ((uint64_t)bx * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)by << 21) ^
                                         ((uint64_t)bz * 0xC2B2AE3D27D4EB4Full);
                    auto it = map.find(key);
                    size_t t;
                    if (it != map.end() && tab[it->second].x == v.x && tab[it->second].y == v.y &&
                        tab[it->second].z == v.z) {
                        t = it->second;
                    } else {
                        for (t = 0; t < tab.size(); ++t)
                            if (tab[t].x == v.x && tab[t].y == v.y && tab[t].z == v.z) break;
                        if (t == tab.size()) {
                            if (tab.size() >= (size_t)kMaxCombo16) { overflow[k] = 1; t = 0; }
                            else { tab.push_back(v); map[key] = (uint32_t)t; }
                        }
                    }
                    id = (uint16_t)t;
                    last = v;
                    last_id = id;
                }
                cid[((size_t)k * NY + j) * pitch + i] = id;
            }
        }
    }
    for (int k = 0; k < NZ; ++k)
        if (overflow[k]) return fail(FDTD_EINVAL, "more than 65536 distinct edge coefficient triples in one plane");
    // merge plane tables into one global table, remap ids
    table.clear();
    std::unordered_map<uint64_t, std::vector<uint32_t>> gmap;
    std::vector<std::vector<uint16_t>> remap(NZ);
    for (int k = 0; k < NZ; ++k) {
        for (const float4 &v : plane_tab[k]) {
            uint32_t bx, by, bz;
            std::memcpy(&bx, &v.x, 4); std::memcpy(&by, &v.y, 4); std::memcpy(&bz, &v.z, 4);
            const uint64_t key = ((uint64_t)bx << 32) ^ ((uint64_t)by * 0x9E3779B97F4A7C15ull) ^ bz;
            std::vector<uint32_t> &cands = gmap[key];
            size_t t = table.size();
            for (uint32_t cnd : cands)
                if (table[cnd].x == v.x && table[cnd].y == v.y && table[cnd].z == v.z) { t = cnd; break; }
            if (t == table.size()) {
                if (table.size() >= (size_t)kMaxCombo16)
                    return fail(FDTD_EINVAL, "more than 65536 distinct edge coefficient triples");
                table.push_back(v);
                cands.push_back((uint32_t)t);
            }
            remap[k].push_back((uint16_t)t);
        }
    }
    ids.wide = table.size() > (size_t)kMaxCombo;
    if (!ids.wide) {
        uint8_t *const c8 = ids.c8;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < NZ; ++k) {
            const uint16_t *row = cid + (size_t)k * NY * pitch;
            uint8_t *out = c8 + (size_t)k * NY * pitch;
            for (int j = 0; j < NY; ++j) {
                for (int i = 0; i < NX; ++i) out[(size_t)j * pitch + i] = (uint8_t)remap[k][row[(size_t)j * pitch + i]];
                for (int i = NX; i < pitch; ++i) out[(size_t)j * pitch + i] = 0;
            }
        }
    } else {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < NZ; ++k) {
            uint16_t *row = cid + (size_t)k * NY * pitch;
            for (int j = 0; j < NY; ++j)
                for (int i = 0; i < NX; ++i) row[(size_t)j * pitch + i] = remap[k][row[(size_t)j * pitch + i]];
        }
    }
    return FDTD_OK;
}

long long node_index(const Board &h, int i, int j, int k) { return (long long)k * h.plane + (long long)j * h.pitch + i; }

bool edge_exists(const fdtd_ctx *c, int i, int j, int k, int comp)
{
    if (i < 0 || j < 0 || k < 0 || i > c->g.nx || j > c->g.ny || k > c->g.nz) return false;
    if (comp == 0) return i < c->g.nx;
    if (comp == 1) return j < c->g.ny;
    if (comp == 2) return k < c->g.nz;
    return false;
}

int upload_board(fdtd_ctx *c)
{
    CK(cudaMemcpyAsync(c->d, &c->h, sizeof(Board), cudaMemcpyHostToDevice, c->cur));
    return FDTD_OK;
}

// Decide the storage scale, upload sources/probes/trace buffers and the
// descriptor; called once before the first step.
int finalize(fdtd_ctx *c)
{
    if (c->started) return FDTD_OK;
    double s = 1.0;
    if (c->prec != FDTD_FP32 && !c->src.empty()) {
        // field magnitude the sources drive: dt J0 / eps0 for a current, V0 / l for a voltage
        const double d[3] = {c->g.dx, c->g.dy, c->g.dz};
        double emax = 0.0;
        for (const Source &S : c->src)
            emax = std::max(emax, S.kind == kSrcCurrent ? c->dt * std::fabs(S.J0) / kEps0 : std::fabs(S.J0) / d[S.comp]);
        if (emax > 0.0) s = std::exp2(std::ceil(std::log2(emax)));
    }
    c->h.scale = (float)s;
    for (Source &S : c->src) {   // coef was stored as ce dt / eps0, gam in V/m per V
        S.coef = S.coef / s;
        S.gam = S.gam / s;
    }
    if (!c->src.empty()) {
        Source *d = nullptr;
        if (int r = dalloc(c, &d, sizeof(Source) * c->src.size())) return r;
        CK(cudaMemcpyAsync(d, c->src.data(), sizeof(Source) * c->src.size(), cudaMemcpyHostToDevice, c->cur));
        c->h.src = d;
    }
    c->h.n_src = (int)c->src.size();
    {
        std::vector<std::pair<long long, int>> edges;
        for (const Source &S : c->src) edges.push_back({S.node, S.comp});
        std::sort(edges.begin(), edges.end());
        c->h.src_distinct = std::adjacent_find(edges.begin(), edges.end()) == edges.end() ? 1 : 0;
    }
    if (!c->probe.empty()) {
        Probe *d = nullptr;
        if (int r = dalloc(c, &d, sizeof(Probe) * c->probe.size())) return r;
        CK(cudaMemcpyAsync(d, c->probe.data(), sizeof(Probe) * c->probe.size(), cudaMemcpyHostToDevice, c->cur));
        c->h.probe = d;
    }
    c->h.n_probe = (int)c->probe.size();
    if (c->h.n_total > 0 && c->h.n_probe > 0) {
        float *tr = nullptr;
        double *dft = nullptr;
        if (int r = dalloc(c, &tr, sizeof(float) * (size_t)c->h.n_probe * c->h.n_total)) return r;
        if (int r = dalloc(c, &dft, sizeof(double) * 2 * (size_t)c->h.n_probe * std::max(c->h.n_bins, 1))) return r;
        CK(cudaMemsetAsync(tr, 0, sizeof(float) * (size_t)c->h.n_probe * c->h.n_total, c->cur));
        CK(cudaMemsetAsync(dft, 0, sizeof(double) * 2 * (size_t)c->h.n_probe * std::max(c->h.n_bins, 1), c->cur));
        c->h.trace = tr;
        c->h.dft = dft;
    }
    c->started = true;
    c->plan_dirty = true;
    return upload_board(c);
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

// 3D tiled map over a [d2][d1][d0] array of es-byte elements, box b0 x b1 x 1.
int encode3d(CUtensorMap *m, CUtensorMapDataType dt, int es, const void *base, uint64_t d0, uint64_t d1, uint64_t d2,
             uint32_t b0, uint32_t b1)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encoder();
    if (!fn) return fail(FDTD_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (((uintptr_t)base & 15) || ((d0 * es) & 15) || ((b0 * (uint64_t)es) & 15))
        return fail(FDTD_EINVAL, "tensor map would break the 16-byte alignment rules");
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {d0 * es, d0 * d1 * es};
    cuuint32_t box[3] = {b0, b1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FDTD_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return FDTD_OK;
}

// (Re)build the board's TMA descriptors for fused tiles of tx x ty columns.
int encode_maps(fdtd_ctx *c, int tx, int ty)
{
    Board &h = c->h;
    if (h.tm && h.tm_ty == ty && h.tm_tx == tx) return FDTD_OK;
    if (h.ix1 <= h.ix0) { h.tm_tx = tx; h.tm_ty = ty; return FDTD_OK; }   // no fused region
    std::vector<CUtensorMap> maps(kNumMaps);
    std::memset(maps.data(), 0, sizeof(CUtensorMap) * kNumMaps);
    const CUtensorMapDataType fdt = c->prec == FDTD_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const int es = elem_size(c->prec);
    const uint64_t d0 = h.pitch, d1 = h.ny + 1, d2 = h.nz + 1;
    for (int set = 0; set < 3; ++set)
        for (int comp = 0; comp < 3 && h.f[set][0]; ++comp) {
            if (int r = encode3d(&maps[tm_e(set, comp)], fdt, es, h.f[set][comp], d0, d1, d2, box_e(tx), ty + 2)) return r;
            if (int r = encode3d(&maps[tm_h(set, comp)], fdt, es, h.f[set][3 + comp], d0, d1, d2, box_h(tx), ty + 1)) return r;
        }
    if (h.f[2][0]) {   // two-step pass: 60 x 8 tiles, boxes of kPairEW columns
        for (int set = 0; set < 2; ++set)
            for (int comp = 0; comp < 3; ++comp) {
                if (int r = encode3d(&maps[tp_e(set, comp)], fdt, es, h.f[set][comp], d0, d1, d2, kPairEW, kPairRows + 4)) return r;
                if (int r = encode3d(&maps[tp_h(set, comp)], fdt, es, h.f[set][3 + comp], d0, d1, d2, kPairEW, kPairRows + 3)) return r;
            }
        for (int comp = 0; comp < 3; ++comp)
            if (int r = encode3d(&maps[tp_t(comp)], fdt, es, h.f[2][comp], d0, d1, d2, kPairEW, kPairRows + 2)) return r;
        if (int r = encode3d(&maps[kTpCid], h.id16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                             h.id16 ? 2 : 1, h.cid, d0, d1, d2, h.id16 ? kPairC16W : kPairC8W, kPairRows + 2))
            return r;
    }
    if (int r = encode3d(&maps[kTmCid], h.id16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                         h.id16 ? 2 : 1, h.cid, d0, d1, d2, h.id16 ? box_c16(tx) : box_c8(tx), ty))
        return r;
    const uint64_t Ly = h.iy1 - h.iy0;
    for (int bx = 0; bx < 2; ++bx) {
        if (!c->zplanes[bx]) continue;
        if (int r = encode3d(&maps[tm_zd(bx)], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h.zD[bx], h.zpitch, Ly,
                             c->zplanes[bx], box_a(tx), ty))
            return r;
        for (int par = 0; par < 2; ++par)
            if (int r = encode3d(&maps[tm_zb(bx, par)], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h.zB[bx][par], h.zpitch,
                                 Ly, c->zplanes[bx], box_a(tx), ty + 1))
                return r;
    }
    // a fresh buffer per encoding: a descriptor address is never rewritten
    // while a kernel may still hold it in its descriptor cache
    if (int r = dalloc(c, &c->tm_dev, sizeof(CUtensorMap) * kNumMaps)) return r;
    CK(cudaMemcpyAsync(c->tm_dev, maps.data(), sizeof(CUtensorMap) * kNumMaps, cudaMemcpyHostToDevice, c->cur));
    CK(cudaStreamSynchronize(c->cur));
    h.tm = c->tm_dev;
    h.tm_tx = tx;
    h.tm_ty = ty;
    return upload_board(c);
}

// Fused-kernel items of a board: (x tile, y tile, z segment), x fastest.  The
// interior launch covers planes [iz0, iz1), the z-UPML launch [zlo, iz0) and
// [max(iz1, iz0), nz); the device decodes items the same way.
long long fused_items(const Board &h, const fdtd_tuning &t, bool zp)
{
    const long long Lx = h.ix1 - h.ix0, Ly = h.iy1 - h.iy0;
    if (Lx <= 0 || Ly <= 0 || h.nz < 2) return 0;
    auto segs = [&](long long k0, long long k1) { return k1 > k0 ? (k1 - k0 + t.zseg - 1) / t.zseg : 0; };
    const long long nseg = zp ? segs(h.zlo, h.iz0) + segs(std::max(h.iz1, h.iz0), h.nz) : segs(h.iz0, h.iz1);
    return ((Lx + t.tile_x - 1) / t.tile_x) * ((Ly + t.tile_y - 1) / t.tile_y) * nseg;
}

// Two-step items of a board: 60 x 8 tiles x z segments of pair_zseg planes of I.
long long pair_items(const Board &h, const fdtd_tuning &t)
{
    if (!h.pair_ok) return 0;
    const long long Lx = h.ix1 - h.ix0, Ly = h.iy1 - h.iy0, Lz = h.iz1 - h.iz0;
    return ((Lx + kPairCols - 1) / kPairCols) * ((Ly + kPairRows - 1) / kPairRows) * ((Lz + t.pair_zseg - 1) / t.pair_zseg);
}

long long dft_items(const Board &h)
{
    if (h.n_total <= 0 || h.n_probe <= 0) return 0;
    return (long long)h.n_bins * ((h.n_probe + kDftProbeGroup - 1) / kDftProbeGroup);
}

// Lay out plan arrays [boards | int_prefix | zp_prefix | slab_prefix | dft_prefix | work | slab blocks] in buf.
int build_plan(const std::vector<fdtd_ctx *> &boards, const fdtd_tuning &t, long long *&buf, size_t &cap,
               Plan &plan, cudaStream_t st, std::vector<long long> &host)
{
    const int nb = (int)boards.size();
    for (int b = 0; b < nb; ++b)
        if (!fused_maps_match(boards[b]->h, t.tile_x, t.tile_y))
            return fail(FDTD_EINVAL, "fused tile " + std::to_string(t.tile_x) + "x" + std::to_string(t.tile_y) +
                                         " does not match the board's tensor maps (" +
                                         std::to_string(boards[b]->h.tm_tx) + "x" + std::to_string(boards[b]->h.tm_ty) +
                                         "); nothing was launched");
    long long n_slab_blk = 0;
    for (int b = 0; b < nb; ++b) n_slab_blk += boards[b]->h.slab_blocks;
    // a single board's band blocks follow its slab blocks (second step of a pair)
    const bool band = nb == 1 && boards[0]->h.pair_ok && boards[0]->h.n_band > 0;
    if (band) n_slab_blk += boards[0]->h.band_blocks;
    static_assert(sizeof(SlabBlock) == 4 * sizeof(long long), "slab block descriptor layout");
    const size_t head = ((size_t)nb + 4 * ((size_t)nb + 1) + 2 + 1) & ~(size_t)1;   // + four work counters, 16-byte aligned
    const size_t words = head + 4 * (size_t)n_slab_blk;
    host.assign(words, 0);
    long long *ptrs = host.data();
    long long *ip = ptrs + nb, *zp = ip + nb + 1, *sp = zp + nb + 1, *dp = sp + nb + 1;
    SlabBlock *sb = reinterpret_cast<SlabBlock *>(ptrs + head);
    // a single board's band blocks come first in the table, E-only boxes then
    // H+E boxes, so that a second-step launch starts them before the slab
    // blocks (their threads march single columns; at the end they would add
    // their latency to the launch)
    const long long nbb = band ? boards[0]->h.band_blocks : 0;
    const long long nbh = band ? boards[0]->h.band_h_blocks : 0;
    for (int b = 0; b < nb; ++b) {
        const Board &h = boards[b]->h;
        ptrs[b] = (long long)(uintptr_t)boards[b]->d;
        ip[b + 1] = ip[b] + fused_items(h, t, false);
        zp[b + 1] = zp[b] + fused_items(h, t, true);
        sp[b + 1] = sp[b] + h.slab_blocks;
        dp[b + 1] = dp[b] + dft_items(h);
        const int ns = h.n_slab + (band ? h.n_band : 0);
        for (int s = 0; s < ns; ++s) {
            const int end = s + 1 < ns ? (int)h.slab[s + 1].block0 : h.slab_blocks + (band ? h.band_blocks : 0);
            for (int k = (int)h.slab[s].block0; k < end; ++k) {
                // table position: slab blocks after the band; band H+E blocks
                // (numbered first) after the E-only ones
                long long at = sp[b] + k + nbb;
                if (band && k >= h.slab_blocks) at = k - h.slab_blocks < nbh ? (nbb - nbh) + (k - h.slab_blocks)
                                                                              : k - h.slab_blocks - nbh;
                SlabBlock &e = sb[at];
                e.B = boards[b]->d;
                e.step = h.step;
                e.stop = h.stop;
                e.slab = s;
                e.t0 = (k - (int)h.slab[s].block0) * kSlabThreads;
            }
        }
    }
    if (words > cap) {
        if (buf) cudaFree(buf);
        buf = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&buf, words * sizeof(long long));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FDTD_ENOMEM, "plan allocation failed");
        }
        cap = words;
    }
    CK(cudaMemcpyAsync(buf, host.data(), words * sizeof(long long), cudaMemcpyHostToDevice, st));
    plan.nb = nb;
    plan.tile_x = t.tile_x;
    plan.tile_y = t.tile_y;
    plan.zseg = t.zseg;
    plan.boards = (Board *const *)buf;
    plan.int_prefix = buf + nb;
    plan.zp_prefix = buf + nb + (nb + 1);
    plan.slab_prefix = buf + nb + 2 * (nb + 1);
    plan.dft_prefix = buf + nb + 3 * (nb + 1);
    plan.n_int = ip[nb];
    plan.n_zp = zp[nb];
    plan.n_slab = sp[nb];
    plan.n_dft = dp[nb];
    plan.work = (int *)(buf + nb + 4 * (nb + 1));
    plan.slab_blk = reinterpret_cast<const SlabBlock *>(buf + head) + nbb;
    plan.pair_zseg = t.pair_zseg;
    plan.n_pair = band ? pair_items(boards[0]->h, t) : 0;
    plan.first_of_pair = 0;
    plan.n_band_h = band ? boards[0]->h.band_h_blocks : 0;
    plan.n_band = band ? boards[0]->h.band_blocks : 0;
    plan.pc = PairConst{};
    if (band) {
        const Board &h = boards[0]->h;
        PairConst &pc = plan.pc;
        for (int a = 0; a < 3; ++a) pc.S[a] = h.S[a];
        pc.ix0 = h.ix0; pc.ix1 = h.ix1; pc.iy0 = h.iy0; pc.iy1 = h.iy1; pc.iz0 = h.iz0; pc.iz1 = h.iz1;
        pc.ny = h.ny; pc.pitch = h.pitch; pc.id16 = h.id16;
        pc.plane = h.plane; pc.nodes = h.nodes;
        pc.ctab = h.ctab;
        pc.mid = h.f[2][0];
    }
    return FDTD_OK;
}

// NVTX range over a host-side call, for profiler timelines (no cost without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Run n steps of `plan` on stream st: CUDA graphs of `chunk` steps (each
// ending with the running-DFT update), direct launches for the remainder.
int run_steps(const Plan &plan, int prec, int grid_cap, int n, int chunk, cudaGraphExec_t &graph, int &graph_chunk,
              cudaStream_t st)
{
    if (n <= 0) return FDTD_OK;
    NvtxRange range(plan.nb > 1 ? "fdtd batch steps" : "fdtd steps");
    if (chunk > 1 && n >= chunk) {
        if (!graph || graph_chunk != chunk) {
            if (graph) cudaGraphExecDestroy(graph);
            graph = nullptr;
            cudaGraph_t gr = nullptr;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int s = 0; s < chunk && e == cudaSuccess; ++s) e = launch_step(plan, prec, grid_cap, st);
            if (e == cudaSuccess) e = launch_dft(plan, grid_cap, st);
            cudaError_t e2 = cudaStreamEndCapture(st, &gr);
            if (e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(e, "capture"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&graph, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) { graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
            graph_chunk = chunk;
        }
        for (int r = 0; r < n / chunk; ++r) CK(cudaGraphLaunch(graph, st));
        n %= chunk;
    }
    if (n > 0) {
        for (int s = 0; s < n; ++s) CK(launch_step(plan, prec, grid_cap, st));
        CK(launch_dft(plan, grid_cap, st));
    }
    return FDTD_OK;
}

// Run n steps of a depth-2 single-board plan: a single step to reach an even
// step, then pairs (CUDA graphs of chunk / 2 pairs), then one or two single
// steps, so that the states after the last two steps are complete in memory
// (the state in the middle of a pair is kept only where later launches read
// it).
int run_depth2(const Plan &plan, int prec, int grid_cap, long long step, int n, int chunk, cudaGraphExec_t &graph2,
               int &graph2_chunk, cudaStream_t st)
{
    if (n <= 0) return FDTD_OK;
    NvtxRange range("fdtd step pairs");
    const PairSplit sp = pair_split(step, n);
    if (sp.lead) CK(launch_step(plan, prec, grid_cap, st));
    const bool direct = sp.lead != 0;
    int pairs = sp.pairs;
    const int left = sp.tail;
    const int cp = std::max(1, chunk / 2);
    if (cp > 1 && pairs >= cp) {
        if (!graph2 || graph2_chunk != cp) {
            if (graph2) cudaGraphExecDestroy(graph2);
            graph2 = nullptr;
            cudaGraph_t gr = nullptr;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int s = 0; s < cp && e == cudaSuccess; ++s) e = launch_pair(plan, prec, grid_cap, st);
            if (e == cudaSuccess) e = launch_dft(plan, grid_cap, st);
            cudaError_t e2 = cudaStreamEndCapture(st, &gr);
            if (e != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(e, "capture"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&graph2, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) { graph2 = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
            graph2_chunk = cp;
        }
        for (int r = 0; r < pairs / cp; ++r) CK(cudaGraphLaunch(graph2, st));
        pairs %= cp;
    }
    for (int p = 0; p < pairs; ++p) CK(launch_pair(plan, prec, grid_cap, st));
    for (int s = 0; s < left; ++s) CK(launch_step(plan, prec, grid_cap, st));
    if (direct || pairs > 0 || left > 0) CK(launch_dft(plan, grid_cap, st));
    return FDTD_OK;
}

// Whether the two-step pass can run on this board (set 2 allocated).  The
// plane above I must be written before the pass by the z-UPML launch, or be
// the zero plane behind a PEC wall; x of the tiles' lane pairs must be even.
bool pair_possible(const fdtd_ctx *c)
{
    const Board &h = c->h;
    return h.ix1 > h.ix0 && h.iy1 > h.iy0 && (h.ix0 % 2) == 0 && h.ix1 - h.ix0 >= 3 && h.iy1 - h.iy0 >= 3 &&
           h.iz1 - h.iz0 >= 3 && h.n_band == 5 && (c->bnd.depth[5] > 0 || c->bnd.wall[5] == FDTD_WALL_PEC);
}

// Field sets for depth d: set 2 is allocated on first use, and the sets are
// renamed so that the states after the last two steps sit where set_of(d, .)
// expects them.
int set_time_depth(fdtd_ctx *c, int d)
{
    Board &h = c->h;
    const int old = h.tdepth;
    if (d == 2 && !h.f[2][0]) {
        unsigned char *blk = nullptr;
        if (int r = dalloc(c, &blk, 6 * c->fbytes)) return r;
        CK(cudaMemsetAsync(blk, 0, 6 * c->fbytes, c->cur));
        for (int f = 0; f < 6; ++f) h.f[2][f] = blk + f * c->fbytes;
    }
    CK(cudaStreamSynchronize(c->cur));
    if (d != old) {
        const long long n = c->host_step;
        int perm[3];
        rename_sets(old, d, n, perm);
        void *f[3][6];
        for (int x = 0; x < 3; ++x)
            for (int q = 0; q < 6; ++q) f[x][q] = h.f[perm[x]][q];
        std::memcpy(h.f, f, sizeof(f));
        h.tdepth = d;
        h.tm_tx = 0;   // the tensor maps name the sets' addresses
        c->plan_dirty = true;
    }
    h.pair_ok = (d == 2 && h.f[2][0] && pair_possible(c)) ? 1 : 0;
    if (c->d) return upload_board(c);
    return FDTD_OK;
}

int check_status(fdtd_ctx *c)
{
    int st = 0;
    CK(cudaMemcpy(&st, c->h.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & 4) return fail(FDTD_EINVAL, "a fused-kernel launch did not match the board's tensor maps; its items were "
                                         "skipped (results of this run are invalid)");
    if (st & 2) return fail(FDTD_ETIMEOUT, "a fused-kernel TMA wait gave up (results of this run are invalid)");
    if (st & 1) return fail(FDTD_EUNSTABLE, "non-finite probe sample (unstable run: check the Courant number)");
    return FDTD_OK;
}

int set_geometry(fdtd_ctx *c, const uint8_t *mat)
{
    IdScratch &scratch = id_scratch();
    std::lock_guard<std::mutex> hold(scratch.lock);
    NodeIds ids;
    ids.n = (size_t)c->h.pitch * (c->g.ny + 1) * (c->g.nz + 1);
    try {
        scratch.reserve(ids.n);
    } catch (const std::bad_alloc &) {
        return fail(FDTD_ENOMEM, "host scratch for the coefficient ids");
    }
    scratch.pin();
    ids.cid = scratch.cid.get();
    ids.c8 = scratch.c8.get();
    std::vector<float4> table;
    if (int r = build_combo(c, mat, ids, table)) return r;
    c->n_combo = (int)table.size();
    const int id16 = table.size() > (size_t)kMaxCombo ? 1 : 0;
    const size_t rows = id16 ? (size_t)kMaxCombo16 : (size_t)kMaxCombo;
    table.resize(rows, make_float4(0, 0, 0, 0));
    c->ctab = table;
    if (id16 != c->h.id16 || !c->h.cid) {
        // id buffers of the other width: allocate once, kept until destroy
        void *d = nullptr;
        float4 *t = nullptr;
        if (int r = dalloc(c, &d, (size_t)c->h.nodes * (id16 ? 2 : 1))) return r;
        if (int r = dalloc(c, &t, sizeof(float4) * rows)) return r;
        c->h.cid = d;
        c->h.ctab = t;
        c->h.id16 = id16;
        c->h.tm_ty = 0;   // the id tensor map must be rebuilt
        c->h.tm_tx = 0;
        c->plan_dirty = true;
    }
    if (id16)
        CK(cudaMemcpyAsync((void *)c->h.cid, ids.cid, ids.n * 2, cudaMemcpyHostToDevice, c->cur));
    else
        CK(cudaMemcpyAsync((void *)c->h.cid, ids.c8, ids.n, cudaMemcpyHostToDevice, c->cur));
    CK(cudaMemcpyAsync((void *)c->h.ctab, table.data(), sizeof(float4) * rows, cudaMemcpyHostToDevice, c->cur));
    // the host copies stay alive until the copies finish
    CK(cudaStreamSynchronize(c->cur));
    if (c->d) return upload_board(c);
    return FDTD_OK;
}

uint32_t edge_combo(const fdtd_ctx *c, long long node)
{
    uint32_t id = 0;
    if (c->h.id16) {
        uint16_t v = 0;
        cudaMemcpy(&v, (const uint16_t *)c->h.cid + node, 2, cudaMemcpyDeviceToHost);
        id = v;
    } else {
        uint8_t v = 0;
        cudaMemcpy(&v, (const uint8_t *)c->h.cid + node, 1, cudaMemcpyDeviceToHost);
        id = v;
    }
    return id;
}

}  // namespace

// =========================================================================== C-ABI

extern "C" {

const char *fdtd_strerror(int code)
{
    switch (code) {
    case FDTD_OK: return "ok";
    case FDTD_EINVAL: return "invalid argument";
    case FDTD_ENOMEM: return "out of memory";
    case FDTD_ECUDA: return "CUDA error";
    case FDTD_EUNSTABLE: return "unstable (non-finite field values)";
    case FDTD_ETIMEOUT: return "device wait timed out";
    case FDTD_ESTATE: return "call not valid in the current state";
    default: return "unknown status";
    }
}

const char *fdtd_last_error(void) { return g_err.c_str(); }

void fdtd_destroy(fdtd_ctx *c);

namespace {

// Argument checks shared by fdtd_create and fdtd_node_coefficients.
int check_problem(const fdtd_grid *grid, const uint8_t *mat_ids, const double *eps_r, int n_mat, const fdtd_box *pec,
                  int n_pec, const fdtd_boundary *bnd)
{
    if (!grid || !mat_ids || !eps_r || !bnd) return fail(FDTD_EINVAL, "NULL grid, mat_ids, eps_r or boundary");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(FDTD_EINVAL, "grid must have at least one cell per axis");
    if (!(grid->dx > 0 && grid->dy > 0 && grid->dz > 0)) return fail(FDTD_EINVAL, "cell sizes must be positive");
    if (grid->dt <= 0 && !(grid->courant > 0)) return fail(FDTD_EINVAL, "need dt > 0 or courant > 0");
    if (n_mat < 1 || n_mat > 256) return fail(FDTD_EINVAL, "n_mat must be in 1..256");
    for (int m = 0; m < n_mat; ++m)
        if (!(eps_r[m] > 0)) return fail(FDTD_EINVAL, "eps_r must be positive");
    if (n_pec < 0 || (n_pec > 0 && !pec)) return fail(FDTD_EINVAL, "bad PEC box list");
    const int N[3] = {grid->nx, grid->ny, grid->nz};
    for (int f = 0; f < 6; ++f) {
        if (bnd->depth[f] < 0 || bnd->depth[f] > N[f / 2]) return fail(FDTD_EINVAL, "bad UPML depth");
        if (bnd->wall[f] != FDTD_WALL_PEC && bnd->wall[f] != FDTD_WALL_PMC) return fail(FDTD_EINVAL, "bad wall type");
        if (bnd->depth[f] > 0 && bnd->wall[f] != FDTD_WALL_PEC)
            return fail(FDTD_EINVAL, "a face with UPML must be backed by a PEC wall");
    }
    for (int w = 0; w < 3; ++w)
        if (bnd->depth[2 * w] + bnd->depth[2 * w + 1] > N[w]) return fail(FDTD_EINVAL, "UPML layers overlap");
    if (bnd->depth[0] + bnd->depth[1] + bnd->depth[2] + bnd->depth[3] + bnd->depth[4] + bnd->depth[5] > 0 &&
        !(bnd->R0 > 0 && bnd->R0 <= 1 && bnd->m >= 0 && bnd->kappa_max >= 1))
        return fail(FDTD_EINVAL, "UPML needs 0 < R0 <= 1, m >= 0, kappa_max >= 1");
    return FDTD_OK;
}

}  // namespace

int fdtd_create(const fdtd_grid *grid, const uint8_t *mat_ids, const double *eps_r, int n_mat, const fdtd_box *pec,
                int n_pec, const uint8_t *pec_mask, const fdtd_boundary *bnd, int precision, void *stream,
                fdtd_ctx **out)
{
    if (!out) return fail(FDTD_EINVAL, "out is NULL");
    *out = nullptr;
    if (precision != FDTD_FP32 && precision != FDTD_FP16_STORE)
        return fail(FDTD_EINVAL, "precision must be FDTD_FP32 or FDTD_FP16_STORE");
    if (int r = check_problem(grid, mat_ids, eps_r, n_mat, pec, n_pec, bnd)) return r;

    fdtd_ctx *c = new fdtd_ctx();
    c->g = *grid;
    c->bnd = *bnd;
    c->eps.assign(eps_r, eps_r + n_mat);
    if (n_pec > 0) c->boxes.assign(pec, pec + n_pec);
    if (pec_mask) c->mask.assign(pec_mask, pec_mask + (size_t)grid->nx * grid->ny * grid->nz);
    c->prec = precision;
    c->dt = grid->dt > 0 ? grid->dt
                         : grid->courant / (kC0 * std::sqrt(1.0 / (grid->dx * grid->dx) + 1.0 / (grid->dy * grid->dy) +
                                                             1.0 / (grid->dz * grid->dz)));
    c->grid_cap = device_grid_cap();
    if (cudaGetDevice(&c->device) != cudaSuccess) { cudaGetLastError(); c->device = 0; }
    static bool smem_limits = false;
    if (!smem_limits) {
        cudaError_t e = fused_set_smem_limits();
        if (e != cudaSuccess) { cudaGetLastError(); return fail(FDTD_ECUDA, std::string("fused kernel shared memory: ") + cudaGetErrorString(e)); }
        smem_limits = true;
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreate"); }
        c->own_stream = true;
    }
    c->cur = c->stream;

    Board &h = c->h;
    h.nx = grid->nx; h.ny = grid->ny; h.nz = grid->nz;
    h.pitch = row_pitch(grid->nx);
    h.plane = (long long)h.pitch * (grid->ny + 1);
    h.nodes = h.plane * (grid->nz + 1);
    if (h.nodes >= (1LL << 31)) { fdtd_destroy(c); return fail(FDTD_EINVAL, "grid too large (>= 2^31 nodes)"); }
    h.prec = precision;
    h.S[0] = (float)(kC0 * c->dt / grid->dx);
    h.S[1] = (float)(kC0 * c->dt / grid->dy);
    h.S[2] = (float)(kC0 * c->dt / grid->dz);
    h.scale = 1.0f;
    h.dt = c->dt;
    for (int f = 0; f < 6; ++f) { h.wall[f] = bnd->wall[f]; h.depth[f] = bnd->depth[f]; }

    int r = FDTD_OK;
    const size_t fbytes = (size_t)h.nodes * elem_size(precision);
    c->fbytes = fbytes;
    h.tdepth = 1;
    h.pair_ok = 0;
    for (int f = 0; f < 6; ++f) h.f[2][f] = nullptr;   // set 2: allocated when two-step passes are enabled
    // the six components of one set are contiguous (component stride = nodes)
    for (int p = 0; p < 2 && !r; ++p) {
        unsigned char *blk = nullptr;
        r = dalloc(c, &blk, 6 * fbytes);
        if (!r) { cudaError_t e = cudaMemsetAsync(blk, 0, 6 * fbytes, c->cur); if (e) r = cuda_fail(e, "memset"); }
        for (int f = 0; f < 6 && !r; ++f) h.f[p][f] = blk + f * fbytes;
    }
    h.cid = nullptr;
    h.ctab = nullptr;
    h.id16 = -1;
    if (r) { fdtd_destroy(c); return r; }
    if ((r = set_geometry(c, mat_ids))) { fdtd_destroy(c); return r; }

    // UPML factors
    Axes A;
    build_axes(c, A);
    for (int w = 0; w < 3 && !r; ++w)
        for (int s = 0; s < 2 && !r; ++s) {
            Coef *d = nullptr;
            r = dalloc(c, &d, sizeof(Coef) * A.cw[w][s].size());
            if (!r) {
                cudaError_t e = cudaMemcpyAsync(d, A.cw[w][s].data(), sizeof(Coef) * A.cw[w][s].size(),
                                                cudaMemcpyHostToDevice, c->cur);
                if (e) r = cuda_fail(e, "upload UPML factors");
            }
            h.cw[w][s] = d;
        }
    if (r) { fdtd_destroy(c); return r; }

    // fused region and slab boxes
    bool aux[kMaxSlab][6];
    if (!layout_board(*grid, *bnd, A, h, aux, c->zplanes)) { fdtd_destroy(c); return fail(FDTD_EINVAL, "internal: too many slab boxes"); }
    layout_band(h);
    for (int s = 0; s < h.n_slab && !r; ++s) {
        Slab &sl = h.slab[s];
        for (int comp = 0; comp < 6 && !r; ++comp) {
            if (!aux[s][comp]) continue;
            r = dalloc(c, &sl.aux[comp], sizeof(float) * (size_t)sl.n);
            if (!r) { cudaError_t e = cudaMemsetAsync(sl.aux[comp], 0, sizeof(float) * (size_t)sl.n, c->cur); if (e) r = cuda_fail(e, "memset"); }
        }
    }
    for (int bx = 0; bx < 2; ++bx) {
        h.zD[bx] = nullptr;
        h.zB[bx][0] = h.zB[bx][1] = nullptr;
        if (!c->zplanes[bx]) continue;
        const size_t n = (size_t)c->zplanes[bx] * h.zpitch * (h.iy1 - h.iy0);
        float *ptr[3] = {nullptr, nullptr, nullptr};   // D~z, B~z (two parities)
        for (int t = 0; t < 3 && !r; ++t) {
            r = dalloc(c, &ptr[t], sizeof(float) * n);
            if (!r) { cudaError_t e = cudaMemsetAsync(ptr[t], 0, sizeof(float) * n, c->cur); if (e) r = cuda_fail(e, "memset"); }
        }
        h.zD[bx] = ptr[0];
        h.zB[bx][0] = ptr[1];
        h.zB[bx][1] = ptr[2];
        c->zaux_n[bx] = n;
    }
    long long *ctr = nullptr;
    const long long init[4] = {0, LLONG_MAX, 0, 0};
    if (!r) r = dalloc(c, &ctr, 4 * sizeof(long long));
    if (!r) {
        h.step = ctr; h.stop = ctr + 1; h.dft_done = ctr + 2; h.status = (int *)(ctr + 3);
        cudaError_t e = cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, c->cur);
        if (e) r = cuda_fail(e, "init counters");
    }
    if (!r) r = dalloc(c, &c->d, sizeof(Board));
    if (!r) {
        c->energy_n = energy_partials(h);
        r = dalloc(c, &c->energy_buf, sizeof(double) * (2 * (size_t)c->energy_n + 2));
    }
    if (!r) r = upload_board(c);
    if (!r) { cudaError_t e = cudaStreamSynchronize(c->cur); if (e) r = cuda_fail(e, "create sync"); }
    if (r) { fdtd_destroy(c); return r; }
    *out = c;
    return FDTD_OK;
}

int fdtd_set_source(fdtd_ctx *c, int i, int j, int k, int comp, double J0, double t0, double tau, int *src_id)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (c->started) return fail(FDTD_ESTATE, "sources must be added before the first step");
    if (!edge_exists(c, i, j, k, comp)) return fail(FDTD_EINVAL, "source edge does not exist");
    if (!(tau > 0)) return fail(FDTD_EINVAL, "tau must be positive");
    // the edge must be outside the UPML: all three factors trivial at its position
    Axes A;
    build_axes(c, A);
    const int idx[3] = {i, j, k};
    for (int a = 0; a < 3; ++a)
        if (!trivial(A.cw[a][a == comp ? 1 : 0][idx[a]]))
            return fail(FDTD_EINVAL, "source edge lies inside the UPML");
    const float4 row = c->ctab[edge_combo(c, node_index(c->h, i, j, k))];
    const float ce = comp == 0 ? row.x : comp == 1 ? row.y : row.z;
    if (ce == 0.0f) return fail(FDTD_EINVAL, "source edge is PEC");
    Source S{};
    S.node = node_index(c->h, i, j, k);
    S.comp = comp;
    S.i = i; S.j = j; S.k = k;
    S.J0 = J0; S.t0 = t0; S.tau = tau;
    S.coef = (double)ce * c->dt / kEps0;
    c->src.push_back(S);
    if (src_id) *src_id = (int)c->src.size() - 1;
    return FDTD_OK;
}

// Lumped-element factors of a resistive voltage source on an edge of length
// l and cross-section area = V / l with permittivity eps0 / ce: Ampere's law
// eps (E' - E)/dt = curl H - (l (E + E')/2 + Vs) / (Rs area) gives
// E' = (E_plain - beta E - gam Vs) / (1 + beta), E_plain = E + dt curl H / eps.
void vsource_coef(const fdtd_ctx *c, Source &S, float ce, double scale)
{
    const double d[3] = {c->g.dx, c->g.dy, c->g.dz};
    const double l = d[S.comp], area = d[0] * d[1] * d[2] / l;
    const double eps = kEps0 / (double)ce;
    S.beta = c->dt * l / (2.0 * eps * S.rs * area);
    S.gam = c->dt / (eps * S.rs * area) / scale;
}

int fdtd_set_voltage_source(fdtd_ctx *c, int i, int j, int k, int comp, double V0, double t0, double tau,
                            double Rs, int *src_id)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (c->started) return fail(FDTD_ESTATE, "sources must be added before the first step");
    if (!edge_exists(c, i, j, k, comp)) return fail(FDTD_EINVAL, "source edge does not exist");
    if (!(tau > 0)) return fail(FDTD_EINVAL, "tau must be positive");
    if (!(Rs > 0)) return fail(FDTD_EINVAL, "Rs must be positive (infinity: an open edge)");
    Axes A;
    build_axes(c, A);
    const int idx[3] = {i, j, k};
    for (int a = 0; a < 3; ++a)
        if (!trivial(A.cw[a][a == comp ? 1 : 0][idx[a]]))
            return fail(FDTD_EINVAL, "source edge lies inside the UPML");
    const float4 row = c->ctab[edge_combo(c, node_index(c->h, i, j, k))];
    const float ce = comp == 0 ? row.x : comp == 1 ? row.y : row.z;
    if (ce == 0.0f) return fail(FDTD_EINVAL, "source edge is PEC");
    Source S{};
    S.node = node_index(c->h, i, j, k);
    S.comp = comp;
    S.i = i; S.j = j; S.k = k;
    S.kind = kSrcResistiveVoltage;
    S.J0 = V0; S.t0 = t0; S.tau = tau;
    S.rs = Rs;
    vsource_coef(c, S, ce, 1.0);
    c->src.push_back(S);
    if (src_id) *src_id = (int)c->src.size() - 1;
    return FDTD_OK;
}

int fdtd_add_probe(fdtd_ctx *c, int i, int j, int k, int comp, int *probe_id)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (c->started) return fail(FDTD_ESTATE, "probes must be added before the first step");
    if (!edge_exists(c, i, j, k, comp)) return fail(FDTD_EINVAL, "probe edge does not exist");
    Probe p{};
    p.node = node_index(c->h, i, j, k);
    p.comp = comp;
    p.i = i; p.j = j; p.k = k;
    c->probe.push_back(p);
    if (probe_id) *probe_id = (int)c->probe.size() - 1;
    return FDTD_OK;
}

int fdtd_set_spectrum(fdtd_ctx *c, double f_max, int n_total_steps)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (c->started) return fail(FDTD_ESTATE, "spectrum must be set before the first step");
    if (n_total_steps < 1) return fail(FDTD_EINVAL, "n_total_steps must be >= 1");
    const int nyq = n_total_steps / 2 + 1;
    int Q = nyq;
    if (f_max > 0) Q = std::min(nyq, (int)std::floor(f_max * n_total_steps * c->dt + 1e-9) + 1);
    c->h.n_total = n_total_steps;
    c->h.n_bins = Q;
    return FDTD_OK;
}

int fdtd_set_tuning(fdtd_ctx *c, const fdtd_tuning *t)
{
    if (!c || !t) return fail(FDTD_EINVAL, "NULL argument");
    fdtd_tuning n = c->tune;
    if (t->tile_x > 0) n.tile_x = t->tile_x;
    if (t->tile_y > 0) n.tile_y = t->tile_y;
    if (t->zseg > 0) n.zseg = t->zseg;
    if (t->graph_chunk > 0) n.graph_chunk = t->graph_chunk;
    if (t->depth > 0) n.depth = t->depth;
    if (t->pair_zseg > 0) n.pair_zseg = t->pair_zseg;
    if (!fused_tile_supported(n.tile_x, n.tile_y))
        return fail(FDTD_EINVAL, "fused tile (tile_x x tile_y) must be 62x4, 62x8, 124x4 or 124x8");
    if (n.depth != 1 && n.depth != 2) return fail(FDTD_EINVAL, "depth must be 1 or 2");
    if (n.pair_zseg < 2) return fail(FDTD_EINVAL, "pair_zseg must be >= 2");
    if (n.depth != c->h.tdepth)
        if (int r = set_time_depth(c, n.depth)) return r;
    c->tune = n;
    c->plan_dirty = true;
    return FDTD_OK;
}

static int prepare_single(fdtd_ctx *c);

int fdtd_step(fdtd_ctx *c, int n)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (n < 0) return fail(FDTD_EINVAL, "n must be >= 0");
    if (c->batch) return fail(FDTD_ESTATE, "context is in a batch; step the batch");
    if (int r = prepare_single(c)) return r;
    if (c->h.pair_ok) {
        if (int r = run_depth2(c->plan, c->prec, c->grid_cap, c->host_step, n, c->tune.graph_chunk, c->graph2,
                               c->graph2_chunk, c->cur))
            return r;
    } else if (int r = run_steps(c->plan, c->prec, c->grid_cap, n, c->tune.graph_chunk, c->graph, c->graph_chunk, c->cur)) {
        return r;
    }
    c->host_step += n;
    return FDTD_OK;
}

static int prepare_single(fdtd_ctx *c)
{
    if (int r = finalize(c)) return r;
    if (int r = encode_maps(c, c->tune.tile_x, c->tune.tile_y)) return r;
    if (c->plan_dirty) {
        std::vector<long long> host;
        std::vector<fdtd_ctx *> one{c};
        if (int r = build_plan(one, c->tune, c->plan_buf, c->plan_cap, c->plan, c->cur, host)) return r;
        CK(cudaStreamSynchronize(c->cur));
        if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
        if (c->graph2) { cudaGraphExecDestroy(c->graph2); c->graph2 = nullptr; }
        c->plan_dirty = false;
    }
    return FDTD_OK;
}

int fdtd_step_profiled(fdtd_ctx *c, int n, double *phase_ms)
{
    if (!c || !phase_ms) return fail(FDTD_EINVAL, "NULL argument");
    if (n < 0) return fail(FDTD_EINVAL, "n must be >= 0");
    if (c->batch) return fail(FDTD_ESTATE, "context is in a batch; step the batch");
    if (int r = prepare_single(c)) return r;
    const size_t need = (size_t)n * (kPairLaunches + 1) + 2;
    while (c->events.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->events.push_back(e);
    }
    for (int p = 0; p <= kNumPhases; ++p) phase_ms[p] = 0.0;
    // the launch sequence: single steps (five launches) and, with depth 2,
    // pairs (nine launches); the same split as fdtd_step
    std::vector<int> unit;   // 1: single step, 2: pair
    if (c->h.pair_ok) {
        const PairSplit sp = pair_split(c->host_step, n);
        unit.assign(sp.lead, 1);
        unit.insert(unit.end(), sp.pairs, 2);
        unit.insert(unit.end(), sp.tail, 1);
    } else {
        unit.assign(n, 1);
    }
    std::vector<int> phase_of;   // phase of each timed launch
    size_t ev = 0;
    for (int u : unit) {
        CK(cudaEventRecord(c->events[ev++], c->cur));
        const int nl = u == 2 ? kPairLaunches : kNumPhases;
        for (int i = 0; i < nl; ++i) {
            if (u == 2) CK(launch_pair_part(c->plan, c->prec, i, c->grid_cap, c->cur));
            else CK(launch_phase(c->plan, c->prec, i, c->grid_cap, c->cur));
            CK(cudaEventRecord(c->events[ev++], c->cur));
            phase_of.push_back(u == 2 ? kPairPhase[i] : i);
        }
    }
    CK(cudaEventRecord(c->events[ev++], c->cur));
    CK(launch_dft(c->plan, c->grid_cap, c->cur));
    CK(cudaEventRecord(c->events[ev++], c->cur));
    CK(cudaStreamSynchronize(c->cur));
    ev = 0;
    size_t li = 0;
    for (int u : unit) {
        const int nl = u == 2 ? kPairLaunches : kNumPhases;
        for (int i = 0; i < nl; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->events[ev + i], c->events[ev + i + 1]));
            phase_ms[phase_of[li++]] += ms;
        }
        ev += nl + 1;
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->events[ev], c->events[ev + 1]));
    phase_ms[kNumPhases] += ms;
    c->host_step += n;
    return check_status(c);
}

int fdtd_sync(fdtd_ctx *c)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    CK(cudaStreamSynchronize(c->cur));
    return check_status(c);
}

int fdtd_probe_spectra(fdtd_ctx *c, double *out, int max_bins, int *n_bins)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (n_bins) *n_bins = c->h.n_bins;
    if (int r = fdtd_sync(c)) return r;
    if (c->h.n_total <= 0 || c->h.n_probe <= 0 || !c->h.dft) return FDTD_OK;
    if (!out || max_bins < c->h.n_bins) return fail(FDTD_EINVAL, "output too small for the spectrum");
    CK(cudaMemcpy(out, c->h.dft, sizeof(double) * 2 * (size_t)c->h.n_probe * c->h.n_bins, cudaMemcpyDeviceToHost));
    return FDTD_OK;
}

int fdtd_probe_trace(fdtd_ctx *c, int probe, float *out, int max_len, int *len)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (probe < 0 || probe >= (int)c->probe.size()) return fail(FDTD_EINVAL, "bad probe index");
    if (int r = fdtd_sync(c)) return r;
    long long n = std::min<long long>(c->host_step, c->h.n_total);
    n = std::min<long long>(n, max_len);
    if (len) *len = (int)n;
    if (n <= 0 || !c->h.trace) return FDTD_OK;
    if (!out) return fail(FDTD_EINVAL, "NULL output");
    CK(cudaMemcpy(out, c->h.trace + (size_t)probe * c->h.n_total, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return FDTD_OK;
}

int fdtd_get_field(fdtd_ctx *c, int field, float *out)
{
    if (!c || !out) return fail(FDTD_EINVAL, "NULL argument");
    if (field < 0 || field > 5) return fail(FDTD_EINVAL, "field must be 0..5");
    if (int r = fdtd_sync(c)) return r;
    const Board &h = c->h;
    const int par = set_of(h.tdepth, c->host_step);
    const int es = elem_size(c->prec);
    std::vector<unsigned char> buf((size_t)h.nodes * es);
    CK(cudaMemcpy(buf.data(), h.f[par][field], buf.size(), cudaMemcpyDeviceToHost));
    const double s = field < 3 ? h.scale : h.scale / kEta0;
    const int NX = h.nx + 1, NY = h.ny + 1, NZ = h.nz + 1;
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j)
            for (int i = 0; i < NX; ++i) {
                const size_t src = ((size_t)k * NY + j) * h.pitch + i;
                float v;
                if (c->prec == FDTD_FP32) v = ((const float *)buf.data())[src];
                else v = __half2float(((const __half *)buf.data())[src]);
                out[((size_t)k * NY + j) * NX + i] = (float)(v * s);
            }
    return FDTD_OK;
}

int fdtd_get_plane(fdtd_ctx *c, int field, int k, float *out)
{
    if (!c || !out) return fail(FDTD_EINVAL, "NULL argument");
    if (field < 0 || field > 5) return fail(FDTD_EINVAL, "field must be 0..5");
    if (k < 0 || k > c->h.nz) return fail(FDTD_EINVAL, "plane index out of range");
    if (int r = fdtd_sync(c)) return r;
    const Board &h = c->h;
    const int par = set_of(h.tdepth, c->host_step);
    const int es = elem_size(c->prec);
    const int NX = h.nx + 1, NY = h.ny + 1;
    std::vector<unsigned char> buf((size_t)NX * NY * es);
    const unsigned char *src = static_cast<const unsigned char *>(h.f[par][field]) + (size_t)k * h.plane * es;
    CK(cudaMemcpy2D(buf.data(), (size_t)NX * es, src, (size_t)h.pitch * es, (size_t)NX * es, NY, cudaMemcpyDeviceToHost));
    const double s = field < 3 ? h.scale : h.scale / kEta0;
    for (size_t t = 0; t < (size_t)NX * NY; ++t) {
        float v;
        if (c->prec == FDTD_FP32) v = ((const float *)buf.data())[t];
        else v = __half2float(((const __half *)buf.data())[t]);
        out[t] = (float)(v * s);
    }
    return FDTD_OK;
}

int fdtd_diagnostics(fdtd_ctx *c, double *energy, double *max_div_b)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (c->host_step < 1) return fail(FDTD_ESTATE, "diagnostics need at least one completed step");
    double *part = c->energy_buf, *res = c->energy_buf + 2 * (size_t)c->energy_n;
    CK(launch_energy(c->d, c->h, part, c->energy_n, res, c->cur));
    if (int r = fdtd_sync(c)) return r;
    double two[2];
    CK(cudaMemcpy(two, res, sizeof(two), cudaMemcpyDeviceToHost));
    const double s = c->h.scale;
    if (energy) *energy = 0.5 * kEps0 * c->g.dx * c->g.dy * c->g.dz * s * s * two[0];
    if (max_div_b) *max_div_b = s / (kC0 * kC0 * c->dt) * two[1];
    return FDTD_OK;
}

int fdtd_reset(fdtd_ctx *c)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    Board &h = c->h;
    const size_t fbytes = (size_t)h.nodes * elem_size(c->prec);
    for (int p = 0; p < 3; ++p)
        for (int f = 0; f < 6; ++f)
            if (h.f[p][f]) CK(cudaMemsetAsync(h.f[p][f], 0, fbytes, c->cur));
    for (int s = 0; s < h.n_slab; ++s)
        for (int a = 0; a < 6; ++a)
            if (h.slab[s].aux[a]) CK(cudaMemsetAsync(h.slab[s].aux[a], 0, sizeof(float) * (size_t)h.slab[s].n, c->cur));
    for (int bx = 0; bx < 2; ++bx) {
        if (h.zD[bx]) CK(cudaMemsetAsync(h.zD[bx], 0, sizeof(float) * c->zaux_n[bx], c->cur));
        for (int p = 0; p < 2; ++p)
            if (h.zB[bx][p]) CK(cudaMemsetAsync(h.zB[bx][p], 0, sizeof(float) * c->zaux_n[bx], c->cur));
    }
    if (h.trace) CK(cudaMemsetAsync(h.trace, 0, sizeof(float) * (size_t)h.n_probe * h.n_total, c->cur));
    if (h.dft) CK(cudaMemsetAsync(h.dft, 0, sizeof(double) * 2 * (size_t)h.n_probe * std::max(h.n_bins, 1), c->cur));
    CK(cudaMemsetAsync(h.step, 0, sizeof(long long), c->cur));
    CK(cudaMemsetAsync(h.dft_done, 0, sizeof(long long), c->cur));
    CK(cudaMemsetAsync(h.status, 0, sizeof(int), c->cur));
    c->host_step = 0;
    return FDTD_OK;
}

namespace {

// Checkpoint header: identifies the board the state belongs to.
struct CkptHeader {
    uint64_t magic;
    int32_t version;
    int32_t nx, ny, nz, pitch, prec, n_probe, n_src, n_total, n_bins, n_slab;
    float scale;
    int32_t pad;
    int64_t nodes, step, dft_done;
    double dt;
};
constexpr uint64_t kCkptMagic = 0x31544b43445446ull;   // "FDTDCKT1"

// Device regions of the state after `step` steps, in checkpoint order: the
// field sets holding the states after steps n and n - 1 (in that order,
// whichever sets they occupy), then the auxiliaries, trace and DFT.
void ckpt_regions(const fdtd_ctx *c, long long step, std::vector<std::pair<void *, size_t>> &out)
{
    const Board &h = c->h;
    const size_t fbytes = (size_t)h.nodes * elem_size(c->prec);
    for (int p : {set_of(h.tdepth, step), set_of(h.tdepth, step - 1)})
        for (int f = 0; f < 6; ++f) out.push_back({h.f[p][f], fbytes});
    for (int s = 0; s < h.n_slab; ++s)
        for (int a = 0; a < 6; ++a)
            if (h.slab[s].aux[a]) out.push_back({h.slab[s].aux[a], sizeof(float) * (size_t)h.slab[s].n});
    for (int bx = 0; bx < 2; ++bx) {
        if (h.zD[bx]) out.push_back({h.zD[bx], sizeof(float) * c->zaux_n[bx]});
        for (int p = 0; p < 2; ++p)
            if (h.zB[bx][p]) out.push_back({h.zB[bx][p], sizeof(float) * c->zaux_n[bx]});
    }
    if (h.trace) out.push_back({h.trace, sizeof(float) * (size_t)h.n_probe * h.n_total});
    if (h.dft) out.push_back({h.dft, sizeof(double) * 2 * (size_t)h.n_probe * std::max(h.n_bins, 1)});
}

CkptHeader ckpt_header(const fdtd_ctx *c)
{
    const Board &h = c->h;
    CkptHeader H{};
    H.magic = kCkptMagic;
    H.version = 2;
    H.nx = h.nx; H.ny = h.ny; H.nz = h.nz; H.pitch = h.pitch; H.prec = c->prec;
    H.n_probe = (int)c->probe.size(); H.n_src = (int)c->src.size();
    H.n_total = h.n_total; H.n_bins = h.n_bins; H.n_slab = h.n_slab;
    H.scale = h.scale;
    H.nodes = h.nodes;
    H.dt = c->dt;
    return H;
}

}  // namespace

int fdtd_save(fdtd_ctx *c, void *buf, size_t cap, size_t *size)
{
    if (!c || !size) return fail(FDTD_EINVAL, "NULL argument");
    if (c->batch) return fail(FDTD_ESTATE, "context is in a batch; remove it first");
    if (int r = finalize(c)) return r;
    std::vector<std::pair<void *, size_t>> reg;
    CK(cudaStreamSynchronize(c->cur));
    ckpt_regions(c, c->host_step, reg);
    size_t need = sizeof(CkptHeader);
    for (auto &g : reg) need += g.second;
    *size = need;
    if (!buf || cap < need) return FDTD_OK;
    CkptHeader H = ckpt_header(c);
    long long ctr[2] = {0, 0};
    CK(cudaMemcpyAsync(&ctr[0], c->h.step, sizeof(long long), cudaMemcpyDeviceToHost, c->cur));
    CK(cudaMemcpyAsync(&ctr[1], c->h.dft_done, sizeof(long long), cudaMemcpyDeviceToHost, c->cur));
    unsigned char *o = static_cast<unsigned char *>(buf) + sizeof(CkptHeader);
    for (auto &g : reg) {
        CK(cudaMemcpyAsync(o, g.first, g.second, cudaMemcpyDeviceToHost, c->cur));
        o += g.second;
    }
    CK(cudaStreamSynchronize(c->cur));
    H.step = ctr[0];
    H.dft_done = ctr[1];
    std::memcpy(buf, &H, sizeof(H));
    return check_status(c);
}

int fdtd_load(fdtd_ctx *c, const void *buf, size_t size)
{
    if (!c || !buf) return fail(FDTD_EINVAL, "NULL argument");
    if (c->batch) return fail(FDTD_ESTATE, "context is in a batch; remove it first");
    if (size < sizeof(CkptHeader)) return fail(FDTD_EINVAL, "checkpoint too small");
    if (int r = finalize(c)) return r;
    CkptHeader H;
    std::memcpy(&H, buf, sizeof(H));
    const CkptHeader M = ckpt_header(c);
    if (H.magic != kCkptMagic || H.version != M.version) return fail(FDTD_EINVAL, "not an fdtd checkpoint");
    if (H.nx != M.nx || H.ny != M.ny || H.nz != M.nz || H.pitch != M.pitch || H.prec != M.prec ||
        H.n_probe != M.n_probe || H.n_src != M.n_src || H.n_total != M.n_total || H.n_bins != M.n_bins ||
        H.n_slab != M.n_slab || H.scale != M.scale || H.nodes != M.nodes || H.dt != M.dt)
        return fail(FDTD_EINVAL, "checkpoint belongs to a different board or settings");
    if (H.step < 0 || H.dft_done < 0 || H.dft_done > H.step) return fail(FDTD_EINVAL, "corrupt checkpoint counters");
    std::vector<std::pair<void *, size_t>> reg;
    ckpt_regions(c, H.step, reg);
    size_t need = sizeof(CkptHeader);
    for (auto &g : reg) need += g.second;
    if (size != need) return fail(FDTD_EINVAL, "checkpoint size does not match this board");
    const unsigned char *in = static_cast<const unsigned char *>(buf) + sizeof(CkptHeader);
    for (auto &g : reg) {
        CK(cudaMemcpyAsync(g.first, in, g.second, cudaMemcpyHostToDevice, c->cur));
        in += g.second;
    }
    const long long ctr[2] = {H.step, H.dft_done};
    CK(cudaMemcpyAsync(c->h.step, &ctr[0], sizeof(long long), cudaMemcpyHostToDevice, c->cur));
    CK(cudaMemcpyAsync(c->h.dft_done, &ctr[1], sizeof(long long), cudaMemcpyHostToDevice, c->cur));
    CK(cudaMemsetAsync(c->h.status, 0, sizeof(int), c->cur));
    CK(cudaStreamSynchronize(c->cur));
    c->host_step = H.step;
    return FDTD_OK;
}

int fdtd_selftest_wait_timeout(void *stream, unsigned max_polls)
{
    cudaStream_t st = (cudaStream_t)stream;
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) { cudaGetLastError(); return fail(FDTD_ECUDA, "selftest allocation failed"); }
    int status = 0;
    e = cudaMemsetAsync(d, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_wait_selftest(d, max_polls ? max_polls : (1u << 21), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    if (status & 2) return fail(FDTD_ETIMEOUT, "bounded device wait gave up (self-test: expected)");
    return FDTD_OK;
}

namespace {

// Node plane `p` along `axis` of one field array as a 2D copy: `height` rows
// of `width` elements, `spitch` elements apart, starting `off` elements in.
// (x planes: one element per (j, k) row, the rows a pitch apart; y planes:
// one x row per k, a plane apart; z planes: the ny+1 x rows of plane p.)
struct PlaneGeom {
    size_t off, width, height, spitch;
};

bool plane_geom(const Board &h, int axis, int p, PlaneGeom &g)
{
    const int n[3] = {h.nx, h.ny, h.nz};
    if (axis < 0 || axis > 2 || p < 0 || p > n[axis]) return false;
    if (axis == 0) g = {(size_t)p, 1, (size_t)(h.ny + 1) * (h.nz + 1), (size_t)h.pitch};
    else if (axis == 1) g = {(size_t)p * h.pitch, (size_t)h.nx + 1, (size_t)h.nz + 1, (size_t)h.plane};
    else g = {(size_t)p * h.plane, (size_t)h.nx + 1, (size_t)h.ny + 1, (size_t)h.pitch};
    return true;
}

int check_halo(const fdtd_ctx *c, int axis, int plane, unsigned mask, PlaneGeom &g)
{
    if (!c) return fail(FDTD_EINVAL, "NULL context");
    if (c->batch) return fail(FDTD_ESTATE, "context is in a batch");
    if (mask == 0 || (mask & ~0x3Fu)) return fail(FDTD_EINVAL, "component mask must be a non-empty subset of 0x3F");
    if (!plane_geom(c->h, axis, plane, g)) return fail(FDTD_EINVAL, "axis must be 0..2 and plane 0..n along it");
    return FDTD_OK;
}

}  // namespace

int fdtd_halo_pack(fdtd_ctx *c, int axis, int plane, unsigned comp_mask, void *dev_buf)
{
    PlaneGeom g{};
    if (int r = check_halo(c, axis, plane, comp_mask, g)) return r;
    if (!dev_buf) return fail(FDTD_EINVAL, "NULL buffer");
    if (int r = finalize(c)) return r;
    const size_t es = elem_size(c->prec);
    const int par = set_of(c->h.tdepth, c->host_step);
    unsigned char *o = static_cast<unsigned char *>(dev_buf);
    for (int f = 0; f < 6; ++f) {
        if (!(comp_mask & (1u << f))) continue;
        const unsigned char *src = static_cast<const unsigned char *>(c->h.f[par][f]) + g.off * es;
        CK(cudaMemcpy2DAsync(o, g.width * es, src, g.spitch * es, g.width * es, g.height, cudaMemcpyDeviceToDevice,
                             c->cur));
        o += g.width * g.height * es;
    }
    return FDTD_OK;
}

int fdtd_halo_unpack(fdtd_ctx *c, int axis, int plane, unsigned comp_mask, const void *dev_buf)
{
    PlaneGeom g{};
    if (int r = check_halo(c, axis, plane, comp_mask, g)) return r;
    if (!dev_buf) return fail(FDTD_EINVAL, "NULL buffer");
    if (int r = finalize(c)) return r;
    const size_t es = elem_size(c->prec);
    const int par = set_of(c->h.tdepth, c->host_step);
    const unsigned char *in = static_cast<const unsigned char *>(dev_buf);
    for (int f = 0; f < 6; ++f) {
        if (!(comp_mask & (1u << f))) continue;
        unsigned char *dst = static_cast<unsigned char *>(c->h.f[par][f]) + g.off * es;
        CK(cudaMemcpy2DAsync(dst, g.spitch * es, in, g.width * es, g.width * es, g.height, cudaMemcpyDeviceToDevice,
                             c->cur));
        in += g.width * g.height * es;
    }
    return FDTD_OK;
}

int fdtd_halo_copy(fdtd_ctx *dst, int dst_plane, fdtd_ctx *src, int src_plane, int axis, unsigned comp_mask)
{
    PlaneGeom gd{}, gs{};
    if (int r = check_halo(dst, axis, dst_plane, comp_mask, gd)) return r;
    if (int r = check_halo(src, axis, src_plane, comp_mask, gs)) return r;
    if (dst == src) return fail(FDTD_EINVAL, "source and destination must be different contexts");
    if (dst->prec != src->prec) return fail(FDTD_EINVAL, "the two contexts store fields in different precisions");
    if (gd.width != gs.width || gd.height != gs.height)
        return fail(FDTD_EINVAL, "the planes differ in shape (the sub-boards must agree on the two other axes)");
    if (dst->host_step != src->host_step) return fail(FDTD_ESTATE, "the two contexts are at different steps");
    if (int r = finalize(dst)) return r;
    if (int r = finalize(src)) return r;
    if (src->h.scale != dst->h.scale) return fail(FDTD_EINVAL, "the two contexts use different storage scales");
    // the copy runs on the destination's stream once the source's queued work is done
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, src->cur);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(dst->cur, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(e, "halo copy ordering");
    const size_t es = elem_size(dst->prec);
    const int spar = set_of(src->h.tdepth, src->host_step), dpar = set_of(dst->h.tdepth, dst->host_step);
    for (int f = 0; f < 6; ++f) {
        if (!(comp_mask & (1u << f))) continue;
        cudaMemcpy3DPeerParms p{};
        p.srcPtr = make_cudaPitchedPtr(static_cast<unsigned char *>(src->h.f[spar][f]) + gs.off * es, gs.spitch * es,
                                       gs.width * es, gs.height);
        p.srcDevice = src->device;
        p.dstPtr = make_cudaPitchedPtr(static_cast<unsigned char *>(dst->h.f[dpar][f]) + gd.off * es, gd.spitch * es,
                                       gd.width * es, gd.height);
        p.dstDevice = dst->device;
        p.extent = make_cudaExtent(gs.width * es, gs.height, 1);
        CK(cudaMemcpy3DPeerAsync(&p, dst->cur));
    }
    return FDTD_OK;
}

int fdtd_set_materials(fdtd_ctx *c, const uint8_t *mat_ids)
{
    if (!c || !mat_ids) return fail(FDTD_EINVAL, "NULL argument");
    if (c->batch) return fail(FDTD_ESTATE, "context is in a batch");
    if (int r = set_geometry(c, mat_ids)) return r;
    // sources keep their edge; refresh their coefficient for the new permittivity
    if (!c->src.empty()) {
        for (Source &S : c->src) {
            const float4 row = c->ctab[edge_combo(c, S.node)];
            const float ce = S.comp == 0 ? row.x : S.comp == 1 ? row.y : row.z;
            if (ce == 0.0f) return fail(FDTD_EINVAL, "a source edge became PEC");
            if (S.kind == kSrcCurrent)
                S.coef = (double)ce * c->dt / kEps0 / (c->started ? c->h.scale : 1.0);
            else
                vsource_coef(c, S, ce, c->started ? c->h.scale : 1.0);
        }
        if (c->started)
            CK(cudaMemcpyAsync((void *)c->h.src, c->src.data(), sizeof(Source) * c->src.size(), cudaMemcpyHostToDevice,
                               c->cur));
    }
    return fdtd_reset(c);
}

int fdtd_node_coefficients(const fdtd_grid *grid, const uint8_t *mat_ids, const double *eps_r, int n_mat,
                           const fdtd_box *pec, int n_pec, const uint8_t *pec_mask, const fdtd_boundary *bnd,
                           uint16_t *ids, float *table, int max_rows, int *n_rows)
{
    if (!ids || !table || !n_rows || max_rows < 1) return fail(FDTD_EINVAL, "NULL output or max_rows < 1");
    if (int r = check_problem(grid, mat_ids, eps_r, n_mat, pec, n_pec, bnd)) return r;
    // a host-only context holding what the id precompute reads; no device work
    fdtd_ctx c;
    c.g = *grid;
    c.bnd = *bnd;
    c.eps.assign(eps_r, eps_r + n_mat);
    if (n_pec > 0) c.boxes.assign(pec, pec + n_pec);
    if (pec_mask) c.mask.assign(pec_mask, pec_mask + (size_t)grid->nx * grid->ny * grid->nz);
    c.h.pitch = row_pitch(grid->nx);
    const int NX = grid->nx + 1, NY = grid->ny + 1, NZ = grid->nz + 1;
    IdScratch &scratch = id_scratch();
    std::lock_guard<std::mutex> hold(scratch.lock);
    NodeIds nid;
    nid.n = (size_t)c.h.pitch * NY * NZ;
    try {
        scratch.reserve(nid.n);
    } catch (const std::bad_alloc &) {
        return fail(FDTD_ENOMEM, "host scratch for the coefficient ids");
    }
    nid.cid = scratch.cid.get();
    nid.c8 = scratch.c8.get();
    std::vector<float4> tab;
    if (int r = build_combo(&c, mat_ids, nid, tab)) return r;
    if ((int)tab.size() > max_rows) return fail(FDTD_EINVAL, "more coefficient triples than max_rows");
    *n_rows = (int)tab.size();
    for (size_t t = 0; t < tab.size(); ++t) {
        table[4 * t] = tab[t].x;
        table[4 * t + 1] = tab[t].y;
        table[4 * t + 2] = tab[t].z;
        table[4 * t + 3] = 0.0f;
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; ++k)
        for (int j = 0; j < NY; ++j) {
            const size_t src = ((size_t)k * NY + j) * c.h.pitch, dst = ((size_t)k * NY + j) * NX;
            for (int i = 0; i < NX; ++i) ids[dst + i] = nid.wide ? nid.cid[src + i] : (uint16_t)nid.c8[src + i];
        }
    return FDTD_OK;
}

int fdtd_device_bytes(const fdtd_grid *grid, const fdtd_boundary *bnd, int precision, int n_sources, int n_probes,
                      int n_total_steps, double f_max, long long *bytes)
{
    if (!grid || !bnd || !bytes) return fail(FDTD_EINVAL, "NULL argument");
    if (precision != FDTD_FP32 && precision != FDTD_FP16_STORE)
        return fail(FDTD_EINVAL, "precision must be FDTD_FP32 or FDTD_FP16_STORE");
    if (n_sources < 0 || n_probes < 0 || n_total_steps < 0) return fail(FDTD_EINVAL, "negative count");
    const double one = 1.0;
    const uint8_t mat0 = 0;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(FDTD_EINVAL, "grid must have at least one cell per axis");
    if (int r = check_problem(grid, &mat0, &one, 1, nullptr, 0, bnd)) return r;
    const long long pitch = row_pitch(grid->nx);
    const long long nodes = pitch * (grid->ny + 1) * (grid->nz + 1);
    const double dt = grid_dt(*grid);
    Axes A;
    build_axes(*grid, *bnd, dt, A);
    std::unique_ptr<Board> hb(new Board());
    Board &h = *hb;
    h.nx = grid->nx; h.ny = grid->ny; h.nz = grid->nz;
    h.prec = precision;
    bool aux[kMaxSlab][6];
    long long zplanes[2] = {0, 0};
    if (!layout_board(*grid, *bnd, A, h, aux, zplanes)) return fail(FDTD_EINVAL, "internal: too many slab boxes");
    auto al = [](long long b) { return b > 0 ? b : 16LL; };   // as the allocator rounds empty requests
    long long t = 2 * al(6 * nodes * elem_size(precision));                    // both field parities
    t += al(nodes * 2) + al((long long)sizeof(float4) * kMaxCombo16);         // 16-bit ids and their table (upper bound)
    for (int w = 0; w < 3; ++w) t += 2 * al((long long)sizeof(Coef) * A.cw[w][0].size());   // UPML factors
    for (int s = 0; s < h.n_slab; ++s)
        for (int comp = 0; comp < 6; ++comp)
            if (aux[s][comp]) t += al(4 * h.slab[s].n);
    for (int bx = 0; bx < 2; ++bx)
        if (zplanes[bx]) t += 3 * al(4 * zplanes[bx] * h.zpitch * (h.iy1 - h.iy0));
    t += al(4 * sizeof(long long)) + al(sizeof(Board));
    t += al((long long)sizeof(double) * (2 * (long long)energy_partials(h) + 2));
    if (h.ix1 > h.ix0) t += al((long long)sizeof(CUtensorMap) * kNumMaps);
    if (n_sources) t += al((long long)sizeof(Source) * n_sources);
    if (n_probes) t += al((long long)sizeof(Probe) * n_probes);
    if (n_total_steps > 0 && n_probes > 0) {
        const int nyq = n_total_steps / 2 + 1;
        int Q = nyq;
        if (f_max > 0) Q = std::min(nyq, (int)std::floor(f_max * n_total_steps * dt + 1e-9) + 1);
        t += al(4LL * n_probes * n_total_steps) + al(16LL * n_probes * std::max(Q, 1));
    }
    *bytes = t;
    return FDTD_OK;
}

int fdtd_info(fdtd_ctx *c, fdtd_info_t *info)
{
    if (!c || !info) return fail(FDTD_EINVAL, "NULL argument");
    CK(cudaStreamSynchronize(c->cur));
    long long st = 0;
    CK(cudaMemcpy(&st, c->h.step, sizeof(st), cudaMemcpyDeviceToHost));
    const Board &h = c->h;
    info->nx = h.nx; info->ny = h.ny; info->nz = h.nz;
    info->dt = c->dt;
    info->step = st;
    info->n_sources = (int)c->src.size();
    info->n_probes = (int)c->probe.size();
    info->n_total_steps = h.n_total;
    info->n_bins = h.n_bins;
    info->precision = c->prec;
    const long long Lx = h.ix1 - h.ix0, Ly = h.iy1 - h.iy0, Lz = (long long)h.nz - h.zlo;
    info->interior_nodes = (Lx > 0 && Ly > 0 && Lz > 0) ? Lx * Ly * Lz : 0;
    info->fused_upml_nodes = info->interior_nodes > 0 ? Lx * Ly * (c->zplanes[0] + c->zplanes[1]) : 0;
    long long sn = 0, sa = 0;
    for (int s = 0; s < h.n_slab; ++s) {
        sn += h.slab[s].n;
        for (int a = 0; a < 6; ++a)
            if (h.slab[s].aux[a]) sa += h.slab[s].n;
    }
    info->slab_nodes = sn;
    info->slab_aux_values = sa;
    info->pitch = h.pitch;
    info->depth = h.pair_ok ? 2 : 1;
    info->device_bytes = c->device_bytes;
    info->n_combo = c->n_combo;
    return FDTD_OK;
}

void fdtd_destroy(fdtd_ctx *c)
{
    if (!c) return;
    if (c->batch) fdtd_batch_remove(c->batch, c);
    if (c->cur) cudaStreamSynchronize(c->cur);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph2) cudaGraphExecDestroy(c->graph2);
    if (c->plan_buf) cudaFree(c->plan_buf);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    for (void *p : c->allocs) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

// --------------------------------------------------------------------------- batch

int fdtd_batch_create(void *stream, fdtd_batch **out)
{
    if (!out) return fail(FDTD_EINVAL, "out is NULL");
    fdtd_batch *b = new fdtd_batch();
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
        b->own_stream = true;
    }
    b->grid_cap = device_grid_cap();
    *out = b;
    return FDTD_OK;
}

int fdtd_batch_set_tuning(fdtd_batch *b, const fdtd_tuning *t)
{
    if (!b || !t) return fail(FDTD_EINVAL, "NULL argument");
    fdtd_tuning n = b->tune;
    if (t->tile_x > 0) n.tile_x = t->tile_x;
    if (t->tile_y > 0) n.tile_y = t->tile_y;
    if (t->zseg > 0) n.zseg = t->zseg;
    if (t->graph_chunk > 0) n.graph_chunk = t->graph_chunk;
    if (t->depth > 1) return fail(FDTD_EINVAL, "a batch steps one leapfrog step per launch set (depth 1)");
    if (!fused_tile_supported(n.tile_x, n.tile_y))
        return fail(FDTD_EINVAL, "fused tile (tile_x x tile_y) must be 62x4, 62x8, 124x4 or 124x8");
    b->tune = n;
    b->dirty = true;
    return FDTD_OK;
}

int fdtd_batch_add(fdtd_batch *b, fdtd_ctx *c, int n_steps)
{
    if (!b || !c) return fail(FDTD_EINVAL, "NULL argument");
    if (c->batch) return fail(FDTD_EINVAL, "context already in a batch");
    if (n_steps < 0) return fail(FDTD_EINVAL, "n_steps must be >= 0");
    if (b->prec >= 0 && !b->members.empty() && c->prec != b->prec)
        return fail(FDTD_EINVAL, "all boards of a batch must share the precision mode");
    CK(cudaStreamSynchronize(c->cur));
    c->cur = b->stream;
    if (int r = finalize(c)) { c->cur = c->stream; return r; }
    CK(launch_set_i64(c->h.stop, c->host_step + n_steps, b->stream));
    c->batch = b;
    b->members.push_back(c);
    b->remaining.push_back(n_steps);
    b->prec = c->prec;
    b->dirty = true;
    return FDTD_OK;
}

int fdtd_batch_remove(fdtd_batch *b, fdtd_ctx *c)
{
    if (!b || !c) return fail(FDTD_EINVAL, "NULL argument");
    auto it = std::find(b->members.begin(), b->members.end(), c);
    if (it == b->members.end()) return fail(FDTD_EINVAL, "context not in this batch");
    CK(cudaStreamSynchronize(b->stream));
    const size_t k = it - b->members.begin();
    b->members.erase(it);
    b->remaining.erase(b->remaining.begin() + k);
    c->batch = nullptr;
    c->cur = c->stream;
    CK(launch_set_i64(c->h.stop, LLONG_MAX, c->cur));
    b->dirty = true;
    return FDTD_OK;
}

int fdtd_batch_step(fdtd_batch *b, int n, int *n_done)
{
    if (!b) return fail(FDTD_EINVAL, "NULL batch");
    if (n < 0) return fail(FDTD_EINVAL, "n must be >= 0");
    long long most = 0;
    for (long long r : b->remaining) most = std::max(most, r);
    const int run = (int)std::min<long long>(n, most);
    if (run > 0 && !b->members.empty()) {
        if (b->dirty) {
            for (fdtd_ctx *m : b->members)
                if (int r = encode_maps(m, b->tune.tile_x, b->tune.tile_y)) return r;
            std::vector<long long> host;
            if (int r = build_plan(b->members, b->tune, b->plan_buf, b->plan_cap, b->plan, b->stream, host)) return r;
            CK(cudaStreamSynchronize(b->stream));
            if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
            b->dirty = false;
        }
        if (int r = run_steps(b->plan, b->prec, b->grid_cap, run, b->tune.graph_chunk, b->graph, b->graph_chunk,
                              b->stream))
            return r;
        for (size_t m = 0; m < b->members.size(); ++m) {
            const long long did = std::min<long long>(run, b->remaining[m]);
            b->remaining[m] -= did;
            b->members[m]->host_step += did;
        }
    }
    if (n_done) {
        int d = 0;
        for (long long r : b->remaining) d += (r == 0);
        *n_done = d;
    }
    return FDTD_OK;
}

int fdtd_batch_remaining(fdtd_batch *b, fdtd_ctx *c, long long *remaining)
{
    if (!b || !c || !remaining) return fail(FDTD_EINVAL, "NULL argument");
    auto it = std::find(b->members.begin(), b->members.end(), c);
    if (it == b->members.end()) return fail(FDTD_EINVAL, "context not in this batch");
    *remaining = b->remaining[it - b->members.begin()];
    return FDTD_OK;
}

int fdtd_batch_sync(fdtd_batch *b)
{
    if (!b) return fail(FDTD_EINVAL, "NULL batch");
    CK(cudaStreamSynchronize(b->stream));
    for (fdtd_ctx *c : b->members)
        if (int r = check_status(c)) return r;
    return FDTD_OK;
}

void fdtd_batch_destroy(fdtd_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (fdtd_ctx *c : b->members) {
        c->batch = nullptr;
        c->cur = c->stream;
        launch_set_i64(c->h.stop, LLONG_MAX, c->cur);
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->plan_buf) cudaFree(b->plan_buf);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
