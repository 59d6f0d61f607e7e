// fdtd_static.cu -- fdtd_energy_static: the discrete field energy and max
// |div B| of caller-owned fields, computed without allocating anything.
//
// Why it exists: some callers cannot allocate device memory at the point
// where they need this check -- code under a memory pool or budget that must
// not grow, real-time loops that forbid allocator calls, or hosts that hand
// the library only pre-registered buffers.  They pass their fields as device
// pointers and get the two numbers back, and this call performs no
// cudaMalloc, cudaFree or other allocation.  It reads the two results back
// into host memory and synchronises the stream before it returns.
//
// The per-block partial sums live in a file-scope static __device__ array of
// a fixed size, which every GPU that loads the library holds until the
// process exits.  Host code may only use the array's device address obtained
// from cudaGetSymbolAddress (the symbol itself is a host-side stand-in): the
// first call on each device looks it up with that device current and caches
// it, so that first call should come before any stream capture.  The cache is
// keyed on the device's current CUDA context as well, so a call after
// cudaDeviceReset (a new primary context, with the array at a possibly new
// address) looks the address up again.  All calls share the array: two calls
// whose kernels overlap on the GPU race and both results are then undefined.
// Every call overwrites each partial it reads, so nothing carries over from
// the previous call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/fdtd.h"
#include "fdtd_internal.h"

namespace {

constexpr int kStaticThreads = 256;
constexpr long long kNodesPerBlock = 8192;
constexpr int kStaticBlocks = 4096;   // -> at most 33,554,432 nodes per call
constexpr int kMaxDevices = 64;

// per block: E sum, H sum, div max; then the reduced triple
static __device__ __align__(256) double g_energy_scratch[3 * kStaticBlocks + 3];

std::mutex g_mu;
struct ScratchAddr {
    CUcontext ctx = nullptr;      // context the address was resolved in
    double *ptr = nullptr;        // device address of the array there
};
ScratchAddr g_scratch_dev[kMaxDevices];   // per device ordinal

struct StaticArgs {
    const float *f[9];      // E^n (x,y,z), H^{n-1/2} (x,y,z), H^{n+1/2} (x,y,z)
    const float *eps[3];    // per-edge eps_r of E_x, E_y, E_z (nullptr = 1)
    int nx, ny, nz, pitch;
    int cx0, cx1, cy0, cy1, cz0, cz1;   // cells outside the UPML
    double ix, iy, iz;      // 1/dx, 1/dy, 1/dz
};

// max that keeps a NaN (fmax would drop it), so a field that has blown up
// shows in max |div B| as well as in the energy
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? NAN : fmax(a, b); }

// One block reduces nodes [b * kNodesPerBlock, (b + 1) * kNodesPerBlock):
// sum of dual-weighted eps_r E.E and H.H' and max |div H'| over cells
// outside the UPML.  A variant of the context's energy kernel on raw
// pointers, with its partials in the static array.
__global__ void __launch_bounds__(kStaticThreads) k_energy_static(StaticArgs a, double *scratch)
{
    const long long total = (long long)(a.nx + 1) * (a.ny + 1) * (a.nz + 1);
    const long long n0 = (long long)blockIdx.x * kNodesPerBlock;
    const long long n1 = n0 + kNodesPerBlock < total ? n0 + kNodesPerBlock : total;
    const long long X = a.pitch, P = (long long)a.pitch * (a.ny + 1);
    double esum = 0.0, hsum = 0.0, dmax = 0.0;
    for (long long t = n0 + threadIdx.x; t < n1; t += blockDim.x) {
        const int i = (int)(t % (a.nx + 1));
        const long long r = t / (a.nx + 1);
        const int j = (int)(r % (a.ny + 1));
        const int k = (int)(r / (a.ny + 1));
        const long long q = (long long)k * P + (long long)j * X + i;
        const double wx = (i == 0 || i == a.nx) ? 0.5 : 1.0;
        const double wy = (j == 0 || j == a.ny) ? 0.5 : 1.0;
        const double wz = (k == 0 || k == a.nz) ? 0.5 : 1.0;
        if (i < a.nx) { const double e = a.f[0][q]; esum += wy * wz * (a.eps[0] ? (double)a.eps[0][q] : 1.0) * e * e; }
        if (j < a.ny) { const double e = a.f[1][q]; esum += wx * wz * (a.eps[1] ? (double)a.eps[1][q] : 1.0) * e * e; }
        if (k < a.nz) { const double e = a.f[2][q]; esum += wx * wy * (a.eps[2] ? (double)a.eps[2][q] : 1.0) * e * e; }
        if (j < a.ny && k < a.nz) hsum += wx * (double)a.f[3][q] * a.f[6][q];
        if (i < a.nx && k < a.nz) hsum += wy * (double)a.f[4][q] * a.f[7][q];
        if (i < a.nx && j < a.ny) hsum += wz * (double)a.f[5][q] * a.f[8][q];
        if (i >= a.cx0 && i < a.cx1 && j >= a.cy0 && j < a.cy1 && k >= a.cz0 && k < a.cz1) {
            const double dv = ((double)a.f[6][q + 1] - a.f[6][q]) * a.ix + ((double)a.f[7][q + X] - a.f[7][q]) * a.iy +
                              ((double)a.f[8][q + P] - a.f[8][q]) * a.iz;
            dmax = nan_max(dmax, fabs(dv));
        }
    }
    __shared__ double se[kStaticThreads], sh[kStaticThreads], sd[kStaticThreads];
    se[threadIdx.x] = esum;
    sh[threadIdx.x] = hsum;
    sd[threadIdx.x] = dmax;
    __syncthreads();
    for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            se[threadIdx.x] += se[threadIdx.x + off];
            sh[threadIdx.x] += sh[threadIdx.x + off];
            sd[threadIdx.x] = nan_max(sd[threadIdx.x], sd[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[3 * blockIdx.x] = se[0];
        scratch[3 * blockIdx.x + 1] = sh[0];
        scratch[3 * blockIdx.x + 2] = sd[0];
    }
}

__global__ void __launch_bounds__(kStaticThreads) k_energy_static_final(double *scratch, int nblk)
{
    __shared__ double se[kStaticThreads], sh[kStaticThreads], sd[kStaticThreads];
    double a = 0.0, b = 0.0, m = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
        a += scratch[3 * t];
        b += scratch[3 * t + 1];
        m = nan_max(m, scratch[3 * t + 2]);
    }
    se[threadIdx.x] = a;
    sh[threadIdx.x] = b;
    sd[threadIdx.x] = m;
    __syncthreads();
    for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            se[threadIdx.x] += se[threadIdx.x + off];
            sh[threadIdx.x] += sh[threadIdx.x + off];
            sd[threadIdx.x] = nan_max(sd[threadIdx.x], sd[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[3 * kStaticBlocks] = se[0];
        scratch[3 * kStaticBlocks + 1] = sh[0];
        scratch[3 * kStaticBlocks + 2] = sd[0];
    }
}

int static_fail(int code, const std::string &m) { return fdtd::set_error(code, m.c_str()); }

// cuCtxGetCurrent from the driver, through the runtime's entry-point query
// (the library links only the runtime).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_getter()
{
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
        cudaGetLastError();
    }
    return fn;
}

// Device address of the static array on the current device, looked up with
// that device current once per (device, context).
int scratch_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(FDTD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(FDTD_EINVAL, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mu);
    CtxGetCurrentFn get_ctx = ctx_getter();
    if (!get_ctx) return static_fail(FDTD_ECUDA, "cuCtxGetCurrent is not available from the driver");
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    ScratchAddr &slot = g_scratch_dev[dev];
    if (!ctx || !slot.ptr || slot.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_scratch);   // makes the device's primary context current if none is
        if (e != cudaSuccess || !p)
            return static_fail(FDTD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx)
            return static_fail(FDTD_ECUDA, "no current CUDA context after cudaGetSymbolAddress");
        slot.ctx = ctx;
        slot.ptr = static_cast<double *>(p);
    }
    *out = slot.ptr;
    return FDTD_OK;
}

}  // namespace

extern "C" int fdtd_energy_static(const float *const fields[9], const float *const eps_r[3], int nx, int ny, int nz,
                                  int pitch, double dx, double dy, double dz, const int upml_depth[6], void *stream,
                                  double *energy, double *max_div_b)
{
    if (!fields) return static_fail(FDTD_EINVAL, "fields is NULL");
    for (int t = 0; t < 9; ++t)
        if (!fields[t]) return static_fail(FDTD_EINVAL, "a field pointer is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || pitch < nx + 1) return static_fail(FDTD_EINVAL, "bad grid size or pitch");
    if (!(dx > 0 && dy > 0 && dz > 0)) return static_fail(FDTD_EINVAL, "cell sizes must be positive");
    if (upml_depth) {
        // the div B window [d_lo, n - d_hi) reads one node past its last cell
        // along each axis, which stays inside the caller's arrays only for
        // depths that are >= 0 and do not overlap
        const int n3[3] = {nx, ny, nz};
        for (int w = 0; w < 3; ++w)
            if (upml_depth[2 * w] < 0 || upml_depth[2 * w + 1] < 0 || upml_depth[2 * w] + upml_depth[2 * w + 1] > n3[w])
                return static_fail(FDTD_EINVAL, "UPML depths must be >= 0 and the two depths of an axis at most its cells");
    }
    const long long total = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    const long long nblk = (total + kNodesPerBlock - 1) / kNodesPerBlock;
    if (nblk > kStaticBlocks)
        return static_fail(FDTD_EINVAL, "grid has " + std::to_string(total) + " nodes; fdtd_energy_static handles at most " +
                                            std::to_string((long long)kStaticBlocks * kNodesPerBlock));
    double *scratch = nullptr;
    if (int r = scratch_address(&scratch)) return r;

    StaticArgs a;
    for (int t = 0; t < 9; ++t) a.f[t] = fields[t];
    for (int t = 0; t < 3; ++t) a.eps[t] = eps_r ? eps_r[t] : nullptr;
    a.nx = nx; a.ny = ny; a.nz = nz; a.pitch = pitch;
    const int d[6] = {upml_depth ? upml_depth[0] : 0, upml_depth ? upml_depth[1] : 0, upml_depth ? upml_depth[2] : 0,
                      upml_depth ? upml_depth[3] : 0, upml_depth ? upml_depth[4] : 0, upml_depth ? upml_depth[5] : 0};
    a.cx0 = d[0]; a.cx1 = nx - d[1];
    a.cy0 = d[2]; a.cy1 = ny - d[3];
    a.cz0 = d[4]; a.cz1 = nz - d[5];
    a.ix = 1.0 / dx; a.iy = 1.0 / dy; a.iz = 1.0 / dz;
    cudaStream_t st = (cudaStream_t)stream;
    k_energy_static<<<(int)nblk, kStaticThreads, 0, st>>>(a, scratch);
    k_energy_static_final<<<1, kStaticThreads, 0, st>>>(scratch, (int)nblk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(FDTD_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    double res[3];
    e = cudaMemcpyAsync(res, scratch + 3 * kStaticBlocks, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_fail(FDTD_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
    const double mu0 = 4.0e-7 * 3.14159265358979323846, c0 = 299792458.0;
    const double eps0 = 1.0 / (mu0 * c0 * c0);
    const double V = dx * dy * dz;
    if (energy) *energy = 0.5 * V * (eps0 * res[0] + mu0 * res[1]);
    if (max_div_b) *max_div_b = mu0 * res[2];
    return FDTD_OK;
}
