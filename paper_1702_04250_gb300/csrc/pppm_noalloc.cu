// Allocation-free mesh charge assignment (particle_map + sort + make_rho).
//
// Some callers cannot allocate device memory at the point where they need a
// charge mesh: a host MD engine that owns all GPU memory through its own pool
// and budget, or a latency-critical step loop that must not pay the implicit
// device-wide synchronisation of cudaMalloc/cudaFree.  For them
// pppm_make_rho_noalloc builds the mesh without any allocation: the sort
// scratch that a plan would own lives in one file-scope device array of fixed
// size, which every GPU that loads this library keeps until the process exits.
// The caller still passes the inputs and the output mesh.
//
// Consequences a caller must respect:
//  - All calls share the same scratch array, so calls that may overlap on the
//    GPU (different streams, or several host threads) race and corrupt each
//    other's result.  Serialise them (one stream is enough).
//  - The first call on each device looks up the array's device address (and
//    sets the kernels' shared-memory limits) and caches both for the life of
//    the process; make that first call before any stream capture, and do not
//    reset the device (cudaDeviceReset) between calls.
//  - Sizes beyond the fixed limits are rejected with PPPM_EINVAL before any
//    GPU work.
//  - Non-finite inputs and failed consistency checks are flagged in an error
//    word inside the array; pppm_make_rho_noalloc_status reads it back.  The
//    next call clears it.
#include <cmath>
#include <mutex>

#include "pppm_common.cuh"

namespace pppm {
namespace {

constexpr int64_t NA_MAX_N = 65536;     // particles per call
constexpr int NA_MAX_TILES = 4096;      // mesh tiles (e.g. up to 128^3 points)
constexpr int NA_MAP_BLOCKS = (int)((NA_MAX_N + 255) / 256);

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t OFF_ANCHOR = 0;
constexpr size_t OFF_RANK = OFF_ANCHOR + align256(4 * NA_MAX_N);
constexpr size_t OFF_PERM = OFF_RANK + align256(4 * NA_MAX_N);
constexpr size_t OFF_CELL = OFF_PERM + align256(4 * NA_MAX_N);
constexpr size_t OFF_REC = OFF_CELL + align256(4 * NA_MAX_N);
constexpr size_t OFF_COUNT = OFF_REC + align256(16 * NA_MAX_N);
constexpr size_t OFF_START = OFF_COUNT + align256(4 * NA_MAX_TILES);
constexpr size_t OFF_BLK = OFF_START + align256(4 * (NA_MAX_TILES + 1));
constexpr size_t OFF_MISC = OFF_BLK + align256(16 * NA_MAP_BLOCKS);  // err, (16 unused), qsum
constexpr size_t NA_BYTES = OFF_MISC + 256;                          // ~2.1 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[NA_MAX_DEVICES] = {nullptr};

int scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return PPPM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return PPPM_ECUDA;
        // kernel attributes (shared-memory sizes) of every order, once per device
        for (int P = 2; P <= MAXP; ++P)
            if (prepare_make_rho<float>(P, true) != cudaSuccess || prepare_make_rho<float>(P, false) != cudaSuccess)
                return PPPM_ECUDA;
        g_addr[dev] = reinterpret_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return PPPM_OK;
}

}  // namespace
}  // namespace pppm

using namespace pppm;

extern "C" int pppm_make_rho_noalloc(const double box[3], const int mesh[3], int order, int precision,
                                     int64_t n, const float *x, const float *q, float *rho,
                                     void *cuda_stream) {
    if (!box || !mesh || !rho) return PPPM_EINVAL;
    if (order < 2 || order > MAXP) return PPPM_EINVAL;
    if (precision != PPPM_FP32 && precision != PPPM_FP32C) return PPPM_EINVAL;
    if (n < 0 || n > NA_MAX_N) return PPPM_EINVAL;
    if (n > 0 && (!x || !q)) return PPPM_EINVAL;
    int T[3], TE[3];
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0) || !std::isfinite(box[d]) || mesh[d] < order || mesh[d] > MAX_MESH) return PPPM_EINVAL;
        // the kernels work with float copies of L, 1/L and M/L: each must be a finite normal float
        const float fl = (float)box[d], fil = (float)(1.0 / box[d]), fih = (float)((double)mesh[d] / box[d]);
        if (!std::isnormal(fl) || !std::isnormal(fil) || !std::isnormal(fih)) return PPPM_EINVAL;
    }
    tile_shape(mesh, false, T, TE);
    const int ntiles = T[0] * T[1] * T[2];
    if (ntiles > NA_MAX_TILES) return PPPM_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PPPM_ECUDA;
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // geometry and the order-P polynomials (host, on the stack)
    double coef[MAXP][MAXP], dcoef[MAXP][MAXP];
    stencil_polynomials(order, coef, dcoef);
    Geom<float> g{};
    double vcell = 1.0;
    for (int d = 0; d < 3; ++d) {
        const double ih = (double)mesh[d] / box[d];
        g.M[d] = mesh[d];
        g.T[d] = T[d];
        g.TE[d] = TE[d];
        g.L[d] = (float)box[d];
        g.iL[d] = (float)(1.0 / box[d]);
        g.ih[d] = (float)ih;
        g.ih_lo[d] = (float)(ih - (double)(float)ih);
        g.h[d] = (float)(box[d] / mesh[d]);
        vcell *= box[d] / mesh[d];
    }
    g.Mzh = mesh[2] / 2 + 1;
    g.ntiles = ntiles;
    g.P = order;
    g.rlo = (order - 1) / 2;
    g.ivcell = (float)(1.0 / vcell);
    for (int k = 0; k < MAXP; ++k)
        for (int l = 0; l < MAXP; ++l) {
            g.coef[k][l] = (float)coef[k][l];
            g.dcoef[k][l] = (float)dcoef[k][l];
        }
    {
        const double wm = stencil_weight_max(order, coef);
        g.wmax3 = (float)(wm * wm * wm * (1.0 + 1e-6));
    }

    SortBufs b{};
    b.anchor = reinterpret_cast<uint32_t *>(base + OFF_ANCHOR);
    b.rank = reinterpret_cast<int *>(base + OFF_RANK);
    b.perm = reinterpret_cast<int *>(base + OFF_PERM);
    b.cell = reinterpret_cast<uint32_t *>(base + OFF_CELL);
    b.rec = base + OFF_REC;
    b.tile_count = reinterpret_cast<int *>(base + OFF_COUNT);
    b.tile_start = reinterpret_cast<int *>(base + OFF_START);
    b.blk = reinterpret_cast<double *>(base + OFF_BLK);
    b.err = reinterpret_cast<int *>(base + OFF_MISC);
    b.qsum = reinterpret_cast<double *>(base + OFF_MISC + 32);

    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(b.tile_count, 0, 4 * (size_t)ntiles, s) != cudaSuccess) return PPPM_ECUDA;
    if (cudaMemsetAsync(base + OFF_MISC, 0, 256, s) != cudaSuccess) return PPPM_ECUDA;
    if (n > 0) launch_sort<float>(g, n, x, q, b, s);
    launch_make_rho<float>(g, n, b, rho, precision == PPPM_FP32C, s);
    return cudaGetLastError() == cudaSuccess ? PPPM_OK : PPPM_ECUDA;
}

extern "C" int pppm_make_rho_noalloc_status(void *cuda_stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PPPM_ECUDA;
    unsigned char *base = nullptr;
    const int rc = scratch_address(dev, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int err = 0;  // host stack word: a pageable copy, complete once the stream is synchronised
    if (cudaMemcpyFromSymbolAsync(&err, g_noalloc_scratch, sizeof(int), OFF_MISC, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return PPPM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PPPM_ECUDA;
    if (err & ERR_NONFINITE) return PPPM_ENONFINITE;
    if (err & ERR_INTERNAL) return PPPM_EINTERNAL;
    return PPPM_OK;
}
