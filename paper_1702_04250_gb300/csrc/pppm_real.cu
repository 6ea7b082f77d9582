// Real-space half of the Ewald split (Sec. 2.1: the short-range part of the
// Coulomb interaction, erfc(g r)/r, summed directly within the cut-off r_C;
// the k-space part is the PPPM path of the other files):
//   E   = (C/2) sum_i sum_{j != i, r_ij < r_C} q_i q_j erfc(g r_ij) / r_ij
//   F_i = C q_i sum_j q_j [erfc(g r)/r + (2g/sqrt(pi)) exp(-g^2 r^2)] r_ij / r^2
//   W_ab = (1/2) sum_i sum_j (F_ij)_a (r_ij)_b
// over minimum images (r_C < L/2).
//
// GB300 layout: the particles are binned into cells at least r_C/2 wide with
// the PPPM sort kernels (order 2: the anchor is the cell, one tile per cell)
// and their wrapped positions written once as float4/double4 (x, y, z, q) in
// cell order.  One warp per cell: its lanes hold the cell's particles (32 at
// a time), and the warp walks the 5^3 cells around it (a dimension with fewer
// than 5 cells is one cell) in step, so every candidate is one broadcast load
// for the whole warp and no lane diverges from the loop.  Each pair is
// computed from both ends (no atomics); per-warp energy/virial partials are
// summed in FP64 in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "pppm_common.cuh"

using namespace pppm;

namespace pppm {
namespace real_detail {

constexpr int REAL_THREADS = 128;

template <typename R>
struct RealGeom {
    int nc[3];        // cells per dimension
    int span[3];      // neighbour cell offsets -span..span (2, or 0 for a single cell)
    R L[3], iL[3];
    R hc[3];          // cell widths
    R rc2;
    R g, g2, c2g;     // g, g^2, 2 g / sqrt(pi)
};

__device__ __forceinline__ float erfc_t(float v) { return erfcf(v); }
__device__ __forceinline__ double erfc_t(double v) { return erfc(v); }
__device__ __forceinline__ float exp_t(float v) { return expf(v); }
__device__ __forceinline__ double exp_t(double v) { return exp(v); }
__device__ __forceinline__ float rint_t(float v) { return rintf(v); }
__device__ __forceinline__ double rint_t(double v) { return rint(v); }
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }

// Wrapped position (and charge) of every particle, in cell order.
template <typename R>
__global__ void __launch_bounds__(256) k_real_positions(RealGeom<R> rg, SortBufs b, int n,
                                                       vec4_t<R> *__restrict__ pos) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const vec4_t<R> r = reinterpret_cast<const vec4_t<R> *>(b.rec)[j];
    int a[3];
    unpack_anchor(b.cell[j], a[0], a[1], a[2]);
    // order-2 anchor: n = floor(u), delta = n - u, so u = n - delta
    vec4_t<R> o;
    o.x = ((R)a[0] - r.x) * rg.hc[0];
    o.y = ((R)a[1] - r.y) * rg.hc[1];
    o.z = ((R)a[2] - r.z) * rg.hc[2];
    o.w = r.w;
    pos[j] = o;
}

constexpr int REAL_WARPS = REAL_THREADS / 32;  // cells per CTA

template <typename R>
__global__ void __launch_bounds__(REAL_THREADS) k_real_pairs(RealGeom<R> rg, SortBufs b, int ncells,
                                                            const vec4_t<R> *__restrict__ pos, R *__restrict__ f,
                                                            int accumulate, R C, double *__restrict__ part) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cell = blockIdx.x * REAL_WARPS + w;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    if (cell < ncells) {
        const int cz = cell % rg.nc[2];
        const int cy = (cell / rg.nc[2]) % rg.nc[1];
        const int cx = cell / (rg.nc[2] * rg.nc[1]);
        const int hs = b.tile_start[cell], he = b.tile_start[cell + 1];
        for (int h0 = hs; h0 < he; h0 += 32) {   // the cell's particles, a warp-full at a time
            const int j = h0 + lane;
            const bool live = j < he;
            const vec4_t<R> pi = pos[live ? j : hs];
            R fx = 0, fy = 0, fz = 0, e = 0, vxx = 0, vyy = 0, vzz = 0, vxy = 0, vxz = 0, vyz = 0;
            for (int ox = -rg.span[0]; ox <= rg.span[0]; ++ox) {
                int nx = cx + ox;
                nx += (nx < 0) ? rg.nc[0] : 0;
                nx -= (nx >= rg.nc[0]) ? rg.nc[0] : 0;
                for (int oy = -rg.span[1]; oy <= rg.span[1]; ++oy) {
                    int ny = cy + oy;
                    ny += (ny < 0) ? rg.nc[1] : 0;
                    ny -= (ny >= rg.nc[1]) ? rg.nc[1] : 0;
                    for (int oz = -rg.span[2]; oz <= rg.span[2]; ++oz) {
                        int nz = cz + oz;
                        nz += (nz < 0) ? rg.nc[2] : 0;
                        nz -= (nz >= rg.nc[2]) ? rg.nc[2] : 0;
                        const int nb = (nx * rg.nc[1] + ny) * rg.nc[2] + nz;
                        const int s = b.tile_start[nb], t = b.tile_start[nb + 1];
                        for (int k = s; k < t; ++k) {   // warp-uniform: one broadcast load per candidate
                            const vec4_t<R> pj = pos[k];
                            R dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                            dx -= rg.L[0] * rint_t(dx * rg.iL[0]);
                            dy -= rg.L[1] * rint_t(dy * rg.iL[1]);
                            dz -= rg.L[2] * rint_t(dz * rg.iL[2]);
                            const R r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < rg.rc2 && k != j && live) {
                                const R ir = rsqrt_t(r2);
                                const R r = r2 * ir;
                                const R qq = pi.w * pj.w;
                                const R et = erfc_t(rg.g * r) * ir;
                                const R fr = qq * (et + rg.c2g * exp_t(-rg.g2 * r2)) * ir * ir;
                                fx += fr * dx;
                                fy += fr * dy;
                                fz += fr * dz;
                                e += qq * et;
                                vxx += fr * dx * dx;
                                vyy += fr * dy * dy;
                                vzz += fr * dz * dz;
                                vxy += fr * dx * dy;
                                vxz += fr * dx * dz;
                                vyz += fr * dy * dz;
                            }
                        }
                    }
                }
            }
            if (live) {
                R *fo = f + 3 * (int64_t)b.perm[j];
                if (accumulate) {
                    fo[0] += C * fx;
                    fo[1] += C * fy;
                    fo[2] += C * fz;
                } else {
                    fo[0] = C * fx;
                    fo[1] = C * fy;
                    fo[2] = C * fz;
                }
            }
            // FP32 paths reduce within the warp in FP32 (GB300's FP64 rate is a
            // small fraction of its FP32 rate), the per-warp values in FP64
            const R vals[7] = {e, vxx, vyy, vzz, vxy, vxz, vyz};
#pragma unroll
            for (int mm = 0; mm < 7; ++mm) acc[mm] += (double)warp_sum_t<R>(vals[mm]);
        }
    }
    __shared__ double sh[7][REAL_WARPS];
    if (lane == 0)
        for (int mm = 0; mm < 7; ++mm) sh[mm][w] = acc[mm];
    __syncthreads();
    if (threadIdx.x < 7) {
        double a = 0.0;
        for (int k = 0; k < REAL_WARPS; ++k) a += sh[threadIdx.x][k];
        part[7 * (int64_t)blockIdx.x + threadIdx.x] = 0.5 * a * (double)C;
    }
}

// Fixed-order sum of the per-CTA partials; one CTA of 7 warps.
__global__ void __launch_bounds__(224) k_real_final(const double *__restrict__ part, int nb, double *ev,
                                                   double *ev_user) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double v = 0.0;
    for (int k = lane; k < nb; k += 32) v += part[7 * k + w];
    v = warp_sum(v);
    if (lane == 0) {
        ev[w] = v;
        if (ev_user) ev_user[w] = v;
    }
}

}  // namespace real_detail
}  // namespace pppm

using namespace pppm::real_detail;

struct pppm_real {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool fp64 = false;
    int64_t n_max = 0;
    double C = 0;
    RealGeom<float> rf{};
    RealGeom<double> rd{};
    Geom<float> gf{};
    Geom<double> gd{};
    SortBufs sb{};
    void *pos = nullptr;
    double *part = nullptr, *ev = nullptr;
    int nb_max = 0;
    std::vector<void *> allocs;
};

namespace {

int rmalloc(pppm_real *r, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return PPPM_ENOMEM;
    }
    r->allocs.push_back(*p);
    return PPPM_OK;
}

void real_release(pppm_real *r) {
    if (!r) return;
    if (r->stream) cudaStreamSynchronize(r->stream);
    else cudaDeviceSynchronize();
    for (void *v : r->allocs) cudaFree(v);
    delete r;
}

template <typename R>
void fill_real(pppm_real *r, RealGeom<R> &rg, Geom<R> &g, const double box[3], const int nc[3], double r_cut,
               double g_ewald) {
    for (int d = 0; d < 3; ++d) {
        rg.nc[d] = nc[d];
        rg.span[d] = nc[d] >= 5 ? 2 : 0;
        rg.L[d] = (R)box[d];
        rg.iL[d] = (R)(1.0 / box[d]);
        rg.hc[d] = (R)(box[d] / nc[d]);
        // the sort sees a "mesh" of cells, order 2, one tile per cell
        g.M[d] = nc[d];
        g.T[d] = nc[d];
        g.TE[d] = 1;
        g.L[d] = (R)box[d];
        g.iL[d] = (R)(1.0 / box[d]);
        const double ih = (double)nc[d] / box[d];
        g.ih[d] = (R)ih;
        g.ih_lo[d] = (R)(ih - (double)(R)ih);
        g.h[d] = (R)(box[d] / nc[d]);
    }
    rg.rc2 = (R)(r_cut * r_cut);
    rg.g = (R)g_ewald;
    rg.g2 = (R)(g_ewald * g_ewald);
    rg.c2g = (R)(2.0 * g_ewald / std::sqrt(M_PI));
    g.Mzh = nc[2] / 2 + 1;
    g.ntiles = nc[0] * nc[1] * nc[2];
    g.P = 2;
    g.rlo = 0;
    g.ivcell = (R)1;
    (void)r;
}

template <typename R>
int real_enqueue(pppm_real *r, const RealGeom<R> &rg, const Geom<R> &g, int64_t n, const void *x, const void *q,
                 void *f, int accumulate, double *ev) {
    cudaStream_t s = r->stream;
    launch_sort<R>(g, n, (const R *)x, (const R *)q, r->sb, s);
    const int nb = (int)((n + 255) / 256);
    k_real_positions<R><<<nb, 256, 0, s>>>(rg, r->sb, (int)n, (vec4_t<R> *)r->pos);
    const int np = (g.ntiles + REAL_WARPS - 1) / REAL_WARPS;  // one warp per cell
    // the sort's histogram is cleared by make_rho in the PPPM step; here after the pairs
    k_real_pairs<R><<<np, REAL_THREADS, 0, s>>>(rg, r->sb, g.ntiles, (const vec4_t<R> *)r->pos, (R *)f,
                                                accumulate, (R)r->C, r->part);
    if (cudaMemsetAsync(r->sb.tile_count, 0, 4 * (size_t)g.ntiles, s) != cudaSuccess) return PPPM_ECUDA;
    k_real_final<<<1, 224, 0, s>>>(r->part, np, r->ev, ev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return PPPM_ECUDA;
    }
    return PPPM_OK;
}

}  // namespace

extern "C" {

int pppm_real_setup(pppm_real **out, const double box[3], int64_t n_max, double r_cut, double g_ewald, int precision,
                    double qqrd2e, void *cuda_stream) {
    if (!out) return PPPM_EINVAL;
    *out = nullptr;
    if (!box || n_max < 0 || n_max > ((int64_t)1 << 30) || !(g_ewald > 0) || !(r_cut > 0)) return PPPM_EINVAL;
    if (precision != PPPM_FP64 && precision != PPPM_FP32 && precision != PPPM_FP32C) return PPPM_EINVAL;
    if (!std::isfinite(qqrd2e) || !std::isfinite(g_ewald) || !std::isfinite(r_cut)) return PPPM_EINVAL;
    int nc[3];
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0) || !std::isfinite(box[d])) return PPPM_EINVAL;
        if (r_cut >= 0.5 * box[d]) return PPPM_EINVAL;  // minimum images
        int c = (int)std::floor(box[d] / (0.5 * r_cut));  // cells at least r_C/2 wide
        c = std::min(c, MAX_MESH);
        nc[d] = c >= 5 ? c : 1;
    }
    pppm_real *r = new (std::nothrow) pppm_real();
    if (!r) return PPPM_ENOMEM;
    cudaGetDevice(&r->device);
    r->stream = (cudaStream_t)cuda_stream;
    r->fp64 = precision == PPPM_FP64;
    r->n_max = n_max;
    r->C = qqrd2e;
    fill_real<float>(r, r->rf, r->gf, box, nc, r_cut, g_ewald);
    fill_real<double>(r, r->rd, r->gd, box, nc, r_cut, g_ewald);
    const size_t rs = r->fp64 ? 8 : 4;
    const int64_t nm = std::max<int64_t>(n_max, 1);
    const int ncell = nc[0] * nc[1] * nc[2];
    r->nb_max = (ncell + REAL_WARPS - 1) / REAL_WARPS;
    int rc = PPPM_OK;
    do {
        if ((rc = rmalloc(r, (void **)&r->sb.anchor, 4 * nm))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.rank, 4 * nm))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.tile_count, 4 * (size_t)ncell))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.tile_start, 4 * ((size_t)ncell + 1)))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.perm, 4 * nm))) break;
        if ((rc = rmalloc(r, &r->sb.rec, 4 * rs * nm))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.cell, 4 * nm))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.blk, sizeof(double) * 2 * ((nm + 255) / 256)))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.qsum, 2 * sizeof(double)))) break;
        if ((rc = rmalloc(r, (void **)&r->sb.err, 4 * sizeof(int)))) break;
        if ((rc = rmalloc(r, &r->pos, 4 * rs * nm))) break;
        if ((rc = rmalloc(r, (void **)&r->part, sizeof(double) * 7 * r->nb_max))) break;
        if ((rc = rmalloc(r, (void **)&r->ev, 8 * sizeof(double)))) break;
    } while (0);
    if (!rc && (cudaMemsetAsync(r->sb.tile_count, 0, 4 * (size_t)ncell, r->stream) != cudaSuccess ||
                cudaMemsetAsync(r->sb.err, 0, 16, r->stream) != cudaSuccess ||
                cudaMemsetAsync(r->ev, 0, 64, r->stream) != cudaSuccess ||
                cudaStreamSynchronize(r->stream) != cudaSuccess))
        rc = PPPM_ECUDA;
    if (rc) {
        real_release(r);
        return rc;
    }
    *out = r;
    return PPPM_OK;
}

int pppm_real_compute(pppm_real *r, int64_t n, const void *x, const void *q, void *f, int accumulate, double *ev) {
    if (!r || n < 0 || n > r->n_max) return PPPM_EINVAL;
    if (n > 0 && (!x || !q || !f)) return PPPM_EINVAL;
    if (n == 0) {
        if (cudaMemsetAsync(r->ev, 0, 64, r->stream) != cudaSuccess) return PPPM_ECUDA;
        if (ev && cudaMemsetAsync(ev, 0, 7 * sizeof(double), r->stream) != cudaSuccess) return PPPM_ECUDA;
        return PPPM_OK;
    }
    if (r->fp64) return real_enqueue<double>(r, r->rd, r->gd, n, x, q, f, accumulate, ev);
    return real_enqueue<float>(r, r->rf, r->gf, n, x, q, f, accumulate, ev);
}

int pppm_real_sync(pppm_real *r) {
    if (!r) return PPPM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(r->stream);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, r->sb.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return PPPM_ECUDA;
    }
    if (err) {
        cudaMemset(r->sb.err, 0, sizeof(int));
        return (err & ERR_INTERNAL) ? PPPM_EINTERNAL : PPPM_ENONFINITE;
    }
    return PPPM_OK;
}

int pppm_real_info(const pppm_real *r, int64_t info[4]) {
    if (!r || !info) return PPPM_EINVAL;
    info[0] = r->rf.nc[0];
    info[1] = r->rf.nc[1];
    info[2] = r->rf.nc[2];
    info[3] = r->n_max;
    return PPPM_OK;
}

int pppm_real_destroy(pppm_real *r) {
    if (!r) return PPPM_EINVAL;
    real_release(r);
    return PPPM_OK;
}

}  // extern "C"
