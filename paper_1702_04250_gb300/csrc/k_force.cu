// Distribute-Force (Sec. 3.1): interpolate the mesh result back to the
// particles with the same P^3 stencil used for Map-Charge.
//  ik: "multiplies the grid values for each spatial dimension at each grid
//      point by the corresponding stencil coefficient, then adds them to three
//      totals"; the totals times the charge and C give the force.  The field is
//      stored interleaved as (Ex, Ey, Ez, 0) per point -- the paper's
//      "repacking" of the Poisson output -- so one 16-byte load serves a point.
//  ad: the scalar potential times three coefficient sets (one derivative
//      factor each), then per-particle work after the loop: scaling and the
//      self-force correction (the paper's "split atom" epilogue, fused here).
//
// Layout: 8 lanes per particle, lane k owning stencil offset k along z (lanes
// k >= P idle: the zero-padded "simd8" inner loop), particles in tile-sorted
// order so a warp's four particles read neighbouring mesh rows; the eight
// partial sums are combined with warp shuffles and the force is written to the
// particle's input position.
//
// ad self force (paper silent; reading of the Ballenegger-Cerda-Holm form):
// F_a -= q^2 sum_{n=1,2} c_{a,n} sin(2 pi n u_a), with u_a = n_a - delta_a the
// grid coordinate, so sin(2 pi n u_a) = -sin(2 pi n delta_a).
#include "pppm_common.cuh"

namespace pppm {

constexpr int FF_THREADS = 256;
constexpr int FGROUP = 8;

__device__ __forceinline__ float ldf(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ldf(const double *p) { return __ldg(p); }
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ double4_32a ld4(const double *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float sin2pi(float x) { return sinpif(2.0f * x); }
__device__ __forceinline__ double sin2pi(double x) { return sinpi(2.0 * x); }

__device__ __forceinline__ int wrap1(int i, int M) { return i < 0 ? i + M : (i >= M ? i - M : i); }

template <typename R, int P, int MODE>  // MODE 0: ik force, 1: ad force, 2: energy gradient
__global__ void __launch_bounds__(FF_THREADS) k_fieldforce(Geom<R> g, SortBufs b, int n,
                                                           const R *__restrict__ field, R *__restrict__ f,
                                                           R *__restrict__ dq, R qC, double c0, double c1,
                                                           double c2, double c3, double c4, double c5,
                                                           R gself, R gbg, const double *__restrict__ qsum) {
    const int lane = threadIdx.x & 31;
    const int k = lane & (FGROUP - 1);
    const int gbase = lane & ~(FGROUP - 1);
    const int64_t gid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / FGROUP;
    const int64_t warp_first = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) / FGROUP;
    if (warp_first >= n) return;  // whole warp idle
    const bool live = gid < n;
    const int j = live ? (int)gid : 0;

    const vec4_t<R> r = reinterpret_cast<const vec4_t<R> *>(b.rec)[j];
    int ax, ay, az;
    unpack_anchor(b.cell[j], ax, ay, az);
    const R dx = r.x, dy = r.y, dz = r.z, qv = r.w;

    R wxl = 0, wyl = 0, wzl = 0, dxl = 0, dyl = 0, dzl = 0;
    if (k < P) {
        wxl = weight<R, P>(g.coef, k, dx);
        wyl = weight<R, P>(g.coef, k, dy);
        wzl = weight<R, P>(g.coef, k, dz);
        if (MODE != 0) {
            dxl = dweight<R, P>(g.dcoef, k, dx);
            dyl = dweight<R, P>(g.dcoef, k, dy);
            dzl = dweight<R, P>(g.dcoef, k, dz);
        }
    }
    R wx[P], wy[P], wdx[P], wdy[P];
#pragma unroll
    for (int t = 0; t < P; ++t) {
        wx[t] = __shfl_sync(0xffffffffu, wxl, gbase + t);
        wy[t] = __shfl_sync(0xffffffffu, wyl, gbase + t);
        if (MODE != 0) {
            wdx[t] = __shfl_sync(0xffffffffu, dxl, gbase + t);
            wdy[t] = __shfl_sync(0xffffffffu, dyl, gbase + t);
        }
    }
    const int My = g.M[1], Mz = g.M[2];
    R e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    if (live && k < P) {
        const int iz = wrap1(az - g.rlo + k, Mz);
        int yoff[P];
#pragma unroll
        for (int c = 0; c < P; ++c) yoff[c] = wrap1(ay - g.rlo + c, My) * Mz + iz;
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const int xoff = wrap1(ax - g.rlo + a, g.M[0]) * (My * Mz);
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const int p = xoff + yoff[c];
                if (MODE == 0) {
                    const vec4_t<R> v = ld4(field + 4 * (int64_t)p);
                    const R w = wx[a] * wy[c];
                    e0 += w * v.x;
                    e1 += w * v.y;
                    e2 += w * v.z;
                } else {
                    const R v = ldf(field + p);
                    e0 += wdx[a] * wy[c] * v;
                    e1 += wx[a] * wdy[c] * v;
                    e2 += wx[a] * wy[c] * v;
                    if (MODE == 2) e3 += wx[a] * wy[c] * v;
                }
            }
        }
        if (MODE == 0) {
            e0 *= wzl; e1 *= wzl; e2 *= wzl;
        } else {
            e0 *= wzl; e1 *= wzl;
            e3 = e2 * wzl;               // potential at the particle (MODE 2)
            e2 *= dzl;
        }
    }
#pragma unroll
    for (int o = FGROUP / 2; o > 0; o >>= 1) {
        e0 += __shfl_xor_sync(0xffffffffu, e0, o);
        e1 += __shfl_xor_sync(0xffffffffu, e1, o);
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        if (MODE == 2) e3 += __shfl_xor_sync(0xffffffffu, e3, o);
    }
    if (!live || k != 0) return;
    const int dst = b.perm[j];
    R F0, F1, F2;
    if (MODE == 0) {
        const R s = qC * qv;
        F0 = s * e0; F1 = s * e1; F2 = s * e2;
    } else {
        // E_a = sum dW/ddelta * W W phi / h_a  (dW/dx = -dW/ddelta / h, E = -grad phi)
        const R s = qC * qv;
        F0 = s * e0 * g.ih[0];
        F1 = s * e1 * g.ih[1];
        F2 = s * e2 * g.ih[2];
        if (MODE == 1) {
            const R q2 = qv * qv;
            F0 += q2 * ((R)c0 * sin2pi(dx) + (R)c1 * sin2pi(R(2) * dx));
            F1 += q2 * ((R)c2 * sin2pi(dy) + (R)c3 * sin2pi(R(2) * dy));
            F2 += q2 * ((R)c4 * sin2pi(dz) + (R)c5 * sin2pi(R(2) * dz));
        } else {
            // gradient of the energy: dE/dx = -(uncorrected ad force)
            F0 = -F0; F1 = -F1; F2 = -F2;
            if (dq) dq[dst] = qC * e3 + gself * qv + gbg * (R)qsum[0];
        }
    }
    if (f) {
        f[3 * (int64_t)dst + 0] = F0;
        f[3 * (int64_t)dst + 1] = F1;
        f[3 * (int64_t)dst + 2] = F2;
    }
}

template <typename R, int P, int MODE>
static void launch_ff(const Geom<R> &g, int64_t n, const SortBufs &b, const R *field, R *f, R *dq, R qC,
                      const double *c, R gs, R gb, cudaStream_t s) {
    // gb multiplies sum(q), read on the device from the sort buffers
    const int64_t threads = n * FGROUP;
    const int nb = (int)((threads + FF_THREADS - 1) / FF_THREADS);
    k_fieldforce<R, P, MODE><<<nb, FF_THREADS, 0, s>>>(g, b, (int)n, field, f, dq, qC, c[0], c[1], c[2], c[3],
                                                       c[4], c[5], gs, gb, b.qsum);
}

template <typename R, int MODE>
static void dispatch(const Geom<R> &g, int64_t n, const SortBufs &b, const R *field, R *f, R *dq, R qC,
                     const double *c, R gs, R gb, cudaStream_t s) {
    switch (g.P) {
        case 2: launch_ff<R, 2, MODE>(g, n, b, field, f, dq, qC, c, gs, gb, s); break;
        case 3: launch_ff<R, 3, MODE>(g, n, b, field, f, dq, qC, c, gs, gb, s); break;
        case 4: launch_ff<R, 4, MODE>(g, n, b, field, f, dq, qC, c, gs, gb, s); break;
        case 5: launch_ff<R, 5, MODE>(g, n, b, field, f, dq, qC, c, gs, gb, s); break;
        case 6: launch_ff<R, 6, MODE>(g, n, b, field, f, dq, qC, c, gs, gb, s); break;
        case 7: launch_ff<R, 7, MODE>(g, n, b, field, f, dq, qC, c, gs, gb, s); break;
        default: break;
    }
}

template <typename R>
void launch_fieldforce(const Geom<R> &g, bool ik, int64_t n, const SortBufs &b, const R *field, R *f, R qC,
                       const double *sf, cudaStream_t s) {
    if (n == 0) return;
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    if (ik)
        dispatch<R, 0>(g, n, b, field, f, nullptr, qC, zero, R(0), R(0), s);
    else
        dispatch<R, 1>(g, n, b, field, f, nullptr, qC, sf ? sf : zero, R(0), R(0), s);
}

template <typename R>
void launch_energy_grad(const Geom<R> &g, int64_t n, const SortBufs &b, const R *phi, R *dEdx, R *dEdq, R C,
                        const double *qsum, double gself, double gbg, cudaStream_t s) {
    (void)qsum;
    if (n == 0) return;
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    dispatch<R, 2>(g, n, b, phi, dEdx, dEdq, C, zero, (R)gself, (R)gbg, s);
}

template void launch_fieldforce<float>(const Geom<float> &, bool, int64_t, const SortBufs &, const float *,
                                       float *, float, const double *, cudaStream_t);
template void launch_fieldforce<double>(const Geom<double> &, bool, int64_t, const SortBufs &, const double *,
                                        double *, double, const double *, cudaStream_t);
template void launch_energy_grad<float>(const Geom<float> &, int64_t, const SortBufs &, const float *, float *,
                                        float *, float, const double *, double, double, cudaStream_t);
template void launch_energy_grad<double>(const Geom<double> &, int64_t, const SortBufs &, const double *,
                                         double *, double *, double, const double *, double, double,
                                         cudaStream_t);

}  // namespace pppm
