// Poisson solve in reciprocal space (Sec. 2.1 step 2, Sec. 3.2): between the
// forward FFT of the mesh charge and the inverse FFT(s), multiply by the
// influence function G(k) -- for ik also by -i k_a, giving the three field
// spectra that need three inverse transforms; for ad only G, giving the
// potential that needs one -- and reduce the energy and virial.
//
// The paper does not print G; this is the Hockney-Eastwood optimal form for
// ik differentiation and the same form without the k.k_m / k^2 factor for ad:
//   G(k) = [sum_m (k.k_m)/k^2 R(k_m) U^2(k_m)] / [sum_m U^2(k_m)]^2 (ik)
//   G(k) = [sum_m R(k_m) U^2(k_m)] / [sum_m U^2(k_m)]^2             (ad)
//   R(k) = 4 pi exp(-k^2/4g^2) / k^2,  U(k) = prod_d sinc^P(k_d h_d / 2),
//   k_m = k + 2 pi m / h, numerator over |m_d| <= 2.
// The denominator's per-dimension sum is evaluated exactly as the finite
// cosine series sum_g M_2P(g) cos(k h g) (Poisson summation).
//
// Energy and virial (paper silent; Ewald's reciprocal-space forms with G in
// place of R):  E = (C/2) vcell^2/V sum_k G|rho_hat|^2 over the full
// spectrum, W_ab = same sum times [delta_ab - 2(1 + k^2/4g^2) k_a k_b / k^2].
// Per-thread sums are taken in the step's type, combined in FP64 with warp
// shuffles; one small kernel reduces the per-CTA partials in a fixed order
// (on a side branch of the step graph, off the critical path).
#include <algorithm>
#include <type_traits>

#include "pppm_common.cuh"

namespace pppm {

constexpr int GREEN_THREADS = 256;
constexpr int GREEN_ZU = 4;  // spectrum elements a lane keeps in flight along a z-row

// ---------------------------------------------------------------------------
// Setup (FP64): G on the half spectrum and the ad self-force sums
//   S[a][n-1] = sum_k w(k) G(k) B_a(k_a h_a, n) prod_{b != a} B_b(k_b h_b, 0)
// where w = 1 for kz = 0 and the z-Nyquist plane, 2 otherwise.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GREEN_THREADS) k_green_setup(GreenSetup gs, double *__restrict__ G64,
                                                               double *__restrict__ sf) {
    __shared__ double sh[6][GREEN_THREADS / 32];
    const int Mx = gs.M[0], My = gs.M[1], Mzh = gs.Mzh;
    const int64_t total = (int64_t)Mx * My * Mzh;
    const int off[3] = {0, Mx, Mx + My};
    const int len = Mx + My + Mzh;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const double twopi = 2.0 * M_PI;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int iz = (int)(e % Mzh);
        const int iy = (int)((e / Mzh) % My);
        const int ix = (int)(e / ((int64_t)Mzh * My));
        const int idx[3] = {ix, iy, iz};
        double k[3];
        for (int d = 0; d < 3; ++d) k[d] = gs.ktab[off[d] + idx[d]];
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double G = 0.0;
        if (k2 > 0.0) {
            double num = 0.0;
            for (int mx = -2; mx <= 2; ++mx) {
                const double kmx = k[0] + twopi * mx / gs.h[0];
                const double axv = gs.atab[(mx + 2) * len + off[0] + ix];
                if (axv == 0.0) continue;
                for (int my = -2; my <= 2; ++my) {
                    const double kmy = k[1] + twopi * my / gs.h[1];
                    const double ayv = gs.atab[(my + 2) * len + off[1] + iy];
                    if (ayv == 0.0) continue;
                    for (int mz = -2; mz <= 2; ++mz) {
                        const double kmz = k[2] + twopi * mz / gs.h[2];
                        const double azv = gs.atab[(mz + 2) * len + off[2] + iz];
                        if (azv == 0.0) continue;
                        const double km2 = kmx * kmx + kmy * kmy + kmz * kmz;
                        double t = 4.0 * M_PI * axv * ayv * azv / km2;
                        if (gs.ik) t *= (k[0] * kmx + k[1] * kmy + k[2] * kmz);
                        num += t;
                    }
                }
            }
            const double D = gs.dtab[off[0] + ix] * gs.dtab[off[1] + iy] * gs.dtab[off[2] + iz];
            double den = D * D;
            if (gs.ik) den *= k2;
            G = num / den;
        }
        G64[e] = G;
        const double w = (iz == 0 || (2 * (Mzh - 1) == gs.M[2] && iz == Mzh - 1)) ? 1.0 : 2.0;
        const double wG = w * G;
        for (int a = 0; a < 3; ++a) {
            for (int n = 1; n <= 2; ++n) {
                double p = wG;
                for (int d = 0; d < 3; ++d) p *= gs.btab[((d == a) ? n : 0) * len + off[d] + idx[d]];
                acc[a * 2 + n - 1] += p;
            }
        }
    }
    for (int c = 0; c < 6; ++c) {
        const double v = warp_sum(acc[c]);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int w = 0; w < GREEN_THREADS / 32; ++w) v += sh[threadIdx.x][w];
        atomicAdd(&sf[threadIdx.x], v);
    }
}

void launch_green_setup(const GreenSetup &gs, double *G64, double *sf_sums, cudaStream_t s) {
    cudaMemsetAsync(sf_sums, 0, 6 * sizeof(double), s);
    const int64_t total = (int64_t)gs.M[0] * gs.M[1] * gs.Mzh;
    int nb = (int)std::min<int64_t>((total + GREEN_THREADS - 1) / GREEN_THREADS, 152 * 16);
    if (nb < 1) nb = 1;
    k_green_setup<<<nb, GREEN_THREADS, 0, s>>>(gs, G64, sf_sums);
}

// ---------------------------------------------------------------------------
// Setup-time k-space error estimate of a mesh (mesh choice for a target
// accuracy): per half-spectrum k != 0, with weight w and
// phi(k) = 4 pi exp(-k^2/4g^2)/k^2,
//  ik: w { sum_m 16 pi^2 exp(-k_m^2/2g^2) / k_m^2
//          - [sum_m U^2(k_m) (k.k_m) phi(k_m)]^2 / (k^2 D(k)^2) }
//      (the Hockney-Eastwood functional of the optimal influence function; D =
//      the full alias sum of U^2);
//  ad: w { G^2 D S2 - 2 G sum_m U^2(k_m) k_m^2 phi(k_m) + sum_m 16 pi^2 exp(-k_m^2/2g^2) / k_m^2 }
//      (the functional of forces taken as the gradient of the interpolated
//      potential, each alias with its own derivative, at the plan's ad
//      influence function G = sum_m U^2(k_m) phi(k_m) / D^2; S2 = the full
//      alias sum of U^2(k_m) k_m^2, which separates over dimensions).
// One FP64 partial per CTA, summed by the host in CTA order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GREEN_THREADS) k_kspace_error(KErrSetup ks, double *__restrict__ part) {
    __shared__ double sh[GREEN_THREADS / 32];
    const int Mx = ks.M[0], My = ks.M[1], Mzh = ks.Mzh;
    const int64_t total = (int64_t)Mx * My * Mzh;
    const int off[3] = {0, Mx, Mx + My};
    const int len = Mx + My + Mzh;
    const double twopi = 2.0 * M_PI;
    double acc = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int iz = (int)(e % Mzh);
        const int iy = (int)((e / Mzh) % My);
        const int ix = (int)(e / ((int64_t)Mzh * My));
        const double k[3] = {ks.ktab[ix], ks.ktab[off[1] + iy], ks.ktab[off[2] + iz]};
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        if (k2 == 0.0) continue;
        double num = 0.0, s1 = 0.0, gnum = 0.0, tsum = 0.0;
        for (int mx = -2; mx <= 2; ++mx) {
            const double kmx = k[0] + twopi * mx / ks.h[0];
            const double ax = ks.atab[(mx + 2) * len + ix], ex = ks.etab[(mx + 2) * len + ix];
            for (int my = -2; my <= 2; ++my) {
                const double kmy = k[1] + twopi * my / ks.h[1];
                const double ay = ks.atab[(my + 2) * len + off[1] + iy], ey = ks.etab[(my + 2) * len + off[1] + iy];
                for (int mz = -2; mz <= 2; ++mz) {
                    const double kmz = k[2] + twopi * mz / ks.h[2];
                    const double az = ks.atab[(mz + 2) * len + off[2] + iz];
                    const double ez = ks.etab[(mz + 2) * len + off[2] + iz];
                    const double km2 = kmx * kmx + kmy * kmy + kmz * kmz;
                    s1 += 16.0 * M_PI * M_PI * ex * ey * ez / km2;
                    if (ks.ad) {
                        const double up = 4.0 * M_PI * ax * ay * az;  // U^2 k_m^2 phi(k_m)
                        gnum += up / km2;                             // U^2 phi(k_m)
                        tsum += up;
                    } else {
                        num += 4.0 * M_PI * ax * ay * az / km2 * (k[0] * kmx + k[1] * kmy + k[2] * kmz);
                    }
                }
            }
        }
        const double dx = ks.dtab[ix], dy = ks.dtab[off[1] + iy], dz = ks.dtab[off[2] + iz];
        const double D = dx * dy * dz;
        const double w = (iz == 0 || (2 * (Mzh - 1) == ks.M[2] && iz == Mzh - 1)) ? 1.0 : 2.0;
        if (ks.ad) {
            const double G = gnum / (D * D);
            const double S2 = ks.s2tab[ix] * dy * dz + dx * ks.s2tab[off[1] + iy] * dz + dx * dy * ks.s2tab[off[2] + iz];
            acc += w * (G * G * D * S2 - 2.0 * G * tsum + s1);
        } else {
            acc += w * (s1 - num * num / (k2 * D * D));
        }
    }
    const double v = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < GREEN_THREADS / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

int launch_kspace_error(const KErrSetup &ks, double *part, cudaStream_t s) {
    const int64_t total = (int64_t)ks.M[0] * ks.M[1] * ks.Mzh;
    int nb = (int)std::min<int64_t>((total + GREEN_THREADS - 1) / GREEN_THREADS, KERR_MAX_BLOCKS);
    if (nb < 1) nb = 1;
    k_kspace_error<<<nb, GREEN_THREADS, 0, s>>>(ks, part);
    return nb;
}

// ---------------------------------------------------------------------------
// Per step
// ---------------------------------------------------------------------------
// One spectrum element e = (kx, ky, kz): the field (ik: three components) or
// potential (ad) spectrum and this element's energy/virial terms (Eq. 5's
// G times |rho_hat|^2, weight w = 1 on the kz = 0 and z-Nyquist planes, 2
// elsewhere for the half spectrum).
template <typename R, bool IK>
__device__ __forceinline__ void green_point(complex_t<R> r, R G, R kx, R ky, R kz, R dkx, R dky, R dkz, R w,
                                            R i4g2, complex_t<R> *__restrict__ spec, int e, int total,
                                            R (&acc)[7]) {
    const R pr = G * r.x, pi = G * r.y;
    if (IK) {
        // E_a = -i k_a G rho_hat / M  ->  (k_a pi, -k_a pr)
        complex_t<R> o;
        o.x = dkx * pi; o.y = -dkx * pr; spec[e] = o;
        o.x = dky * pi; o.y = -dky * pr; spec[total + e] = o;
        o.x = dkz * pi; o.y = -dkz * pr; spec[2 * total + e] = o;
    } else {
        complex_t<R> o;
        o.x = pr; o.y = pi;
        spec[e] = o;
    }
    const R s = w * G * (r.x * r.x + r.y * r.y);
    const R k2 = kx * kx + ky * ky + kz * kz;
    const R fac = (k2 > R(0)) ? R(2) * (R(1) + k2 * i4g2) / k2 : R(0);
    const R sf = s * fac;
    acc[0] += s;
    acc[1] += s - sf * kx * kx;
    acc[2] += s - sf * ky * ky;
    acc[3] += s - sf * kz * kz;
    acc[4] -= sf * kx * ky;
    acc[5] -= sf * kx * kz;
    acc[6] -= sf * ky * kz;
}

// the CTA's seven energy/virial partials, summed in a fixed order
template <typename R>
__device__ __forceinline__ void green_partials(R (&acc)[7], double (&sh)[7][GREEN_THREADS / 32], double *part,
                                               int lb) {
    const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;
    for (int c = 0; c < 7; ++c) {
        const R v = warp_sum_t<R>(acc[c]);
        if (lane == 0) sh[c][wrow] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = 0.0;
        for (int w = 0; w < GREEN_THREADS / 32; ++w) v += sh[threadIdx.x][w];
        part[7 * lb + threadIdx.x] = v;
    }
}

template <typename R, bool IK>
__device__ __forceinline__ void green_body(const Geom<R> &g, const complex_t<R> *__restrict__ rhat,
                                           complex_t<R> *__restrict__ spec, const GreenBufs &b,
                                           const EnergyConsts &ec, int lb, int nlb) {
    __shared__ double sh[7][GREEN_THREADS / 32];
    pdl_wait();  // the forward transform is complete
    const int Mx = g.M[0], My = g.M[1], Mzh = g.Mzh;
    const int rows = Mx * My;
    const int total = rows * Mzh;
    const R *__restrict__ Gs = reinterpret_cast<const R *>(b.Gs);
    const R *__restrict__ kv = reinterpret_cast<const R *>(b.kvec);
    const R *__restrict__ kd = reinterpret_cast<const R *>(b.kdiff);
    const bool evenz = (2 * (Mzh - 1) == g.M[2]);
    const R i4g2 = (R)ec.inv4g2;
    const int lane = threadIdx.x & 31;
    const int wrow = threadIdx.x >> 5;
    R acc[7] = {0, 0, 0, 0, 0, 0, 0};
    // one warp per z-row: row = (kx, ky), lanes along kz
    const int rows_per_cta = GREEN_THREADS / 32;
    for (int row = lb * rows_per_cta + wrow; row < rows; row += nlb * rows_per_cta) {
        const int ix = row / My, iy = row - ix * My;
        const R kx = kv[ix], ky = kv[Mx + iy];
        const R dkx = kd[ix], dky = kd[Mx + iy];
        // GREEN_ZU elements a lane, every load issued before any is used (the
        // kernel streams rho_hat and G once: its time is bytes in flight)
        for (int iz0 = lane; iz0 < Mzh; iz0 += GREEN_ZU * 32) {
            complex_t<R> rv[GREEN_ZU];
            R Gv[GREEN_ZU];
#pragma unroll
            for (int u = 0; u < GREEN_ZU; ++u) {
                const int iz = iz0 + 32 * u;
                if (iz < Mzh) {
                    rv[u] = rhat[row * Mzh + iz];
                    Gv[u] = Gs[row * Mzh + iz];
                } else {
                    rv[u].x = rv[u].y = R(0);
                    Gv[u] = R(0);
                }
            }
#pragma unroll
            for (int u = 0; u < GREEN_ZU; ++u) {
                const int iz = iz0 + 32 * u;
                if (iz >= Mzh) continue;
                const R w = (iz == 0 || (evenz && iz == Mzh - 1)) ? R(1) : R(2);
                green_point<R, IK>(rv[u], Gv[u], kx, ky, kv[Mx + My + iz], dkx, dky, IK ? kd[Mx + My + iz] : R(0),
                                   w, i4g2, spec, row * Mzh + iz, total, acc);
            }
        }
    }
    green_partials<R>(acc, sh, b.part, lb);
}

// The same over the spectrum as one flat array (element e = row Mzh + kz):
// consecutive threads take consecutive elements whatever the row length, for
// meshes whose half rows (Mzh = M_z / 2 + 1) are short against a warp (the
// batch's 16^3 - 64^3 meshes: 9 - 33 elements, where a warp a row leaves up
// to 23 of its 32 lanes idle).  Each thread keeps GREEN_ZU elements, a grid
// stride apart, in flight.
template <typename R, bool IK>
__device__ __forceinline__ void green_flat_body(const Geom<R> &g, const complex_t<R> *__restrict__ rhat,
                                                complex_t<R> *__restrict__ spec, const GreenBufs &b,
                                                const EnergyConsts &ec, int lb, int nlb) {
    __shared__ double sh[7][GREEN_THREADS / 32];
    pdl_wait();  // the forward transform is complete
    const int Mx = g.M[0], My = g.M[1], Mzh = g.Mzh;
    const int total = Mx * My * Mzh;
    const R *__restrict__ Gs = reinterpret_cast<const R *>(b.Gs);
    const R *__restrict__ kv = reinterpret_cast<const R *>(b.kvec);
    const R *__restrict__ kd = reinterpret_cast<const R *>(b.kdiff);
    const bool evenz = (2 * (Mzh - 1) == g.M[2]);
    const R i4g2 = (R)ec.inv4g2;
    R acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const int stride = nlb * GREEN_THREADS;
    for (int e0 = lb * GREEN_THREADS + (int)threadIdx.x; e0 < total; e0 += GREEN_ZU * stride) {
        complex_t<R> rv[GREEN_ZU];
        R Gv[GREEN_ZU];
#pragma unroll
        for (int u = 0; u < GREEN_ZU; ++u) {
            const int e = e0 + u * stride;
            if (e < total) {
                rv[u] = rhat[e];
                Gv[u] = Gs[e];
            } else {
                rv[u].x = rv[u].y = R(0);
                Gv[u] = R(0);
            }
        }
#pragma unroll
        for (int u = 0; u < GREEN_ZU; ++u) {
            const int e = e0 + u * stride;
            if (e >= total) continue;
            const int row = e / Mzh, iz = e - row * Mzh;
            const int ix = row / My, iy = row - ix * My;
            const R w = (iz == 0 || (evenz && iz == Mzh - 1)) ? R(1) : R(2);
            green_point<R, IK>(rv[u], Gv[u], kv[ix], kv[Mx + iy], kv[Mx + My + iz], IK ? kd[ix] : R(0),
                               IK ? kd[Mx + iy] : R(0), IK ? kd[Mx + My + iz] : R(0), w, i4g2, spec, e, total, acc);
        }
    }
    green_partials<R>(acc, sh, b.part, lb);
}

template <typename R, bool IK>
__global__ void __launch_bounds__(GREEN_THREADS) k_green(Geom<R> g, const complex_t<R> *__restrict__ rhat,
                                                         complex_t<R> *__restrict__ spec, GreenBufs b,
                                                         EnergyConsts ec) {
    green_body<R, IK>(g, rhat, spec, b, ec, blockIdx.x, gridDim.x);
}

template <typename R, bool IK>
__global__ void __launch_bounds__(GREEN_THREADS) k_batch_green(const BatchSys<R> *__restrict__ sys, BatchList bl) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<R> &S = sys[bl.ids[e]];
    green_flat_body<R, IK>(S.g, reinterpret_cast<const complex_t<R> *>(S.rho_hat),
                           reinterpret_cast<complex_t<R> *>(S.spec), S.gb, S.ec, blockIdx.x - bl.boff[e],
                           bl.boff[e + 1] - bl.boff[e]);
}

template <typename R>
void launch_batch_green(const BatchSys<R> *sys, const BatchList &bl, bool ik, cudaStream_t s) {
    if (bl.nblocks == 0) return;
    if (ik)
        k_batch_green<R, true><<<bl.nblocks, GREEN_THREADS, 0, s>>>(sys, bl);
    else
        k_batch_green<R, false><<<bl.nblocks, GREEN_THREADS, 0, s>>>(sys, bl);
}
template void launch_batch_green<float>(const BatchSys<float> *, const BatchList &, bool, cudaStream_t);
template void launch_batch_green<double>(const BatchSys<double> *, const BatchList &, bool, cudaStream_t);

// CTAs of k_green the GPU holds at once (SMs x resident CTAs per SM), per
// step type, found once per process before any capture.
static int g_green_wave[2] = {0, 0};

template <typename R>
cudaError_t prepare_green() {
    const int t = std::is_same<R, float>::value ? 0 : 1;
    if (g_green_wave[t] > 0) return cudaSuccess;
    int dev = 0, sms = 0, a = 0, b = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_green<R, true>, GREEN_THREADS, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_green<R, false>, GREEN_THREADS, 0);
    if (e == cudaSuccess) g_green_wave[t] = std::max(1, sms * std::min(a, b));
    return e;
}
template cudaError_t prepare_green<float>();
template cudaError_t prepare_green<double>();

template <typename R>
int launch_green(const Geom<R> &g, bool ik, const void *rho_hat, void *spec, const GreenBufs &b,
                 const EnergyConsts &ec, cudaStream_t s) {
    const int rows = g.M[0] * g.M[1];
    const int per_cta = GREEN_THREADS / 32;
    // eight z rows per warp before the CTA's energy/virial reduction, but at
    // least two CTAs per SM while there are rows for them; at most one wave of
    // resident CTAs (on 256^3, 1,024 CTAs of eight rows a warp took 1.35
    // waves and left the SMs idle for 12 % of the kernel) and at most
    // 152 x 8 CTAs (the partials buffer)
    int nb = std::max((rows + 8 * per_cta - 1) / (8 * per_cta), std::min(2 * 152, (rows + per_cta - 1) / per_cta));
    const int wave = g_green_wave[std::is_same<R, float>::value ? 0 : 1];
    if (wave > 0) nb = std::min(nb, wave);
    nb = std::min(std::max(nb, 1), 152 * 8);
    const auto *rh = reinterpret_cast<const complex_t<R> *>(rho_hat);
    auto *sp = reinterpret_cast<complex_t<R> *>(spec);
    const bool pdl = (g.launch_flags & LF_PDL_GREEN) != 0;
    if (ik) {
        if (pdl) launch_pdl(k_green<R, true>, dim3(nb), dim3(GREEN_THREADS), 0, s, g, rh, sp, b, ec);
        else k_green<R, true><<<nb, GREEN_THREADS, 0, s>>>(g, rh, sp, b, ec);
    } else {
        if (pdl) launch_pdl(k_green<R, false>, dim3(nb), dim3(GREEN_THREADS), 0, s, g, rh, sp, b, ec);
        else k_green<R, false><<<nb, GREEN_THREADS, 0, s>>>(g, rh, sp, b, ec);
    }
    return nb;
}

__global__ void __launch_bounds__(256) k_energy_final(GreenBufs b, EnergyConsts ec, int gn, int mn,
                                                      double *ev_user) {
    energy_final_body(b, ec, gn, mn, ev_user);
}

template <typename R>
__global__ void __launch_bounds__(256) k_batch_energy_final(const BatchSys<R> *__restrict__ sys, double *ev) {
    const BatchSys<R> &S = sys[blockIdx.x];
    energy_final_body(S.gb, S.ec, S.green_nb, S.map_nb, ev ? ev + 7 * blockIdx.x : nullptr);
}

template <typename R>
void launch_batch_energy_final(const BatchSys<R> *sys, int nsys, double *ev, cudaStream_t s) {
    if (nsys > 0) k_batch_energy_final<R><<<nsys, 256, 0, s>>>(sys, ev);
}
template void launch_batch_energy_final<float>(const BatchSys<float> *, int, double *, cudaStream_t);
template void launch_batch_energy_final<double>(const BatchSys<double> *, int, double *, cudaStream_t);

void launch_energy_final(const GreenBufs &b, const EnergyConsts &ec, int green_nblk, int map_nblk,
                         double *ev_user, cudaStream_t s) {
    k_energy_final<<<1, 256, 0, s>>>(b, ec, green_nblk, map_nblk, ev_user);
}

template int launch_green<float>(const Geom<float> &, bool, const void *, void *, const GreenBufs &,
                                 const EnergyConsts &, cudaStream_t);
template int launch_green<double>(const Geom<double> &, bool, const void *, void *, const GreenBufs &,
                                  const EnergyConsts &, cudaStream_t);

}  // namespace pppm
