// The Poisson solve of Sec. 2.1 step 2 / Sec. 3.2 -- forward 3-D FFT of the
// mesh charge, multiply by the influence function, one (ad) or three (ik)
// inverse 3-D FFTs -- as three kernels for FP32 plans whose mesh edges are
// powers of two from 16 to 128, or cubic meshes of edge 48, 96 or 256:
//   plane forward   CTA per x-plane: z real-to-complex of every row (two
//                   rows packed in one complex transform), then the y
//                   transform of every kz column         rho -> A[x][ky][kz]
//   x + Green       a group of lanes per (ky, kz) line and component: x
//                   transform, energy/virial partials (component 0), multiply
//                   by G (and -i k_a for ik), x inverse A -> S_a[x][ky][kz]
//   plane inverse   CTA per (x-plane, component): y inverse of every column,
//                   then z complex-to-real of every row pair
//                                                       S_a -> field / phi
// Same conventions as the cuFFT path (both directions unnormalised, G/M
// carries the 1/M), the same spectrum buffers, energy partials, final sums
// and field layout (ik: interleaved (E_x, E_y, E_z, pad) per point; ad and
// the potential: one value per point).  cuFFT serves other meshes and FP64.
// A 256 x 256 plane's spectrum (264 KB) exceeds one CTA's shared memory, so
// at edge 256 each plane pass runs on a cluster of four CTAs that split the
// plane's kz columns and exchange rows through distributed shared memory
// (k_fft_plane_fwd_cl / k_fft_plane_inv_cl below).
//
// One 1-D transform of length N = E L runs on a group of L lanes holding E
// points each (E = 8; 16 for N = 128 and 256, 12 for 48, 24 for 96), as the
// four-step factorisation
// with n = j + L a and k = b + E c (j: lane in the group):
//   X[b + E c] = sum_j W_L^(j c) W_N^(j b) sum_a W_E^(a b) x[j + L a]
// i.e. an E-point DFT in registers, the twiddle W_N^(j b), a transpose
// through shared memory, and L-point DFTs in registers.  "In" layout: lane j
// register a holds index j + L a; "out" layout: lane j' holds the E/L lines
// b = j' E/L + u, register u L + c holds index b + E c.  The forward runs in
// -> out, and the inverse runs the same steps backwards (out -> in), so a
// forward transform, a pointwise product and an inverse need no permutation.
#include <cmath>
#include <type_traits>

#include <cooperative_groups.h>

#include "pppm_common.cuh"

namespace pppm {

constexpr int FFT_THREADS = 256;
constexpr int FFT_WARPS = FFT_THREADS / 32;

template <int N>
struct Fft {
    static_assert(N == 16 || N == 32 || N == 64 || N == 128 || N == 256 || N == 48 || N == 96, "supported lengths");
    static constexpr int E = (N >= 128) ? 16 : (N == 96) ? 24 : (N == 48) ? 12 : 8;  // points per lane
    static constexpr int L = N / E;                 // lanes per line
    static constexpr int LINES = E / L;             // b-lines per lane in the out layout
    static constexpr int G = 32 / L;                // lines per warp
    static constexpr int P = L + 1;                 // transpose scratch: pitch of a b-row
    // a line's scratch, E*P complex rounded up to 8 mod 16, so that the two
    // halves of a 64-bit shared access touch disjoint banks
    static constexpr int S = E * P + (((8 - E * P) % 16) + 16) % 16;
    static constexpr int WARP_SCRATCH = G * S;      // complex per warp
};

// cos / sin of 2 pi q / 16, q = 0..7
__device__ __forceinline__ constexpr float c16(int q) {
    return q == 0 ? 1.0f : q == 1 ? 0.923879532511286756f : q == 2 ? 0.707106781186547524f
         : q == 3 ? 0.382683432365089772f : q == 4 ? 0.0f : q == 5 ? -0.382683432365089772f
         : q == 6 ? -0.707106781186547524f : -0.923879532511286756f;
}
__device__ __forceinline__ constexpr float s16(int q) {
    return q == 0 ? 0.0f : q == 1 ? 0.382683432365089772f : q == 2 ? 0.707106781186547524f
         : q == 3 ? 0.923879532511286756f : q == 4 ? 1.0f : q == 5 ? 0.923879532511286756f
         : q == 6 ? 0.707106781186547524f : 0.382683432365089772f;
}
// i with its low `bits` (<= 4) bits reversed
__host__ __device__ constexpr int brev_bits(int i, int bits) {
    return (((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3)) >> (4 - bits);
}

// cos and sin of 2 pi q / m at compile time (Taylor series of the reduced
// angle, double precision) for the twiddles of the mixed-radix stages
__host__ __device__ constexpr double cx_angle(int q, int m) {
    const int r = ((q % m) + m) % m;                       // [0, m)
    const double a = 6.283185307179586476925 * r / m;      // [0, 2 pi)
    return a > 3.141592653589793238463 ? a - 6.283185307179586476925 : a;  // (-pi, pi]
}
__host__ __device__ constexpr double cx_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n < 24; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double cx_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 24; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
template <int Q, int M>
struct Twiddle {
    static constexpr float c = (float)cx_cos(cx_angle(Q, M));
    static constexpr float s = (float)cx_sin(cx_angle(Q, M));
};

// f(std::integral_constant<int, I>) for I = B .. E-1, in order
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// a * W_16^q with W = exp(-2 pi i q / 16) (forward) or its conjugate (INV)
template <bool INV>
__device__ __forceinline__ float2 mul_w16(float2 a, int q) {
    if (q == 0) return a;
    if (q == 4) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);  // * (+i) / * (-i)
    const float c = c16(q), s = INV ? s16(q) : -s16(q);
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

// One radix-2 stage (butterfly span H) of an M-point in-register transform.
template <int M, int H, bool INV>
__device__ __forceinline__ void dit_stage(float2 (&t)[M]) {
#pragma unroll
    for (int k = 0; k < M; k += 2 * H) {
#pragma unroll
        for (int q = 0; q < H; ++q) {
            const float2 u = t[k + q];
            const float2 w = mul_w16<INV>(t[k + q + H], q * (8 / H));
            t[k + q] = cadd(u, w);
            t[k + q + H] = csub(u, w);
        }
    }
}

// a * W_M^Q, W = exp(-2 pi i / M) (forward) or its conjugate (INV); compile-time twiddle
template <bool INV, int Q, int M>
__device__ __forceinline__ float2 mul_tw(float2 a) {
    if constexpr (Q % M == 0) {
        return a;
    } else {
        constexpr float c = Twiddle<Q, M>::c, sn = Twiddle<Q, M>::s;
        const float s = INV ? sn : -sn;
        return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

template <int M, bool INV, int OFF = 0, int K>
__device__ __forceinline__ void dft_reg(float2 (&v)[K]);

// M = 3 m: three m-point DFTs of the stride-3 subsequences, the twiddles
// W_M^(n1 k2), and a 3-point DFT for every k2 (decimation in time).
template <int M, bool INV, int OFF, int K>
__device__ __forceinline__ void dft_radix3(float2 (&v)[K]) {
    constexpr int m = M / 3;
    float2 s0[m], s1[m], s2[m];
#pragma unroll
    for (int n = 0; n < m; ++n) {
        s0[n] = v[OFF + 3 * n];
        s1[n] = v[OFF + 3 * n + 1];
        s2[n] = v[OFF + 3 * n + 2];
    }
    dft_reg<m, INV>(s0);
    dft_reg<m, INV>(s1);
    dft_reg<m, INV>(s2);
    constexpr float h3 = 0.866025403784438646764f;  // sqrt(3) / 2
    static_for<0, m>([&](auto ic) {
        constexpr int k = decltype(ic)::value;
        const float2 a = s0[k];
        const float2 b = mul_tw<INV, k, M>(s1[k]);
        const float2 c = mul_tw<INV, 2 * k, M>(s2[k]);
        const float2 t1 = cadd(b, c);
        const float2 t2 = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
        const float2 d = csub(b, c);
        // -i sqrt(3)/2 (b - c) forward, +i sqrt(3)/2 (b - c) inverse
        const float2 t3 = INV ? make_float2(-h3 * d.y, h3 * d.x) : make_float2(h3 * d.y, -h3 * d.x);
        v[OFF + k] = cadd(a, t1);
        v[OFF + k + m] = cadd(t2, t3);
        v[OFF + k + 2 * m] = csub(t2, t3);
    });
}

// In-register DFT of M points at v[OFF .. OFF + M), natural order in and
// out: M = 2, 4, 8, 16 radix 2 (the bit reversal is a renaming of
// registers), M = 3 * 2^k by one radix-3 split over those.
template <int M, bool INV, int OFF, int K>
__device__ __forceinline__ void dft_reg(float2 (&v)[K]) {
    if constexpr (M % 3 == 0) {
        dft_radix3<M, INV, OFF>(v);
        return;
    } else {
    constexpr int LOGM = M == 1 ? 0 : M == 2 ? 1 : M == 4 ? 2 : M == 8 ? 3 : 4;
    float2 t[M];
#pragma unroll
    for (int i = 0; i < M; ++i) t[i] = v[OFF + brev_bits(i, LOGM)];
    if constexpr (M >= 2) dit_stage<M, 1, INV>(t);
    if constexpr (M >= 4) dit_stage<M, 2, INV>(t);
    if constexpr (M >= 8) dit_stage<M, 4, INV>(t);
    if constexpr (M >= 16) dit_stage<M, 8, INV>(t);
#pragma unroll
    for (int i = 0; i < M; ++i) v[OFF + i] = t[i];
    }
}

// dft_reg<L> on each of the LINES consecutive L-register lines of v
template <int L, int LINES, bool INV, int K>
__device__ __forceinline__ void line_dfts(float2 (&v)[K]) {
    static_for<0, LINES>([&](auto ic) { dft_reg<L, INV, decltype(ic)::value * L>(v); });
}

// index held by register r of lane j in the out layout
template <int N>
__device__ __forceinline__ int out_index(int j, int r) {
    using F = Fft<N>;
    return (j * F::LINES + r / F::L) + F::E * (r % F::L);
}

// in layout -> out layout (forward with INV = false).  scr: this line's
// scratch (Fft<N>::S complex); tw[t] = W_N^t, t < N.  Every lane of the warp
// calls it (it synchronises the warp).
template <int N, bool INV>
__device__ __forceinline__ void fft_in_out(float2 (&v)[Fft<N>::E], float2 *scr, const float2 *tw, int j) {
    using F = Fft<N>;
    dft_reg<F::E, INV>(v);
#pragma unroll
    for (int b = 1; b < F::E; ++b) {
        float2 w = tw[j * b];
        if (INV) w.y = -w.y;
        v[b] = cmul(v[b], w);
    }
#pragma unroll
    for (int b = 0; b < F::E; ++b) scr[b * F::P + j] = v[b];
    __syncwarp();
#pragma unroll
    for (int u = 0; u < F::LINES; ++u)
#pragma unroll
        for (int c = 0; c < F::L; ++c) v[u * F::L + c] = scr[(j * F::LINES + u) * F::P + c];
    __syncwarp();
    line_dfts<F::L, F::LINES, INV>(v);
}

// out layout -> in layout: the steps of fft_in_out backwards (the inverse
// transform with INV = true).
template <int N, bool INV>
__device__ __forceinline__ void fft_out_in(float2 (&v)[Fft<N>::E], float2 *scr, const float2 *tw, int j) {
    using F = Fft<N>;
    line_dfts<F::L, F::LINES, INV>(v);
#pragma unroll
    for (int u = 0; u < F::LINES; ++u)
#pragma unroll
        for (int c = 0; c < F::L; ++c) scr[(j * F::LINES + u) * F::P + c] = v[u * F::L + c];
    __syncwarp();
#pragma unroll
    for (int b = 0; b < F::E; ++b) v[b] = scr[b * F::P + j];
    __syncwarp();
#pragma unroll
    for (int b = 1; b < F::E; ++b) {
        float2 w = tw[j * b];
        if (INV) w.y = -w.y;
        v[b] = cmul(v[b], w);
    }
    dft_reg<F::E, INV>(v);
}

// tw[t] = W_N^t = exp(-2 pi i t / N), t < N (whole CTA; the caller synchronises)
template <int N>
__device__ __forceinline__ void fill_twiddles(float2 *tw) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        float s, c;
        sincospif(-2.0f * (float)t / (float)N, &s, &c);
        tw[t] = make_float2(c, s);
    }
}

// dst[di(e)] = src(e) for e < NEL by the whole CTA, up to eight loads in
// flight per thread before their stores (the sources sit in L2).
template <int NEL, int NT, typename T, typename F, typename D>
__device__ __forceinline__ void stage(T *dst, F src, D di) {
    constexpr int IT = (NEL + NT - 1) / NT;
    constexpr int CH = IT < 8 ? IT : 8;
#pragma unroll
    for (int k0 = 0; k0 < IT; k0 += CH) {
        T v[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int e = threadIdx.x + (k0 + k) * NT;
            if (k0 + k < IT && e < NEL) v[k] = src(e);
        }
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int e = threadIdx.x + (k0 + k) * NT;
            if (k0 + k < IT && e < NEL) dst[di(e)] = v[k];
        }
    }
}

template <int A, int B>
__host__ __device__ constexpr int imax() {
    return A > B ? A : B;
}

// Warps of a plane CTA: enough that the z row pairs (NY / 2) and the kz
// columns (NZ / 2 + 1) each take one pass.
template <int NY, int NZ>
__host__ __device__ constexpr int plane_warps() {
    return imax<(NZ / 2 + 1 + Fft<NY>::G - 1) / Fft<NY>::G, (NY / 2 + Fft<NZ>::G - 1) / Fft<NZ>::G>();
}

// ---- shared-memory budgets (bytes) ----------------------------------------
template <int NY, int NZ>
constexpr size_t plane_fwd_smem() {  // complex tile, real plane (pitch NZ + 8), line scratch
    return sizeof(float2) * (size_t)NY * (NZ / 2 + 1) + sizeof(float) * (size_t)NY * (NZ + 8) +
           sizeof(float2) * (size_t)plane_warps<NY, NZ>() * imax<Fft<NY>::WARP_SCRATCH, Fft<NZ>::WARP_SCRATCH>();
}
template <int NY, int NZ>
constexpr size_t plane_inv_smem() {  // complex tile, line scratch
    return sizeof(float2) * (size_t)NY * (NZ / 2 + 1) +
           sizeof(float2) * (size_t)plane_warps<NY, NZ>() * imax<Fft<NY>::WARP_SCRATCH, Fft<NZ>::WARP_SCRATCH>();
}
template <int NX>
constexpr size_t x_green_smem() {  // line scratch
    return sizeof(float2) * (size_t)FFT_WARPS * Fft<NX>::WARP_SCRATCH;
}

// ---- plane forward: z real-to-complex rows, then y columns ----------------
template <int NY, int NZ>
__global__ void __launch_bounds__(32 * plane_warps<NY, NZ>()) k_fft_plane_fwd(const float *__restrict__ rho,
                                                                            float2 *__restrict__ A) {
    using FZ = Fft<NZ>;
    using FY = Fft<NY>;
    constexpr int MZH = NZ / 2 + 1, RP = NZ + 8;  // RP: real-plane pitch
    constexpr int NW = plane_warps<NY, NZ>(), NT = 32 * NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);                      // [NY][MZH]
    float *real = reinterpret_cast<float *>(tile + NY * MZH);                  // [NY][RP]
    float2 *scr_all = reinterpret_cast<float2 *>(real + NY * RP);             // per warp
    __shared__ float2 twz[NZ];
    __shared__ float2 twy[NY];
    fill_twiddles<NZ>(twz);
    fill_twiddles<NY>(twy);
    pdl_wait();  // the mesh charge of make_rho is complete
    pdl_trigger();
    const int x = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *wscr = scr_all + warp * imax<FY::WARP_SCRATCH, FZ::WARP_SCRATCH>();
    {
        const float4 *plane = reinterpret_cast<const float4 *>(rho + (int64_t)x * NY * NZ);
        float4 *r4 = reinterpret_cast<float4 *>(real);
        stage<NY * NZ / 4, NT>(r4, [&](int e) { return __ldg(plane + e); },
                           [](int e) { return (e / (NZ / 4)) * (RP / 4) + e % (NZ / 4); });
    }
    __syncthreads();

    // z: rows 2p and 2p + 1 as the real and imaginary parts of one transform
    {
        const int g = lane / FZ::L, j = lane % FZ::L;
        float2 *scr = wscr + g * FZ::S;
        for (int p0 = warp * FZ::G; p0 < NY / 2; p0 += NW * FZ::G) {
            const int p = p0 + g;
            const bool ok = p < NY / 2;
            float2 v[FZ::E];
#pragma unroll
            for (int a = 0; a < FZ::E; ++a) {
                const int n = j + FZ::L * a;
                v[a] = ok ? make_float2(real[(2 * p) * RP + n], real[(2 * p + 1) * RP + n]) : make_float2(0.f, 0.f);
            }
            fft_in_out<NZ, false>(v, scr, twz, j);
            // Z[k] in natural order, then X1 = (Z[k] + conj Z[-k]) / 2, X2 = (Z[k] - conj Z[-k]) / 2i
#pragma unroll
            for (int r = 0; r < FZ::E; ++r) scr[out_index<NZ>(j, r)] = v[r];
            __syncwarp();
            constexpr int T = (MZH + FZ::L - 1) / FZ::L;
            float2 x1[T], x2[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int k = j + FZ::L * t;
                if (k < MZH) {
                    const float2 zk = scr[k], zm = scr[k == 0 ? 0 : NZ - k];  // Z[-k]
                    x1[t] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                    x2[t] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
                }
            }
            __syncwarp();
            if (ok) {
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const int k = j + FZ::L * t;
                    if (k < MZH) {
                        tile[(2 * p) * MZH + k] = x1[t];
                        tile[(2 * p + 1) * MZH + k] = x2[t];
                    }
                }
            }
        }
    }
    __syncthreads();

    // y: every kz column
    {
        const int g = lane / FY::L, j = lane % FY::L;
        float2 *scr = wscr + g * FY::S;
        for (int c0 = warp * FY::G; c0 < MZH; c0 += NW * FY::G) {
            const int col = c0 + g;
            const bool ok = col < MZH;
            float2 v[FY::E];
#pragma unroll
            for (int a = 0; a < FY::E; ++a) v[a] = ok ? tile[(j + FY::L * a) * MZH + col] : make_float2(0.f, 0.f);
            fft_in_out<NY, false>(v, scr, twy, j);
            if (ok) {
#pragma unroll
                for (int r = 0; r < FY::E; ++r) tile[out_index<NY>(j, r) * MZH + col] = v[r];
            }
        }
    }
    __syncthreads();
    float2 *o = A + (int64_t)x * NY * MZH;
    for (int e = threadIdx.x; e < NY * MZH; e += NT) o[e] = tile[e];
}

// ---- x transform, influence function, energy/virial, x inverse ------------
// A group of lanes per (ky, kz) line; CTA (line block lb < nlb, component a),
// grid nlb * ncomp.  A = [NX][My][MZH], S = [ncomp][NX][My][MZH].
template <int NX, int MZH, bool IK>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_green(int My, int nlb, const float2 *__restrict__ A,
                                                            float2 *__restrict__ S, GreenBufs b, EnergyConsts ec) {
    using F = Fft<NX>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float2 tw[NX];
    __shared__ float kvx[NX], kdx[NX];
    __shared__ double sh[7][FFT_WARPS];
    fill_twiddles<NX>(tw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / F::L, j = lane % F::L;
    float2 *scr = reinterpret_cast<float2 *>(smem_raw) + warp * F::WARP_SCRATCH + g * F::S;
    const int lb = blockIdx.x % nlb, a = blockIdx.x / nlb;
    const int line = (lb * FFT_WARPS + warp) * F::G + g;
    const bool ok = line < My * MZH;
    const int ky = ok ? line / MZH : 0, kz = ok ? line - ky * MZH : 0;
    const float *__restrict__ Gs = reinterpret_cast<const float *>(b.Gs);
    const float *__restrict__ kv = reinterpret_cast<const float *>(b.kvec);
    const float *__restrict__ kd = reinterpret_cast<const float *>(b.kdiff);
    const int64_t total = (int64_t)NX * My * MZH;
    // plan constants (nothing in the step writes them), loaded before the
    // wait: G / M of this lane's out-layout points, the x wavenumbers and
    // derivative factors (shared), this line's y and z ones
    float Gk[F::E];
#pragma unroll
    for (int r = 0; r < F::E; ++r) {
        const int k = out_index<NX>(j, r);
        Gk[r] = ok ? __ldg(Gs + ((int64_t)k * My + ky) * MZH + kz) : 0.0f;
    }
    for (int t = threadIdx.x; t < NX; t += FFT_THREADS) {
        kvx[t] = __ldg(kv + t);
        kdx[t] = __ldg(kd + t);
    }
    const float kyv = __ldg(kv + NX + ky), kzv = __ldg(kv + NX + My + kz);
    const float dky = __ldg(kd + NX + ky), dkz = __ldg(kd + NX + My + kz);
    __syncthreads();  // twiddles and wavenumber tables
    pdl_wait();
    pdl_trigger();
    float2 v[F::E];
#pragma unroll
    for (int q = 0; q < F::E; ++q)
        v[q] = ok ? A[((int64_t)(j + F::L * q) * My + ky) * MZH + kz] : make_float2(0.f, 0.f);
    fft_in_out<NX, false>(v, scr, tw, j);

    if (a == 0) {
        // the energy/virial sums of k_green (Mz is even: kz = 0 and kz = Mz/2
        // count once, the others twice)
        const float i4g2 = (float)ec.inv4g2;
        const float w = (kz == 0 || kz == MZH - 1) ? 1.0f : 2.0f;
        float acc[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int r = 0; r < F::E; ++r) {
            const float s = w * Gk[r] * (v[r].x * v[r].x + v[r].y * v[r].y);
            const float kxv = kvx[out_index<NX>(j, r)];
            const float k2 = kxv * kxv + kyv * kyv + kzv * kzv;
            const float fac = (k2 > 0.0f) ? 2.0f * (1.0f + k2 * i4g2) / k2 : 0.0f;
            const float sf = s * fac;
            acc[0] += s;
            acc[1] += s - sf * kxv * kxv;
            acc[2] += s - sf * kyv * kyv;
            acc[3] += s - sf * kzv * kzv;
            acc[4] -= sf * kxv * kyv;
            acc[5] -= sf * kxv * kzv;
            acc[6] -= sf * kyv * kzv;
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const float t = warp_sum_t<float>(acc[c]);
            if (lane == 0) sh[c][warp] = (double)t;
        }
        __syncthreads();
        if (threadIdx.x < 7) {
            double t = 0.0;
            for (int w2 = 0; w2 < FFT_WARPS; ++w2) t += sh[threadIdx.x][w2];
            b.part[7 * lb + threadIdx.x] = t;
        }
    }

#pragma unroll
    for (int r = 0; r < F::E; ++r) {
        const float pr = Gk[r] * v[r].x, pi = Gk[r] * v[r].y;
        if (IK) {
            // E_a = -i k_a G rho_hat / M  ->  (k_a pi, -k_a pr), Nyquist zeroed
            const float dk = (a == 0) ? kdx[out_index<NX>(j, r)] : ((a == 1) ? dky : dkz);
            v[r] = make_float2(dk * pi, -dk * pr);
        } else {
            v[r] = make_float2(pr, pi);
        }
    }
    fft_out_in<NX, true>(v, scr, tw, j);
    if (ok) {
        float2 *o = S + a * total;
#pragma unroll
        for (int q = 0; q < F::E; ++q) o[((int64_t)(j + F::L * q) * My + ky) * MZH + kz] = v[q];
    }
}

// ---- x pass with staged lines (large meshes) --------------------------------
// The same work as k_fft_x_green, but a CTA's XL_LINES consecutive lines
// (line = ky MZH + kz, contiguous in A, S and G) come in and go out as
// 16-byte copies of each x plane's run (XL_LINES x 8 bytes of A and S,
// XL_LINES x 4 bytes of G) through shared memory, instead of one 8-byte load
// per lane and point.  Needs nlines = My MZH even (16-byte aligned runs).
constexpr int XL_LINES = 16;  // lines of a CTA: FFT_WARPS warps x 2 groups of 16 lanes (N = 256)
template <int NX>
struct XStage {
    static constexpr int AP = XL_LINES + 1;  // complex pitch of an x row of the A / S tile
    static constexpr int GP = XL_LINES + 1;  // float pitch of an x row of the G tile
    static constexpr size_t A_BYTES = sizeof(float2) * NX * AP;
    static constexpr size_t G_BYTES = (sizeof(float) * NX * GP + 15) / 16 * 16;
    static constexpr size_t SMEM = A_BYTES + G_BYTES + sizeof(float2) * FFT_WARPS * Fft<NX>::WARP_SCRATCH;
    static_assert(FFT_WARPS * Fft<NX>::G == XL_LINES, "one line per group");
};

template <int NX, bool IK>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_green_st(int My, int MZH, int nlb, const float2 *__restrict__ A,
                                                                float2 *__restrict__ S, GreenBufs b, EnergyConsts ec) {
    using F = Fft<NX>;
    using X = XStage<NX>;
    constexpr int AP = X::AP, GP = X::GP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *at = reinterpret_cast<float2 *>(smem_raw);                                        // [NX][AP]
    float *gt = reinterpret_cast<float *>(smem_raw + X::A_BYTES);                              // [NX][GP]
    float2 *scr_all = reinterpret_cast<float2 *>(smem_raw + X::A_BYTES + X::G_BYTES);
    __shared__ float2 tw[NX];
    __shared__ float kvx[NX], kdx[NX];
    __shared__ double sh[7][FFT_WARPS];
    fill_twiddles<NX>(tw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / F::L, j = lane % F::L;
    float2 *scr = scr_all + warp * F::WARP_SCRATCH + g * F::S;
    const int lb = blockIdx.x % nlb, a = blockIdx.x / nlb;
    const int nlines = My * MZH;
    const int line0 = lb * XL_LINES;
    const int nl = min(XL_LINES, nlines - line0);  // even: nlines and line0 are
    const int l = warp * F::G + g;                 // this group's line in the CTA
    const int line = line0 + l;
    const bool ok = l < nl;
    const int ky = ok ? line / MZH : 0, kz = ok ? line - ky * MZH : 0;
    const float *__restrict__ Gs = reinterpret_cast<const float *>(b.Gs);
    const float *__restrict__ kv = reinterpret_cast<const float *>(b.kvec);
    const float *__restrict__ kd = reinterpret_cast<const float *>(b.kdiff);
    const int64_t total = (int64_t)NX * nlines;
    // plan constants first (nothing in the step writes them): G of the
    // CTA's lines in 16-byte pieces (4 lines each), wavenumber tables
    {
        const int gq = nl / 4, gr = nl % 4;  // whole 4-line pieces, then the 2-line rest
        for (int e = threadIdx.x; e < NX * (gq + (gr ? 1 : 0)); e += FFT_THREADS) {
            const int x = e / (gq + (gr ? 1 : 0)), c = e % (gq + (gr ? 1 : 0));
            const float *src = Gs + (int64_t)x * nlines + line0 + 4 * c;
            if (c < gq) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
                float *d = gt + x * GP + 4 * c;
                d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
            } else {
                const float2 v = __ldg(reinterpret_cast<const float2 *>(src));
                float *d = gt + x * GP + 4 * c;
                d[0] = v.x; d[1] = v.y;
            }
        }
    }
    for (int t = threadIdx.x; t < NX; t += FFT_THREADS) {
        kvx[t] = __ldg(kv + t);
        kdx[t] = __ldg(kd + t);
    }
    const float kyv = __ldg(kv + NX + ky), kzv = __ldg(kv + NX + My + kz);
    const float dky = __ldg(kd + NX + ky), dkz = __ldg(kd + NX + My + kz);
    pdl_wait();
    pdl_trigger();
    // this CTA's lines of every x plane of A: nl / 2 16-byte pieces per plane
    {
        const int pc = nl / 2;
        for (int e = threadIdx.x; e < NX * pc; e += FFT_THREADS) {
            const int x = e / pc, c = e % pc;
            const float4 v = *reinterpret_cast<const float4 *>(A + (int64_t)x * nlines + line0 + 2 * c);
            float2 *d = at + x * AP + 2 * c;
            d[0] = make_float2(v.x, v.y);
            d[1] = make_float2(v.z, v.w);
        }
    }
    __syncthreads();  // tiles, twiddles and wavenumber tables

    float2 v[F::E];
#pragma unroll
    for (int q = 0; q < F::E; ++q) v[q] = ok ? at[(j + F::L * q) * AP + l] : make_float2(0.f, 0.f);
    fft_in_out<NX, false>(v, scr, tw, j);
    float Gk[F::E];
#pragma unroll
    for (int r = 0; r < F::E; ++r) Gk[r] = ok ? gt[out_index<NX>(j, r) * GP + l] : 0.0f;

    if (a == 0) {
        // the energy/virial sums of k_green (Mz even: kz = 0 and Mz/2 count once)
        const float i4g2 = (float)ec.inv4g2;
        const float w = (kz == 0 || kz == MZH - 1) ? 1.0f : 2.0f;
        float acc[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int r = 0; r < F::E; ++r) {
            const float s = w * Gk[r] * (v[r].x * v[r].x + v[r].y * v[r].y);
            const float kxv = kvx[out_index<NX>(j, r)];
            const float k2 = kxv * kxv + kyv * kyv + kzv * kzv;
            const float fac = (k2 > 0.0f) ? 2.0f * (1.0f + k2 * i4g2) / k2 : 0.0f;
            const float sf = s * fac;
            acc[0] += s;
            acc[1] += s - sf * kxv * kxv;
            acc[2] += s - sf * kyv * kyv;
            acc[3] += s - sf * kzv * kzv;
            acc[4] -= sf * kxv * kyv;
            acc[5] -= sf * kxv * kzv;
            acc[6] -= sf * kyv * kzv;
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const float t = warp_sum_t<float>(acc[c]);
            if (lane == 0) sh[c][warp] = (double)t;
        }
    }
#pragma unroll
    for (int r = 0; r < F::E; ++r) {
        const float pr = Gk[r] * v[r].x, pi = Gk[r] * v[r].y;
        if (IK) {
            const float dk = (a == 0) ? kdx[out_index<NX>(j, r)] : ((a == 1) ? dky : dkz);
            v[r] = make_float2(dk * pi, -dk * pr);
        } else {
            v[r] = make_float2(pr, pi);
        }
    }
    fft_out_in<NX, true>(v, scr, tw, j);
#pragma unroll
    for (int q = 0; q < F::E; ++q) at[(j + F::L * q) * AP + l] = v[q];
    __syncthreads();  // every line back in the tile (and the energy partials in sh)
    if (a == 0 && threadIdx.x < 7) {
        double t = 0.0;
        for (int w2 = 0; w2 < FFT_WARPS; ++w2) t += sh[threadIdx.x][w2];
        b.part[7 * lb + threadIdx.x] = t;
    }
    {
        float2 *o = S + a * total;
        const int pc = nl / 2;
        for (int e = threadIdx.x; e < NX * pc; e += FFT_THREADS) {
            const int x = e / pc, c = e % pc;
            const float2 *sv = at + x * AP + 2 * c;
            *reinterpret_cast<float4 *>(o + (int64_t)x * nlines + line0 + 2 * c) = make_float4(sv[0].x, sv[0].y, sv[1].x, sv[1].y);
        }
    }
}

// ---- plane inverse: y columns, then z complex-to-real row pairs ------------
// Grid Mx * ncomp; CTA (x, a).  Output: out[((x NY + y) NZ + z) * stride + a].
template <int NY, int NZ>
__global__ void __launch_bounds__(32 * plane_warps<NY, NZ>()) k_fft_plane_inv(const float2 *__restrict__ S,
                                                                            float *__restrict__ out, int Mx,
                                                                            int64_t comp_stride, int stride) {
    using FZ = Fft<NZ>;
    using FY = Fft<NY>;
    constexpr int MZH = NZ / 2 + 1;
    constexpr int NW = plane_warps<NY, NZ>(), NT = 32 * NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);  // [NY][MZH]
    float2 *scr_all = tile + NY * MZH;
    __shared__ float2 twz[NZ];
    __shared__ float2 twy[NY];
    fill_twiddles<NZ>(twz);
    fill_twiddles<NY>(twy);
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x % Mx, a = blockIdx.x / Mx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *wscr = scr_all + warp * imax<FY::WARP_SCRATCH, FZ::WARP_SCRATCH>();
    {
        const float2 *g = S + a * comp_stride + (int64_t)x * NY * MZH;
        stage<NY * MZH, NT>(tile, [&](int e) { return g[e]; }, [](int e) { return e; });
    }
    __syncthreads();

    // y inverse: every kz column (out layout in, in layout out)
    {
        const int g = lane / FY::L, j = lane % FY::L;
        float2 *scr = wscr + g * FY::S;
        for (int c0 = warp * FY::G; c0 < MZH; c0 += NW * FY::G) {
            const int col = c0 + g;
            const bool ok = col < MZH;
            float2 v[FY::E];
#pragma unroll
            for (int r = 0; r < FY::E; ++r)
                v[r] = ok ? tile[out_index<NY>(j, r) * MZH + col] : make_float2(0.f, 0.f);
            fft_out_in<NY, true>(v, scr, twy, j);
            if (ok) {
#pragma unroll
                for (int q = 0; q < FY::E; ++q) tile[(j + FY::L * q) * MZH + col] = v[q];
            }
        }
    }
    __syncthreads();

    // z: rows 2p, 2p + 1 from one inverse of Z = X1 + i X2 (both Hermitian-
    // extended; the imaginary parts of the k = 0 and k = Mz/2 terms, which a
    // real row cannot carry, are dropped)
    {
        const int g = lane / FZ::L, j = lane % FZ::L;
        float2 *scr = wscr + g * FZ::S;
        float *plane = out + (int64_t)x * NY * NZ * stride + a;
        for (int p0 = warp * FZ::G; p0 < NY / 2; p0 += NW * FZ::G) {
            const int p = p0 + g;
            const bool ok = p < NY / 2;
            float2 v[FZ::E];
#pragma unroll
            for (int r = 0; r < FZ::E; ++r) {
                const int k = out_index<NZ>(j, r);
                float2 x1 = make_float2(0.f, 0.f), x2 = make_float2(0.f, 0.f);
                if (ok) {
                    const int kk = (k < MZH) ? k : NZ - k;
                    x1 = tile[(2 * p) * MZH + kk];
                    x2 = tile[(2 * p + 1) * MZH + kk];
                    if (k >= MZH) {
                        x1.y = -x1.y;
                        x2.y = -x2.y;
                    }
                    if (k == 0 || k == NZ / 2) {
                        x1.y = 0.f;
                        x2.y = 0.f;
                    }
                }
                v[r] = make_float2(x1.x - x2.y, x1.y + x2.x);
            }
            fft_out_in<NZ, true>(v, scr, twz, j);
            if (ok) {
#pragma unroll
                for (int q = 0; q < FZ::E; ++q) {
                    const int n = j + FZ::L * q;
                    plane[(int64_t)((2 * p) * NZ + n) * stride] = v[q].x;
                    plane[(int64_t)((2 * p + 1) * NZ + n) * stride] = v[q].y;
                }
            }
        }
    }
}

// ---- edge 256: plane passes on clusters of CTAs ------------------------------
// A plane's kz columns 0 .. NZ/2 are split CL ways: rank r of the cluster
// holds columns [r CW, (r + 1) CW) (CW = NZ / 2CL) of all NY rows in a shared
// tile [NY][CW + 1], and rank 0 also the Nyquist column kz = NZ/2 in its tile
// column CW.  Columns kz = 0 and kz = NZ/2 of a plane are real sequences over
// y before the forward y transform and after the inverse one (the z
// transform of a real row is real there), so rank 0 transforms the two
// together as one complex line, the same packing as two real rows in z, and
// every rank runs exactly CW y transforms.  The z transforms of a rank's
// NY/CL rows read (inverse) or write (forward) the other ranks' tiles through
// distributed shared memory.  Cluster sizes as measured at 256^3 on GB300:
// the forward pass on eight CTAs (the smallest tiles: two CTAs an SM, 82 us
// against 88 us on four), the inverse on four (80 us against 106 us on
// eight, whose z transforms read seven eighths of their input remotely).
namespace cg = cooperative_groups;
constexpr int FFT_CL_FWD = 8, FFT_CL_INV = 4;  // CTAs of a plane's cluster

template <int NY, int NZ, int CL>
struct PlaneCl {
    static constexpr int MZH = NZ / 2 + 1;
    static constexpr int CW = NZ / (2 * CL);       // kz columns per rank
    static constexpr int TP = CW + 1;              // tile pitch (complex)
    static constexpr int ROWS = NY / CL;           // z rows per rank
    static constexpr int SP = NZ + 8;              // staged real row pitch (floats): the two row pairs of a
                                                   // warp's groups sit 16 banks apart
    static constexpr int NW = 8, NT = 32 * NW;
    static constexpr int SCR = imax<Fft<NY>::WARP_SCRATCH, Fft<NZ>::WARP_SCRATCH>();
    static constexpr size_t TILE = sizeof(float2) * NY * TP;
    static constexpr size_t STAGE = sizeof(float) * ROWS * SP;  // forward: this rank's real rows
    static constexpr size_t SCRB = sizeof(float2) * NW * SCR;
    static constexpr size_t FWD_SMEM = TILE + STAGE + SCRB;
    static constexpr size_t INV_SMEM = TILE + SCRB;
    static_assert(CW * 2 * CL == NZ && ROWS * CL == NY, "edges split evenly over the cluster");
    static_assert((ROWS / 2) % (NW * Fft<NZ>::G) == 0 && CW % (NW * Fft<NY>::G) == 0, "whole passes");
    static_assert(TILE % 16 == 0 && STAGE % 16 == 0 && (SP * 4) % 16 == 0, "16-byte aligned regions");
};

// rank and tile column of spectrum column kz (0 <= kz <= CL CW)
template <int CW, int CL>
__device__ __forceinline__ void kz_home(int kz, int &rank, int &col) {
    if (kz == CL * CW) {
        rank = 0;
        col = CW;
    } else {
        rank = kz / CW;
        col = kz % CW;
    }
}

// asynchronous global -> shared copies (16 bytes: both addresses 16-byte
// aligned; 8 bytes: 8-byte aligned)
__device__ __forceinline__ void fft_cp16(void *smem, const void *gmem) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void fft_cp8(void *smem, const void *gmem) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void fft_cp_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Forward plane pass, cluster (x-plane x, rank r): z real-to-complex of rows
// [r NY/CL, (r + 1) NY/CL) into every rank's tile, then the y transform of
// this rank's columns.  Grid CL Mx.
template <int NY, int NZ, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(PlaneCl<NY, NZ, CL>::NT)
    k_fft_plane_fwd_cl(const float *__restrict__ rho, float2 *__restrict__ A) {
    using C = PlaneCl<NY, NZ, CL>;
    using FZ = Fft<NZ>;
    using FY = Fft<NY>;
    constexpr int MZH = C::MZH, CW = C::CW, TP = C::TP, SP = C::SP, NW = C::NW, NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);                           // [NY][TP]
    float *stg = reinterpret_cast<float *>(smem_raw + C::TILE);                     // [ROWS][SP]
    float2 *scr_all = reinterpret_cast<float2 *>(smem_raw + C::TILE + C::STAGE);   // per warp
    __shared__ float2 twz[NZ];
    __shared__ float2 twy[NY];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int x = blockIdx.x / CL;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *wscr = scr_all + warp * C::SCR;
    fill_twiddles<NZ>(twz);
    fill_twiddles<NY>(twy);
    pdl_wait();  // the mesh charge of make_rho is complete
    {
        const float *src = rho + ((int64_t)x * NY + rank * C::ROWS) * NZ;
        for (int e = threadIdx.x; e < C::ROWS * NZ / 4; e += NT) {
            const int row = e / (NZ / 4), c4 = e % (NZ / 4);
            fft_cp16(stg + row * SP + 4 * c4, src + 4 * e);
        }
    }
    pdl_trigger();
    cl.sync();  // every rank runs before the first store into its tile; orders the twiddles
    fft_cp_wait_all();
    __syncthreads();

    // z: local rows 2p and 2p + 1 as the real and imaginary parts of one transform
    {
        const int g = lane / FZ::L, j = lane % FZ::L;
        float2 *scr = wscr + g * FZ::S;
        constexpr int T = (MZH + FZ::L - 1) / FZ::L;
        for (int p0 = warp * FZ::G; p0 < C::ROWS / 2; p0 += NW * FZ::G) {
            const int p = p0 + g;
            float2 v[FZ::E];
#pragma unroll
            for (int a = 0; a < FZ::E; ++a) {
                const int n = j + FZ::L * a;
                v[a] = make_float2(stg[(2 * p) * SP + n], stg[(2 * p + 1) * SP + n]);
            }
            fft_in_out<NZ, false>(v, scr, twz, j);
#pragma unroll
            for (int r = 0; r < FZ::E; ++r) scr[out_index<NZ>(j, r)] = v[r];
            __syncwarp();
            const int y0 = rank * C::ROWS + 2 * p;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int k = j + FZ::L * t;
                if (k < MZH) {
                    const float2 zk = scr[k], zm = scr[k == 0 ? 0 : NZ - k];  // Z[-k]
                    int hr, hc;
                    kz_home<CW, CL>(k, hr, hc);
                    float2 *h = cl.map_shared_rank(tile + y0 * TP + hc, hr);
                    h[0] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                    h[TP] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
                }
            }
            __syncwarp();
        }
    }
    cl.sync();  // every rank's tile holds its columns of all NY rows

    // y: this rank's CW columns (rank 0's first line carries kz = 0 and NZ/2)
    {
        const int g = lane / FY::L, j = lane % FY::L;
        float2 *scr = wscr + g * FY::S;
        for (int c0 = warp * FY::G; c0 < CW; c0 += NW * FY::G) {
            const int col = c0 + g;
            const bool pk = (rank == 0 && col == 0);
            float2 v[FY::E];
#pragma unroll
            for (int a = 0; a < FY::E; ++a) {
                const int y = j + FY::L * a;
                v[a] = pk ? make_float2(tile[y * TP].x, tile[y * TP + CW].x) : tile[y * TP + col];
            }
            fft_in_out<NY, false>(v, scr, twy, j);
#pragma unroll
            for (int r = 0; r < FY::E; ++r) scr[out_index<NY>(j, r)] = v[r];
            __syncwarp();
#pragma unroll
            for (int t = 0; t < FY::E; ++t) {
                const int k = j + FY::L * t;
                const float2 zk = scr[k];
                if (pk) {
                    const float2 zm = scr[k == 0 ? 0 : NY - k];
                    tile[k * TP] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                    tile[k * TP + CW] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
                } else {
                    tile[k * TP + col] = zk;
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    float2 *o = A + (int64_t)x * NY * MZH + rank * CW;
    for (int e = threadIdx.x; e < NY * CW; e += NT) {
        const int ky = e / CW, c = e % CW;
        o[(int64_t)ky * MZH + c] = tile[ky * TP + c];
    }
    if (rank == 0)
        for (int ky = threadIdx.x; ky < NY; ky += NT) A[((int64_t)x * NY + ky) * MZH + NZ / 2] = tile[ky * TP + CW];
}

// Inverse plane pass, cluster (x-plane x, component a, rank r): y inverse of
// this rank's columns, then z complex-to-real of rows [r NY/CL, (r + 1) NY/CL)
// from every rank's tile.  Grid CL Mx ncomp.  Output as k_fft_plane_inv.
template <int NY, int NZ, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(PlaneCl<NY, NZ, CL>::NT)
    k_fft_plane_inv_cl(const float2 *__restrict__ S, float *__restrict__ out, int Mx, int64_t comp_stride,
                       int stride) {
    using C = PlaneCl<NY, NZ, CL>;
    using FZ = Fft<NZ>;
    using FY = Fft<NY>;
    constexpr int MZH = C::MZH, CW = C::CW, TP = C::TP, NW = C::NW, NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);                // [NY][TP]
    float2 *scr_all = reinterpret_cast<float2 *>(smem_raw + C::TILE);   // per warp
    __shared__ float2 twz[NZ];
    __shared__ float2 twy[NY];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int pl = blockIdx.x / CL;
    const int x = pl % Mx, a = pl / Mx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *wscr = scr_all + warp * C::SCR;
    fill_twiddles<NZ>(twz);
    fill_twiddles<NY>(twy);
    pdl_wait();
    {
        const float2 *src = S + a * comp_stride + (int64_t)x * NY * MZH;
        for (int e = threadIdx.x; e < NY * CW; e += NT) {
            const int ky = e / CW, c = e % CW;
            fft_cp8(tile + ky * TP + c, src + (int64_t)ky * MZH + rank * CW + c);
        }
        if (rank == 0)
            for (int ky = threadIdx.x; ky < NY; ky += NT) fft_cp8(tile + ky * TP + CW, src + (int64_t)ky * MZH + NZ / 2);
    }
    pdl_trigger();
    fft_cp_wait_all();
    __syncthreads();

    // y inverse: this rank's columns (out layout in, natural y order back
    // into the tile); rank 0's first line carries kz = 0 and NZ/2
    {
        const int g = lane / FY::L, j = lane % FY::L;
        float2 *scr = wscr + g * FY::S;
        for (int c0 = warp * FY::G; c0 < CW; c0 += NW * FY::G) {
            const int col = c0 + g;
            const bool pk = (rank == 0 && col == 0);
            float2 v[FY::E];
#pragma unroll
            for (int r = 0; r < FY::E; ++r) {
                const int ky = out_index<NY>(j, r);
                if (pk) {
                    const float2 z0 = tile[ky * TP], zn = tile[ky * TP + CW];
                    v[r] = make_float2(z0.x - zn.y, z0.y + zn.x);  // Z0 + i ZN
                } else {
                    v[r] = tile[ky * TP + col];
                }
            }
            fft_out_in<NY, true>(v, scr, twy, j);
#pragma unroll
            for (int q = 0; q < FY::E; ++q) {
                const int y = j + FY::L * q;
                if (pk) {
                    tile[y * TP] = make_float2(v[q].x, 0.f);
                    tile[y * TP + CW] = make_float2(v[q].y, 0.f);
                } else {
                    tile[y * TP + col] = v[q];
                }
            }
        }
    }
    cl.sync();  // every rank's columns are in natural y order

    // z: rows 2p, 2p + 1 from one inverse of Z = X1 + i X2 (imaginary parts
    // of the k = 0 and k = NZ/2 terms dropped, as in k_fft_plane_inv)
    {
        const int g = lane / FZ::L, j = lane % FZ::L;
        float2 *scr = wscr + g * FZ::S;
        float *plane = out + (int64_t)x * NY * NZ * stride + a;
        for (int p0 = warp * FZ::G; p0 < C::ROWS / 2; p0 += NW * FZ::G) {
            const int p = p0 + g;
            const int y0 = rank * C::ROWS + 2 * p;
            float2 v[FZ::E];
#pragma unroll
            for (int r = 0; r < FZ::E; ++r) {
                const int k = out_index<NZ>(j, r);
                const int kk = (k < MZH) ? k : NZ - k;
                int hr, hc;
                kz_home<CW, CL>(kk, hr, hc);
                const float2 *h = cl.map_shared_rank(tile + y0 * TP + hc, hr);
                float2 x1 = h[0], x2 = h[TP];
                if (k >= MZH) {
                    x1.y = -x1.y;
                    x2.y = -x2.y;
                }
                if (k == 0 || k == NZ / 2) {
                    x1.y = 0.f;
                    x2.y = 0.f;
                }
                v[r] = make_float2(x1.x - x2.y, x1.y + x2.x);
            }
            fft_out_in<NZ, true>(v, scr, twz, j);
#pragma unroll
            for (int q = 0; q < FZ::E; ++q) {
                const int n = j + FZ::L * q;
                plane[(int64_t)(y0 * NZ + n) * stride] = v[q].x;
                plane[(int64_t)((y0 + 1) * NZ + n) * stride] = v[q].y;
            }
        }
    }
    cl.sync();  // no rank leaves while another still reads its tile
}

// ---------------------------------------------------------------------------
// host side: dispatch over the mesh edges
// ---------------------------------------------------------------------------
// Cubic meshes of these edges use the mixed-radix lengths (one instantiation
// per edge rather than one per combination of edges).
bool cubic_mixed(const int M[3]) { return M[0] == M[1] && M[1] == M[2] && (M[0] == 48 || M[0] == 96); }

// Cubic meshes of edge 256 run the plane passes on clusters (PlaneCl).
bool cubic_256(const int M[3]) { return M[0] == 256 && M[1] == 256 && M[2] == 256; }

bool custom_fft_supported(const int M[3]) {
    if (cubic_mixed(M) || cubic_256(M)) return true;
    for (int d = 0; d < 3; ++d)
        if (M[d] != 16 && M[d] != 32 && M[d] != 64 && M[d] != 128) return false;
    return true;
}

// The plan's default: the hand-written solve wherever it runs, except at
// 256^3, where on GB300 the three passes took 82 + 82 + 80 us against cuFFT's
// 86 + 47 (influence function) + 84 us: at this size the six 1-D transforms
// per point cost about as many issue slots as the memory traffic, and the
// cluster passes hold only 16 to 24 warps an SM.
bool custom_fft_default(const int M[3]) { return custom_fft_supported(M) && !cubic_256(M); }

namespace {

template <typename... KArgs, typename... Args>
void launch_k(void (*kernel)(KArgs...), bool pdl, int grid, int threads, size_t smem, cudaStream_t s,
              Args... args) {
    if (pdl)
        launch_pdl(kernel, dim3(grid), dim3(threads), smem, s, args...);
    else
        kernel<<<grid, threads, smem, s>>>(args...);
}

// fn(std::integral_constant<int, n>) for n in {16, 32, 64, 128}
template <typename F>
void pow2_dispatch(int n, F &&fn) {
    switch (n) {
        case 16: fn(std::integral_constant<int, 16>{}); break;
        case 32: fn(std::integral_constant<int, 32>{}); break;
        case 64: fn(std::integral_constant<int, 64>{}); break;
        default: fn(std::integral_constant<int, 128>{}); break;
    }
}

template <int NX>
int x_line_blocks(int My, int mzh) {
    const int lines_per_cta = FFT_WARPS * Fft<NX>::G;
    return (My * mzh + lines_per_cta - 1) / lines_per_cta;
}

}  // namespace

template <int N>
cudaError_t prepare_cubic() {
    constexpr int MZH = N / 2 + 1;
    cudaError_t e = cudaFuncSetAttribute(k_fft_plane_fwd<N, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plane_fwd_smem<N, N>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_plane_inv<N, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)plane_inv_smem<N, N>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_x_green<N, MZH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)x_green_smem<N>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_x_green<N, MZH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)x_green_smem<N>());
    return e;
}

// fn(std::integral_constant<int, N>) for the cubic mixed-radix edge of M
template <typename F>
void cubic_dispatch(const int M[3], F &&fn) {
    if (M[0] == 48) fn(std::integral_constant<int, 48>{});
    else fn(std::integral_constant<int, 96>{});
}

cudaError_t prepare_cubic_256() {
    using CF = PlaneCl<256, 256, FFT_CL_FWD>;
    using CI = PlaneCl<256, 256, FFT_CL_INV>;
    cudaError_t e = cudaFuncSetAttribute(k_fft_plane_fwd_cl<256, 256, FFT_CL_FWD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::FWD_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_plane_inv_cl<256, 256, FFT_CL_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CI::INV_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_x_green_st<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)XStage<256>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_x_green_st<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)XStage<256>::SMEM);
    return e;
}

int custom_fft_parts(const int M[3]) {
    if (!custom_fft_supported(M)) return 0;
    const int mzh = M[2] / 2 + 1;
    int nlb = 0;
    if (cubic_256(M)) return (M[1] * mzh + XL_LINES - 1) / XL_LINES;
    if (cubic_mixed(M)) {
        cubic_dispatch(M, [&](auto nn) { nlb = x_line_blocks<decltype(nn)::value>(M[1], mzh); });
        return nlb;
    }
    pow2_dispatch(M[0], [&](auto nx) { nlb = x_line_blocks<decltype(nx)::value>(M[1], mzh); });
    return nlb;
}

cudaError_t prepare_custom_fft(const int M[3]) {
    if (!custom_fft_supported(M)) return cudaErrorInvalidValue;
    if (cubic_256(M)) return prepare_cubic_256();
    if (cubic_mixed(M)) return M[0] == 48 ? prepare_cubic<48>() : prepare_cubic<96>();
    cudaError_t e = cudaSuccess;
    pow2_dispatch(M[1], [&](auto ny) {
        pow2_dispatch(M[2], [&](auto nz) {
            constexpr int NY = decltype(ny)::value, NZ = decltype(nz)::value;
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_fft_plane_fwd<NY, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plane_fwd_smem<NY, NZ>());
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_fft_plane_inv<NY, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plane_inv_smem<NY, NZ>());
        });
    });
    pow2_dispatch(M[0], [&](auto nx) {
        pow2_dispatch(M[2], [&](auto nz) {
            constexpr int NX = decltype(nx)::value, MZH = decltype(nz)::value / 2 + 1;
            const int sm = (int)x_green_smem<NX>();
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_fft_x_green<NX, MZH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sm);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_fft_x_green<NX, MZH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sm);
        });
    });
    return e;
}

int launch_custom_fft(int step, const Geom<float> &g, bool ik_spec, const float *rho, void *rho_hat, void *spec,
                      float *field, const GreenBufs &b, const EnergyConsts &ec, bool pdl, cudaStream_t s) {
    float2 *A = reinterpret_cast<float2 *>(rho_hat);
    float2 *S = reinterpret_cast<float2 *>(spec);
    const int Mx = g.M[0], My = g.M[1];
    const int ncomp = ik_spec ? 3 : 1;
    const int64_t total = (int64_t)Mx * My * (g.M[2] / 2 + 1);
    int nparts = 0;
    if (cubic_256(g.M)) {
        using CF = PlaneCl<256, 256, FFT_CL_FWD>;
        using CI = PlaneCl<256, 256, FFT_CL_INV>;
        if (step == 0) {
            launch_k(k_fft_plane_fwd_cl<256, 256, FFT_CL_FWD>, pdl, FFT_CL_FWD * Mx, CF::NT, CF::FWD_SMEM, s, rho, A);
        } else if (step == 1) {
            const int nlb = (My * 129 + XL_LINES - 1) / XL_LINES;
            if (ik_spec)
                launch_k(k_fft_x_green_st<256, true>, pdl, nlb * ncomp, FFT_THREADS, XStage<256>::SMEM, s, My, 129, nlb,
                         (const float2 *)A, S, b, ec);
            else
                launch_k(k_fft_x_green_st<256, false>, pdl, nlb * ncomp, FFT_THREADS, XStage<256>::SMEM, s, My, 129,
                         nlb, (const float2 *)A, S, b, ec);
            nparts = nlb;
        } else {
            launch_k(k_fft_plane_inv_cl<256, 256, FFT_CL_INV>, pdl, FFT_CL_INV * Mx * ncomp, CI::NT, CI::INV_SMEM, s,
                     (const float2 *)S, field, Mx, total, ncomp == 3 ? 4 : 1);
        }
        return nparts;
    }
    if (cubic_mixed(g.M)) {
        cubic_dispatch(g.M, [&](auto nn) {
            constexpr int N = decltype(nn)::value, MZH = N / 2 + 1;
            if (step == 0) {
                launch_k(k_fft_plane_fwd<N, N>, pdl, Mx, 32 * plane_warps<N, N>(), plane_fwd_smem<N, N>(), s, rho, A);
            } else if (step == 1) {
                const int nlb = x_line_blocks<N>(My, MZH);
                if (ik_spec)
                    launch_k(k_fft_x_green<N, MZH, true>, pdl, nlb * ncomp, FFT_THREADS, x_green_smem<N>(), s, My, nlb,
                             (const float2 *)A, S, b, ec);
                else
                    launch_k(k_fft_x_green<N, MZH, false>, pdl, nlb * ncomp, FFT_THREADS, x_green_smem<N>(), s, My,
                             nlb, (const float2 *)A, S, b, ec);
                nparts = nlb;
            } else {
                launch_k(k_fft_plane_inv<N, N>, pdl, Mx * ncomp, 32 * plane_warps<N, N>(), plane_inv_smem<N, N>(), s,
                         (const float2 *)S, field, Mx, total, ncomp == 3 ? 4 : 1);
            }
        });
        return nparts;
    }
    if (step == 0) {
        pow2_dispatch(My, [&](auto ny) {
            pow2_dispatch(g.M[2], [&](auto nz) {
                constexpr int NY = decltype(ny)::value, NZ = decltype(nz)::value;
                launch_k(k_fft_plane_fwd<NY, NZ>, pdl, Mx, 32 * plane_warps<NY, NZ>(), plane_fwd_smem<NY, NZ>(), s,
                         rho, A);
            });
        });
    } else if (step == 1) {
        pow2_dispatch(Mx, [&](auto nx) {
            pow2_dispatch(g.M[2], [&](auto nz) {
                constexpr int NX = decltype(nx)::value, MZH = decltype(nz)::value / 2 + 1;
                const int nlb = x_line_blocks<NX>(My, MZH);
                const size_t sm = x_green_smem<NX>();
                if (ik_spec)
                    launch_k(k_fft_x_green<NX, MZH, true>, pdl, nlb * ncomp, FFT_THREADS, sm, s, My, nlb,
                             (const float2 *)A, S, b, ec);
                else
                    launch_k(k_fft_x_green<NX, MZH, false>, pdl, nlb * ncomp, FFT_THREADS, sm, s, My, nlb,
                             (const float2 *)A, S, b, ec);
                nparts = nlb;
            });
        });
    } else {
        pow2_dispatch(My, [&](auto ny) {
            pow2_dispatch(g.M[2], [&](auto nz) {
                constexpr int NY = decltype(ny)::value, NZ = decltype(nz)::value;
                launch_k(k_fft_plane_inv<NY, NZ>, pdl, Mx * ncomp, 32 * plane_warps<NY, NZ>(),
                         plane_inv_smem<NY, NZ>(), s, (const float2 *)S, field, Mx, total, ncomp == 3 ? 4 : 1);
            });
        });
    }
    return nparts;
}

}  // namespace pppm
