// The Poisson solve of Sec. 2.1 step 2 / Sec. 3.2 -- forward 3-D FFT of the
// mesh charge, multiply by the influence function, one (ad) or three (ik)
// inverse 3-D FFTs -- as three kernels for FP32 plans whose mesh edges are
// powers of two from 16 to 128, or cubic meshes of edge 48 or 96:
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
//
// One 1-D transform of length N = E L runs on a group of L lanes holding E
// points each (E = 8; 16 for N = 128, 12 for 48, 24 for 96), as the
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

#include "pppm_common.cuh"

namespace pppm {

constexpr int FFT_THREADS = 256;
constexpr int FFT_WARPS = FFT_THREADS / 32;

template <int N>
struct Fft {
    static_assert(N == 16 || N == 32 || N == 64 || N == 128 || N == 48 || N == 96, "supported lengths");
    static constexpr int E = (N == 128) ? 16 : (N == 96) ? 24 : (N == 48) ? 12 : 8;  // points per lane
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

// ---------------------------------------------------------------------------
// host side: dispatch over the mesh edges
// ---------------------------------------------------------------------------
// Cubic meshes of these edges use the mixed-radix lengths (one instantiation
// per edge rather than one per combination of edges).
bool cubic_mixed(const int M[3]) { return M[0] == M[1] && M[1] == M[2] && (M[0] == 48 || M[0] == 96); }

bool custom_fft_supported(const int M[3]) {
    if (cubic_mixed(M)) return true;
    for (int d = 0; d < 3; ++d)
        if (M[d] != 16 && M[d] != 32 && M[d] != 64 && M[d] != 128) return false;
    return true;
}

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

cudaError_t prepare_custom_fft(const int M[3]) {
    if (!custom_fft_supported(M)) return cudaErrorInvalidValue;
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
