// The Poisson solve of Sec. 2.1 step 2 / Sec. 3.2 -- forward 3-D FFT of the
// mesh charge, multiply by the influence function, one (ad) or three (ik)
// inverse 3-D FFTs -- as three kernels for FP32 plans whose mesh edges are
// powers of two from 16 to 128:
//   plane forward   CTA per x-plane: z real-to-complex of every row, then the
//                   y transform of every kz column      rho -> A[x][ky][kz]
//   x + Green       CTA per (ky, component): x transform, energy/virial
//                   partials (component 0; the last such CTA also sums them),
//                   multiply by G (and -i k_a for ik), x inverse
//                                                       A -> S_a[x][ky][kz]
//   plane inverse   CTA per (x-plane, component): y inverse of every column,
//                   then z complex-to-real of every row
//                                                       S_a -> field / phi
// Same conventions as the cuFFT path (both directions unnormalised, G/M
// carries the 1/M), the same spectrum buffers, energy partials, final sums
// and field layout (ik: interleaved (E_x, E_y, E_z, pad) per point; ad and
// the potential: one value per point).  cuFFT serves other meshes and FP64.
//
// One 1-D transform of length N per warp: element i lives in lane i % 32,
// register i / 32, loaded in bit-reversed order; log2(N) radix-2
// decimation-in-time stages follow, a stage whose butterfly partner is in
// another lane exchanging through a shuffle and one whose partner is in the
// same lane working in registers.  Twiddles w_N^t = exp(-2 pi i t / N) come
// from a per-CTA table filled with sincospif.
#include <cmath>
#include <type_traits>

#include "pppm_common.cuh"

namespace pppm {

constexpr int FFT_THREADS = 256;
constexpr int FFT_WARPS = FFT_THREADS / 32;

template <int N>
struct FftLen {
    static_assert(N == 16 || N == 32 || N == 64 || N == 128, "power-of-two length 16..128");
    static constexpr int R = N >= 32 ? N / 32 : 1;  // elements per lane
    static constexpr int LOG = N == 16 ? 4 : N == 32 ? 5 : N == 64 ? 6 : 7;
};

template <int N>
__device__ __forceinline__ int bitrev(int i) {
    return (int)(__brev((unsigned)i) >> (32 - FftLen<N>::LOG));
}

// tw[t] = exp(-2 pi i t / N), t < N/2 (whole CTA; the caller synchronises)
template <int N>
__device__ __forceinline__ void fill_twiddles(float2 *tw) {
    for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
        float s, c;
        sincospif(-2.0f * (float)t / (float)N, &s, &c);
        tw[t] = make_float2(c, s);
    }
}

// In-place length-N transform of this warp's elements (bit-reversed input,
// natural-order output); INV takes exp(+2 pi i ...).  For N = 16 lanes 16..31
// carry no element but take part in the shuffles.
template <int N, bool INV>
__device__ __forceinline__ void warp_fft(float (&re)[FftLen<N>::R], float (&im)[FftLen<N>::R],
                                         const float2 *__restrict__ tw, int lane) {
    constexpr int R = FftLen<N>::R, LOG = FftLen<N>::LOG;
#pragma unroll
    for (int s = 1; s <= LOG; ++s) {
        const int half = 1 << (s - 1);
        const int tstep = N >> s;  // w_{2 half}^t = w_N^(t tstep)
        float nre[R], nim[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            float pre, pim;
            if (half < 32) {
                pre = __shfl_xor_sync(0xffffffffu, re[r], half);
                pim = __shfl_xor_sync(0xffffffffu, im[r], half);
            } else {
                const int rp = r ^ (half >> 5);
                pre = re[rp];
                pim = im[rp];
            }
            const float2 w = tw[(i & (half - 1)) * tstep];
            const float wr = w.x, wi = INV ? -w.y : w.y;
            if ((i & half) == 0) {  // upper: self + w * partner
                nre[r] = re[r] + (wr * pre - wi * pim);
                nim[r] = im[r] + (wr * pim + wi * pre);
            } else {                // lower: partner - w * self
                nre[r] = pre - (wr * re[r] - wi * im[r]);
                nim[r] = pim - (wr * im[r] + wi * re[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            re[r] = nre[r];
            im[r] = nim[r];
        }
    }
}

// Transform every column of a [N][ld] complex tile in shared memory in
// place, one warp per column.
template <int N, bool INV>
__device__ __forceinline__ void tile_columns(float2 *tile, int ld, const float2 *tw) {
    constexpr int R = FftLen<N>::R;
    const int lane = threadIdx.x & 31;
    for (int col = threadIdx.x >> 5; col < ld; col += FFT_WARPS) {
        float re[R], im[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            const float2 v = (i < N) ? tile[bitrev<N>(i & (N - 1)) * ld + col] : make_float2(0.f, 0.f);
            re[r] = v.x;
            im[r] = v.y;
        }
        __syncwarp();
        warp_fft<N, INV>(re, im, tw, lane);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            if (i < N) tile[i * ld + col] = make_float2(re[r], im[r]);
        }
    }
}

template <int N>
__host__ __device__ constexpr size_t tile_bytes(int ld) {
    return sizeof(float2) * (size_t)N * ld;
}

// dst[e] = src(e) for e < NEL by the whole CTA, up to eight loads in flight
// per thread before their stores (the sources sit in L2: one round trip per
// eight elements a thread instead of one per element).
template <int NEL, typename T, typename F>
__device__ __forceinline__ void stage(T *dst, F src) {
    constexpr int IT = (NEL + FFT_THREADS - 1) / FFT_THREADS;
    constexpr int CH = IT < 8 ? IT : 8;
#pragma unroll
    for (int k0 = 0; k0 < IT; k0 += CH) {
        T v[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int e = threadIdx.x + (k0 + k) * FFT_THREADS;
            if (k0 + k < IT && e < NEL) v[k] = src(e);
        }
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const int e = threadIdx.x + (k0 + k) * FFT_THREADS;
            if (k0 + k < IT && e < NEL) dst[e] = v[k];
        }
    }
}

template <int NY, int NZ>
constexpr size_t plane_fwd_smem() {  // complex tile + the real plane
    return tile_bytes<NY>(NZ / 2 + 1) + sizeof(float) * (size_t)NY * NZ;
}
template <int NX, int MZH>
constexpr size_t x_green_smem() {  // complex tile + G of the ky plane
    return tile_bytes<NX>(MZH) + sizeof(float) * (size_t)NX * MZH;
}

// ---- plane forward: z real-to-complex rows, then y columns ----------------
template <int NY, int NZ>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_plane_fwd(const float *__restrict__ rho,
                                                              float2 *__restrict__ A) {
    constexpr int RZ = FftLen<NZ>::R, MZH = NZ / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);                    // [NY][MZH]
    float *real = reinterpret_cast<float *>(smem_raw + tile_bytes<NY>(MZH));  // [NY][NZ]
    __shared__ float2 twz[NZ / 2];
    __shared__ float2 twy[NY / 2];
    fill_twiddles<NZ>(twz);
    fill_twiddles<NY>(twy);
    pdl_wait();  // the mesh charge of make_rho is complete
    pdl_trigger();
    const int x = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const float4 *plane = reinterpret_cast<const float4 *>(rho + (int64_t)x * NY * NZ);
    stage<NY * NZ / 4>(reinterpret_cast<float4 *>(real), [&](int e) { return __ldg(plane + e); });
    __syncthreads();
    for (int y = threadIdx.x >> 5; y < NY; y += FFT_WARPS) {
        const float *row = real + y * NZ;
        float re[RZ], im[RZ];
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = lane + 32 * r;
            re[r] = (i < NZ) ? row[bitrev<NZ>(i & (NZ - 1))] : 0.0f;
            im[r] = 0.0f;
        }
        warp_fft<NZ, false>(re, im, twz, lane);
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = lane + 32 * r;
            if (i < MZH) tile[y * MZH + i] = make_float2(re[r], im[r]);
        }
    }
    __syncthreads();
    tile_columns<NY, false>(tile, MZH, twy);
    __syncthreads();
    float2 *o = A + (int64_t)x * NY * MZH;
    for (int e = threadIdx.x; e < NY * MZH; e += FFT_THREADS) o[e] = tile[e];
}

// ---- x transform, influence function, energy/virial, x inverse ------------
// Grid My * ncomp; CTA (ky, a).  A = [NX][My][MZH], S = [ncomp][NX][My][MZH].
template <int NX, int MZH, bool IK>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_x_green(int My, const float2 *__restrict__ A,
                                                            float2 *__restrict__ S, GreenBufs b, EnergyConsts ec,
                                                            int map_nblk, double *ev_user) {
    constexpr int NEL = NX * MZH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);                   // [NX][MZH]
    float *gpl = reinterpret_cast<float *>(smem_raw + tile_bytes<NX>(MZH));  // [NX][MZH] G / M
    __shared__ float2 tw[NX / 2];
    __shared__ float kvx[NX], kdx[NX], kvz[MZH], kdz[MZH];
    __shared__ double sh[7][FFT_WARPS];
    __shared__ int last;
    fill_twiddles<NX>(tw);
    const int ky = blockIdx.x % My, a = blockIdx.x / My;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *__restrict__ Gs = reinterpret_cast<const float *>(b.Gs);
    const float *__restrict__ kv = reinterpret_cast<const float *>(b.kvec);
    const float *__restrict__ kd = reinterpret_cast<const float *>(b.kdiff);
    // plan constants (not written by the step): before the wait
    for (int t = threadIdx.x; t < NX; t += FFT_THREADS) {
        kvx[t] = __ldg(kv + t);
        kdx[t] = __ldg(kd + t);
    }
    for (int t = threadIdx.x; t < MZH; t += FFT_THREADS) {
        kvz[t] = __ldg(kv + NX + My + t);
        kdz[t] = __ldg(kd + NX + My + t);
    }
    const float kyv = __ldg(kv + NX + ky), dky = __ldg(kd + NX + ky);
    stage<NEL>(gpl, [&](int e) {
        const int x = e / MZH, kz = e - x * MZH;
        return __ldg(Gs + ((int64_t)x * My + ky) * MZH + kz);
    });
    pdl_wait();
    pdl_trigger();
    const int64_t total = (int64_t)NX * My * MZH;
    stage<NEL>(tile, [&](int e) {
        const int x = e / MZH, kz = e - x * MZH;
        return A[((int64_t)x * My + ky) * MZH + kz];
    });
    __syncthreads();
    tile_columns<NX, false>(tile, MZH, tw);
    __syncthreads();

    if (a == 0) {
        // the energy/virial sums of k_green over this ky plane (Mz is even:
        // kz = 0 and kz = Mz/2 count once, the others twice)
        const float i4g2 = (float)ec.inv4g2;
        float acc[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int e = threadIdx.x; e < NEL; e += FFT_THREADS) {
            const int kx = e / MZH, kz = e - kx * MZH;
            const float2 r = tile[e];
            const float G = gpl[e];
            const float w = (kz == 0 || kz == MZH - 1) ? 1.0f : 2.0f;
            const float s = w * G * (r.x * r.x + r.y * r.y);
            const float kxv = kvx[kx], kzv = kvz[kz];
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
            const float v = warp_sum_t<float>(acc[c]);
            if (lane == 0) sh[c][warp] = (double)v;
        }
        __syncthreads();
        if (threadIdx.x < 7) {
            double v = 0.0;
            for (int w2 = 0; w2 < FFT_WARPS; ++w2) v += sh[threadIdx.x][w2];
            b.part[7 * ky + threadIdx.x] = v;
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) last = (atomicAdd(b.counter, 1u) == (unsigned)(My - 1)) ? 1 : 0;
        __syncthreads();
        if (last) {  // every ky plane's partials are written: the final sums, fixed order
            __threadfence();
            energy_final_body(b, ec, My, map_nblk, ev_user);
            if (threadIdx.x == 0) *b.counter = 0u;
        }
    }

    // multiply and inverse, column by column in place (each warp owns its
    // columns; the energy pass above read the tile before its barrier)
    {
        constexpr int R = FftLen<NX>::R;
        for (int col = warp; col < MZH; col += FFT_WARPS) {
            const float dkz = kdz[col];
            float re[R], im[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = lane + 32 * r;
                const int kx = bitrev<NX>(i & (NX - 1));
                float vr = 0.f, vi = 0.f;
                if (i < NX) {
                    const float2 v = tile[kx * MZH + col];
                    const float G = gpl[kx * MZH + col];
                    const float pr = G * v.x, pi = G * v.y;
                    if (IK) {
                        // E_a = -i k_a G rho_hat / M  ->  (k_a pi, -k_a pr), Nyquist zeroed
                        const float dk = (a == 0) ? kdx[kx] : ((a == 1) ? dky : dkz);
                        vr = dk * pi;
                        vi = -dk * pr;
                    } else {
                        vr = pr;
                        vi = pi;
                    }
                }
                re[r] = vr;
                im[r] = vi;
            }
            __syncwarp();
            warp_fft<NX, true>(re, im, tw, lane);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = lane + 32 * r;
                if (i < NX) tile[i * MZH + col] = make_float2(re[r], im[r]);
            }
        }
    }
    __syncthreads();
    float2 *o = S + a * total;
    for (int e = threadIdx.x; e < NEL; e += FFT_THREADS) {
        const int x = e / MZH, kz = e - x * MZH;
        o[((int64_t)x * My + ky) * MZH + kz] = tile[e];
    }
}

// ---- plane inverse: y columns, then z complex-to-real rows -----------------
// Grid Mx * ncomp; CTA (x, a).  Output: out[((x NY + y) NZ + z) * stride + a].
template <int NY, int NZ>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_plane_inv(const float2 *__restrict__ S, float *__restrict__ out,
                                                              int Mx, int64_t comp_stride, int stride) {
    constexpr int RZ = FftLen<NZ>::R, MZH = NZ / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);  // [NY][MZH]
    __shared__ float2 twz[NZ / 2];
    __shared__ float2 twy[NY / 2];
    fill_twiddles<NZ>(twz);
    fill_twiddles<NY>(twy);
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x % Mx, a = blockIdx.x / Mx;
    const int lane = threadIdx.x & 31;
    const float2 *g = S + a * comp_stride + (int64_t)x * NY * MZH;
    stage<NY * MZH>(tile, [&](int e) { return g[e]; });
    __syncthreads();
    tile_columns<NY, true>(tile, MZH, twy);
    __syncthreads();
    float *plane = out + (int64_t)x * NY * NZ * stride + a;
    for (int y = threadIdx.x >> 5; y < NY; y += FFT_WARPS) {
        float re[RZ], im[RZ];
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = lane + 32 * r;
            const int k = bitrev<NZ>(i & (NZ - 1));
            float2 v = make_float2(0.f, 0.f);
            if (i < NZ) {  // the Hermitian extension of the half spectrum
                if (k < MZH) {
                    v = tile[y * MZH + k];
                } else {
                    v = tile[y * MZH + (NZ - k)];
                    v.y = -v.y;
                }
            }
            re[r] = v.x;
            im[r] = v.y;
        }
        warp_fft<NZ, true>(re, im, twz, lane);
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = lane + 32 * r;
            if (i < NZ) plane[(int64_t)(y * NZ + i) * stride] = re[r];
        }
    }
}

// ---------------------------------------------------------------------------
// host side: dispatch over the mesh edges
// ---------------------------------------------------------------------------
bool custom_fft_supported(const int M[3]) {
    for (int d = 0; d < 3; ++d)
        if (M[d] != 16 && M[d] != 32 && M[d] != 64 && M[d] != 128) return false;
    return true;
}

namespace {

template <typename... KArgs, typename... Args>
void launch_k(void (*kernel)(KArgs...), bool pdl, int grid, size_t smem, cudaStream_t s, Args... args) {
    if (pdl)
        launch_pdl(kernel, dim3(grid), dim3(FFT_THREADS), smem, s, args...);
    else
        kernel<<<grid, FFT_THREADS, smem, s>>>(args...);
}

// Calls fn.template operator()<N>() for N = n in {16, 32, 64, 128}.
template <typename F>
void pow2_dispatch(int n, F &&fn) {
    switch (n) {
        case 16: fn(std::integral_constant<int, 16>{}); break;
        case 32: fn(std::integral_constant<int, 32>{}); break;
        case 64: fn(std::integral_constant<int, 64>{}); break;
        default: fn(std::integral_constant<int, 128>{}); break;
    }
}

}  // namespace

cudaError_t prepare_custom_fft(const int M[3]) {
    if (!custom_fft_supported(M)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    pow2_dispatch(M[1], [&](auto ny) {
        pow2_dispatch(M[2], [&](auto nz) {
            constexpr int NY = decltype(ny)::value, NZ = decltype(nz)::value;
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_fft_plane_fwd<NY, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plane_fwd_smem<NY, NZ>());
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_fft_plane_inv<NY, NZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tile_bytes<NY>(NZ / 2 + 1));
        });
    });
    pow2_dispatch(M[0], [&](auto nx) {
        pow2_dispatch(M[2], [&](auto nz) {
            constexpr int NX = decltype(nx)::value, MZH = decltype(nz)::value / 2 + 1;
            const int sm = (int)x_green_smem<NX, MZH>();
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

void launch_custom_fft(int step, const Geom<float> &g, bool ik_spec, const float *rho, void *rho_hat, void *spec,
                       float *field, const GreenBufs &b, const EnergyConsts &ec, int map_nblk, double *ev_user,
                       bool pdl, cudaStream_t s) {
    float2 *A = reinterpret_cast<float2 *>(rho_hat);
    float2 *S = reinterpret_cast<float2 *>(spec);
    const int Mx = g.M[0], My = g.M[1];
    const int ncomp = ik_spec ? 3 : 1;
    const int64_t total = (int64_t)Mx * My * (g.M[2] / 2 + 1);
    if (step == 0) {
        pow2_dispatch(My, [&](auto ny) {
            pow2_dispatch(g.M[2], [&](auto nz) {
                constexpr int NY = decltype(ny)::value, NZ = decltype(nz)::value;
                launch_k(k_fft_plane_fwd<NY, NZ>, pdl, Mx, plane_fwd_smem<NY, NZ>(), s, rho, A);
            });
        });
    } else if (step == 1) {
        pow2_dispatch(Mx, [&](auto nx) {
            pow2_dispatch(g.M[2], [&](auto nz) {
                constexpr int NX = decltype(nx)::value, MZH = decltype(nz)::value / 2 + 1;
                const size_t sm = x_green_smem<NX, MZH>();
                if (ik_spec)
                    launch_k(k_fft_x_green<NX, MZH, true>, pdl, My * ncomp, sm, s, My, (const float2 *)A, S, b,
                             ec, map_nblk, ev_user);
                else
                    launch_k(k_fft_x_green<NX, MZH, false>, pdl, My * ncomp, sm, s, My, (const float2 *)A, S, b,
                             ec, map_nblk, ev_user);
            });
        });
    } else {
        pow2_dispatch(My, [&](auto ny) {
            pow2_dispatch(g.M[2], [&](auto nz) {
                constexpr int NY = decltype(ny)::value, NZ = decltype(nz)::value;
                launch_k(k_fft_plane_inv<NY, NZ>, pdl, Mx * ncomp, tile_bytes<NY>(NZ / 2 + 1), s,
                         (const float2 *)S, field, Mx, total, ncomp == 3 ? 4 : 1);
            });
        });
    }
}

}  // namespace pppm
