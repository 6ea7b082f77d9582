// Internal definitions shared by the PPPM kernels and the C-ABI layer.
//
// Stencil convention (the order-P charge-assignment stencil of Sec. 3.1,
// "product of three polynomials of order equal to the stencil size"):
//   u = x_wrapped / h (grid coordinate), anchor n = floor(u + 1/2) for odd P
//   and floor(u) for even P, delta = n - u.  The P stencil points are
//   n - rlo + k (k = 0..P-1, rlo = (P-1)/2, wrapped mod M) with weight
//   W_k(delta) = sum_l coef[k][l] delta^l, the order-P B-spline restricted to
//   the unit piece that point k sees.
//
// Tiles: each mesh dimension of M points is cut into T = ceil(M/B) tiles with
// boundaries floor(t*M/T); every tile is between floor(M/T) and B points wide,
// which is >= 4 > rlo for the supported sizes, so a particle only reaches the
// 27 tiles around the tile of its anchor.  B = 8, or 16 along z for "long
// tiles" (compensated FP32 at order >= 6, see tile_shape).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include <cufft.h>

#include "../../include/pppm_gb300.h"

namespace pppm {

constexpr int MAXP = 7;
constexpr int TILE_B = 8;           // tile edge in mesh points
constexpr int MAX_MESH = 1024;

// Device error word bits (SortBufs::err): reported by pppm_sync.
constexpr int ERR_NONFINITE = 1;  // a non-finite position or charge
constexpr int ERR_INTERNAL = 2;   // a consistency check failed; the offending work was skipped

// Remembers a failed CUDA runtime call for pppm_last_cuda_error.
void note_cuda_error(cudaError_t e);

// ---------------------------------------------------------------------------
// Geometry and per-order constants passed to kernels by value.
// ---------------------------------------------------------------------------
template <typename R>
struct Geom {
    int M[3];
    int Mzh;            // Mz/2 + 1
    int T[3];           // tiles per dimension
    int TE[3];          // widest tile per dimension, ceil(M / T)
    int ntiles;
    int P, rlo;
    R L[3], iL[3];
    R ih[3];            // 1/h, and its rounding remainder (float path only)
    R ih_lo[3];
    R ivcell;           // 1 / (hx hy hz)
    R h[3];
    R coef[MAXP][MAXP];   // coef[k][l]: weight of stencil point k, power l of delta
    R dcoef[MAXP][MAXP];  // d/ddelta of the same polynomials
    int ff_tiled;         // fieldforce variant: 0 per-particle through L1, 1 tile-staged brick (one CTA a
                          // tile), 2 persistent double-buffered tile-staged brick (FP32 step types)
    int rho_copies;       // make_rho brick: 0 one, tile strides; 1 four interleaved copies (FP32C);
                          // 2 one, strides of the largest tile; 4 one per z-pair of tiles, those strides
    int lut_bins;         // coefficient table entries (0: exact polynomials), see pppm_set_lut
    int launch_flags;     // host side: LF_* launch options of this step
    int planar_stride;    // ik field layout: 0 interleaved (Ex,Ey,Ez,pad); > 0 three planes this far apart
    float wmax3;          // bound on a stencil point's weight product wx wy wz (0: use 1)
};

// Geom::launch_flags: green / fieldforce may use a programmatic dependent
// launch (their stream predecessor is a kernel, no event node in between).
constexpr int LF_PDL_GREEN = 1, LF_PDL_FF = 2;

template <typename R> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };
template <typename R> using vec4_t = typename Vec4<R>::type;

template <typename R> struct Complex;
template <> struct Complex<float> { using type = cufftComplex; };
template <> struct Complex<double> { using type = cufftDoubleComplex; };
template <typename R> using complex_t = typename Complex<R>::type;

__host__ __device__ inline int tile_of(int n, int T, int M) { return ((n + 1) * T - 1) / M; }

// Tiles per dimension (T) and the widest tile (TE) for tile edge TILE_B, or
// 2 TILE_B along z when long_z, or TILE_B / 2 when small.  Long tiles would
// halve the tile count and cut the halo share of the make_rho brick flush,
// but no dispatched make_rho takes bricks deeper than 16 points (one brick
// column per thread of its flush), so they are refused.  Small tiles give
// meshes with few 8^3 tiles enough CTAs for the GPU, at the price of a
// larger halo share.
inline void tile_shape(const int M[3], bool long_z, int T[3], int TE[3], bool small = false) {
    for (int d = 0; d < 3; ++d) {
        const int e = small ? TILE_B / 2 : ((d == 2 && long_z) ? 2 * TILE_B : TILE_B);
        T[d] = (M[d] + e - 1) / e;
        TE[d] = (M[d] + T[d] - 1) / T[d];
    }
}
inline bool long_tiles_allowed(int P, bool compensated) {
    (void)P;
    (void)compensated;
    return false;  // no make_rho brick deeper than 16 points (see tile_shape)
}
__host__ __device__ inline int tile_origin(int t, int T, int M) { return (t * M) / T; }

__host__ __device__ inline uint32_t pack_anchor(int a, int b, int c) {
    return (uint32_t)a | ((uint32_t)b << 10) | ((uint32_t)c << 20);
}
__host__ __device__ inline void unpack_anchor(uint32_t v, int &a, int &b, int &c) {
    a = (int)(v & 1023u);
    b = (int)((v >> 10) & 1023u);
    c = (int)((v >> 20) & 1023u);
}

// Rounded arithmetic that the compiler may not contract, so that two kernels
// computing the same anchor from the same position agree bit for bit.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Wrap one coordinate into [0, L) and return the anchor (wrapped to [0, M))
// and delta = n - u (n unwrapped).  The float path carries 1/h as hi + lo so
// that delta keeps ~1e-7 absolute accuracy even for u ~ 1000.
template <typename R>
__device__ __forceinline__ void grid_anchor(R x, R L, R iL, R ih, R ih_lo, int M, int P,
                                            int &n_out, R &delta) {
    R t = floor(mul_rn(x, iL));
    R xw = fma_rn(-t, L, x);
    if (xw < R(0)) xw = add_rn(xw, L);
    if (xw >= L) xw = add_rn(xw, -L);
    if (xw >= L || xw < R(0)) xw = R(0);
    R uh = mul_rn(xw, ih);
    R ul = add_rn(fma_rn(xw, ih, -uh), mul_rn(xw, ih_lo));
    R nf = (P & 1) ? floor(add_rn(add_rn(uh, R(0.5)), ul)) : floor(add_rn(uh, ul));
    delta = add_rn(add_rn(nf, -uh), -ul);
    int n = (int)nf;
    if (n >= M) n -= M;
    if (n < 0) n += M;
    n_out = n;
}

// Horner evaluation of stencil weight k at delta.
template <typename R, int P>
__device__ __forceinline__ R weight(const R (&c)[MAXP][MAXP], int k, R d) {
    R w = c[k][P - 1];
#pragma unroll
    for (int l = P - 2; l >= 0; --l) w = fma_rn(w, d, c[k][l]);
    return w;
}
template <typename R, int P>
__device__ __forceinline__ R dweight(const R (&c)[MAXP][MAXP], int k, R d) {
    R w = c[k][P - 2];
#pragma unroll
    for (int l = P - 3; l >= 0; --l) w = fma_rn(w, d, c[k][l]);
    return w;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while its stream predecessor (a kernel) is still running; it must call
// pdl_wait() before it reads anything the predecessor writes or writes
// anything the predecessor reads.  pdl_trigger() lets the successor start
// early; it changes scheduling only (the successor's pdl_wait still waits for
// the whole predecessor grid).  Both are no-ops for ordinary launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Warp reduction of a double (full warp).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Warp reduction in the step's type: on GB300 the FP64 pipe is ~2 DFMA per
// clock per SM, so FP32 paths reduce within the warp in FP32 and combine only
// the per-warp values in FP64.
template <typename R>
__device__ __forceinline__ R warp_sum_t(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Host-side coefficient/table builders (coeffs.cpp): independent exact
// arithmetic, no device code.
// ---------------------------------------------------------------------------
// coef[k][l], dcoef[k][l] of the order-P stencil in delta (see top comment).
void stencil_polynomials(int P, double coef[MAXP][MAXP], double dcoef[MAXP][MAXP]);
// An upper bound on every stencil weight W_k(delta) of the polynomials above.
double stencil_weight_max(int P, const double coef[MAXP][MAXP]);
// M_{2P}(g) for g = 0..P (values at the integers of the order-2P B-spline).
void spline2p_at_integers(int P, double out[MAXP + 1]);
// Grid-unit wavenumber of mesh index m (Nyquist index taken as -M/2).
double grid_kappa(int m, int M);
// sum_{|m| <= mmax} U1(kappa + 2 pi m) U1(kappa + 2 pi (m - n)), U1 = sinc^P(./2).
double alias_cross(double kappa, int n, int P, int mmax);

// ---------------------------------------------------------------------------
// Kernel launchers (one per .cu file), all enqueue on `s`.
// ---------------------------------------------------------------------------
struct SortBufs {
    uint32_t *anchor;      // [n] packed wrapped anchor, input order
    int *rank;             // [n] rank within its tile
    int *tile_count;       // [ntiles], zero between steps
    int *tile_start;       // [ntiles + 1]
    int *perm;             // [n] sorted -> input index
    void *rec;             // [n] vec4 (delta_x, delta_y, delta_z, q/vcell or q), sorted
    uint32_t *cell;        // [n] packed anchor, sorted
    double *blk;           // [2 * nblk] per-block sum q, sum q^2
    double *qsum;          // [2] sum q, sum q^2
    unsigned int *queue;   // [2] the persistent ad fieldforce's unit queue: ticket, CTAs done (zero between steps)
    int *err;              // [1] device error word
};

// rho_zero (nullable, mtot values) is cleared by the same launch, so that
// make_rho can follow with mesh_zeroed = true.
template <typename R>
void launch_sort(const Geom<R> &g, int64_t n, const R *x, const R *q, const SortBufs &b,
                 cudaStream_t s, R *rho_zero = nullptr, int64_t mtot = 0, R *x_copy = nullptr,
                 R *q_copy = nullptr);
// Particles per thread of launch_sort's k_particle_map: one, or four on
// systems large enough to fill the GPU with a quarter of the blocks (fewer
// blocks: fewer per-block charge sums, FP64 adds and histogram-scan tickets).
constexpr int MAP_NPT_BIG = 4;
constexpr int64_t MAP_NPT_MIN_N = 1 << 19;
inline int map_npt(int64_t n) { return n >= MAP_NPT_MIN_N ? MAP_NPT_BIG : 1; }
// k_particle_map's blocks (its per-block q, q^2 partials) for n particles
inline int map_blocks(int64_t n) { return (int)((n + 256LL * map_npt(n) - 1) / (256LL * map_npt(n))); }

template <typename R>
cudaError_t prepare_make_rho(int P, bool compensated);  // once per process/device, before capture
// mesh_zeroed: rho was cleared by launch_sort (no memset here); pdl: the
// launch directly follows launch_sort's kernels in the stream and may use a
// programmatic dependent launch.
template <typename R>
void launch_make_rho(const Geom<R> &g, int64_t n, const SortBufs &b, R *rho, bool compensated,
                     cudaStream_t s, bool mesh_zeroed = false, bool pdl = false);

struct GreenBufs {
    const double *G64;     // [Mx*My*Mzh] unscaled G
    const void *Gs;        // [Mx*My*Mzh] G / M in the step type
    const void *kvec;      // [Mx + My + Mzh] wavenumbers (step type), Nyquist negative
    const void *kdiff;     // same with the Nyquist entries zeroed (ik differentiation)
    double *part;          // [7 * nblk] per-block partial energy/virial
    double *qsum;          // [2] sum q, sum q^2 (written by k_energy_final)
    const double *map_part;// [2 * map_nblk] per-block sum q, sum q^2 of k_particle_map
    double *ev;            // [8] energy + virial
};
struct EnergyConsts {
    double epref;  // (C/2) vcell^2 / V * M  (energy of sum w Gs |rho_hat|^2)
    double inv4g2;
    double eself;  // -C g / sqrt(pi), times sum q^2
    double ebg;    // -C pi / (2 g^2 V), times Q^2
};

// Final energy/virial of one system, by one whole 256-thread CTA: warp c < 7
// sums energy/virial component c over the gn green partials, warp 7 sums q
// and q^2 over the mn particle_map partials; fixed order.
__device__ __forceinline__ void energy_final_body(const GreenBufs &b, const EnergyConsts &ec, int gn, int mn,
                                                  double *ev_user) {
    __shared__ double qs[2];
    __shared__ double comp[7];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // each lane adds its entries k = lane, lane + 32, ... in order, loading
    // eight of them before adding (one memory round trip per eight)
    if (w == 7) {
        double a = 0.0, c = 0.0;
        for (int k0 = lane; k0 < mn; k0 += 256) {
            double va[8], vc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + 32 * u;
                va[u] = (k < mn) ? b.map_part[2 * k] : 0.0;
                vc[u] = (k < mn) ? b.map_part[2 * k + 1] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                a += va[u];
                c += vc[u];
            }
        }
        a = warp_sum(a);
        c = warp_sum(c);
        if (lane == 0) {
            qs[0] = a;
            qs[1] = c;
            b.qsum[0] = a;
            b.qsum[1] = c;
        }
    } else {
        double v = 0.0;
        for (int k0 = lane; k0 < gn; k0 += 256) {
            double vv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) vv[u] = (k0 + 32 * u < gn) ? b.part[7 * (k0 + 32 * u) + w] : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) v += vv[u];
        }
        v = warp_sum(v);
        if (lane == 0) comp[w] = v * ec.epref;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = comp[threadIdx.x];
        if (threadIdx.x == 0) v += ec.eself * qs[1] + ec.ebg * qs[0] * qs[0];
        b.ev[threadIdx.x] = v;
        if (ev_user) ev_user[threadIdx.x] = v;
    }
}

// Returns the number of CTAs launched (the count of energy/virial partials).
template <typename R>
int launch_green(const Geom<R> &g, bool ik, const void *rho_hat, void *spec,
                 const GreenBufs &b, const EnergyConsts &ec, cudaStream_t s);
// Final energy/virial (and sum q, sum q^2) from the per-CTA partials, in a
// fixed order; one CTA.  ev_user may be NULL.
void launch_energy_final(const GreenBufs &b, const EnergyConsts &ec, int green_nblk, int map_nblk,
                         double *ev_user, cudaStream_t s);

// Hand-written Poisson solve for FP32 plans with power-of-two mesh edges
// 16..128, or cubic meshes of edge 48, 96 or 256 (k_fft.cu): step 0 forward
// plane pass (rho -> rho_hat), step 1 x
// pass with the influence function and the energy/virial partials (in place
// of launch_green; returns the number of partials, for launch_energy_final),
// step 2 inverse plane pass (spec -> field).  pdl: the launch directly
// follows its stream predecessor kernel.
bool custom_fft_supported(const int M[3]);
cudaError_t prepare_custom_fft(const int M[3]);  // shared-memory opt-in, before capture
int custom_fft_parts(const int M[3]);            // energy/virial partials of step 1 (0: unsupported mesh)
bool custom_fft_default(const int M[3]);         // the plan's default variants include the hand-written solve
int launch_custom_fft(int step, const Geom<float> &g, bool ik_spec, const float *rho, void *rho_hat, void *spec,
                      float *field, const GreenBufs &b, const EnergyConsts &ec, bool pdl, cudaStream_t s);

// Particles one fieldforce CTA of the per-particle kernel serves (groups of
// P lanes, 32 / P per warp, 8 warps).
inline int ff_particles_per_cta(int P) { return 8 * (32 / P); }
template <typename R>
cudaError_t prepare_fieldforce(int P);  // shared-memory opt-in of the tile-staged kernels
template <typename R>
cudaError_t prepare_green();  // k_green's resident-CTA count (its grid), before capture
template <typename R>
void launch_fieldforce(const Geom<R> &g, bool ik, int64_t n, const SortBufs &b, const R *field,
                       R *f, R qC, const double *sf_coeff, cudaStream_t s);

template <typename R>
void launch_energy_grad(const Geom<R> &g, int64_t n, const SortBufs &b, const R *phi, R *dEdx,
                        R *dEdq, R C, const double *qsum, double gself, double gbg,
                        cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched path: many independent systems in one launch per stage.  Each
// system has its own geometry, sort buffers and mesh slices; a batched launch
// covers a list of systems (ids) whose CTAs are laid out back to back
// (boff = prefix sums of per-system CTA counts, length L + 1), and every CTA
// finds its system by binary search and runs the single-system body with its
// local CTA index.
// ---------------------------------------------------------------------------
template <typename R>
struct BatchSys {
    Geom<R> g;
    SortBufs sb;
    GreenBufs gb;
    EnergyConsts ec;
    double sf[6];          // ad self-force coefficients c[a][n-1]
    R *rho;                // [M] mesh slice
    void *rho_hat;         // [Mhalf] complex
    void *spec;            // [3 or 1][Mhalf] complex
    R *field;              // [M][4] (ik) or [M]
    int64_t poff;          // first particle of this system in the caller's arrays
    int n;                 // particles
    int map_nb, green_nb;  // CTAs of its map/scatter and green launches
};
struct BatchList {
    const int *ids;   // [L] system ids
    const int *boff;  // [L + 1] CTA offsets
    int L;
    int nblocks;      // boff[L]
};

__device__ __forceinline__ int batch_entry(const int *__restrict__ boff, int L, int b) {
    int lo = 0, hi = L;  // largest e with boff[e] <= b
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&boff[mid]) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename R>
void launch_batch_sort(const BatchSys<R> *sys, const BatchList &all, const R *x, const R *q, cudaStream_t s);
template <typename R>
void launch_batch_make_rho(const BatchSys<R> *sys, const BatchList &byP, int P, bool compensated, bool copies4,
                           bool pairs, cudaStream_t s);
template <typename R>
void launch_batch_green(const BatchSys<R> *sys, const BatchList &all, bool ik, cudaStream_t s);
template <typename R>
void launch_batch_energy_final(const BatchSys<R> *sys, int nsys, double *ev, cudaStream_t s);
template <typename R>
void launch_batch_fieldforce(const BatchSys<R> *sys, const BatchList &byP, int P, bool ik, bool tiled, R *f, R qC,
                             cudaStream_t s);

// Setup: G(k) in FP64 over the half spectrum and the ad self-force sums.
struct GreenSetup {
    int M[3], Mzh, P;
    bool ik;
    double h[3], g;
    const double *ktab;    // [Mx + My + Mzh] FP64 wavenumbers (Nyquist negative)
    const double *atab;    // [5][Mx + My + Mzh] exp(-km^2/4g^2) U^2(km) for alias m = -2..2
    const double *dtab;    // [Mx + My + Mzh] per-dimension denominator sum U^2
    const double *btab;    // [3 n][Mx + My + Mzh] self-force alias sums, n = 0,1,2
};
void launch_green_setup(const GreenSetup &gs, double *G64, double *sf_sums, cudaStream_t s);
// Setup-time k-space error estimate of an ik or ad mesh: tables as for
// GreenSetup plus etab[5][Mx + My + Mzh] = exp(-k_m^2 / 2g^2) per dimension
// and alias, and (ad) s2tab[Mx + My + Mzh] = the full alias sum of
// U1^2(k_m) k_m^2 per dimension.  Writes one partial sum of the error
// functional per CTA (at most KERR_MAX_BLOCKS) and returns the CTA count.
constexpr int KERR_MAX_BLOCKS = 152 * 8;
struct KErrSetup {
    int M[3], Mzh;
    int ad;  // 1: forces as the gradient of the interpolated potential
    double h[3];
    const double *ktab, *atab, *dtab, *etab, *s2tab;
};
int launch_kspace_error(const KErrSetup &ks, double *part, cudaStream_t s);
// Host driver of the above for one system (pppm_api.cu): G64 on the device,
// the ad self-force coefficients c[a][n-1] and the wavenumber tables on the host.
int green_setup_fp64(const int M[3], const double h[3], double V, int P, bool ik, double g, double C,
                     double *G64, double sf_out[6], std::vector<double> &ktab, std::vector<double> &kdiff,
                     cudaStream_t stream);

}  // namespace pppm
