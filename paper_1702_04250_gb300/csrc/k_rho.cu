// make_rho: Map-Charge of Sec. 3.1 -- "multiplies the particle charge by the
// stencil coefficient and adds that value to a point on the grid", over the
// P^3 stencil whose coefficients are a product of three 1-D polynomials.
//
// GB300 layout: one CTA per mesh tile (particles already sorted by the tile
// of their stencil anchor).  The CTA accumulates its particles' full stencils
// into a private shared-memory brick that covers the tile plus its P-1 halo
// (the paper's thread-private grid copies, "rethread"), then adds the brick
// to the global mesh once.  Within a warp, 8 lanes serve one particle: lane k
// owns stencil offset k along z (unit stride) and lanes k >= P carry no work
// -- the paper's padding of the 7-long inner loop to 8 ("simd8").
//
// Accumulators (ACC):
//  ACC_NATIVE  atomics in the step type (FP64, FP32).  On sm_103a shared
//              float/double atomic adds are compare-and-swap loops whose
//              round trip serialises each thread's updates.
//  ACC_FIXED   FP32C: error-free accumulation in two 32-bit integer words per
//              brick point, hi = sum rint(v s) and lo = sum of the rounded
//              16-bit fractions, with the power of two s chosen per tile so
//              that one contribution stays below 2^21 and any point's sum
//              (bounded by sum|q_j| / vcell) below 2^30.  The split uses only
//              full-rate float adds (magic-number rounding), integer shared
//              atomics are native and need no return value, and the sum is
//              exact and independent of order to 2^-37 of the largest
//              contribution -- the hi/lo compensation carried in integers.
//              lo is folded into hi every 32768 particles, so neither word
//              can overflow.
#include "pppm_common.cuh"

namespace pppm {

constexpr int RHO_THREADS = 256;
constexpr int GROUP = 8;
constexpr int ACC_NATIVE = 0, ACC_FIXED = 1;
constexpr int LO_CHUNK = 32768;
constexpr float MAGIC = 12582912.0f;      // 1.5 * 2^23
constexpr int MAGIC_BITS = 0x4B400000;    // its bit pattern

template <typename R, int P>
__device__ __forceinline__ R horner(const R (&c)[P], R d) {
    R w = c[P - 1];
#pragma unroll
    for (int l = P - 2; l >= 0; --l) w = fma_rn(w, d, c[l]);
    return w;
}

__device__ __forceinline__ float absval(float v) { return fabsf(v); }
__device__ __forceinline__ double absval(double v) { return fabs(v); }

template <typename R, int P, int ACC>
__device__ __forceinline__ void make_rho_body(const Geom<R> &g, const SortBufs &b, R *__restrict__ rho,
                                              int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float sh_red[RHO_THREADS / 32];
    __shared__ float sh_max[RHO_THREADS / 32];

    const int start = b.tile_start[tile], end = b.tile_start[tile + 1];
    if (threadIdx.x == 0) b.tile_count[tile] = 0;  // histogram is clean for the next step
    if (start == end) return;

    const int tz = tile % g.T[2];
    const int ty = (tile / g.T[2]) % g.T[1];
    const int tx = tile / (g.T[2] * g.T[1]);
    const int ox = tile_origin(tx, g.T[0], g.M[0]);
    const int oy = tile_origin(ty, g.T[1], g.M[1]);
    const int oz = tile_origin(tz, g.T[2], g.M[2]);
    const int Ex = tile_origin(tx + 1, g.T[0], g.M[0]) - ox + P - 1;
    const int Ey = tile_origin(ty + 1, g.T[1], g.M[1]) - oy + P - 1;
    const int Ez = tile_origin(tz + 1, g.T[2], g.M[2]) - oz + P - 1;
    const int vol = Ex * Ey * Ez;

    R *accr = reinterpret_cast<R *>(smem_raw);
    int *acch = reinterpret_cast<int *>(smem_raw);
    unsigned int *accl = reinterpret_cast<unsigned int *>(smem_raw) + vol;
    const R *__restrict__ recp = reinterpret_cast<const R *>(b.rec);

    // fixed-point scale s = 2^e: every contribution |v s| < 2^21 (so it can be
    // split with the float magic-number trick) and every brick point's sum
    // |sum v s| < 2^30 (so the hi word cannot overflow)
    float fs = 1.0f, ifs = 1.0f;
    if (ACC == ACC_FIXED) {
        float part = 0.0f, pmax = 0.0f;
        for (int j = start + threadIdx.x; j < end; j += blockDim.x) {
            const float a = absval((float)reinterpret_cast<const vec4_t<R> *>(recp)[j].w);
            part += a;
            pmax = fmaxf(pmax, a);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            part += __shfl_xor_sync(0xffffffffu, part, o);
            pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            sh_red[threadIdx.x >> 5] = part;
            sh_max[threadIdx.x >> 5] = pmax;
        }
        __syncthreads();
        float bound = 0.0f, bmax = 0.0f;
#pragma unroll
        for (int w = 0; w < RHO_THREADS / 32; ++w) {
            bound += sh_red[w];
            bmax = fmaxf(bmax, sh_max[w]);
        }
        bound = bound * (float)g.ivcell * 1.0001f + 1e-30f;
        bmax = bmax * (float)g.ivcell * 1.0001f + 1e-30f;
        int es, em;
        frexpf(bound, &es);  // bound < 2^es
        frexpf(bmax, &em);   // largest contribution < 2^em
        const int e = min(30 - es, 21 - em);
        fs = ldexpf(1.0f, e);
        ifs = ldexpf(1.0f, -e);
    }

    {
        const int words = (ACC == ACC_FIXED ? 2 * vol : vol * (int)(sizeof(R) / 4));
        int *w = reinterpret_cast<int *>(smem_raw);
        for (int e = threadIdx.x; e < words; e += blockDim.x) w[e] = 0;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int k = lane & (GROUP - 1);            // z stencil offset of this lane
    const int gbase = lane & ~(GROUP - 1);
    const int grp = threadIdx.x / GROUP;         // particle slot in the CTA
    const int ngrp = blockDim.x / GROUP;
    const R qscale = (ACC == ACC_FIXED) ? (R)(g.ivcell * (R)fs) : g.ivcell;
    // this lane's polynomial (stencil offset k), held in registers for the CTA
    R ck[P];
#pragma unroll
    for (int l = 0; l < P; ++l) ck[l] = (k < P) ? g.coef[k][l] : R(0);

    for (int chunk = start; chunk < end; chunk += LO_CHUNK) {
        const int cend = min(end, chunk + LO_CHUNK);
        // warp-uniform trip count: all 32 lanes take part in the shuffles
        for (int base = chunk; base < cend; base += ngrp) {
            const int j = base + grp;
            const bool live = j < cend;
            R dx = R(0), dy = R(0), dz = R(0), qv = R(0);
            int ax = 0, ay = 0, az = 0;
            if (live) {
                const vec4_t<R> r = reinterpret_cast<const vec4_t<R> *>(recp)[j];
                dx = r.x; dy = r.y; dz = r.z; qv = r.w * qscale;
                unpack_anchor(b.cell[j], ax, ay, az);
                ax -= ox; ay -= oy; az -= oz;        // local anchor in [0, tile size)
            }
            // lane k < P evaluates the three weights of stencil offset k
            const R wx = horner<R, P>(ck, dx), wy = horner<R, P>(ck, dy), wz = horner<R, P>(ck, dz);
            R wxq[P], wyk[P];
#pragma unroll
            for (int t = 0; t < P; ++t) {
                wxq[t] = __shfl_sync(0xffffffffu, wx, gbase + t) * qv;
                wyk[t] = __shfl_sync(0xffffffffu, wy, gbase + t);
            }
            if (live && k < P) {
                const int row = (ax * Ey + ay) * Ez + az + k;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const R wa = wxq[a] * wz;
#pragma unroll
                    for (int c = 0; c < P; ++c) {
                        const R v = wa * wyk[c];
                        const int e = row + (a * Ey + c) * Ez;
                        if (ACC == ACC_FIXED) {
                            // t = v s = hi + lo / 2^16 with full-rate float ops:
                            // adding 1.5 * 2^23 rounds |t| < 2^22 to an integer
                            // held in the mantissa bits
                            const float t = (float)v;
                            const float r1 = __fadd_rn(t, MAGIC);
                            const float fr = __fadd_rn(t, -__fadd_rn(r1, -MAGIC));  // exact
                            const float r2 = __fmaf_rn(fr, 65536.0f, MAGIC);
                            atomicAdd(&acch[e], __float_as_int(r1) - MAGIC_BITS);
                            atomicAdd(&accl[e], (unsigned int)(__float_as_int(r2) - MAGIC_BITS));
                        } else {
                            atomicAdd(&accr[e], v);
                        }
                    }
                }
            }
        }
        if (ACC == ACC_FIXED && cend < end) {  // fold lo into hi before it can overflow
            __syncthreads();
            for (int e = threadIdx.x; e < vol; e += blockDim.x) {
                const int l = (int)accl[e];  // signed sum of fractions in [-2^15, 2^15] each
                acch[e] += l >> 16;          // floor division by 2^16
                accl[e] = (unsigned int)(l & 0xffff);
            }
        }
        __syncthreads();
    }

    // flush the brick (tile + halo) into the global mesh: 16 lanes per z row
    // (Ez <= 14), 16 rows per pass; every wrap is a single conditional since
    // the brick is never wider than the mesh plus one period.
    const int lz = threadIdx.x & 15, ry = threadIdx.x >> 4;
    if (lz < Ez) {
        int gz = oz - g.rlo + lz;
        gz += (gz < 0) ? g.M[2] : 0;
        gz -= (gz >= g.M[2]) ? g.M[2] : 0;
        for (int ex = 0; ex < Ex; ++ex) {
            int gx = ox - g.rlo + ex;
            gx += (gx < 0) ? g.M[0] : 0;
            gx -= (gx >= g.M[0]) ? g.M[0] : 0;
            for (int ey = ry; ey < Ey; ey += RHO_THREADS / 16) {
                int gy = oy - g.rlo + ey;
                gy += (gy < 0) ? g.M[1] : 0;
                gy -= (gy >= g.M[1]) ? g.M[1] : 0;
                const int e = (ex * Ey + ey) * Ez + lz;
                R v;
                if (ACC == ACC_FIXED) {
                    // normalise in integers (exact), then one FP32 rounding
                    const int l = (int)accl[e];
                    const int h = acch[e] + (l >> 16);
                    v = (R)(fmaf((float)(l & 0xffff), 1.0f / 65536.0f, (float)h) * ifs);
                } else {
                    v = accr[e];
                }
                if (v != R(0)) atomicAdd(&rho[(gx * g.M[1] + gy) * g.M[2] + gz], v);
            }
        }
    }
}

template <typename R, int P, int ACC>
__global__ void __launch_bounds__(RHO_THREADS) k_make_rho(Geom<R> g, SortBufs b, R *__restrict__ rho) {
    make_rho_body<R, P, ACC>(g, b, rho, blockIdx.x);
}

template <typename R, int P, int ACC>
__global__ void __launch_bounds__(RHO_THREADS) k_batch_make_rho(const BatchSys<R> *__restrict__ sys, BatchList bl) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<R> &S = sys[bl.ids[e]];
    make_rho_body<R, P, ACC>(S.g, S.sb, S.rho, blockIdx.x - bl.boff[e]);
}

template <typename R, int P>
static size_t brick_bytes(int acc) {
    const int E = TILE_B + P - 1;
    return (size_t)E * E * E * (acc == ACC_FIXED ? 8 : sizeof(R));
}

template <typename R, int P>
static void launch_p(const Geom<R> &g, const SortBufs &b, R *rho, int acc, cudaStream_t s) {
    const size_t bytes = brick_bytes<R, P>(acc);
    if (acc == ACC_FIXED)
        k_make_rho<R, P, ACC_FIXED><<<g.ntiles, RHO_THREADS, bytes, s>>>(g, b, rho);
    else
        k_make_rho<R, P, ACC_NATIVE><<<g.ntiles, RHO_THREADS, bytes, s>>>(g, b, rho);
}

template <typename R, int P>
static cudaError_t prepare_p(int acc) {
    const int bytes = (int)brick_bytes<R, P>(acc);
    cudaError_t e;
    if (acc == ACC_FIXED) {
        e = cudaFuncSetAttribute(k_make_rho<R, P, ACC_FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_make_rho<R, P, ACC_FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     bytes);
        return e;
    }
    e = cudaFuncSetAttribute(k_make_rho<R, P, ACC_NATIVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_make_rho<R, P, ACC_NATIVE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    return e;
}

template <typename R, int P>
static void launch_batch_p(const BatchSys<R> *sys, const BatchList &bl, int acc, cudaStream_t s) {
    const size_t bytes = brick_bytes<R, P>(acc);
    if (acc == ACC_FIXED)
        k_batch_make_rho<R, P, ACC_FIXED><<<bl.nblocks, RHO_THREADS, bytes, s>>>(sys, bl);
    else
        k_batch_make_rho<R, P, ACC_NATIVE><<<bl.nblocks, RHO_THREADS, bytes, s>>>(sys, bl);
}

// The meshes of the systems in the list must have been cleared.
template <typename R>
void launch_batch_make_rho(const BatchSys<R> *sys, const BatchList &bl, int P, bool comp, cudaStream_t s) {
    if (bl.nblocks == 0) return;
    const int acc = comp ? ACC_FIXED : ACC_NATIVE;
    switch (P) {
        case 2: launch_batch_p<R, 2>(sys, bl, acc, s); break;
        case 3: launch_batch_p<R, 3>(sys, bl, acc, s); break;
        case 4: launch_batch_p<R, 4>(sys, bl, acc, s); break;
        case 5: launch_batch_p<R, 5>(sys, bl, acc, s); break;
        case 6: launch_batch_p<R, 6>(sys, bl, acc, s); break;
        case 7: launch_batch_p<R, 7>(sys, bl, acc, s); break;
        default: break;
    }
}
template void launch_batch_make_rho<float>(const BatchSys<float> *, const BatchList &, int, bool, cudaStream_t);
template void launch_batch_make_rho<double>(const BatchSys<double> *, const BatchList &, int, bool, cudaStream_t);

template <typename R>
cudaError_t prepare_make_rho(int P, bool comp) {
    const int acc = comp ? ACC_FIXED : ACC_NATIVE;
    switch (P) {
        case 2: return prepare_p<R, 2>(acc);
        case 3: return prepare_p<R, 3>(acc);
        case 4: return prepare_p<R, 4>(acc);
        case 5: return prepare_p<R, 5>(acc);
        case 6: return prepare_p<R, 6>(acc);
        case 7: return prepare_p<R, 7>(acc);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
void launch_make_rho(const Geom<R> &g, int64_t n, const SortBufs &b, R *rho, bool comp, cudaStream_t s) {
    cudaMemsetAsync(rho, 0, sizeof(R) * (size_t)g.M[0] * g.M[1] * g.M[2], s);
    if (n == 0) return;
    const int acc = comp ? ACC_FIXED : ACC_NATIVE;
    switch (g.P) {
        case 2: launch_p<R, 2>(g, b, rho, acc, s); break;
        case 3: launch_p<R, 3>(g, b, rho, acc, s); break;
        case 4: launch_p<R, 4>(g, b, rho, acc, s); break;
        case 5: launch_p<R, 5>(g, b, rho, acc, s); break;
        case 6: launch_p<R, 6>(g, b, rho, acc, s); break;
        case 7: launch_p<R, 7>(g, b, rho, acc, s); break;
        default: break;
    }
}

template cudaError_t prepare_make_rho<float>(int, bool);
template cudaError_t prepare_make_rho<double>(int, bool);
template void launch_make_rho<float>(const Geom<float> &, int64_t, const SortBufs &, float *, bool, cudaStream_t);
template void launch_make_rho<double>(const Geom<double> &, int64_t, const SortBufs &, double *, bool, cudaStream_t);

}  // namespace pppm
