// make_rho: Map-Charge of Sec. 3.1 -- "multiplies the particle charge by the
// stencil coefficient and adds that value to a point on the grid", over the
// P^3 stencil whose coefficients are a product of three 1-D polynomials.
//
// GB300 layout: one CTA per mesh tile (particles already sorted by the tile
// of their stencil anchor).  The CTA accumulates its particles' full stencils
// into a private shared-memory brick that covers the tile plus its P-1 halo
// (the paper's thread-private grid copies, "rethread"), then adds the brick
// to the global mesh once.  Within a warp, 8 lanes serve one particle: lane k
// owns stencil row offset k along z (unit stride) and lanes k >= P carry zero
// weight -- the paper's padding of the 7-long inner loop to 8 ("simd8").
// Consecutive lanes therefore hit consecutive shared-memory words.
//
// FP32C keeps a compensated (hi, lo) pair per brick point: the rounding error
// of every shared atomic add is recovered exactly with TwoSum from the value
// the atomic returns and accumulated in lo.
#include "pppm_common.cuh"

namespace pppm {

constexpr int RHO_THREADS = 128;
constexpr int GROUP = 8;

template <typename R, int P, bool COMP>
__global__ void __launch_bounds__(RHO_THREADS) k_make_rho(Geom<R> g, SortBufs b, R *__restrict__ rho) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *acc = reinterpret_cast<R *>(smem_raw);

    const int tile = blockIdx.x;
    const int tz = tile % g.T[2];
    const int ty = (tile / g.T[2]) % g.T[1];
    const int tx = tile / (g.T[2] * g.T[1]);
    const int start = b.tile_start[tile], end = b.tile_start[tile + 1];
    if (start == end) return;

    const int ox = tile_origin(tx, g.T[0], g.M[0]);
    const int oy = tile_origin(ty, g.T[1], g.M[1]);
    const int oz = tile_origin(tz, g.T[2], g.M[2]);
    const int Ex = tile_origin(tx + 1, g.T[0], g.M[0]) - ox + P - 1;
    const int Ey = tile_origin(ty + 1, g.T[1], g.M[1]) - oy + P - 1;
    const int Ez = tile_origin(tz + 1, g.T[2], g.M[2]) - oz + P - 1;
    const int vol = Ex * Ey * Ez;
    R *lo = acc + vol;

    for (int e = threadIdx.x; e < (COMP ? 2 : 1) * vol; e += blockDim.x) acc[e] = R(0);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int k = lane & (GROUP - 1);            // z stencil offset of this lane
    const int grp = threadIdx.x / GROUP;         // particle slot in the CTA
    const int ngrp = blockDim.x / GROUP;
    const R *__restrict__ recp = reinterpret_cast<const R *>(b.rec);

    // warp-uniform trip count: all 32 lanes take part in the shuffles
    for (int base = start; base < end; base += ngrp) {
        const int j = base + grp;
        const bool live = j < end;
        R dx = R(0), dy = R(0), dz = R(0), qv = R(0);
        int ax = 0, ay = 0, az = 0;
        if (live) {
            const vec4_t<R> r = reinterpret_cast<const vec4_t<R> *>(recp)[j];
            dx = r.x; dy = r.y; dz = r.z; qv = r.w * g.ivcell;
            unpack_anchor(b.cell[j], ax, ay, az);
            ax -= ox; ay -= oy; az -= oz;        // local anchor in [0, tile size)
        }
        // lane k < P evaluates the three weights of stencil offset k
        R wx = R(0), wy = R(0), wz = R(0);
        if (k < P) {
            wx = weight<R, P>(g.coef, k, dx);
            wy = weight<R, P>(g.coef, k, dy);
            wz = weight<R, P>(g.coef, k, dz);
        }
        R wxq[P], wyk[P];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            wxq[t] = __shfl_sync(0xffffffffu, wx, (lane & ~(GROUP - 1)) + t) * qv;
            wyk[t] = __shfl_sync(0xffffffffu, wy, (lane & ~(GROUP - 1)) + t);
        }
        if (live && k < P) {
            R *row = acc + ((ax * Ey + ay) * Ez + az + k);
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const R wa = wxq[a] * wz;
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const R v = wa * wyk[c];
                    R *p = row + (a * Ey + c) * Ez;
                    if (COMP) {
                        const R old = atomicAdd(p, v);
                        const R s = old + v;
                        const R bb = s - old;
                        const R err = (old - (s - bb)) + (v - bb);
                        atomicAdd(p + vol, err);
                    } else {
                        atomicAdd(p, v);
                    }
                }
            }
        }
    }
    __syncthreads();

    // flush the brick (tile + halo) into the global mesh
    const int bx0 = ox - g.rlo, by0 = oy - g.rlo, bz0 = oz - g.rlo;
    for (int e = threadIdx.x; e < vol; e += blockDim.x) {
        R v = acc[e];
        if (COMP) v = v + lo[e];
        if (v == R(0)) continue;
        const int ez = e % Ez, ey = (e / Ez) % Ey, ex = e / (Ez * Ey);
        int gx = bx0 + ex, gy = by0 + ey, gz = bz0 + ez;
        gx = (gx + 2 * g.M[0]) % g.M[0];
        gy = (gy + 2 * g.M[1]) % g.M[1];
        gz = (gz + 2 * g.M[2]) % g.M[2];
        atomicAdd(&rho[((int64_t)gx * g.M[1] + gy) * g.M[2] + gz], v);
    }
}

template <typename R, int P>
static size_t brick_bytes(bool comp) {
    const int E = TILE_B + P - 1;
    return (size_t)E * E * E * sizeof(R) * (comp ? 2 : 1);
}

template <typename R, int P>
static void launch_p(const Geom<R> &g, const SortBufs &b, R *rho, bool comp, cudaStream_t s) {
    const size_t bytes = brick_bytes<R, P>(comp);
    if (comp)
        k_make_rho<R, P, true><<<g.ntiles, RHO_THREADS, bytes, s>>>(g, b, rho);
    else
        k_make_rho<R, P, false><<<g.ntiles, RHO_THREADS, bytes, s>>>(g, b, rho);
}

template <typename R, int P>
static cudaError_t prepare_p(bool comp) {
    const int bytes = (int)brick_bytes<R, P>(comp);
    if (comp) return cudaFuncSetAttribute(k_make_rho<R, P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return cudaFuncSetAttribute(k_make_rho<R, P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename R>
cudaError_t prepare_make_rho(int P, bool comp) {
    switch (P) {
        case 2: return prepare_p<R, 2>(comp);
        case 3: return prepare_p<R, 3>(comp);
        case 4: return prepare_p<R, 4>(comp);
        case 5: return prepare_p<R, 5>(comp);
        case 6: return prepare_p<R, 6>(comp);
        case 7: return prepare_p<R, 7>(comp);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
void launch_make_rho(const Geom<R> &g, int64_t n, const SortBufs &b, R *rho, bool comp, cudaStream_t s) {
    cudaMemsetAsync(rho, 0, sizeof(R) * (size_t)g.M[0] * g.M[1] * g.M[2], s);
    if (n == 0) return;
    switch (g.P) {
        case 2: launch_p<R, 2>(g, b, rho, comp, s); break;
        case 3: launch_p<R, 3>(g, b, rho, comp, s); break;
        case 4: launch_p<R, 4>(g, b, rho, comp, s); break;
        case 5: launch_p<R, 5>(g, b, rho, comp, s); break;
        case 6: launch_p<R, 6>(g, b, rho, comp, s); break;
        case 7: launch_p<R, 7>(g, b, rho, comp, s); break;
        default: break;
    }
}

template cudaError_t prepare_make_rho<float>(int, bool);
template cudaError_t prepare_make_rho<double>(int, bool);
template void launch_make_rho<float>(const Geom<float> &, int64_t, const SortBufs &, float *, bool, cudaStream_t);
template void launch_make_rho<double>(const Geom<double> &, int64_t, const SortBufs &, double *, bool, cudaStream_t);

}  // namespace pppm
