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
// Layout: P lanes per particle (32 / P particles per warp), lane k owning
// stencil offset k along z -- no lane spent on the paper's zero padding of the
// inner loop to 8 ("simd8").  Each lane sums its z column separably -- first
// over y into per-x partials, then over x -- so the ad gather costs two FMAs
// per stencil point; the P lane partials are combined with warp shuffles and
// the force is written to the particle's input position.
//
// Two variants (chosen per plan, see pppm_autotune):
//  k_fieldforce        particles in tile order, field rows read through L1.
//  k_fieldforce_tiled  one CTA per mesh tile copies the field over the tile
//                      plus its P-1 halo (<= 14^3 points) into shared memory
//                      with asynchronous copies (cp.async, all in flight at
//                      once), then its particles gather from shared memory.
//
// ad self force (paper silent; reading of the Ballenegger-Cerda-Holm form):
// F_a -= q^2 sum_{n=1,2} c_{a,n} sin(2 pi n u_a), with u_a = n_a - delta_a the
// grid coordinate, so sin(2 pi n u_a) = -sin(2 pi n delta_a).
#include <type_traits>

#include "pppm_common.cuh"

namespace pppm {

constexpr int FF_THREADS = 256;

__device__ __forceinline__ float ldf(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ldf(const double *p) { return __ldg(p); }
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ double4_32a ld4(const double *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}
// sin(2 pi x) and cos(2 pi x) in one call
__device__ __forceinline__ void sincos2pi(float x, float &s, float &c) { sincospif(2.0f * x, &s, &c); }
__device__ __forceinline__ void sincos2pi(double x, double &s, double &c) { sincospi(2.0 * x, &s, &c); }

// The ad self force along one axis, q^2 (c1 sin(2 pi d) + c2 sin(4 pi d)), with
// sin(4 pi d) = 2 sin(2 pi d) cos(2 pi d) from one sin/cos evaluation.
template <typename R>
__device__ __forceinline__ R self_force_axis(R c1, R c2, R d) {
    R sn, cs;
    sincos2pi(d, sn, cs);
    return sn * (c1 + R(2) * c2 * cs);
}

__device__ __forceinline__ int wrap1(int i, int M) { return i < 0 ? i + M : (i >= M ? i - M : i); }

// Asynchronous global -> shared copy of `bytes` (4, 8 or 16).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem);
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename R, int P>
__device__ __forceinline__ R horner_r(const R (&c)[P], R d) {
    R w = c[P - 1];
#pragma unroll
    for (int l = P - 2; l >= 0; --l) w = fma_rn(w, d, c[l]);
    return w;
}

// This lane's stencil polynomial (offset k) and its derivative, in registers.
template <typename R, int P>
struct LaneCoef {
    R cw[P], cd[P];
    __device__ __forceinline__ void load(const Geom<R> &g, int k) {
#pragma unroll
        for (int l = 0; l < P; ++l) {
            cw[l] = (k < P) ? g.coef[k][l] : R(0);
            cd[l] = (k < P && l < P - 1) ? g.dcoef[k][l] : R(0);
        }
    }
};

// Per-particle weights shared inside a group of P lanes (32 / P groups per
// warp; the lanes past the last whole group idle): lane t evaluates stencil
// offset t, every lane receives the x and y sets.
template <typename R, int P, int MODE>
struct GroupWeights {
    R wx[P], wy[P], wdx[P], wdy[P];
    R wz, dwz;  // this lane's z offset
    __device__ __forceinline__ void build(const LaneCoef<R, P> &lc, int gbase, R dx, R dy, R dz) {
        const R wxl = horner_r<R, P>(lc.cw, dx);
        const R wyl = horner_r<R, P>(lc.cw, dy);
        wz = horner_r<R, P>(lc.cw, dz);
        R dxl = 0, dyl = 0;
        dwz = 0;
        if (MODE != 0) {
            dxl = horner_r<R, P>(lc.cd, dx);
            dyl = horner_r<R, P>(lc.cd, dy);
            dwz = horner_r<R, P>(lc.cd, dz);
        }
        share(gbase, wxl, wyl, dxl, dyl);
    }
    // same, reading this lane's coefficients from the plan's table (fewer
    // live registers: the better choice when a thread sees one particle)
    __device__ __forceinline__ void build(const Geom<R> &g, int k, int gbase, R dx, R dy, R dz) {
        R wxl = 0, wyl = 0, dxl = 0, dyl = 0;
        wz = 0;
        dwz = 0;
        if (k < P) {
            wxl = weight<R, P>(g.coef, k, dx);
            wyl = weight<R, P>(g.coef, k, dy);
            wz = weight<R, P>(g.coef, k, dz);
            if (MODE != 0) {
                dxl = dweight<R, P>(g.dcoef, k, dx);
                dyl = dweight<R, P>(g.dcoef, k, dy);
                dwz = dweight<R, P>(g.dcoef, k, dz);
            }
        }
        share(gbase, wxl, wyl, dxl, dyl);
    }
    __device__ __forceinline__ void share(int gbase, R wxl, R wyl, R dxl, R dyl) {
#pragma unroll
        for (int t = 0; t < P; ++t) {
            // an idle lane's source wraps within the warp; it is not used
            const int src = (gbase + t) & 31;
            wx[t] = __shfl_sync(0xffffffffu, wxl, src);
            wy[t] = __shfl_sync(0xffffffffu, wyl, src);
            if (MODE != 0) {
                wdx[t] = __shfl_sync(0xffffffffu, dxl, src);
                wdy[t] = __shfl_sync(0xffffffffu, dyl, src);
            }
        }
    }
};

// Separable gather of one lane's z column.  load(a, c) returns the field at
// stencil offsets (a, c, this lane's k).  Results, before the z weight:
//  MODE 0: e0..e2 = sum_a wx[a] sum_c wy[c] E_{x,y,z}
//  MODE 1/2: e0 = sum_a wdx[a] S0[a], e1 = sum_a wx[a] S1[a], e2 = sum_a wx[a] S0[a]
//            with S0[a] = sum_c wy[c] phi, S1[a] = sum_c wdy[c] phi.
template <typename R, int P, int MODE, typename Load>
__device__ __forceinline__ void gather_column(const GroupWeights<R, P, MODE> &w, Load load, R &e0, R &e1, R &e2) {
    e0 = e1 = e2 = R(0);
#pragma unroll
    for (int a = 0; a < P; ++a) {
        if (MODE == 0) {
            R sx = 0, sy = 0, sz = 0;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const vec4_t<R> v = load(a, c);
                sx += w.wy[c] * v.x;
                sy += w.wy[c] * v.y;
                sz += w.wy[c] * v.z;
            }
            e0 += w.wx[a] * sx;
            e1 += w.wx[a] * sy;
            e2 += w.wx[a] * sz;
        } else {
            R s0 = 0, s1 = 0;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const R v = load(a, c).x;
                s0 += w.wy[c] * v;
                s1 += w.wdy[c] * v;
            }
            e0 += w.wdx[a] * s0;
            e1 += w.wx[a] * s1;
            e2 += w.wx[a] * s0;
        }
    }
}

// Combine the group's P lanes into its lane 0, finish the per-particle
// epilogue and store.
template <typename R, int P, int MODE>
__device__ __forceinline__ void finish_particle(const Geom<R> &g, const SortBufs &b, bool live, int k, int j,
                                                const GroupWeights<R, P, MODE> &w, R e0, R e1, R e2, R dx, R dy,
                                                R dz, R qv, R *__restrict__ f, R *__restrict__ dq, R qC,
                                                const double *c, R gself, R gbg) {
    R e3 = R(0);
    if (MODE == 0) {
        e0 *= w.wz; e1 *= w.wz; e2 *= w.wz;
    } else {
        e0 *= w.wz; e1 *= w.wz;
        e3 = e2 * w.wz;  // potential at the particle (MODE 2)
        e2 *= w.dwz;
    }
    // tree over offsets 4, 2, 1: lane k adds lane k + o while that lane is in
    // its group (k + o < P); lane 0 ends with the sum of all P (P <= 8)
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        if (o >= P) continue;
        const R v0 = __shfl_down_sync(0xffffffffu, e0, o);
        const R v1 = __shfl_down_sync(0xffffffffu, e1, o);
        const R v2 = __shfl_down_sync(0xffffffffu, e2, o);
        R v3 = R(0);
        if (MODE == 2) v3 = __shfl_down_sync(0xffffffffu, e3, o);
        if (k + o < P) {
            e0 += v0;
            e1 += v1;
            e2 += v2;
            if (MODE == 2) e3 += v3;
        }
    }
    if (!live || k != 0) return;
    const int dst = b.perm[j];
    R F0, F1, F2;
    const R s = qC * qv;
    if (MODE == 0) {
        F0 = s * e0; F1 = s * e1; F2 = s * e2;
    } else {
        // E_a = sum dW/ddelta W W phi / h_a  (dW/dx = -dW/ddelta / h, E = -grad phi)
        F0 = s * e0 * g.ih[0];
        F1 = s * e1 * g.ih[1];
        F2 = s * e2 * g.ih[2];
        if (MODE == 1) {
            const R q2 = qv * qv;
            F0 += q2 * self_force_axis<R>((R)c[0], (R)c[1], dx);
            F1 += q2 * self_force_axis<R>((R)c[2], (R)c[3], dy);
            F2 += q2 * self_force_axis<R>((R)c[4], (R)c[5], dz);
        } else {
            // gradient of the energy: dE/dx = -(uncorrected ad force)
            F0 = -F0; F1 = -F1; F2 = -F2;
            if (dq) dq[dst] = qC * e3 + gself * qv + gbg * (R)b.qsum[0];
        }
    }
    if (f) {
        f[3 * (int64_t)dst + 0] = F0;
        f[3 * (int64_t)dst + 1] = F1;
        f[3 * (int64_t)dst + 2] = F2;
    }
}

struct SelfCoef {
    double c[6];
};

template <typename R>
__device__ __forceinline__ vec4_t<R> as_vec(R v) {
    vec4_t<R> o;
    o.x = v;
    o.y = o.z = o.w = R(0);
    return o;
}

// MODE 0: ik force, 1: ad force, 2: energy gradient; lb = this CTA's index
// within its system's launch; c = the six ad self-force coefficients.
template <typename R, int P, int MODE>
__device__ __forceinline__ void fieldforce_body(const Geom<R> &g, const SortBufs &b, int n,
                                                const R *__restrict__ field, R *__restrict__ f,
                                                R *__restrict__ dq, R qC, const double *c, R gself, R gbg,
                                                int lb) {
    constexpr int NG = 32 / P;  // particles per warp
    const int lane = threadIdx.x & 31;
    const int k = lane % P;
    const int gbase = lane - k;
    const int64_t gwarp = (lb * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t gid = gwarp * NG + lane / P;
    const int64_t warp_first = gwarp * NG;
    if (warp_first >= n) return;  // whole warp idle
    const bool live = lane < NG * P && gid < n;
    const int j = live ? (int)gid : 0;

    const vec4_t<R> r = reinterpret_cast<const vec4_t<R> *>(b.rec)[j];
    int ax, ay, az;
    unpack_anchor(b.cell[j], ax, ay, az);
    const bool inmesh = (unsigned)ax < (unsigned)g.M[0] && (unsigned)ay < (unsigned)g.M[1] &&
                        (unsigned)az < (unsigned)g.M[2];
    if (live && !inmesh && k == 0) atomicOr(b.err, ERR_INTERNAL);  // skipped, reported
    GroupWeights<R, P, MODE> w;
    w.build(g, k, gbase, r.x, r.y, r.z);
    pdl_wait();  // weights come from the sort's records; the field from the inverse transform
    R e0 = 0, e1 = 0, e2 = 0;
    if (live && inmesh) {
        const int My = g.M[1], Mz = g.M[2];
        const int iz = wrap1(az - g.rlo + k, Mz);
        int yoff[P], xoff[P];
#pragma unroll
        for (int c = 0; c < P; ++c) yoff[c] = wrap1(ay - g.rlo + c, My) * Mz + iz;
#pragma unroll
        for (int a = 0; a < P; ++a) xoff[a] = wrap1(ax - g.rlo + a, g.M[0]) * (My * Mz);
        const int ps = g.planar_stride;
        gather_column<R, P, MODE>(w, [&](int a, int c) {
            const int p = xoff[a] + yoff[c];
            if (MODE == 0) {
                if (ps == 0) return ld4(field + 4 * (int64_t)p);
                vec4_t<R> v;  // three planes (batched path)
                v.x = ldf(field + p);
                v.y = ldf(field + p + ps);
                v.z = ldf(field + p + 2 * (int64_t)ps);
                v.w = R(0);
                return v;
            }
            return as_vec<R>(ldf(field + p));
        }, e0, e1, e2);
    }
    finish_particle<R, P, MODE>(g, b, live, k, j, w, e0, e1, e2, r.x, r.y, r.z, r.w, f, dq, qC, c, gself, gbg);
}

template <typename R, int P, int MODE>
__global__ void __launch_bounds__(FF_THREADS) k_fieldforce(Geom<R> g, SortBufs b, int n,
                                                           const R *__restrict__ field, R *__restrict__ f,
                                                           R *__restrict__ dq, R qC, SelfCoef sc, R gself, R gbg) {
    fieldforce_body<R, P, MODE>(g, b, n, field, f, dq, qC, sc.c, gself, gbg, blockIdx.x);
}

template <typename R, int P, int MODE>
__global__ void __launch_bounds__(FF_THREADS) k_batch_fieldforce(const BatchSys<R> *__restrict__ sys, BatchList bl,
                                                                 R *__restrict__ f, R qC) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<R> &S = sys[bl.ids[e]];
    fieldforce_body<R, P, MODE>(S.g, S.sb, S.n, S.field, f + 3 * S.poff, nullptr, qC, S.sf, R(0), R(0),
                                blockIdx.x - bl.boff[e]);
}

// One CTA per mesh tile (tile = the CTA's index within its system): stage the
// field brick, then gather.  An ik field in three planes (g.planar_stride > 0,
// the batched path) is staged point by point into the same float4 brick.
template <typename R, int P, int MODE>
__device__ __forceinline__ void fieldforce_tiled_body(const Geom<R> &g, const SortBufs &b,
                                                      const R *__restrict__ field, R *__restrict__ f,
                                                      R *__restrict__ dq, R qC, const double *c, R gself, R gbg,
                                                      int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *brick = reinterpret_cast<R *>(smem_raw);

    const int start = b.tile_start[tile], end = b.tile_start[tile + 1];
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

    pdl_wait();  // the field of the inverse transform is complete
    // stage the brick: 16 lanes along z (Ez <= 14), 16 rows per pass, every
    // copy issued before any is awaited
    {
        const int lz = threadIdx.x & 15, ry = threadIdx.x >> 4;
        if (lz < Ez) {
            const int gz = wrap1(oz - g.rlo + lz, g.M[2]);
            for (int ex = 0; ex < Ex; ++ex) {
                const int gx = wrap1(ox - g.rlo + ex, g.M[0]);
                for (int ey = ry; ey < Ey; ey += FF_THREADS / 16) {
                    const int gy = wrap1(oy - g.rlo + ey, g.M[1]);
                    const int64_t p = ((int64_t)gx * g.M[1] + gy) * g.M[2] + gz;
                    const int e = (ex * Ey + ey) * Ez + lz;
                    if (MODE == 0) {
                        if (g.planar_stride > 0) {  // three planes: one copy per component
                            const int64_t ps = g.planar_stride;
                            cp_async<sizeof(R)>(brick + 4 * e, field + p);
                            cp_async<sizeof(R)>(brick + 4 * e + 1, field + p + ps);
                            cp_async<sizeof(R)>(brick + 4 * e + 2, field + p + 2 * ps);
                        } else if (sizeof(R) == 4) {
                            cp_async<16>(brick + 4 * e, field + 4 * p);
                        } else {
                            cp_async<16>(brick + 4 * e, field + 4 * p);
                            cp_async<16>(brick + 4 * e + 2, field + 4 * p + 2);
                        }
                    } else {
                        cp_async<sizeof(R)>(brick + e, field + p);
                    }
                }
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();

    constexpr int NG = 32 / P;  // particles per warp
    const int lane = threadIdx.x & 31;
    const int k = lane % P;
    const int gbase = lane - k;
    const int grp = (threadIdx.x >> 5) * NG + lane / P;
    const int ngrp = (FF_THREADS >> 5) * NG;
    const bool lane_on = lane < NG * P;
    LaneCoef<R, P> lc;
    lc.load(g, k);
    for (int base = start; base < end; base += ngrp) {
        const int j = base + grp;
        const bool live = lane_on && j < end;
        const int jj = live ? j : start;
        const vec4_t<R> r = reinterpret_cast<const vec4_t<R> *>(b.rec)[jj];
        int ax, ay, az;
        unpack_anchor(b.cell[jj], ax, ay, az);
        ax -= ox; ay -= oy; az -= oz;  // local anchor; brick index of stencil point = anchor + offset
        const bool intile = (unsigned)ax <= (unsigned)(Ex - P) && (unsigned)ay <= (unsigned)(Ey - P) &&
                            (unsigned)az <= (unsigned)(Ez - P);
        if (live && !intile && k == 0) atomicOr(b.err, ERR_INTERNAL);  // skipped, reported
        GroupWeights<R, P, MODE> w;
        w.build(lc, gbase, r.x, r.y, r.z);
        R e0 = 0, e1 = 0, e2 = 0;
        if (live && intile) {
            const int row0 = (ax * Ey + ay) * Ez + az + k;
            gather_column<R, P, MODE>(w, [&](int a, int c) {
                const int e = row0 + (a * Ey + c) * Ez;
                if (MODE == 0) return reinterpret_cast<const vec4_t<R> *>(brick)[e];
                return as_vec<R>(brick[e]);
            }, e0, e1, e2);
        }
        finish_particle<R, P, MODE>(g, b, live, k, j, w, e0, e1, e2, r.x, r.y, r.z, r.w, f, dq, qC, c, gself, gbg);
    }
}

template <typename R, int P, int MODE>
__global__ void __launch_bounds__(FF_THREADS) k_fieldforce_tiled(Geom<R> g, SortBufs b,
                                                                 const R *__restrict__ field, R *__restrict__ f,
                                                                 R *__restrict__ dq, R qC, SelfCoef sc, R gself,
                                                                 R gbg) {
    fieldforce_tiled_body<R, P, MODE>(g, b, field, f, dq, qC, sc.c, gself, gbg, blockIdx.x);
}

template <typename R, int P, int MODE>
__global__ void __launch_bounds__(FF_THREADS) k_batch_fieldforce_tiled(const BatchSys<R> *__restrict__ sys,
                                                                       BatchList bl, R *__restrict__ f, R qC) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<R> &S = sys[bl.ids[e]];
    fieldforce_tiled_body<R, P, MODE>(S.g, S.sb, S.field, f + 3 * S.poff, nullptr, qC, S.sf, R(0), R(0),
                                      blockIdx.x - bl.boff[e]);
}

// ---------------------------------------------------------------------------
// Persistent, double-buffered tile-staged fieldforce (FP32 step types,
// variant bit 6).  One CTA per SM slot walks the work units u = blockIdx.x,
// blockIdx.x + gridDim.x, ...; while it gathers unit u from one shared-memory
// buffer, the copies of unit u + gridDim.x (field brick over the unit plus
// its P-1 halo, and the unit's particle records, anchors and input indices)
// are in flight into the other buffer with cp.async, so the HBM/L2 latency
// of the staging hides behind the gather instead of preceding it.  Each
// stencil read is a shared-memory load at a compile-time offset from the
// particle's run start (brick strides of the widest tile).
//
// ik (this kernel): the unit is one mesh tile; the brick holds float4 field
// points, [x][y][z] with E = TILE_B + P - 1 points per edge, and the groups
// of P lanes per particle gather as k_fieldforce_tiled does.  The ad form
// (k_fieldforce_ad_thread, below) runs one particle per thread.  Particles
// of one unit are handled in sub-chunks of CH (the first one staged with
// the brick, any further one copied when reached).
// ---------------------------------------------------------------------------
template <int P>
struct PersistGeom {
    static constexpr int NT = 256;
    static constexpr int E = TILE_B + P - 1;            // brick edge of the widest tile
    static constexpr int BRICK_BYTES = E * E * E * 16;  // float4 points
    static constexpr int CH = 256;                      // particles per sub-chunk
    static constexpr int REC_OFF = BRICK_BYTES;         // float4 records [CH]
    static constexpr int CELL_OFF = REC_OFF + 16 * CH;  // packed anchors [CH]
    static constexpr int PERM_OFF = CELL_OFF + 4 * CH;  // input indices [CH]
    static constexpr int BUF_BYTES = PERM_OFF + 4 * CH;
    static constexpr size_t BYTES = 2 * (size_t)BUF_BYTES;
    static_assert(BRICK_BYTES % 16 == 0 && BUF_BYTES % 16 == 0, "16-byte aligned buffer parts");
};

struct TileBox {
    int ox, oy, oz, Ex, Ey, Ez;  // origin and brick extents (tile width + P - 1)
};
// Tile origins per dimension, tile_origin(t) for t = 0..T, in shared memory
// (one table per CTA: no integer division per tile).
constexpr int PERSIST_MAX_T = MAX_MESH / (TILE_B / 2);
struct OriginTable {
    int o[3][PERSIST_MAX_T + 1];
};
// a / b for 0 <= a < 2^24 and 1 <= b: the float quotient, corrected by one
__device__ __forceinline__ int div_small(int a, int b, float ib) {
    int qq = __float2int_rz(__int2float_rn(a) * ib);
    const int r = a - qq * b;
    qq += (r >= b) ? 1 : 0;
    qq -= (r < 0) ? 1 : 0;
    return qq;
}
__device__ __forceinline__ TileBox tile_box(const Geom<float> &g, int tile, const OriginTable &ot, float iT2,
                                            float iT1) {
    TileBox t;
    const int r1 = div_small(tile, g.T[2], iT2);  // tile / T2
    const int tz = tile - r1 * g.T[2];
    const int tx = div_small(r1, g.T[1], iT1);
    const int ty = r1 - tx * g.T[1];
    t.ox = ot.o[0][tx];
    t.oy = ot.o[1][ty];
    t.oz = ot.o[2][tz];
    t.Ex = ot.o[0][tx + 1] - t.ox + g.P - 1;
    t.Ey = ot.o[1][ty + 1] - t.oy + g.P - 1;
    t.Ez = ot.o[2][tz + 1] - t.oz + g.P - 1;
    return t;
}

// The six ad self-force coefficients in the step type.
struct SelfCoefF {
    float c[6];
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Issue (do not await) the copies of the tile whose box is tb into buffer
// `buf`: its field brick and its first min(n, CH) particles [s0, s0 + n).
template <int P>
__device__ __forceinline__ void persist_stage(const Geom<float> &g, const SortBufs &b, const float *__restrict__ field,
                                              const TileBox &tb, int s0, int n, unsigned char *buf) {
    using PG = PersistGeom<P>;
    if (n <= 0) return;  // an empty tile needs no brick
    float *brick = reinterpret_cast<float *>(buf);
    const int tid = threadIdx.x;
    const int My = g.M[1], Mz = g.M[2];
    // one 16-byte point per copy: 16 lanes along z (Ez <= 14), 16 rows per pass
    const int lz = tid & 15, ry = tid >> 4;
    if (lz < tb.Ez) {
        const int gz = wrap1(tb.oz - g.rlo + lz, Mz);
        for (int ex = 0; ex < tb.Ex; ++ex) {
            const int gx = wrap1(tb.ox - g.rlo + ex, g.M[0]);
            for (int ey = ry; ey < tb.Ey; ey += PG::NT / 16) {
                const int gy = wrap1(tb.oy - g.rlo + ey, My);
                const int64_t p = ((int64_t)gx * My + gy) * Mz + gz;
                cp_async<16>(brick + 4 * ((ex * PG::E + ey) * PG::E + lz), field + 4 * p);
            }
        }
    }
    const int m = min(n, PG::CH);
    for (int i = tid; i < m; i += PG::NT) {
        cp_async<16>(buf + PG::REC_OFF + 16 * i, reinterpret_cast<const float4 *>(b.rec) + s0 + i);
        cp_async<4>(buf + PG::CELL_OFF + 4 * i, b.cell + s0 + i);
        cp_async<4>(buf + PG::PERM_OFF + 4 * i, b.perm + s0 + i);
    }
}

template <int P>
__global__ void __launch_bounds__(256, 1)
    k_fieldforce_persist(Geom<float> g, SortBufs b, const float *__restrict__ field, float *__restrict__ f, float qC) {
    using PG = PersistGeom<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ OriginTable s_org;

    constexpr int NG = 32 / P;  // particle groups per warp
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int k = lane % P;
    const int gbase = lane - k;
    const int q = lane / P;  // this group's place in its warp
    const bool lane_on = lane < NG * P;
    constexpr int NGRP = (PG::NT / 32) * NG;  // particle slots per pass
    LaneCoef<float, P> lc;
    lc.load(g, k);
    for (int d = 0; d < 3; ++d)
        for (int i = tid; i <= g.T[d]; i += PG::NT) s_org.o[d][i] = tile_origin(i, g.T[d], g.M[d]);
    const float iT2 = 1.0f / (float)g.T[2], iT1 = 1.0f / (float)g.T[1];
    __syncthreads();

    const int stride = gridDim.x;
    int t = blockIdx.x;
    pdl_wait();  // the field, the sorted records and the tile offsets are complete
    if (t >= g.ntiles) return;
    // tile ranges (and boxes) one and two tiles ahead are found an iteration early
    int cs = __ldg(&b.tile_start[t]), ce = __ldg(&b.tile_start[t + 1]);
    TileBox tb = tile_box(g, t, s_org, iT2, iT1);
    persist_stage<P>(g, b, field, tb, cs, ce - cs, smem_raw);
    cp_async_commit();
    int ns = 0, ne = 0;
    if (t + stride < g.ntiles) {
        ns = __ldg(&b.tile_start[t + stride]);
        ne = __ldg(&b.tile_start[t + stride + 1]);
    }
    for (int it = 0; t < g.ntiles; ++it, t += stride) {
        unsigned char *cur = smem_raw + (it & 1) * PG::BUF_BYTES;
        unsigned char *nxt = smem_raw + ((it + 1) & 1) * PG::BUF_BYTES;
        const int tn = t + stride;
        TileBox tbn = tb;
        if (tn < g.ntiles) {
            tbn = tile_box(g, tn, s_org, iT2, iT1);
            persist_stage<P>(g, b, field, tbn, ns, ne - ns, nxt);
        }
        cp_async_commit();
        int n2s = 0, n2e = 0;
        if (tn + stride < g.ntiles) {
            n2s = __ldg(&b.tile_start[tn + stride]);
            n2e = __ldg(&b.tile_start[tn + stride + 1]);
        }
        cp_async_wait_prev();  // tile t's copies (the older group) have landed
        __syncthreads();

        const float4 *brick = reinterpret_cast<const float4 *>(cur);
        const float4 *srec = reinterpret_cast<const float4 *>(cur + PG::REC_OFF);
        const uint32_t *scell = reinterpret_cast<const uint32_t *>(cur + PG::CELL_OFF);
        const int *sperm = reinterpret_cast<const int *>(cur + PG::PERM_OFF);
        const int n = ce - cs;
        for (int sub = 0; sub < n; sub += PG::CH) {
            const int nch = min(PG::CH, n - sub);
            if (sub > 0) {  // a tile with more than CH particles: copy the next sub-chunk
                __syncthreads();
                for (int i = tid; i < nch; i += PG::NT) {
                    reinterpret_cast<float4 *>(cur + PG::REC_OFF)[i] = reinterpret_cast<const float4 *>(b.rec)[cs + sub + i];
                    reinterpret_cast<uint32_t *>(cur + PG::CELL_OFF)[i] = b.cell[cs + sub + i];
                    reinterpret_cast<int *>(cur + PG::PERM_OFF)[i] = b.perm[cs + sub + i];
                }
                __syncthreads();
            }
            const int Q = (nch + NG - 1) / NG;  // positions per group place
            // warp-uniform trip count: all 32 lanes take part in the shuffles
            for (int base = 0; base < NG * Q; base += NGRP) {
                const int col = base / NG + warp;
                const int pos = q * Q + col;
                const bool live = lane_on && col < Q && pos < nch;
                const int idx = live ? pos : 0;
                const float4 r = srec[idx];
                int ax, ay, az;
                unpack_anchor(scell[idx], ax, ay, az);
                ax -= tb.ox; ay -= tb.oy; az -= tb.oz;
                const bool intile = (unsigned)ax <= (unsigned)(tb.Ex - P) && (unsigned)ay <= (unsigned)(tb.Ey - P) &&
                                    (unsigned)az <= (unsigned)(tb.Ez - P);
                if (live && !intile && k == 0) atomicOr(b.err, ERR_INTERNAL);  // skipped, reported
                const bool use = live && intile;
                // lane k: z offset k; rows along x (a) and y (c)
                GroupWeights<float, P, 0> w;
                w.build(lc, gbase, r.x, r.y, r.z);
                float e0 = 0.f, e1 = 0.f, e2 = 0.f;
                if (use) {
                    const int row0 = (ax * PG::E + ay) * PG::E + az + k;
                    gather_column<float, P, 0>(w, [&](int a, int c) { return brick[row0 + (a * PG::E + c) * PG::E]; },
                                               e0, e1, e2);
                }
                e0 *= w.wz; e1 *= w.wz; e2 *= w.wz;
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) {
                    if (o >= P) continue;
                    const float v0 = __shfl_down_sync(0xffffffffu, e0, o);
                    const float v1 = __shfl_down_sync(0xffffffffu, e1, o);
                    const float v2 = __shfl_down_sync(0xffffffffu, e2, o);
                    if (k + o < P) {
                        e0 += v0;
                        e1 += v1;
                        e2 += v2;
                    }
                }
                if (use && k == 0) {
                    const int dst = sperm[idx];
                    const float s = qC * r.w;
                    f[3 * (int64_t)dst + 0] = s * e0;
                    f[3 * (int64_t)dst + 1] = s * e1;
                    f[3 * (int64_t)dst + 2] = s * e2;
                }
            }
        }
        __syncthreads();  // the buffer is free for the next copies
        cs = ns; ce = ne;
        ns = n2s; ne = n2e;
        tb = tbn;
    }
}

// ---------------------------------------------------------------------------
// Persistent ad fieldforce with one particle per thread (FP32 step types;
// the ad form of variant bit 6).  The work unit is a "super-tile": ZT = 2
// consecutive mesh tiles along z (their particles are consecutive in the
// sorted order), staged as one brick of the scalar potential (x, y: tile +
// P - 1 halo; z: 24 floats per row from oz - 4, four-byte aligned rows of
// six 16-byte copies when the z tiles are 8 wide) plus the unit's particle
// records, double-buffered like k_fieldforce_persist.  Each thread
// then evaluates its particle's three weight sets and their derivatives
// itself (no shuffles) and sums the P^3 stencil separably from shared
// memory at compile-time offsets: z runs into two partial sums (weight and
// derivative), those into three per x slice, those into the three
// components -- 2 FMAs per stencil point and no cross-lane reduction.
//
// Bank order: the 32 lanes of a warp read the same stencil offset of 32
// different particles, so they hit distinct banks exactly when their brick
// base addresses differ mod 32.  Each sub-chunk is ordered rank-major by that
// residue (every residue's first particle, then every residue's second, ...)
// and a warp takes 32 consecutive particles of that order.
// ---------------------------------------------------------------------------
struct AdThreadGeom {
    static constexpr int NT = 128;         // threads per CTA (4 warps)
    static constexpr int ZT = 2;           // mesh tiles per work unit along z
    static constexpr int RZ = 24;          // z row length and stride (floats) from oz - 4
    static constexpr int CH = 256;         // particles per staged sub-chunk
    static constexpr int EMAX = TILE_B + MAXP - 1;
    static constexpr int BRICK_BYTES = EMAX * EMAX * RZ * 4;
    static constexpr int REC_OFF = BRICK_BYTES;
    static constexpr int CELL_OFF = REC_OFF + 16 * CH;
    static constexpr int PERM_OFF = CELL_OFF + 4 * CH;
    static constexpr int BUF_BYTES = PERM_OFF + 4 * CH;
    static constexpr size_t BYTES = 2 * (size_t)BUF_BYTES;
    static_assert(BRICK_BYTES % 16 == 0 && BUF_BYTES % 16 == 0, "16-byte aligned buffer parts");
    static_assert(4 + ZT * TILE_B + (MAXP - 1) / 2 <= RZ, "a row covers the unit's z range");
};

// Work unit u: tiles (tx, ty, tz0 .. tz0 + nz - 1), nz = min(ZT, T2 - tz0).
struct UnitBox {
    int t0, nz;                  // first tile, tiles in the unit
    int ox, oy, oz, Ex, Ey, Ez;  // origin and brick extents (unit width + P - 1)
};
__device__ __forceinline__ UnitBox unit_box(const Geom<float> &g, int u, int U2, float iU2, float iT1) {
    using AG = AdThreadGeom;
    UnitBox b;
    const int r1 = div_small(u, U2, iU2);
    const int uz = u - r1 * U2;
    const int tx = div_small(r1, g.T[1], iT1);
    const int ty = r1 - tx * g.T[1];
    const int tz0 = uz * AG::ZT;
    b.nz = min(AG::ZT, g.T[2] - tz0);
    b.t0 = (tx * g.T[1] + ty) * g.T[2] + tz0;
    b.ox = tile_origin(tx, g.T[0], g.M[0]);
    b.oy = tile_origin(ty, g.T[1], g.M[1]);
    b.oz = tile_origin(tz0, g.T[2], g.M[2]);
    b.Ex = tile_origin(tx + 1, g.T[0], g.M[0]) - b.ox + g.P - 1;
    b.Ey = tile_origin(ty + 1, g.T[1], g.M[1]) - b.oy + g.P - 1;
    b.Ez = tile_origin(tz0 + b.nz, g.T[2], g.M[2]) - b.oz + g.P - 1;
    return b;
}

// Issue the copies of one unit into `buf`: brick rows of the potential and the
// first min(n, CH) particle records from s0.
template <int P>
__device__ __forceinline__ void adthread_stage(const Geom<float> &g, const SortBufs &b, const float *__restrict__ phi,
                                               const UnitBox &ub, int s0, int n, unsigned char *buf, bool aligned) {
    using AG = AdThreadGeom;
    constexpr int E = TILE_B + P - 1;  // brick z index i holds global z = oz - 4 + i (wrapped)
    if (n <= 0) return;
    float *brick = reinterpret_cast<float *>(buf);
    const int tid = threadIdx.x;
    const int My = g.M[1], Mz = g.M[2];
    const int rows = ub.Ex * ub.Ey;
    const unsigned int inv = (65536u + (unsigned)ub.Ey - 1u) / (unsigned)ub.Ey;  // r / Ey = (r inv) >> 16, r < 256
    if (aligned) {
        // six aligned 16-byte chunks per row from z = oz - 4 (wrapped; Mz % 8 == 0)
        constexpr int NCH = AG::RZ / 4;
        for (int i = tid; i < rows * NCH; i += AG::NT) {
            const int r = i / NCH, j = i - r * NCH;
            const int ex = (int)(((unsigned)r * inv) >> 16), ey = r - ex * ub.Ey;
            const int gx = wrap1(ub.ox - g.rlo + ex, g.M[0]);
            const int gy = wrap1(ub.oy - g.rlo + ey, My);
            int gz = ub.oz - 4 + 4 * j;
            gz += (gz < 0) ? Mz : 0;
            gz -= (gz >= Mz) ? Mz : 0;
            cp_async<16>(brick + (ex * E + ey) * AG::RZ + 4 * j, phi + ((int64_t)gx * My + gy) * Mz + gz);
        }
    } else {
        // one point per copy: 32 lanes along z, 4 rows per pass; the whole row
        // (z = oz - 4 .. oz + 19, wrapped as often as a small mesh needs) is
        // copied, so that the spare word of a run's last pair is a finite value
        const int lz = tid & 31, ry = tid >> 5;
        if (lz < AG::RZ) {
            int gz = (ub.oz - 4 + lz) % Mz;
            gz += (gz < 0) ? Mz : 0;
            for (int r = ry; r < rows; r += AG::NT / 32) {
                const int ex = (int)(((unsigned)r * inv) >> 16), ey = r - ex * ub.Ey;
                const int gx = wrap1(ub.ox - g.rlo + ex, g.M[0]);
                const int gy = wrap1(ub.oy - g.rlo + ey, My);
                cp_async<4>(brick + (ex * E + ey) * AG::RZ + lz, phi + ((int64_t)gx * My + gy) * Mz + gz);
            }
        }
    }
    const int m = min(n, AG::CH);
    for (int i = tid; i < m; i += AG::NT) {
        cp_async<16>(buf + AG::REC_OFF + 16 * i, reinterpret_cast<const float4 *>(b.rec) + s0 + i);
        cp_async<4>(buf + AG::CELL_OFF + 4 * i, b.cell + s0 + i);
        cp_async<4>(buf + AG::PERM_OFF + 4 * i, b.perm + s0 + i);
    }
}

template <int P>
__global__ void __launch_bounds__(AdThreadGeom::NT, 4)
    k_fieldforce_ad_thread(Geom<float> g, SortBufs b, const float *__restrict__ phi, float *__restrict__ f, float qC,
                           SelfCoefF sc, int aligned, int nunits, int U2, unsigned int *__restrict__ queue) {
    using AG = AdThreadGeom;
    constexpr int E = TILE_B + P - 1;
    constexpr int ZOFF = 4 - (P - 1) / 2;
    constexpr int NW = AG::NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_bins[32], s_off[16];
    __shared__ int s_list[AG::CH];
    __shared__ int s_unit[2];  // the unit after next, by iteration parity

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid < 32) s_bins[tid] = 0;
    const float iU2 = 1.0f / (float)U2, iT1 = 1.0f / (float)g.T[1];

    // Units: blockIdx.x, then blockIdx.x + gridDim.x, then from a queue
    // (2 gridDim.x + a ticket of queue[0]), so that CTAs that drew light units
    // take more: static striding left the SMs idle for 5.6 % of the kernel.
    const int stride = gridDim.x;
    int u = blockIdx.x;
    pdl_wait();  // the potential, the sorted records and the tile offsets are complete
    UnitBox ub{}, ubn{};
    int cs = 0, ce = 0, ns = 0, ne = 0, un = u + stride;
    if (u < nunits) {
        ub = unit_box(g, u, U2, iU2, iT1);
        cs = __ldg(&b.tile_start[ub.t0]);
        ce = __ldg(&b.tile_start[ub.t0 + ub.nz]);
        adthread_stage<P>(g, b, phi, ub, cs, ce - cs, smem_raw, aligned);
    }
    cp_async_commit();
    if (un < nunits) {
        ubn = unit_box(g, un, U2, iU2, iT1);
        ns = __ldg(&b.tile_start[ubn.t0]);
        ne = __ldg(&b.tile_start[ubn.t0 + ubn.nz]);
    }
    for (int it = 0; u < nunits; ++it) {
        unsigned char *cur = smem_raw + (it & 1) * AG::BUF_BYTES;
        unsigned char *nxt = smem_raw + ((it + 1) & 1) * AG::BUF_BYTES;
        if (un < nunits) adthread_stage<P>(g, b, phi, ubn, ns, ne - ns, nxt, aligned);
        cp_async_commit();
        if (tid == 0) s_unit[it & 1] = (un < nunits) ? 2 * stride + (int)atomicAdd(queue, 1u) : nunits;
        cp_async_wait_prev();  // this unit's copies (the older group) have landed
        __syncthreads();
        // the unit after next: its box and particle range, for the next iteration
        const int u2 = s_unit[it & 1];
        UnitBox ub2 = ubn;
        int n2s = 0, n2e = 0;
        if (u2 < nunits) {
            ub2 = unit_box(g, u2, U2, iU2, iT1);
            n2s = __ldg(&b.tile_start[ub2.t0]);
            n2e = __ldg(&b.tile_start[ub2.t0 + ub2.nz]);
        }

        const float *brick = reinterpret_cast<const float *>(cur);
        const float4 *srec = reinterpret_cast<const float4 *>(cur + AG::REC_OFF);
        const uint32_t *scell = reinterpret_cast<const uint32_t *>(cur + AG::CELL_OFF);
        const int *sperm = reinterpret_cast<const int *>(cur + AG::PERM_OFF);
        const int n = ce - cs;
        for (int sub = 0; sub < n; sub += AG::CH) {
            const int nch = min(AG::CH, n - sub);
            if (sub > 0) {  // a unit with more than CH particles: copy the next sub-chunk
                __syncthreads();
                for (int i = tid; i < nch; i += AG::NT) {
                    reinterpret_cast<float4 *>(cur + AG::REC_OFF)[i] = reinterpret_cast<const float4 *>(b.rec)[cs + sub + i];
                    reinterpret_cast<uint32_t *>(cur + AG::CELL_OFF)[i] = b.cell[cs + sub + i];
                    reinterpret_cast<int *>(cur + AG::PERM_OFF)[i] = b.perm[cs + sub + i];
                }
                __syncthreads();
            }
            // Bank order: each particle reads its z runs as 8-byte pairs from the
            // even word at or below its run start b; a warp's 64-bit shared load
            // is served per half-warp, whose 16 lanes are conflict-free when
            // their (b / 2) mod 16 differ.  Counting-sort the sub-chunk by that
            // class; below, the 16 lanes of a half-warp take positions spread
            // over the whole sorted list.
            int my_item[AG::CH / AG::NT];
#pragma unroll
            for (int j = 0; j < AG::CH / AG::NT; ++j) {
                const int i = tid + j * AG::NT;
                my_item[j] = -1;
                if (i < nch) {
                    int ax, ay, az;
                    unpack_anchor(scell[i], ax, ay, az);
                    const int key =
                        ((((ax - ub.ox) * E + (ay - ub.oy)) * AG::RZ + (az - ub.oz) + ZOFF) >> 1) & 15;
                    my_item[j] = (key << 16) | atomicAdd(&s_bins[key], 1);  // class and rank
                }
            }
            __syncthreads();
            if (tid < 32) {
                const int v = (tid < 16) ? s_bins[tid] : 0;
                int incl = v;
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    const int w = __shfl_up_sync(0xffffffffu, incl, o);
                    if (tid >= o) incl += w;
                }
                if (tid < 16) s_off[tid] = incl - v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < AG::CH / AG::NT; ++j)
                if (my_item[j] >= 0) s_list[s_off[my_item[j] >> 16] + (my_item[j] & 0xffff)] = tid + j * AG::NT;
            if (tid < 16) s_bins[tid] = 0;  // clean for the next sub-chunk (s_off holds the offsets)
            __syncthreads();
            const int npass = (nch + AG::NT - 1) / AG::NT;
            const int hw = 2 * warp + (lane >> 4);  // half-warp of the CTA
            for (int pass = 0; pass < npass; ++pass) {
                // the 16 lanes of a half-warp take sorted positions 2 NW npass apart
                const int pos = ((lane & 15) * (2 * NW) + hw) * npass + pass;
                if (pos >= nch) continue;
                const int idx = s_list[pos];
                const float4 r = srec[idx];
                int ax, ay, az;
                unpack_anchor(scell[idx], ax, ay, az);
                ax -= ub.ox; ay -= ub.oy; az -= ub.oz;
                const bool inunit = (unsigned)ax <= (unsigned)(ub.Ex - P) &&
                                    (unsigned)ay <= (unsigned)(ub.Ey - P) && (unsigned)az <= (unsigned)(ub.Ez - P);
                if (!inunit) {  // not this unit's particle: skipped, reported
                    atomicOr(b.err, ERR_INTERNAL);
                    continue;
                }
                // the three weight sets and their derivatives (Horner, this thread alone)
                float wx[P], wy[P], wz[P], vx[P], vy[P], vz[P];
#pragma unroll
                for (int t = 0; t < P; ++t) {
                    wx[t] = weight<float, P>(g.coef, t, r.x);
                    wy[t] = weight<float, P>(g.coef, t, r.y);
                    wz[t] = weight<float, P>(g.coef, t, r.z);
                    vx[t] = dweight<float, P>(g.dcoef, t, r.x);
                    vy[t] = dweight<float, P>(g.dcoef, t, r.y);
                    vz[t] = dweight<float, P>(g.dcoef, t, r.z);
                }
                // z runs as NPR 8-byte pairs from the even word at or below the run
                // start; the z weights shifted to match (zero on the spare word,
                // which is a finite staged value)
                constexpr int NPR = (P + 2) / 2;
                const int b0 = (ax * E + ay) * AG::RZ + az + ZOFF;
                const int sh = b0 & 1;
                const float2 *bp = reinterpret_cast<const float2 *>(brick + (b0 - sh));
                float wz2[2 * NPR], vz2[2 * NPR];
#pragma unroll
                for (int j = 0; j < 2 * NPR; ++j) {
                    const float w0 = (j < P) ? wz[j] : 0.f, w1 = (j >= 1 && j - 1 < P) ? wz[j - 1] : 0.f;
                    const float d0 = (j < P) ? vz[j] : 0.f, d1 = (j >= 1 && j - 1 < P) ? vz[j - 1] : 0.f;
                    wz2[j] = sh ? w1 : w0;
                    vz2[j] = sh ? d1 : d0;
                }
                float ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    float y00 = 0.f, y10 = 0.f, y01 = 0.f;
#pragma unroll
                    for (int c = 0; c < P; ++c) {
                        float z0 = 0.f, z1 = 0.f;
#pragma unroll
                        for (int m = 0; m < NPR; ++m) {
                            const float2 v = bp[((a * E + c) * AG::RZ) / 2 + m];
                            z0 = fmaf(wz2[2 * m], v.x, z0);
                            z0 = fmaf(wz2[2 * m + 1], v.y, z0);
                            z1 = fmaf(vz2[2 * m], v.x, z1);
                            z1 = fmaf(vz2[2 * m + 1], v.y, z1);
                        }
                        y00 = fmaf(wy[c], z0, y00);  // sum wy wz phi
                        y10 = fmaf(vy[c], z0, y10);  // sum dwy wz phi
                        y01 = fmaf(wy[c], z1, y01);  // sum wy dwz phi
                    }
                    ex = fmaf(vx[a], y00, ex);
                    ey = fmaf(wx[a], y10, ey);
                    ez = fmaf(wx[a], y01, ez);
                }
                const float s = qC * r.w, q2 = r.w * r.w;
                const int dst = sperm[idx];
                f[3 * (int64_t)dst + 0] = s * ex * g.ih[0] + q2 * self_force_axis<float>(sc.c[0], sc.c[1], r.x);
                f[3 * (int64_t)dst + 1] = s * ey * g.ih[1] + q2 * self_force_axis<float>(sc.c[2], sc.c[3], r.y);
                f[3 * (int64_t)dst + 2] = s * ez * g.ih[2] + q2 * self_force_axis<float>(sc.c[4], sc.c[5], r.z);
            }
        }
        __syncthreads();  // the buffer and the order list are free for the next copies
        cs = ns; ce = ne; ub = ubn;
        ns = n2s; ne = n2e; ubn = ub2;
        u = un;
        un = u2;
    }
    // the last CTA out (every ticket drawn) clears the queue for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
            queue[0] = 0u;
            queue[1] = 0u;
        }
    }
}

template <typename R, int P, int MODE>
static size_t ff_brick_bytes() {
    const int E = TILE_B + P - 1;
    return (size_t)E * E * E * sizeof(R) * ((MODE == 0) ? 4 : 1);
}

// Persistent fieldforce: CTAs per SM at its shared-memory size, found once
// per process (prepare_fieldforce) for each order and mode, and the SM count.
static int g_persist_ctas[2][MAXP + 1];
static int g_num_sms = 0;

template <int P, int MODE>
static cudaError_t prepare_persist() {
    cudaError_t e;
    int nb = 0;
    if constexpr (MODE == 0) {
        using PG = PersistGeom<P>;
        e = cudaFuncSetAttribute(k_fieldforce_persist<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PG::BYTES);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fieldforce_persist<P>, PG::NT, PG::BYTES);
    } else {  // the ad form runs one particle per thread
        using AG = AdThreadGeom;
        e = cudaFuncSetAttribute(k_fieldforce_ad_thread<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)AG::BYTES);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fieldforce_ad_thread<P>, AG::NT, AG::BYTES);
    }
    if (e == cudaSuccess && g_num_sms == 0) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e == cudaSuccess) g_persist_ctas[MODE][P] = nb > 0 ? nb : 1;
    return e;
}

// The ad brick's rows are six aligned 16-byte copies when every z tile is 8
// points wide (tile origins and Mz multiples of 8).
inline bool persist_rows_aligned(const Geom<float> &g) { return g.M[2] % 8 == 0 && g.T[2] * 8 == g.M[2]; }

template <int P, int MODE>
static void launch_persist(const Geom<float> &g, const SortBufs &b, const float *field, float *f, float qC,
                           const SelfCoef &scd, bool pdl, cudaStream_t s) {
    const int slots = (g_num_sms > 0 ? g_num_sms : 152) * (g_persist_ctas[MODE][P] > 0 ? g_persist_ctas[MODE][P] : 1);
    if constexpr (MODE == 1) {
        using AG = AdThreadGeom;
        SelfCoefF sc;
        for (int i = 0; i < 6; ++i) sc.c[i] = (float)scd.c[i];
        const int aligned = persist_rows_aligned(g) ? 1 : 0;
        const int U2 = (g.T[2] + AG::ZT - 1) / AG::ZT;
        const int nunits = g.T[0] * g.T[1] * U2;
        const int grid = nunits < slots ? nunits : slots;
        if (pdl)
            launch_pdl(k_fieldforce_ad_thread<P>, dim3(grid), dim3(AG::NT), AG::BYTES, s, g, b, field, f, qC, sc, aligned,
                       nunits, U2, b.queue);
        else
            k_fieldforce_ad_thread<P><<<grid, AG::NT, AG::BYTES, s>>>(g, b, field, f, qC, sc, aligned, nunits, U2,
                                                                      b.queue);
    } else {
        using PG = PersistGeom<P>;
        (void)scd;
        const int grid = g.ntiles < slots ? g.ntiles : slots;
        if (pdl)
            launch_pdl(k_fieldforce_persist<P>, dim3(grid), dim3(PG::NT), PG::BYTES, s, g, b, field, f, qC);
        else
            k_fieldforce_persist<P><<<grid, PG::NT, PG::BYTES, s>>>(g, b, field, f, qC);
    }
}

template <typename R, int P, int MODE>
static void launch_ff(const Geom<R> &g, int64_t n, const SortBufs &b, const R *field, R *f, R *dq, R qC,
                      const double *c, R gs, R gb, cudaStream_t s) {
    // gb multiplies sum(q), read on the device from the sort buffers
    SelfCoef sc;
    for (int i = 0; i < 6; ++i) sc.c[i] = c[i];
    const bool pdl = (g.launch_flags & LF_PDL_FF) != 0;
    // the energy gradient (MODE 2) gathers a scalar potential, which reads
    // best through L1 on every measured workload; the plan's tuned variant
    // is chosen on force steps and applies to MODE 0 / 1 only
    if constexpr (std::is_same<R, float>::value && MODE != 2) {
        if (g.ff_tiled == 2) {
            launch_persist<P, MODE>(g, b, field, f, qC, sc, pdl, s);
            return;
        }
    }
    if (g.ff_tiled && MODE != 2) {
        if (pdl)
            launch_pdl(k_fieldforce_tiled<R, P, MODE>, dim3(g.ntiles), dim3(FF_THREADS), ff_brick_bytes<R, P, MODE>(),
                       s, g, b, field, f, dq, qC, sc, gs, gb);
        else
            k_fieldforce_tiled<R, P, MODE><<<g.ntiles, FF_THREADS, ff_brick_bytes<R, P, MODE>(), s>>>(
                g, b, field, f, dq, qC, sc, gs, gb);
        return;
    }
    // one group of P lanes per particle, a full grid
    const int64_t per_cta = ff_particles_per_cta(P);
    const int nb = (int)((n + per_cta - 1) / per_cta);
    if (pdl)
        launch_pdl(k_fieldforce<R, P, MODE>, dim3(nb), dim3(FF_THREADS), 0, s, g, b, (int)n, field, f, dq, qC, sc,
                   gs, gb);
    else
        k_fieldforce<R, P, MODE><<<nb, FF_THREADS, 0, s>>>(g, b, (int)n, field, f, dq, qC, sc, gs, gb);
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

template <typename R, int P>
static cudaError_t prepare_ff_p() {
    cudaError_t e = cudaFuncSetAttribute(k_fieldforce_tiled<R, P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ff_brick_bytes<R, P, 0>());
    if constexpr (std::is_same<R, float>::value) {
        if (e == cudaSuccess) e = prepare_persist<P, 0>();
        if (e == cudaSuccess) e = prepare_persist<P, 1>();
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fieldforce_tiled<R, P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ff_brick_bytes<R, P, 1>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fieldforce_tiled<R, P, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ff_brick_bytes<R, P, 2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_fieldforce_tiled<R, P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ff_brick_bytes<R, P, 0>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_fieldforce_tiled<R, P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ff_brick_bytes<R, P, 1>());
    return e;
}

template <typename R>
cudaError_t prepare_fieldforce(int P) {
    switch (P) {
        case 2: return prepare_ff_p<R, 2>();
        case 3: return prepare_ff_p<R, 3>();
        case 4: return prepare_ff_p<R, 4>();
        case 5: return prepare_ff_p<R, 5>();
        case 6: return prepare_ff_p<R, 6>();
        case 7: return prepare_ff_p<R, 7>();
        default: return cudaErrorInvalidValue;
    }
}

template <typename R, int P>
static void launch_batch_ff(const BatchSys<R> *sys, const BatchList &bl, bool ik, bool tiled, R *f, R qC,
                            cudaStream_t s) {
    if (tiled) {
        if (ik)
            k_batch_fieldforce_tiled<R, P, 0><<<bl.nblocks, FF_THREADS, ff_brick_bytes<R, P, 0>(), s>>>(sys, bl, f, qC);
        else
            k_batch_fieldforce_tiled<R, P, 1><<<bl.nblocks, FF_THREADS, ff_brick_bytes<R, P, 1>(), s>>>(sys, bl, f, qC);
        return;
    }
    if (ik)
        k_batch_fieldforce<R, P, 0><<<bl.nblocks, FF_THREADS, 0, s>>>(sys, bl, f, qC);
    else
        k_batch_fieldforce<R, P, 1><<<bl.nblocks, FF_THREADS, 0, s>>>(sys, bl, f, qC);
}

// CTA counts in bl: ceil(n / ff_particles_per_cta(P)) per system (one group of
// P lanes per particle), or the system's tile count when tiled.
template <typename R>
void launch_batch_fieldforce(const BatchSys<R> *sys, const BatchList &bl, int P, bool ik, bool tiled, R *f, R qC,
                             cudaStream_t s) {
    if (bl.nblocks == 0) return;
    switch (P) {
        case 2: launch_batch_ff<R, 2>(sys, bl, ik, tiled, f, qC, s); break;
        case 3: launch_batch_ff<R, 3>(sys, bl, ik, tiled, f, qC, s); break;
        case 4: launch_batch_ff<R, 4>(sys, bl, ik, tiled, f, qC, s); break;
        case 5: launch_batch_ff<R, 5>(sys, bl, ik, tiled, f, qC, s); break;
        case 6: launch_batch_ff<R, 6>(sys, bl, ik, tiled, f, qC, s); break;
        case 7: launch_batch_ff<R, 7>(sys, bl, ik, tiled, f, qC, s); break;
        default: break;
    }
}
template void launch_batch_fieldforce<float>(const BatchSys<float> *, const BatchList &, int, bool, bool, float *,
                                             float, cudaStream_t);
template void launch_batch_fieldforce<double>(const BatchSys<double> *, const BatchList &, int, bool, bool, double *,
                                              double, cudaStream_t);

template cudaError_t prepare_fieldforce<float>(int);
template cudaError_t prepare_fieldforce<double>(int);
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
