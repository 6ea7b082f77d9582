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
__device__ __forceinline__ float sin2pi(float x) { return sinpif(2.0f * x); }
__device__ __forceinline__ double sin2pi(double x) { return sinpi(2.0 * x); }

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
            F0 += q2 * ((R)c[0] * sin2pi(dx) + (R)c[1] * sin2pi(R(2) * dx));
            F1 += q2 * ((R)c[2] * sin2pi(dy) + (R)c[3] * sin2pi(R(2) * dy));
            F2 += q2 * ((R)c[4] * sin2pi(dz) + (R)c[5] * sin2pi(R(2) * dz));
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

template <typename R, int P, int MODE>
__global__ void __launch_bounds__(FF_THREADS) k_fieldforce_tiled(Geom<R> g, SortBufs b,
                                                                 const R *__restrict__ field, R *__restrict__ f,
                                                                 R *__restrict__ dq, R qC, SelfCoef sc, R gself,
                                                                 R gbg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *brick = reinterpret_cast<R *>(smem_raw);

    const int tile = blockIdx.x;
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
                        if (sizeof(R) == 4) {
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
        finish_particle<R, P, MODE>(g, b, live, k, j, w, e0, e1, e2, r.x, r.y, r.z, r.w, f, dq, qC, sc.c, gself,
                                    gbg);
    }
}

template <typename R, int P, int MODE>
static size_t ff_brick_bytes() {
    const int E = TILE_B + P - 1;
    return (size_t)E * E * E * sizeof(R) * ((MODE == 0) ? 4 : 1);
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
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fieldforce_tiled<R, P, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ff_brick_bytes<R, P, 1>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fieldforce_tiled<R, P, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ff_brick_bytes<R, P, 2>());
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
static void launch_batch_ff(const BatchSys<R> *sys, const BatchList &bl, bool ik, R *f, R qC, cudaStream_t s) {
    if (ik)
        k_batch_fieldforce<R, P, 0><<<bl.nblocks, FF_THREADS, 0, s>>>(sys, bl, f, qC);
    else
        k_batch_fieldforce<R, P, 1><<<bl.nblocks, FF_THREADS, 0, s>>>(sys, bl, f, qC);
}

// CTA counts in bl are ceil(n / ff_particles_per_cta(P)) per system (one group of P lanes per particle).
template <typename R>
void launch_batch_fieldforce(const BatchSys<R> *sys, const BatchList &bl, int P, bool ik, R *f, R qC,
                             cudaStream_t s) {
    if (bl.nblocks == 0) return;
    switch (P) {
        case 2: launch_batch_ff<R, 2>(sys, bl, ik, f, qC, s); break;
        case 3: launch_batch_ff<R, 3>(sys, bl, ik, f, qC, s); break;
        case 4: launch_batch_ff<R, 4>(sys, bl, ik, f, qC, s); break;
        case 5: launch_batch_ff<R, 5>(sys, bl, ik, f, qC, s); break;
        case 6: launch_batch_ff<R, 6>(sys, bl, ik, f, qC, s); break;
        case 7: launch_batch_ff<R, 7>(sys, bl, ik, f, qC, s); break;
        default: break;
    }
}
template void launch_batch_fieldforce<float>(const BatchSys<float> *, const BatchList &, int, bool, float *, float,
                                             cudaStream_t);
template void launch_batch_fieldforce<double>(const BatchSys<double> *, const BatchList &, int, bool, double *,
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
