// make_rho: Map-Charge of Sec. 3.1 -- "multiplies the particle charge by the
// stencil coefficient and adds that value to a point on the grid", over the
// P^3 stencil whose coefficients are a product of three 1-D polynomials.
//
// GB300 layout: one CTA per mesh tile (particles already sorted by the tile
// of their stencil anchor).  The CTA accumulates its particles' full stencils
// into a private shared-memory brick that covers the tile plus its P-1 halo
// (the paper's thread-private grid copies, "rethread"), then adds the brick
// to the global mesh once.  Within a warp, P lanes serve one particle and lane
// k owns stencil offset k along z (unit stride); 32 / P particles share a
// warp, so for P < 7 no lane is spent on the paper's padding of the inner
// loop to 8 ("simd8").  At P = 7 the groups keep 8 lanes (four particles a
// warp either way); so does the four-copy brick kernel below.
//
// Accumulators (ACC):
//  ACC_NATIVE  atomics in the step type (FP64).  On sm_103a shared
//              float/double atomic adds are compare-and-swap loops whose
//              round trip serialises each thread's updates.
//  ACC_FIXED1  FP32: one 32-bit integer word per brick point, sum rint(v s)
//              with s chosen per tile so that a contribution stays below
//              2^22 and any point's sum below 2^30: one FMA, one integer
//              add and one native integer atomic a point, exact and
//              independent of order for the rounded contributions (each
//              rounded once, to 2^-23 of the tile's largest possible
//              contribution -- the rounding FP32 float accumulation makes
//              against a running sum of that size).  A tile whose charge sum
//              would cost that resolution more than two bits (e.g. tens of
//              thousands of charges in one tile) takes the two-word ACC_FIXED
//              accumulation instead; the choice is per tile, CTA-uniform.
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
#include <type_traits>

#include "pppm_common.cuh"

namespace pppm {

constexpr int RHO_THREADS = 256;
constexpr int GROUP = 8;
constexpr int ACC_NATIVE = 0, ACC_FIXED = 1, ACC_FIXED1 = 2;
constexpr int LO_CHUNK = 32768;
constexpr int ORDER_CHUNK = RHO_THREADS;  // particles per bank-ordered sub-chunk (one per thread)
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

// Power-of-two fixed-point scale for one tile's particles [start, end):
// s = 2^e with every contribution |q W s / vcell| < 2^21 (W <= 1) and every
// brick point's sum < 2^30.  With one_word non-null (ACC_FIXED1): W <= wmax3
// (the largest weight product of the stencil), and the one-word scale,
// contributions below 2^22, where the sum bound costs that at most two bits
// (*one_word = true), else the two-word scale.
// Whole CTA; ends with the CTA synchronised.
template <typename R, int NT = RHO_THREADS>
__device__ __forceinline__ void fixed_scale(const R *__restrict__ recp, int start, int end, float ivcell,
                                            float &fs, float &ifs, bool *one_word = nullptr, float wmax3 = 1.0f) {
    static_assert(NT / 32 <= 32, "one warp combines the warps' partials");
    __shared__ float sh_red[NT / 32];
    __shared__ float sh_max[NT / 32];
    __shared__ int sh_e[2];  // the scale exponent, the one-word choice
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
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        sh_red[threadIdx.x >> 5] = part;
        sh_max[threadIdx.x >> 5] = pmax;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // warp 0 combines the partials and picks the scale
        float bound = (lane < NT / 32) ? sh_red[lane] : 0.0f, bmax = (lane < NT / 32) ? sh_max[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bound += __shfl_xor_sync(0xffffffffu, bound, o);
            bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        }
        if (lane == 0) {
            // one_word: every weight product is at most wmax3 (< 1), which
            // bounds both the contributions and the point sums more tightly
            const float wb = one_word ? wmax3 : 1.0f;
            bound = bound * ivcell * wb * 1.0001f + 1e-30f;
            bmax = bmax * ivcell * wb * 1.0001f + 1e-30f;
            int es, em;
            frexpf(bound, &es);  // bound < 2^es
            frexpf(bmax, &em);   // largest contribution < 2^em
            int e = min(30 - es, 21 - em), one = 0;
            if (one_word) {
                const int e1 = min(30 - es, 22 - em);
                one = (22 - em) - e1 <= 2;
                if (one) e = e1;
            }
            sh_e[0] = e;
            sh_e[1] = one;
        }
    }
    __syncthreads();
    const int e = sh_e[0];
    if (one_word) *one_word = sh_e[1] != 0;
    fs = __int_as_float((127 + e) << 23);   // 2^e, |e| < 127
    ifs = __int_as_float((127 - e) << 23);  // 2^-e
}

// a / b for 0 <= a and 1 <= b: a shift when b is a power of two (the usual
// tile counts), else the integer division.  CTA-uniform operands.
__device__ __forceinline__ int div_tiles(int a, int b) { return (b & (b - 1)) == 0 ? a >> (__ffs(b) - 1) : a / b; }

// Origin and brick extents (tile plus P - 1 halo) of a tile, as tile_of /
// tile_origin define them: multiplications where the dimension's tiles are
// all TE wide (M = T TE), the divisions of tile_origin otherwise.
template <typename R, int P>
__device__ __forceinline__ void tile_extent(const Geom<R> &g, int tile, int &ox, int &oy, int &oz, int &Ex, int &Ey,
                                            int &Ez) {
    const int r1 = div_tiles(tile, g.T[2]);
    const int tz = tile - r1 * g.T[2];
    const int tx = div_tiles(r1, g.T[1]);
    const int ty = r1 - tx * g.T[1];
    const int t[3] = {tx, ty, tz};
    int o[3], e[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (g.T[d] * g.TE[d] == g.M[d]) {
            o[d] = t[d] * g.TE[d];
            e[d] = g.TE[d] + P - 1;
        } else {
            o[d] = tile_origin(t[d], g.T[d], g.M[d]);
            e[d] = tile_origin(t[d] + 1, g.T[d], g.M[d]) - o[d] + P - 1;
        }
    }
    ox = o[0]; oy = o[1]; oz = o[2];
    Ex = e[0]; Ey = e[1]; Ez = e[2];
}

// CS: the brick's strides are those of the largest tile (TILE_B + P - 1 per
// edge, compile-time), so every stencil point's offset is an immediate;
// otherwise they are this tile's own extents.  NZT = 2 (with CS; the plan's
// variant bit 7): `unit` is a z-pair of tiles, row r = unit / ceil(T_z / 2),
// pair k = unit mod ceil(T_z / 2): tiles r T_z + 2k and, unless T_z is odd
// and k the last pair, r T_z + 2k + 1, z neighbours whose particles are
// contiguous in the sorted order, in one brick TILE_B + P - 1 by TILE_B +
// P - 1 by 2 TILE_B + P - 1 (z tiles are at most TILE_B deep): the pair's
// shared halo reaches the mesh's atomics once instead of twice, and a CTA's
// fixed costs (scale, order, clearing) serve twice the particles.  NZT = 1:
// `unit` is the tile.
template <typename R, int P, int ACC, bool CS = false, int NZT = 1>
__device__ __forceinline__ void make_rho_body(const Geom<R> &g, const SortBufs &b, R *__restrict__ rho,
                                              int unit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(NZT == 1 || (NZT == 2 && CS), "tile pairs use the compile-time-stride brick");

    int tile = unit, ntz = 1;  // first tile and tiles of this CTA
    // (an even number of uniform z tiles, c3's case, takes the short path:
    // the index arithmetic runs in all of the CTA's threads)
    const bool zpaired = NZT == 2 && (g.T[2] & 1) == 0 && g.T[2] * g.TE[2] == g.M[2];
    if (zpaired) {
        tile = 2 * unit;
        ntz = 2;
    } else if (NZT == 2) {
        const int pairs = (g.T[2] + 1) >> 1;
        const int row = div_tiles(unit, pairs);
        const int k = unit - row * pairs;
        tile = row * g.T[2] + 2 * k;
        ntz = min(2, g.T[2] - 2 * k);
    }
    int ox, oy, oz, Ex, Ey, Ez;
    tile_extent<R, P>(g, tile, ox, oy, oz, Ex, Ey, Ez);
    if (zpaired) {
        Ez += g.TE[2];
    } else if (NZT == 2 && ntz == 2) {  // the pair's brick: through the end of the second tile
        const int tz = tile - div_tiles(tile, g.T[2]) * g.T[2];
        Ez = tile_origin(tz + 2, g.T[2], g.M[2]) - oz + P - 1;
    }
    constexpr int EB = TILE_B + P - 1;          // widest brick edge
    constexpr int EBZ = NZT * TILE_B + P - 1;   // ... along z
    const int SZ = CS ? EBZ : Ez;               // brick row (z) stride
    const int SY = CS ? EB * EBZ : Ey * Ez;     // brick plane stride
    const int vol = CS ? EB * EB * EBZ : Ex * Ey * Ez;

    // bank-ordering scratch: particles of a sub-chunk counted by the shared
    // bank of their first stencil point, then listed in that order
    __shared__ int s_bins[32], s_off[32];
    __shared__ int s_list[ORDER_CHUNK];

    // the brick is this CTA's own shared memory: cleared while the sort may
    // still be finishing (ordered before the atomics by the barrier below)
    {
        const int words = (ACC != ACC_NATIVE ? 2 * vol : vol * (int)(sizeof(R) / 4));
        int4 *w4 = reinterpret_cast<int4 *>(smem_raw);
        const int n4 = words >> 2;
        for (int e = threadIdx.x; e < n4; e += blockDim.x) w4[e] = make_int4(0, 0, 0, 0);
        int *w = reinterpret_cast<int *>(smem_raw);
        for (int e = 4 * n4 + (int)threadIdx.x; e < words; e += blockDim.x) w[e] = 0;
        if (threadIdx.x < 32) s_bins[threadIdx.x] = 0;
    }

    pdl_wait();  // the sort's outputs (and its reads of the histogram) are complete
    const int start = b.tile_start[tile], end = b.tile_start[tile + ntz];
    if ((int)threadIdx.x < ntz) b.tile_count[tile + threadIdx.x] = 0;  // histogram is clean for the next step
    if (start == end) return;

    R *accr = reinterpret_cast<R *>(smem_raw);
    int *acch = reinterpret_cast<int *>(smem_raw);
    unsigned int *accl = reinterpret_cast<unsigned int *>(smem_raw) + vol;
    const R *__restrict__ recp = reinterpret_cast<const R *>(b.rec);

    // fixed-point scale s = 2^e: every contribution |v s| < 2^21 (so it can be
    // split with the float magic-number trick) and every brick point's sum
    // |sum v s| < 2^30 (so the hi word cannot overflow)
    float fs = 1.0f, ifs = 1.0f;
    bool one = false;  // ACC_FIXED1: this tile accumulates in one word
    if (ACC == ACC_FIXED) fixed_scale<R>(recp, start, end, (float)g.ivcell, fs, ifs);
    else if (ACC == ACC_FIXED1)
        fixed_scale<R>(recp, start, end, (float)g.ivcell, fs, ifs, &one, g.wmax3 > 0.0f ? fminf(g.wmax3, 1.0f) : 1.0f);
    else __syncthreads();  // (fixed_scale ends with one)

    // GS lanes serve one particle (32 / GS particles per warp; the lanes past
    // the last whole group idle).  GS = P, except 8 at P = 7: the warp holds
    // four particles either way and the power of two indexes cheaper
    // (measured 5 % faster at 2M charges).
    constexpr int GS = (P == 7) ? 8 : P;
    constexpr int NG = 32 / GS;
    const int lane = threadIdx.x & 31;
    const int k = lane % GS;                     // z stencil offset of this lane
    const int gbase = lane - k;
    const bool lane_on = lane < NG * GS && k < P;
    const int q = lane / GS;                     // this group's place in its warp
    const int warp = threadIdx.x >> 5;
    const int ngrp = (blockDim.x >> 5) * NG;     // particle slots per pass of the CTA
    const R qscale = (ACC != ACC_NATIVE) ? (R)(g.ivcell * (R)fs) : g.ivcell;
    // this lane's polynomial (stencil offset k), held in registers for the CTA
    R ck[P];
#pragma unroll
    for (int l = 0; l < P; ++l) ck[l] = (k < P) ? g.coef[k][l] : R(0);

    for (int chunk = start; chunk < end; chunk += LO_CHUNK) {
        const int cend = min(end, chunk + LO_CHUNK);
        for (int sub = chunk; sub < cend; sub += ORDER_CHUNK) {
            const int nch = min(ORDER_CHUNK, cend - sub);
            // Bank order: a group's z run starts at brick word row0 = anchor
            // index, so its atomics hit banks row0 + k + (a, c offset) mod 32
            // and two groups of one warp collide iff their row0 are closer
            // than P mod 32, whatever (a, c).  Counting-sort the sub-chunk by
            // row0 mod 32 and hand the warp's groups particles a quarter (an
            // NG-th) of the sorted list apart: their runs then start about
            // 32 / NG >= P banks apart.  The accumulation is exact integer
            // arithmetic (ACC_FIXED, ACC_FIXED1), so the order changes no
            // result bit.
            {
                int key = 0, rank = 0;
                if ((int)threadIdx.x < nch) {
                    int ax, ay, az;
                    unpack_anchor(b.cell[sub + threadIdx.x], ax, ay, az);
                    key = ((ax - ox) * SY + (ay - oy) * SZ + (az - oz)) & 31;
                    rank = atomicAdd(&s_bins[key], 1);
                }
                __syncthreads();
                if (threadIdx.x < 32) {
                    const int v = s_bins[threadIdx.x];
                    int incl = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, incl, o);
                        if ((int)threadIdx.x >= o) incl += u;
                    }
                    s_off[threadIdx.x] = incl - v;
                    s_bins[threadIdx.x] = 0;  // clean for the next sub-chunk
                }
                __syncthreads();
                if ((int)threadIdx.x < nch) s_list[s_off[key] + rank] = threadIdx.x;
                __syncthreads();
            }
            const int Q = (nch + NG - 1) / NG;   // sorted positions per group place
            // warp-uniform trip count: all 32 lanes take part in the shuffles
            for (int base = 0; base < NG * Q; base += ngrp) {
                const int col = base / NG + warp;   // slot (base + warp NG + q) -> position q Q + col
                const int pos = q * Q + col;
                const bool live = lane_on && col < Q && pos < nch;
                R dx = R(0), dy = R(0), dz = R(0), qv = R(0);
                int ax = 0, ay = 0, az = 0;
                if (live) {
                    const int j = sub + s_list[pos];
                    const vec4_t<R> r = reinterpret_cast<const vec4_t<R> *>(recp)[j];
                    dx = r.x; dy = r.y; dz = r.z; qv = r.w * qscale;
                    unpack_anchor(b.cell[j], ax, ay, az);
                    ax -= ox; ay -= oy; az -= oz;        // local anchor in [0, tile size)
                    if ((unsigned)ax > (unsigned)(Ex - P) || (unsigned)ay > (unsigned)(Ey - P) ||
                        (unsigned)az > (unsigned)(Ez - P)) {  // not this tile's particle: skip, report
                        if (k == 0) atomicOr(b.err, ERR_INTERNAL);
                        ax = ay = az = 0;
                        qv = R(0);
                    }
                }
                // lane k evaluates the three weights of stencil offset k (an idle
                // lane's shuffle source wraps within the warp; it is not used)
                const R wx = horner<R, P>(ck, dx), wy = horner<R, P>(ck, dy), wz = horner<R, P>(ck, dz);
                R wxq[P], wyk[P];
#pragma unroll
                for (int t = 0; t < P; ++t) {
                    wxq[t] = __shfl_sync(0xffffffffu, wx, (gbase + t) & 31) * qv;
                    wyk[t] = __shfl_sync(0xffffffffu, wy, (gbase + t) & 31);
                }
                if (live && ACC == ACC_FIXED1 && one) {
                    // t = wa wy s rounded to an integer inside the FMA (|t| < 2^22)
                    const int row = ax * SY + ay * SZ + az + k;
#pragma unroll
                    for (int a = 0; a < P; ++a) {
                        const float fa = (float)(wxq[a] * wz);
#pragma unroll
                        for (int c = 0; c < P; ++c) {
                            const float r1 = __fmaf_rn(fa, (float)wyk[c], MAGIC);
                            atomicAdd(&acch[row + a * SY + c * SZ], __float_as_int(r1) - MAGIC_BITS);
                        }
                    }
                } else if (live) {
                    const int row = ax * SY + ay * SZ + az + k;
#pragma unroll
                    for (int a = 0; a < P; ++a) {
                        const R wa = wxq[a] * wz;
#pragma unroll
                        for (int c = 0; c < P; ++c) {
                            const int e = row + a * SY + c * SZ;
                            if (ACC != ACC_NATIVE) {
                                // t = wa wy s = hi + lo / 2^16, the product never
                                // rounded on its own: adding 1.5 * 2^23 inside the
                                // FMA rounds |t| < 2^22 to an integer held in the
                                // mantissa bits, and the second FMA takes the exact
                                // remainder (|.| <= 1/2) before its one rounding
                                const float fa = (float)wa, fy = (float)wyk[c];
                                const float r1 = __fmaf_rn(fa, fy, MAGIC);
                                const float hi = __fadd_rn(r1, -MAGIC);  // exact
                                const float fr = __fmaf_rn(fa, fy, -hi);
                                const float r2 = __fmaf_rn(fr, 65536.0f, MAGIC);
                                atomicAdd(&acch[e], __float_as_int(r1) - MAGIC_BITS);
                                atomicAdd(&accl[e], (unsigned int)(__float_as_int(r2) - MAGIC_BITS));
                            } else {
                                atomicAdd(&accr[e], wa * wyk[c]);
                            }
                        }
                    }
                }
            }
            __syncthreads();  // the list is rewritten by the next sub-chunk
        }
        if (ACC != ACC_NATIVE && !one && cend < end) {  // fold lo into hi before it can overflow
            for (int e = threadIdx.x; e < vol; e += blockDim.x) {
                const int l = (int)accl[e];  // signed sum of fractions in [-2^15, 2^15] each
                acch[e] += l >> 16;          // floor division by 2^16
                accl[e] = (unsigned int)(l & 0xffff);
            }
            __syncthreads();
        }
    }

    // flush the brick (tile + halo) into the global mesh: thread (ry, lz) owns
    // brick column (y = ry, z = lz) -- edges are at most TILE_B + P - 1 <= 16
    // points -- and walks it along x; every wrap is a single conditional since
    // the brick is never wider than the mesh plus one period.
    // (a tile pair's 2 TILE_B + P - 1 deep columns: every thread takes columns
    // a CTA apart)
    static_assert(TILE_B + 7 - 1 <= 16 && RHO_THREADS == 256, "one brick column per thread");
    auto flush_column = [&](int ry, int lz) {
        int gz = oz - g.rlo + lz;
        gz += (gz < 0) ? g.M[2] : 0;
        gz -= (gz >= g.M[2]) ? g.M[2] : 0;
        int gy = oy - g.rlo + ry;
        gy += (gy < 0) ? g.M[1] : 0;
        gy -= (gy >= g.M[1]) ? g.M[1] : 0;
        R *__restrict__ col = rho + gy * g.M[2] + gz;
        const int plane = g.M[1] * g.M[2];
        const int e0 = ry * SZ + lz;
        int gx = ox - g.rlo;
        gx += (gx < 0) ? g.M[0] : 0;
        for (int ex = 0; ex < Ex; ++ex) {
            const int e = e0 + ex * SY;
            R v;
            if (ACC == ACC_FIXED1 && one) {
                v = (R)((float)acch[e] * ifs);
            } else if (ACC != ACC_NATIVE) {
                // normalise in integers (exact), then one FP32 rounding
                const int l = (int)accl[e];
                const int h = acch[e] + (l >> 16);
                v = (R)(fmaf((float)(l & 0xffff), 1.0f / 65536.0f, (float)h) * ifs);
            } else {
                v = accr[e];
            }
            if (v != R(0)) atomicAdd(col + gx * plane, v);
            gx = (gx + 1 == g.M[0]) ? 0 : gx + 1;
        }
    };
    if (NZT == 1) {
        const int lz = threadIdx.x & 15, ry = threadIdx.x >> 4;
        if (lz < Ez && ry < Ey) flush_column(ry, lz);
    } else {
        for (int c = threadIdx.x; c < Ey * EBZ; c += blockDim.x) {
            const int lz = c % EBZ;
            if (zpaired || lz < Ez) flush_column(c / EBZ, lz);
        }
    }
}

// ---------------------------------------------------------------------------
// FP32C, 8-lane particle groups, four-copy brick (variant bit 2 of a plan,
// chosen by pppm_autotune; in the batch, the kernel for P <= 5).  Measured
// on GB300: level with make_rho_body at P = 5 (32k and 100k charges, where
// make_rho waits on latency, not on the atomic unit), slower at P = 7 on
// 2M charges (824 vs 685 us: zeroing and flushing four 2744-point copies per
// 8^3 tile of ~62 particles outweighs the bank conflicts it removes).
//
// Same work split and accumulators as make_rho_body<ACC_FIXED>, with four
// interleaved copies of the brick: the particle group in lanes 8g..8g+7 adds
// into copy g, word 4e + g of brick point e.  A group's z run e0..e0+7 then
// covers banks 4(e0 + k) + g, distinct within the group and disjoint between
// the four groups of a warp, so the atomics never replay on bank conflicts
// (with one shared brick, the four particles of a warp collided on 60 % of
// the atomic wavefronts).  The flush sums the copies exactly in integers.
// Strides are compile-time (E = TILE_B + P - 1 points per dimension, tiles at
// most TILE_B wide), every atomic is a red.shared.add.u32 at one register
// plus a compile-time offset, and the contribution t = wa * wy is never
// rounded on its own (both FMAs of the split see the exact product).
// ---------------------------------------------------------------------------
template <int P>
struct GBrick {
    static constexpr int NT = RHO_THREADS;
    static constexpr int E = TILE_B + P - 1;
    static constexpr int RS = E;          // z row stride (points)
    static constexpr int PS = E * E;      // x plane stride
    static constexpr int VOL = E * E * E;
    static constexpr int COPIES = 4;
    static constexpr int WORDS = COPIES * VOL;  // per accumulator array (hi or lo)
    static constexpr size_t BYTES = 2 * WORDS * sizeof(int);
};

template <int OFF>
__device__ __forceinline__ void red_shared_s32(unsigned int addr, int v) {
    asm volatile("red.shared.add.u32 [%0+%2], %1;" ::"r"(addr), "r"(v), "n"(OFF));
}

// Stencil point I = a * P + c of this lane's z column: hi = rint(t) and
// lo = rint(frac 2^16), each added as a signed integer.
template <int I, int P>
struct Scatter8 {
    static __device__ __forceinline__ void run(const float (&wa)[P], const float (&wy)[P], unsigned int addr) {
        using BR = GBrick<P>;
        constexpr int a = I / P, c = I % P;
        constexpr int off = 4 * BR::COPIES * (a * BR::PS + c * BR::RS);  // bytes
        const float r1 = __fmaf_rn(wa[a], wy[c], MAGIC);
        const float hi = __fadd_rn(r1, -MAGIC);
        const float fr = __fmaf_rn(wa[a], wy[c], -hi);  // |fr| <= 1/2, rounded once
        const float r2 = __fmaf_rn(fr, 65536.0f, MAGIC);
        red_shared_s32<off>(addr, __float_as_int(r1) - MAGIC_BITS);
        red_shared_s32<off + 4 * BR::WORDS>(addr, __float_as_int(r2) - MAGIC_BITS);
        Scatter8<I + 1, P>::run(wa, wy, addr);
    }
};
template <int P>
struct Scatter8<P * P, P> {
    static __device__ __forceinline__ void run(const float (&)[P], const float (&)[P], unsigned int) {}
};

template <int P>
__device__ __forceinline__ void make_rho_fixed_body(const Geom<float> &g, const SortBufs &b,
                                                    float *__restrict__ rho, int tile) {
    using BR = GBrick<P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *acch = reinterpret_cast<int *>(smem_raw);
    int *accl = acch + BR::WORDS;

    const int tz = tile % g.T[2];
    const int ty = (tile / g.T[2]) % g.T[1];
    const int tx = tile / (g.T[2] * g.T[1]);
    const int ox = tile_origin(tx, g.T[0], g.M[0]);
    const int oy = tile_origin(ty, g.T[1], g.M[1]);
    const int oz = tile_origin(tz, g.T[2], g.M[2]);
    const int Ex = tile_origin(tx + 1, g.T[0], g.M[0]) - ox + P - 1;
    const int Ey = tile_origin(ty + 1, g.T[1], g.M[1]) - oy + P - 1;
    const int Ez = tile_origin(tz + 1, g.T[2], g.M[2]) - oz + P - 1;

    pdl_wait();  // the sort's outputs (and its reads of the histogram) are complete
    const int start = b.tile_start[tile], end = b.tile_start[tile + 1];
    if (threadIdx.x == 0) b.tile_count[tile] = 0;  // histogram is clean for the next step
    if (start == end) return;

    const float4 *__restrict__ rec = reinterpret_cast<const float4 *>(b.rec);
    float fs, ifs;
    fixed_scale<float, BR::NT>(reinterpret_cast<const float *>(b.rec), start, end, g.ivcell, fs, ifs);
    for (int e = threadIdx.x; e < 2 * BR::WORDS; e += BR::NT) acch[e] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int k = lane & (GROUP - 1);            // z stencil offset of this lane
    const int gbase = lane & ~(GROUP - 1);
    const int copy = lane >> 3;                  // this group's brick copy
    const int grp = threadIdx.x / GROUP;         // particle slot in the CTA
    constexpr int NGRP = BR::NT / GROUP;
    const float qscale = g.ivcell * fs;
    float ck[P];
#pragma unroll
    for (int l = 0; l < P; ++l) ck[l] = (k < P) ? g.coef[k][l] : 0.0f;
    const unsigned int sbase = (unsigned int)__cvta_generic_to_shared(acch) + 4u * (unsigned int)copy;
    bool bad = false;  // a particle outside this tile (an inconsistent sort)

    for (int chunk = start; chunk < end; chunk += LO_CHUNK) {
        const int cend = min(end, chunk + LO_CHUNK);
        // warp-uniform trip count: all 32 lanes take part in the shuffles
        for (int base = chunk; base < cend; base += NGRP) {
            const int j = base + grp;
            const bool live = j < cend;
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            int ax = 0, ay = 0, az = 0;
            if (live) {
                r = rec[j];
                unpack_anchor(b.cell[j], ax, ay, az);
                ax -= ox; ay -= oy; az -= oz;        // local anchor in [0, tile size)
            }
            const bool out = (unsigned)ax > (unsigned)(Ex - P) || (unsigned)ay > (unsigned)(Ey - P) ||
                             (unsigned)az > (unsigned)(Ez - P);
            bad |= live && out;
            const bool use = live && !out;
            const float qv = use ? r.w * qscale : 0.0f;
            // lane k < P evaluates the three weights of stencil offset k
            const float wx = horner<float, P>(ck, r.x), wy = horner<float, P>(ck, r.y);
            const float wz = horner<float, P>(ck, r.z);
            float wa[P], wyk[P];
#pragma unroll
            for (int t = 0; t < P; ++t) {
                wa[t] = __shfl_sync(0xffffffffu, wx, gbase + t) * qv * wz;
                wyk[t] = __shfl_sync(0xffffffffu, wy, gbase + t);
            }
            if (use && k < P) {
                const unsigned int addr =
                    sbase + 4u * BR::COPIES * (unsigned int)(ax * BR::PS + ay * BR::RS + az + k);
                Scatter8<0, P>::run(wa, wyk, addr);
            }
        }
        if (cend < end) {  // fold lo into hi (every copy) before it can overflow
            __syncthreads();
            for (int e = threadIdx.x; e < BR::WORDS; e += BR::NT) {
                const int l = accl[e];       // signed sum of fractions in [-2^15, 2^15] each
                acch[e] += l >> 16;          // floor division by 2^16
                accl[e] = l & 0xffff;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(b.err, ERR_INTERNAL);

    // flush the brick (tile + halo) into the global mesh: 16 lanes per z row
    // (Ez <= 14), 16 rows per pass; every wrap is a single conditional since
    // the brick is never wider than the mesh plus one period
    // rows (ex, ey) dealt out over NT / 16 row slots
    const int lz = threadIdx.x & 15, rslot = threadIdx.x >> 4;
    if (lz < Ez) {
        int gz = oz - g.rlo + lz;
        gz += (gz < 0) ? g.M[2] : 0;
        gz -= (gz >= g.M[2]) ? g.M[2] : 0;
        for (int row = rslot; row < Ex * Ey; row += BR::NT / 16) {
            const int ex = row / Ey, ey = row - ex * Ey;
            int gx = ox - g.rlo + ex;
            gx += (gx < 0) ? g.M[0] : 0;
            gx -= (gx >= g.M[0]) ? g.M[0] : 0;
            {
                int gy = oy - g.rlo + ey;
                gy += (gy < 0) ? g.M[1] : 0;
                gy -= (gy >= g.M[1]) ? g.M[1] : 0;
                const int w = BR::COPIES * (ex * BR::PS + ey * BR::RS + lz);
                // the four copies, normalised in integers (exact), then one FP32 rounding
                int h = 0, fr = 0;
#pragma unroll
                for (int cp = 0; cp < BR::COPIES; ++cp) {
                    const int l = accl[w + cp];
                    h += acch[w + cp] + (l >> 16);
                    fr += l & 0xffff;
                }
                h += fr >> 16;
                const float v = fmaf((float)(fr & 0xffff), 1.0f / 65536.0f, (float)h) * ifs;
                if (v != 0.0f) atomicAdd(&rho[(gx * g.M[1] + gy) * g.M[2] + gz], v);
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(GBrick<P>::NT) k_make_rho_fixed(Geom<float> g, SortBufs b, float *__restrict__ rho) {
    make_rho_fixed_body<P>(g, b, rho, blockIdx.x);
}

template <int P>
__global__ void __launch_bounds__(GBrick<P>::NT) k_batch_make_rho_fixed(const BatchSys<float> *__restrict__ sys,
                                                                        BatchList bl) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<float> &S = sys[bl.ids[e]];
    make_rho_fixed_body<P>(S.g, S.sb, S.rho, blockIdx.x - bl.boff[e]);
}

template <typename R, int P, int ACC, bool CS = false, int NZT = 1>
__global__ void __launch_bounds__(RHO_THREADS) k_make_rho(Geom<R> g, SortBufs b, R *__restrict__ rho) {
    make_rho_body<R, P, ACC, CS, NZT>(g, b, rho, blockIdx.x);
}

// (NZT = 2: the list counts each system's z-pairs of tiles)
template <typename R, int P, int ACC, int NZT = 1>
__global__ void __launch_bounds__(RHO_THREADS) k_batch_make_rho(const BatchSys<R> *__restrict__ sys, BatchList bl) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<R> &S = sys[bl.ids[e]];
    make_rho_body<R, P, ACC, true, NZT>(S.g, S.sb, S.rho, blockIdx.x - bl.boff[e]);  // compile-time brick strides
}

// Dynamic shared memory of make_rho_body: one tile's brick, or a z-pair's
template <typename R, int P>
static size_t brick_bytes(int acc, int nzt = 1) {
    const int E = TILE_B + P - 1;
    return (size_t)E * E * (E + (nzt - 1) * TILE_B) * (acc != ACC_NATIVE ? 8 : sizeof(R));
}

template <typename K, typename R>
static void launch_one(K kernel, bool pdl, dim3 grid, size_t bytes, cudaStream_t s, const Geom<R> &g,
                       const SortBufs &b, R *rho, int threads = RHO_THREADS) {
    if (pdl)
        launch_pdl(kernel, grid, dim3(threads), bytes, s, g, b, rho);
    else
        kernel<<<grid, threads, bytes, s>>>(g, b, rho);
}

template <typename R, int P>
static void launch_p(const Geom<R> &g, const SortBufs &b, R *rho, int acc, cudaStream_t s, bool pdl) {
    const size_t bytes = brick_bytes<R, P>(acc);
    if constexpr (std::is_same<R, float>::value) {
        if (acc == ACC_FIXED && g.rho_copies == 1) {
            launch_one(k_make_rho_fixed<P>, pdl, dim3(g.ntiles), GBrick<P>::BYTES, s, g, b, rho, GBrick<P>::NT);
            return;
        }
    }
    const bool cs = g.rho_copies == 2;  // one brick with compile-time strides
    if (g.rho_copies == 4) {            // ... over a z-pair of tiles
        const size_t b2 = brick_bytes<R, P>(acc, 2);
        const dim3 grid(g.T[0] * g.T[1] * ((g.T[2] + 1) / 2));
        if (acc == ACC_FIXED) {
            launch_one(k_make_rho<R, P, ACC_FIXED, true, 2>, pdl, grid, b2, s, g, b, rho);
        } else if (acc == ACC_FIXED1) {
            if constexpr (std::is_same<R, float>::value)
                launch_one(k_make_rho<R, P, ACC_FIXED1, true, 2>, pdl, grid, b2, s, g, b, rho);
        } else {
            launch_one(k_make_rho<R, P, ACC_NATIVE, true, 2>, pdl, grid, b2, s, g, b, rho);
        }
        return;
    }
    if (acc == ACC_FIXED) {
        if (cs) launch_one(k_make_rho<R, P, ACC_FIXED, true>, pdl, dim3(g.ntiles), bytes, s, g, b, rho);
        else launch_one(k_make_rho<R, P, ACC_FIXED>, pdl, dim3(g.ntiles), bytes, s, g, b, rho);
    } else if (acc == ACC_FIXED1) {
        if constexpr (std::is_same<R, float>::value) {
            if (cs) launch_one(k_make_rho<R, P, ACC_FIXED1, true>, pdl, dim3(g.ntiles), bytes, s, g, b, rho);
            else launch_one(k_make_rho<R, P, ACC_FIXED1>, pdl, dim3(g.ntiles), bytes, s, g, b, rho);
        }
    } else {
        if (cs) launch_one(k_make_rho<R, P, ACC_NATIVE, true>, pdl, dim3(g.ntiles), bytes, s, g, b, rho);
        else launch_one(k_make_rho<R, P, ACC_NATIVE>, pdl, dim3(g.ntiles), bytes, s, g, b, rho);
    }
}

template <typename R, int P>
static cudaError_t prepare_p(int acc) {
    const int bytes = (int)brick_bytes<R, P>(acc);
    cudaError_t e;
    if constexpr (std::is_same<R, float>::value) {
        if (acc == ACC_FIXED) {
            e = cudaFuncSetAttribute(k_make_rho_fixed<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)GBrick<P>::BYTES);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_batch_make_rho_fixed<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GBrick<P>::BYTES);
            return e;
        }
    }
    if (acc == ACC_FIXED) {
        e = cudaFuncSetAttribute(k_make_rho<R, P, ACC_FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_batch_make_rho<R, P, ACC_FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     bytes);
        return e;
    }
    if constexpr (std::is_same<R, float>::value) {
        if (acc == ACC_FIXED1) {
            e = cudaFuncSetAttribute(k_make_rho<R, P, ACC_FIXED1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_make_rho<R, P, ACC_FIXED1, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_batch_make_rho<R, P, ACC_FIXED1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            return e;
        }
    }
    e = cudaFuncSetAttribute(k_make_rho<R, P, ACC_NATIVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_make_rho<R, P, ACC_NATIVE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    return e;
}

template <typename R, int P>
static void launch_batch_p(const BatchSys<R> *sys, const BatchList &bl, int acc, bool copies4, bool pairs,
                           cudaStream_t s) {
    const size_t bytes = brick_bytes<R, P>(acc);
    if constexpr (std::is_same<R, float>::value) {
        if (acc == ACC_FIXED && copies4) {
            k_batch_make_rho_fixed<P><<<bl.nblocks, GBrick<P>::NT, GBrick<P>::BYTES, s>>>(sys, bl);
            return;
        }
    }
    if (pairs) {  // (a pair's brick stays below the default 48 KB of dynamic shared memory)
        const size_t b2 = brick_bytes<R, P>(acc, 2);
        if (acc == ACC_FIXED) {
            k_batch_make_rho<R, P, ACC_FIXED, 2><<<bl.nblocks, RHO_THREADS, b2, s>>>(sys, bl);
        } else if (acc == ACC_FIXED1) {
            if constexpr (std::is_same<R, float>::value)
                k_batch_make_rho<R, P, ACC_FIXED1, 2><<<bl.nblocks, RHO_THREADS, b2, s>>>(sys, bl);
        } else {
            k_batch_make_rho<R, P, ACC_NATIVE, 2><<<bl.nblocks, RHO_THREADS, b2, s>>>(sys, bl);
        }
        return;
    }
    if (acc == ACC_FIXED) {
        k_batch_make_rho<R, P, ACC_FIXED><<<bl.nblocks, RHO_THREADS, bytes, s>>>(sys, bl);
    } else if (acc == ACC_FIXED1) {
        if constexpr (std::is_same<R, float>::value)
            k_batch_make_rho<R, P, ACC_FIXED1><<<bl.nblocks, RHO_THREADS, bytes, s>>>(sys, bl);
    } else {
        k_batch_make_rho<R, P, ACC_NATIVE><<<bl.nblocks, RHO_THREADS, bytes, s>>>(sys, bl);
    }
}

// The meshes of the systems in the list must have been cleared.
template <typename R>
void launch_batch_make_rho(const BatchSys<R> *sys, const BatchList &bl, int P, bool comp, bool copies4, bool pairs,
                           cudaStream_t s) {
    if (bl.nblocks == 0) return;
    const int acc = comp ? ACC_FIXED : (std::is_same<R, float>::value ? ACC_FIXED1 : ACC_NATIVE);
    switch (P) {
        case 2: launch_batch_p<R, 2>(sys, bl, acc, copies4, pairs, s); break;
        case 3: launch_batch_p<R, 3>(sys, bl, acc, copies4, pairs, s); break;
        case 4: launch_batch_p<R, 4>(sys, bl, acc, copies4, pairs, s); break;
        case 5: launch_batch_p<R, 5>(sys, bl, acc, copies4, pairs, s); break;
        case 6: launch_batch_p<R, 6>(sys, bl, acc, copies4, pairs, s); break;
        case 7: launch_batch_p<R, 7>(sys, bl, acc, copies4, pairs, s); break;
        default: break;
    }
}
template void launch_batch_make_rho<float>(const BatchSys<float> *, const BatchList &, int, bool, bool, bool,
                                           cudaStream_t);
template void launch_batch_make_rho<double>(const BatchSys<double> *, const BatchList &, int, bool, bool, bool,
                                            cudaStream_t);

template <typename R>
cudaError_t prepare_make_rho(int P, bool comp) {
    const int acc = comp ? ACC_FIXED : (std::is_same<R, float>::value ? ACC_FIXED1 : ACC_NATIVE);
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
void launch_make_rho(const Geom<R> &g, int64_t n, const SortBufs &b, R *rho, bool comp, cudaStream_t s,
                     bool mesh_zeroed, bool pdl) {
    if (!mesh_zeroed) {
        cudaMemsetAsync(rho, 0, sizeof(R) * (size_t)g.M[0] * g.M[1] * g.M[2], s);
        pdl = false;  // the memset now sits between the sort and this launch
    }
    if (n == 0) return;
    const int acc = comp ? ACC_FIXED : (std::is_same<R, float>::value ? ACC_FIXED1 : ACC_NATIVE);
    switch (g.P) {
        case 2: launch_p<R, 2>(g, b, rho, acc, s, pdl); break;
        case 3: launch_p<R, 3>(g, b, rho, acc, s, pdl); break;
        case 4: launch_p<R, 4>(g, b, rho, acc, s, pdl); break;
        case 5: launch_p<R, 5>(g, b, rho, acc, s, pdl); break;
        case 6: launch_p<R, 6>(g, b, rho, acc, s, pdl); break;
        case 7: launch_p<R, 7>(g, b, rho, acc, s, pdl); break;
        default: break;
    }
}

template cudaError_t prepare_make_rho<float>(int, bool);
template cudaError_t prepare_make_rho<double>(int, bool);
template void launch_make_rho<float>(const Geom<float> &, int64_t, const SortBufs &, float *, bool, cudaStream_t,
                                     bool, bool);
template void launch_make_rho<double>(const Geom<double> &, int64_t, const SortBufs &, double *, bool,
                                      cudaStream_t, bool, bool);

}  // namespace pppm
