// particle_map: the "loop over all atoms" that starts every mapping function
// (Sec. 3.1).  Each particle is wrapped into the box, its stencil anchor and
// offset delta are computed, and the particles are counting-sorted by the
// mesh tile of their anchor, so that make_rho and fieldforce see each tile's
// particles contiguously.
//
// Kernels:
//  k_particle_map  anchor + tile histogram (atomic ranks, one atomic per run
//                  of consecutive lanes with the same tile) and per-block
//                  sums of q and q^2; one particle per thread, or
//                  MAP_NPT_BIG on large systems.
//  k_tile_scan     with more than SMALL_TILES tiles: one CTA turns the
//                  histogram into tile offsets (exclusive scan).
//  k_scatter       with at most SMALL_TILES tiles every block first scans the
//                  histogram in shared memory (no grid-wide step in between);
//                  then each particle's (delta, q) record, packed anchor and
//                  input index are written at its sorted position.
// make_rho clears each tile's histogram entry for the next step.
#include "pppm_common.cuh"

namespace pppm {

constexpr int MAP_THREADS = 256;
constexpr int SMALL_TILES = 4096;  // histogram scanned per scatter block up to this many tiles

template <typename R>
__device__ __forceinline__ bool load_particle(const R *__restrict__ x, const R *__restrict__ q,
                                              int i, R (&xi)[3], R &qi) {
    xi[0] = x[3 * (int64_t)i + 0];
    xi[1] = x[3 * (int64_t)i + 1];
    xi[2] = x[3 * (int64_t)i + 2];
    qi = q[i];
    const bool ok = isfinite(xi[0]) && isfinite(xi[1]) && isfinite(xi[2]) && isfinite(qi);
    if (!ok) {  // keep the kernels in bounds; the host reports PPPM_ENONFINITE
        xi[0] = xi[1] = xi[2] = R(0);
        qi = R(0);
    }
    return ok;
}

template <typename R>
__device__ __forceinline__ void anchors(const Geom<R> &g, const R (&xi)[3], int (&a)[3], R (&d)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        grid_anchor<R>(xi[k], g.L[k], g.iL[k], g.ih[k], g.ih_lo[k], g.M[k], g.P, a[k], d[k]);
}

// tile_of without a division where the tiles are all TE = 8 (or 4) wide:
// with M = T TE, ((n + 1) T - 1) / M = n / TE for every 0 <= n < M
template <typename R>
__device__ __forceinline__ int tile_of_dim(const Geom<R> &g, int d, int n) {
    if (g.T[d] * g.TE[d] == g.M[d]) {
        if (g.TE[d] == TILE_B) return n >> 3;
        if (g.TE[d] == TILE_B / 2) return n >> 2;
    }
    return tile_of(n, g.T[d], g.M[d]);
}
template <typename R>
__device__ __forceinline__ int tile_index(const Geom<R> &g, const int (&a)[3]) {
    return (tile_of_dim(g, 0, a[0]) * g.T[1] + tile_of_dim(g, 1, a[1])) * g.T[2] + tile_of_dim(g, 2, a[2]);
}

// Block sums of two values: warps reduce in the step type, the per-warp
// values in FP64 (one barrier).  Valid in thread 0.
template <typename R>
__device__ void block_sum2(R a, R b, double *sh, double &sa, double &sb) {
    a = warp_sum_t<R>(a);
    b = warp_sum_t<R>(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[2 * w] = (double)a;
        sh[2 * w + 1] = (double)b;
    }
    __syncthreads();
    sa = sb = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            sa += sh[2 * k];
            sb += sh[2 * k + 1];
        }
}

// lb / nlb: this CTA's index and the CTA count of its system's launch.
// Grid-stride clear of the mesh (mtot values, 16-byte stores for the bulk).
template <typename R>
__device__ __forceinline__ void clear_mesh(R *__restrict__ rho, int64_t mtot, int lb, int nlb) {
    constexpr int V = 16 / sizeof(R);
    const int64_t nv = mtot / V;
    const int64_t t0 = (int64_t)lb * blockDim.x + threadIdx.x, stride = (int64_t)nlb * blockDim.x;
    for (int64_t k = t0; k < nv; k += stride) reinterpret_cast<uint4 *>(rho)[k] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t k = nv * V + t0; k < mtot; k += stride) rho[k] = R(0);
}

// NPT particles per thread: the block takes particles [lb, lb + 1) x
// NPT blockDim.x, pass u the u-th blockDim.x of them (coalesced).
// x_copy, q_copy (nullable): device copies of the inputs written on the way,
// for inputs read over the host link (the scatter then reads the copies).
template <typename R, int NPT = 1>
__device__ __forceinline__ void particle_map_body(const Geom<R> &g, int n, const R *__restrict__ x,
                                                  const R *__restrict__ q, const SortBufs &b, int lb, int nlb,
                                                  R *__restrict__ rho_zero = nullptr, int64_t mtot = 0,
                                                  R *__restrict__ x_copy = nullptr, R *__restrict__ q_copy = nullptr) {
    __shared__ double sh[32];
    if (rho_zero) clear_mesh<R>(rho_zero, mtot, lb, nlb);
    const int lane = threadIdx.x & 31;
    const unsigned int upto = 0xffffffffu >> (31 - lane);  // lanes 0 .. lane
    R qs = R(0), qq = R(0);
    // every particle's loads in flight before any is used (the kernel waits
    // on them: c3 particle_map 31.4 -> 28.6 us)
    R px[NPT][3], pq[NPT];
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        const int i = (lb * NPT + u) * (int)blockDim.x + (int)threadIdx.x;
        px[u][0] = px[u][1] = px[u][2] = pq[u] = R(0);
        if (i < n) {
            px[u][0] = x[3 * (int64_t)i + 0];
            px[u][1] = x[3 * (int64_t)i + 1];
            px[u][2] = x[3 * (int64_t)i + 2];
            pq[u] = q[i];
        }
    }
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        const int i = (lb * NPT + u) * (int)blockDim.x + (int)threadIdx.x;
        int tile = -1 - lane;  // a key no other lane or tile has
        if (i < n) {
            R xi[3] = {px[u][0], px[u][1], px[u][2]}, qi = pq[u];
            if (!(isfinite(xi[0]) && isfinite(xi[1]) && isfinite(xi[2]) && isfinite(qi))) {
                xi[0] = xi[1] = xi[2] = R(0);  // in bounds; the host reports PPPM_ENONFINITE
                qi = R(0);
                atomicOr(b.err, ERR_NONFINITE);
            }
            if (x_copy) {  // (a non-finite input is copied as zeros; the step reports it)
                x_copy[3 * (int64_t)i + 0] = xi[0];
                x_copy[3 * (int64_t)i + 1] = xi[1];
                x_copy[3 * (int64_t)i + 2] = xi[2];
                q_copy[i] = qi;
            }
            int a[3];
            R d[3];
            anchors<R>(g, xi, a, d);
            tile = tile_index<R>(g, a);
            b.anchor[i] = pack_anchor(a[0], a[1], a[2]);
            qs += qi;
            qq += qi * qi;
        }
        // ranks within the tile: one atomic per run of lanes with the same
        // tile (the atoms of a molecule are consecutive and usually share
        // one), handed out in lane order; lanes with the same tile in
        // different runs take separate atomics
        const int prev = __shfl_up_sync(0xffffffffu, tile, 1);
        const unsigned int starts = __ballot_sync(0xffffffffu, lane == 0 || tile != prev);
        const int rs = 31 - __clz(starts & upto);                   // first lane of this lane's run
        const unsigned int after = starts & ~upto;
        const int re = after ? __ffs(after) - 1 : 32;               // one past its last lane
        int base = 0;
        if (i < n && lane == rs) base = atomicAdd(&b.tile_count[tile], re - rs);
        base = __shfl_sync(0xffffffffu, base, rs);
        if (i < n) b.rank[i] = base + lane - rs;
    }
    // per-block sums of q and q^2, reduced later off the critical path
    double s1, s2;
    block_sum2<R>(qs, qq, sh, s1, s2);
    if (threadIdx.x == 0) {
        b.blk[2 * lb] = s1;
        b.blk[2 * lb + 1] = s2;
    }
    pdl_trigger();
}

template <typename R, int NPT>
__global__ void __launch_bounds__(MAP_THREADS) k_particle_map(Geom<R> g, int n, const R *__restrict__ x,
                                                              const R *__restrict__ q, SortBufs b,
                                                              R *__restrict__ rho_zero, int64_t mtot,
                                                              R *__restrict__ x_copy, R *__restrict__ q_copy) {
    particle_map_body<R, NPT>(g, n, x, q, b, blockIdx.x, gridDim.x, rho_zero, mtot, x_copy, q_copy);
}

// Exclusive scan of the tile histogram into tile offsets (more than
// SMALL_TILES tiles): one CTA of SCAN_THREADS threads.  Warp w owns a
// contiguous segment of the histogram's int4 groups (the histogram comes
// from cudaMalloc, 16-byte aligned) and its lanes read it 32 groups at a
// time, coalesced; up to SCAN_V groups a lane stay in registers between the
// sum and the write (32,768 tiles and fewer: one load round trip).  The
// nt % 4 tiles past the last whole group follow all groups.  The step waits
// on this CTA alone, so its time is L2 round trips.
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_V = 8;
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const int *__restrict__ count, int *__restrict__ start,
                                                            int nt) {
    __shared__ int sh_w[SCAN_THREADS / 32];
    pdl_wait();  // every histogram atomic of particle_map is complete
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nt4 = nt / 4;
    const int seg = ((nt4 + SCAN_THREADS / 32 - 1) / (SCAN_THREADS / 32) + 31) & ~31;  // groups per warp
    const int g0 = min(nt4, w * seg), g1 = min(nt4, g0 + seg);
    const int4 *c4 = reinterpret_cast<const int4 *>(count);
    int4 *s4 = reinterpret_cast<int4 *>(start);
    const bool held = seg <= 32 * SCAN_V;  // the whole segment in registers
    int4 v[SCAN_V];
    // pass 1: the segment's total
    int wsum = 0;
    for (int b0 = g0; b0 < g1; b0 += 32 * SCAN_V) {
#pragma unroll
        for (int k = 0; k < SCAN_V; ++k) {
            const int i = b0 + 32 * k + lane;
            v[k] = (i < g1) ? __ldcg(c4 + i) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < SCAN_V; ++k) wsum += v[k].x + v[k].y + v[k].z + v[k].w;
    }
    pdl_trigger();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if (lane == 0) sh_w[w] = wsum;
    __syncthreads();
    if (w == 0) {
        const int t = sh_w[lane];
        int it = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, it, o);
            if (lane >= o) it += y;
        }
        sh_w[lane] = it - t;  // exclusive prefix of warp segments
        if (lane == 31) {
            // the tail tiles after every whole group, and the total
            int run = it;
            for (int k = 4 * nt4; k < nt; ++k) {
                start[k] = run;
                run += __ldcg(count + k);
            }
            start[nt] = run;
        }
    }
    __syncthreads();
    // pass 2: group by group in segment order, lanes of a row of 32 groups
    // scanned with shuffles, the row totals carried
    int carry = sh_w[w];
    for (int b0 = g0; b0 < g1; b0 += 32 * SCAN_V) {
        if (!held) {
#pragma unroll
            for (int k = 0; k < SCAN_V; ++k) {
                const int i = b0 + 32 * k + lane;
                v[k] = (i < g1) ? __ldcg(c4 + i) : make_int4(0, 0, 0, 0);
            }
        }
#pragma unroll
        for (int k = 0; k < SCAN_V; ++k) {
            const int sk = v[k].x + v[k].y + v[k].z + v[k].w;
            int incl = sk;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int i = b0 + 32 * k + lane;
            if (i < g1) {
                int4 o;
                o.x = carry + incl - sk;
                o.y = o.x + v[k].x;
                o.z = o.y + v[k].y;
                o.w = o.z + v[k].z;
                s4[i] = o;
            }
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// Block-wide exclusive scan of the tile histogram into shared memory
// (small tile counts only): every block of k_scatter does it redundantly, so
// no grid-wide step sits between the histogram and the scatter.
__device__ void scan_tiles_smem(const int *__restrict__ count, int nt, int *sh_start, int *sh_warp) {
    const int chunk = (nt + blockDim.x - 1) / blockDim.x;
    const int lo = min(nt, (int)threadIdx.x * chunk), hi = min(nt, lo + chunk);
    int local = 0;
    for (int k = lo; k < hi; ++k) local += count[k];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) sh_warp[w] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = (lane < (int)(blockDim.x >> 5)) ? sh_warp[lane] : 0;
        int iv = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, iv, o);
            if (lane >= o) iv += t;
        }
        if (lane < (int)(blockDim.x >> 5)) sh_warp[lane] = iv - v;
    }
    __syncthreads();
    int run = sh_warp[w] + incl - local;
    for (int k = lo; k < hi; ++k) {
        sh_start[k] = run;
        run += count[k];
    }
    if (hi == nt && lo < hi) sh_start[nt] = run;
    __syncthreads();
}

// staged: x, q are particle_map's copies, readable only after the wait
template <typename R>
__device__ __forceinline__ void scatter_body(const Geom<R> &g, int n, const R *__restrict__ x,
                                             const R *__restrict__ q, const SortBufs &b, int big, int lb,
                                             bool staged = false) {
    __shared__ int sh_start[SMALL_TILES + 1];
    __shared__ int sh_warp[MAP_THREADS / 32];
    // the record comes from the inputs alone: computed before the histogram is final
    const int i = lb * blockDim.x + threadIdx.x;
    R xi[3], qi = R(0);
    int a[3];
    R d[3] = {R(0), R(0), R(0)};
    if (i < n && !staged) {
        load_particle<R>(x, q, i, xi, qi);
        anchors<R>(g, xi, a, d);
    }
    pdl_wait();
    if (i < n && staged) {
        load_particle<R>(x, q, i, xi, qi);
        anchors<R>(g, xi, a, d);
    }
    // this particle's rank from particle_map, requested before the scan
    const int rank = (i < n) ? b.rank[i] : 0;
    const int *starts = b.tile_start;
    if (!big) {
        scan_tiles_smem(b.tile_count, g.ntiles, sh_start, sh_warp);
        if (lb == 0)
            for (int k = threadIdx.x; k <= g.ntiles; k += blockDim.x) b.tile_start[k] = sh_start[k];
        starts = sh_start;
    }
    pdl_trigger();
    if (i >= n) return;
    if (g.lut_bins > 0) {
        // table coefficients (Sec. 3.1 "precompute"): the offset rounded to
        // the centre of its bin, so every later use reads the table's entry
        const R lo = (g.P & 1) ? R(-0.5) : R(-1), K = (R)g.lut_bins;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R bin = floor((d[k] - lo) * K);
            bin = bin < R(0) ? R(0) : (bin > K - R(1) ? K - R(1) : bin);
            d[k] = lo + (bin + R(0.5)) / K;
        }
    }
    // the anchor is particle_map's: the same function of the same inputs
    const uint32_t packed = pack_anchor(a[0], a[1], a[2]);
    const int dest = starts[tile_index<R>(g, a)] + rank;
    if ((unsigned int)dest >= (unsigned int)n) {  // a stale histogram: skip, report
        atomicOr(b.err, ERR_INTERNAL);
        return;
    }
    vec4_t<R> r;
    r.x = d[0];
    r.y = d[1];
    r.z = d[2];
    r.w = qi;
    reinterpret_cast<vec4_t<R> *>(b.rec)[dest] = r;
    b.cell[dest] = packed;
    b.perm[dest] = i;
}

template <typename R>
__global__ void __launch_bounds__(MAP_THREADS) k_scatter(Geom<R> g, int n, const R *__restrict__ x,
                                                         const R *__restrict__ q, SortBufs b, int big, int staged) {
    scatter_body<R>(g, n, x, q, b, big, blockIdx.x, staged != 0);
}

// Batched: every system of the list in one launch (small tile counts only).
template <typename R>
__global__ void __launch_bounds__(MAP_THREADS) k_batch_map(const BatchSys<R> *__restrict__ sys, BatchList bl,
                                                           const R *__restrict__ x, const R *__restrict__ q) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<R> &S = sys[bl.ids[e]];
    particle_map_body<R>(S.g, S.n, x + 3 * S.poff, q + S.poff, S.sb, blockIdx.x - bl.boff[e],
                         bl.boff[e + 1] - bl.boff[e]);
}
template <typename R>
__global__ void __launch_bounds__(MAP_THREADS) k_batch_scatter(const BatchSys<R> *__restrict__ sys, BatchList bl,
                                                               const R *__restrict__ x, const R *__restrict__ q) {
    const int e = batch_entry(bl.boff, bl.L, blockIdx.x);
    const BatchSys<R> &S = sys[bl.ids[e]];
    scatter_body<R>(S.g, S.n, x + 3 * S.poff, q + S.poff, S.sb, 0, blockIdx.x - bl.boff[e]);
}

template <typename R>
void launch_batch_sort(const BatchSys<R> *sys, const BatchList &all, const R *x, const R *q, cudaStream_t s) {
    if (all.nblocks == 0) return;
    k_batch_map<R><<<all.nblocks, MAP_THREADS, 0, s>>>(sys, all, x, q);
    k_batch_scatter<R><<<all.nblocks, MAP_THREADS, 0, s>>>(sys, all, x, q);
}
template void launch_batch_sort<float>(const BatchSys<float> *, const BatchList &, const float *, const float *,
                                       cudaStream_t);
template void launch_batch_sort<double>(const BatchSys<double> *, const BatchList &, const double *,
                                        const double *, cudaStream_t);

template <typename R>
void launch_sort(const Geom<R> &g, int64_t n, const R *x, const R *q, const SortBufs &b,
                 cudaStream_t s, R *rho_zero, int64_t mtot, R *x_copy, R *q_copy) {
    static_assert(MAP_THREADS == 256, "map_blocks counts blocks of 256 threads");
    const int nb = (int)((n + MAP_THREADS - 1) / MAP_THREADS);
    const int nbm = map_blocks(n);
    const int big = g.ntiles > SMALL_TILES;
    const int staged = (x_copy && q_copy) ? 1 : 0;
    if (!staged) x_copy = q_copy = nullptr;
    if (map_npt(n) == MAP_NPT_BIG)
        k_particle_map<R, MAP_NPT_BIG><<<nbm, MAP_THREADS, 0, s>>>(g, (int)n, x, q, b, rho_zero, mtot, x_copy,
                                                                   q_copy);
    else
        k_particle_map<R, 1><<<nbm, MAP_THREADS, 0, s>>>(g, (int)n, x, q, b, rho_zero, mtot, x_copy, q_copy);
    if (big) launch_pdl(k_tile_scan, dim3(1), dim3(SCAN_THREADS), 0, s, (const int *)b.tile_count, b.tile_start,
                        g.ntiles);
    launch_pdl(k_scatter<R>, dim3(nb), dim3(MAP_THREADS), 0, s, g, (int)n, staged ? (const R *)x_copy : x,
               staged ? (const R *)q_copy : q, b, big, staged);
}

template void launch_sort<float>(const Geom<float> &, int64_t, const float *, const float *,
                                 const SortBufs &, cudaStream_t, float *, int64_t, float *, float *);
template void launch_sort<double>(const Geom<double> &, int64_t, const double *, const double *,
                                  const SortBufs &, cudaStream_t, double *, int64_t, double *, double *);

}  // namespace pppm
