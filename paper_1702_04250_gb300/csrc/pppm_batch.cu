// Batched k-space path: many independent systems (uneven particle counts,
// meshes and orders) advanced together, one launch per stage for all of
// them, the whole step captured as one CUDA graph.
//
// Each stage runs the single-system kernel bodies (Sec. 3.1 Map-Charge and
// Distribute-Force, Sec. 3.2 Poisson solve) on a list of systems: CTAs of all
// systems are laid out back to back and every CTA finds its system by binary
// search.  Stages templated on the order P run once per order present.  The
// 3-D FFTs run as one batched cuFFT transform per mesh-size class and
// direction (systems with the same mesh are stored contiguously; the ik
// inverse batches the three field components of every system).  The energy/virial sums run on
// a forked stream beside the inverse FFTs and fieldforce.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <vector>

#include "pppm_common.cuh"

using namespace pppm;

namespace {

constexpr int BATCH_SMALL_TILES = 4096;  // per system (the in-block scan of the sort)

struct MeshClass {
    int M[3];
    std::vector<int> members;  // system ids, in slot order
    int64_t Mtot = 0, Mhalf = 0;
    int64_t Mpad = 0;          // ik field plane stride: Mtot rounded up to 256 bytes
    void *rho = nullptr, *rho_hat = nullptr, *spec = nullptr, *field = nullptr, *Gs = nullptr;
    cufftHandle r2c = 0, c2r = 0;
    bool have_r2c = false, have_c2r = false;
};

__global__ void k_scale_copy(const double *__restrict__ G, float *__restrict__ out32, double *__restrict__ out64,
                             int64_t n, double s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = G[i] * s;
        if (out32) out32[i] = (float)v;
        if (out64) out64[i] = v;
    }
}

}  // namespace

struct pppm_batch {
    int nsys = 0;
    bool fp64 = false, comp = false, ik = true;
    int prec = 0, mode = 0;
    double C = 0;
    int64_t ntot = 0;
    cudaStream_t stream = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // parallel branches for independent launches (one per mesh class or
    // order): up to kLanes streams, forked from and joined back to `stream`
    static constexpr int kLanes = 8;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_done;
    cudaEvent_t fan = nullptr;
    void *d_sys = nullptr;              // BatchSys<R>[nsys]
    int *d_lists = nullptr;
    BatchList map_list{}, green_list{};
    BatchList rho_list[MAXP + 1] = {}, rho_pair_list[MAXP + 1] = {}, ff_list[MAXP + 1] = {},
              ff_tile_list[MAXP + 1] = {};
    std::vector<MeshClass> classes;
    int *err = nullptr;
    bool graph_on = false;
    cudaGraphExec_t gexec = nullptr;
    const void *gkey[4] = {nullptr, nullptr, nullptr, nullptr};
    // bit P: FP32C make_rho of order P in four brick copies; bit 8 + P:
    // tile-staged fieldforce for order P; bit 16 + P: make_rho of order P over
    // z-pairs of tiles (the default for every order: 256 systems of 16^3 -
    // 64^3 meshes, FP32C, 1.36 -> 1.24 ms a call)
    int variants = 0xFC0000;
    std::vector<void *> allocs;
};

namespace {

int bmalloc(pppm_batch *b, void **ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return PPPM_ENOMEM;
    }
    b->allocs.push_back(*ptr);
    return PPPM_OK;
}

void batch_release(pppm_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto &c : b->classes) {
        if (c.have_r2c) cufftDestroy(c.r2c);
        if (c.have_c2r) cufftDestroy(c.c2r);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->fan) cudaEventDestroy(b->fan);
    for (auto e : b->lane_done) cudaEventDestroy(e);
    for (auto st : b->lanes) cudaStreamDestroy(st);
    for (void *v : b->allocs) cudaFree(v);
    delete b;
}

template <typename R>
void fill_geom_b(Geom<R> &g, const double box[3], const int M[3], int P, bool comp) {
    double coef[MAXP][MAXP], dcoef[MAXP][MAXP];
    stencil_polynomials(P, coef, dcoef);
    double vcell = 1.0;
    for (int d = 0; d < 3; ++d) {
        const double ih = (double)M[d] / box[d];
        g.M[d] = M[d];
        g.L[d] = (R)box[d];
        g.iL[d] = (R)(1.0 / box[d]);
        g.ih[d] = (R)ih;
        g.ih_lo[d] = (R)(ih - (double)(R)ih);
        g.h[d] = (R)(box[d] / M[d]);
        vcell *= box[d] / M[d];
    }
    tile_shape(M, long_tiles_allowed(P, comp), g.T, g.TE);
    g.Mzh = M[2] / 2 + 1;
    g.ntiles = g.T[0] * g.T[1] * g.T[2];
    g.P = P;
    g.rlo = (P - 1) / 2;
    g.ivcell = (R)(1.0 / vcell);
    g.ff_tiled = 0;
    g.rho_copies = 0;
    g.lut_bins = 0;
    g.launch_flags = 0;
    g.planar_stride = 0;
    for (int k = 0; k < MAXP; ++k)
        for (int l = 0; l < MAXP; ++l) {
            g.coef[k][l] = (R)coef[k][l];
            g.dcoef[k][l] = (R)dcoef[k][l];
        }
    const double wm = stencil_weight_max(P, coef);
    g.wmax3 = (float)(wm * wm * wm * (1.0 + 1e-6));
}

// Builds every per-system descriptor, the mesh classes and the launch lists.
template <typename R>
int batch_build(pppm_batch *b, const double *box, const int64_t *n, const int *order, const int *mesh,
                const double *gew) {
    const int ns = b->nsys;
    const size_t rs = sizeof(R);
    std::vector<BatchSys<R>> hs(ns);
    // mesh classes (systems with the same mesh share batched transforms)
    std::map<std::vector<int>, int> cls_of;
    std::vector<int> cls(ns), slot(ns);
    for (int s = 0; s < ns; ++s) {
        std::vector<int> key = {mesh[3 * s], mesh[3 * s + 1], mesh[3 * s + 2]};
        auto it = cls_of.find(key);
        if (it == cls_of.end()) {
            MeshClass mc;
            for (int d = 0; d < 3; ++d) mc.M[d] = key[d];
            mc.Mtot = (int64_t)key[0] * key[1] * key[2];
            mc.Mhalf = (int64_t)key[0] * key[1] * (key[2] / 2 + 1);
            mc.Mpad = (mc.Mtot + 63) / 64 * 64;
            it = cls_of.emplace(key, (int)b->classes.size()).first;
            b->classes.push_back(mc);
        }
        cls[s] = it->second;
        slot[s] = (int)b->classes[cls[s]].members.size();
        b->classes[cls[s]].members.push_back(s);
    }
    int rc;
    for (auto &mc : b->classes) {
        const size_t k = mc.members.size();
        if ((rc = bmalloc(b, &mc.rho, rs * mc.Mtot * k))) return rc;
        if ((rc = bmalloc(b, &mc.rho_hat, 2 * rs * mc.Mhalf * k))) return rc;
        if ((rc = bmalloc(b, &mc.spec, 2 * rs * mc.Mhalf * k * (b->ik ? 3 : 1)))) return rc;
        if ((rc = bmalloc(b, &mc.field, rs * (b->ik ? 3 * mc.Mpad : mc.Mtot) * k))) return rc;
        if ((rc = bmalloc(b, &mc.Gs, rs * mc.Mhalf * k))) return rc;
    }
    // per-system sort/green buffers in one arena each
    int64_t poff = 0;
    std::vector<double> ktab, kdiff;
    double *G64 = nullptr;
    int64_t maxhalf = 0;
    for (auto &mc : b->classes) maxhalf = std::max(maxhalf, mc.Mhalf);
    if ((rc = bmalloc(b, (void **)&G64, sizeof(double) * maxhalf))) return rc;
    for (int s = 0; s < ns; ++s) {
        BatchSys<R> &S = hs[s];
        const int *M = mesh + 3 * s;
        const double *bx = box + 3 * s;
        fill_geom_b<R>(S.g, bx, M, order[s], b->comp);
        if (S.g.ntiles > BATCH_SMALL_TILES) return PPPM_EINVAL;
        S.n = (int)n[s];
        S.poff = poff;
        poff += n[s];
        S.map_nb = (int)((n[s] + 255) / 256);
        // the flat green: eight spectrum elements a thread (256 a CTA) before
        // the CTA's energy/virial reduction
        const int64_t half = (int64_t)M[0] * M[1] * (M[2] / 2 + 1);
        S.green_nb = (int)std::min<int64_t>(std::max<int64_t>((half + 2047) / 2048, 1), 152 * 8);
        const int64_t nn = std::max<int64_t>(n[s], 1);
        void *p;
        if ((rc = bmalloc(b, &p, 4 * nn))) return rc;
        S.sb.anchor = (uint32_t *)p;
        if ((rc = bmalloc(b, &p, 4 * nn))) return rc;
        S.sb.rank = (int *)p;
        if ((rc = bmalloc(b, &p, 4 * (size_t)S.g.ntiles))) return rc;
        S.sb.tile_count = (int *)p;
        cudaMemset(p, 0, 4 * (size_t)S.g.ntiles);
        if ((rc = bmalloc(b, &p, 4 * ((size_t)S.g.ntiles + 1)))) return rc;
        S.sb.tile_start = (int *)p;
        if ((rc = bmalloc(b, &p, 4 * nn))) return rc;
        S.sb.perm = (int *)p;
        if ((rc = bmalloc(b, &p, 4 * rs * nn))) return rc;
        S.sb.rec = p;
        if ((rc = bmalloc(b, &p, 4 * nn))) return rc;
        S.sb.cell = (uint32_t *)p;
        if ((rc = bmalloc(b, &p, sizeof(double) * 2 * std::max(S.map_nb, 1)))) return rc;
        S.sb.blk = (double *)p;
        if ((rc = bmalloc(b, &p, 64))) return rc;  // (16 bytes unused) | qsum | ev
        S.sb.qsum = (double *)((char *)p + 16);
        S.sb.err = b->err;
        // mesh slices
        const MeshClass &mc = b->classes[cls[s]];
        const int sl = slot[s];
        S.rho = (R *)mc.rho + (size_t)sl * mc.Mtot;
        S.rho_hat = (char *)mc.rho_hat + 2 * rs * mc.Mhalf * sl;
        S.spec = (char *)mc.spec + 2 * rs * mc.Mhalf * sl * (b->ik ? 3 : 1);
        S.field = (R *)mc.field + (size_t)sl * (b->ik ? 3 * mc.Mpad : mc.Mtot);
        S.g.planar_stride = b->ik ? (int)mc.Mpad : 0;
        // influence function and self-force coefficients (FP64, then G/M in R)
        double h[3] = {bx[0] / M[0], bx[1] / M[1], bx[2] / M[2]};
        const double V = bx[0] * bx[1] * bx[2];
        if ((rc = green_setup_fp64(M, h, V, order[s], b->ik, gew[s], b->C, G64, S.sf, ktab, kdiff, b->stream)))
            return rc;
        R *Gs = (R *)mc.Gs + (size_t)sl * mc.Mhalf;
        k_scale_copy<<<128, 256, 0, b->stream>>>(G64, b->fp64 ? nullptr : (float *)Gs,
                                                  b->fp64 ? (double *)Gs : nullptr, mc.Mhalf, 1.0 / (double)mc.Mtot);
        const int len = M[0] + M[1] + M[2] / 2 + 1;
        std::vector<R> kv(len), kd(len);
        for (int i = 0; i < len; ++i) {
            kv[i] = (R)ktab[i];
            kd[i] = (R)kdiff[i];
        }
        if ((rc = bmalloc(b, &p, 2 * rs * len))) return rc;
        if (cudaMemcpyAsync(p, kv.data(), rs * len, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
            cudaMemcpyAsync((char *)p + rs * len, kd.data(), rs * len, cudaMemcpyHostToDevice, b->stream) !=
                cudaSuccess)
            return PPPM_ECUDA;
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return PPPM_ECUDA;
        S.gb.G64 = nullptr;
        S.gb.Gs = Gs;
        S.gb.kvec = p;
        S.gb.kdiff = (char *)p + rs * len;
        if ((rc = bmalloc(b, &p, sizeof(double) * (7 * S.green_nb + 8)))) return rc;
        S.gb.part = (double *)p;
        S.gb.ev = (double *)p + 7 * S.green_nb;
        S.gb.qsum = S.sb.qsum;
        S.gb.map_part = S.sb.blk;
        S.ec.epref = 0.5 * b->C * (h[0] * h[1] * h[2]) * (h[0] * h[1] * h[2]) / V * (double)mc.Mtot;
        S.ec.inv4g2 = 1.0 / (4.0 * gew[s] * gew[s]);
        S.ec.eself = -b->C * gew[s] / std::sqrt(M_PI);
        S.ec.ebg = -b->C * M_PI / (2.0 * gew[s] * gew[s] * V);
    }
    b->ntot = poff;
    if ((rc = bmalloc(b, &b->d_sys, sizeof(BatchSys<R>) * ns))) return rc;
    if (cudaMemcpy(b->d_sys, hs.data(), sizeof(BatchSys<R>) * ns, cudaMemcpyHostToDevice) != cudaSuccess)
        return PPPM_ECUDA;

    // launch lists: ids + CTA offsets, all in one device array
    std::vector<int> host;
    auto add_list = [&](BatchList &bl, const std::vector<int> &ids, auto ctas) {
        bl.L = (int)ids.size();
        const int at = (int)host.size();
        for (int id : ids) host.push_back(id);
        int acc = 0;
        for (int id : ids) {
            host.push_back(acc);
            acc += ctas(id);
        }
        host.push_back(acc);
        bl.nblocks = acc;
        return at;  // ids at [at, at+L), boff at [at+L, at+2L+1)
    };
    std::vector<int> live;
    for (int s = 0; s < ns; ++s)
        if (n[s] > 0) live.push_back(s);
    std::vector<int> all(ns);
    for (int s = 0; s < ns; ++s) all[s] = s;
    struct Pending {
        BatchList *bl;
        int at;
    };
    std::vector<Pending> pend;
    pend.push_back({&b->map_list, add_list(b->map_list, live, [&](int s) { return hs[s].map_nb; })});
    pend.push_back({&b->green_list, add_list(b->green_list, all, [&](int s) { return hs[s].green_nb; })});
    for (int P = 2; P <= MAXP; ++P) {
        std::vector<int> ids;
        for (int s : live)
            if (order[s] == P) ids.push_back(s);
        if (ids.empty()) continue;
        pend.push_back({&b->rho_list[P], add_list(b->rho_list[P], ids, [&](int s) { return hs[s].g.ntiles; })});
        pend.push_back({&b->rho_pair_list[P], add_list(b->rho_pair_list[P], ids, [&](int s) {
                           const Geom<R> &g = hs[s].g;
                           return g.T[0] * g.T[1] * ((g.T[2] + 1) / 2);
                       })});
        pend.push_back({&b->ff_list[P], add_list(b->ff_list[P], ids, [&](int s) {
                           return (hs[s].n + ff_particles_per_cta(P) - 1) / ff_particles_per_cta(P);
                       })});
        pend.push_back({&b->ff_tile_list[P], add_list(b->ff_tile_list[P], ids, [&](int s) { return hs[s].g.ntiles; })});
    }
    if ((rc = bmalloc(b, (void **)&b->d_lists, sizeof(int) * std::max<size_t>(host.size(), 1)))) return rc;
    if (!host.empty() &&
        cudaMemcpy(b->d_lists, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return PPPM_ECUDA;
    for (auto &pd : pend) {
        pd.bl->ids = b->d_lists + pd.at;
        pd.bl->boff = b->d_lists + pd.at + pd.bl->L;
    }

    // batched transforms per mesh class
    const cufftType tr2c = b->fp64 ? CUFFT_D2Z : CUFFT_R2C;
    const cufftType tc2r = b->fp64 ? CUFFT_Z2D : CUFFT_C2R;
    for (auto &mc : b->classes) {
        const int k = (int)mc.members.size();
        int nn[3] = {mc.M[0], mc.M[1], mc.M[2]};
        int inemb[3] = {mc.M[0], mc.M[1], mc.M[2]};
        int hemb[3] = {mc.M[0], mc.M[1], mc.M[2] / 2 + 1};
        if (cufftPlanMany(&mc.r2c, 3, nn, inemb, 1, (int)mc.Mtot, hemb, 1, (int)mc.Mhalf, tr2c, k) != CUFFT_SUCCESS)
            return PPPM_ECUFFT;
        mc.have_r2c = true;
        cufftResult r;
        if (b->ik)  // the 3 components of every system as one batch: spectra [sys][3][Mhalf] in,
                    // padded planes [sys][3][Mpad] out
            r = cufftPlanMany(&mc.c2r, 3, nn, hemb, 1, (int)mc.Mhalf, inemb, 1, (int)mc.Mpad, tc2r, 3 * k);
        else
            r = cufftPlanMany(&mc.c2r, 3, nn, hemb, 1, (int)mc.Mhalf, inemb, 1, (int)mc.Mtot, tc2r, k);
        if (r != CUFFT_SUCCESS) return PPPM_ECUFFT;
        mc.have_c2r = true;
        if (cufftSetStream(mc.r2c, b->stream) != CUFFT_SUCCESS || cufftSetStream(mc.c2r, b->stream) != CUFFT_SUCCESS)
            return PPPM_ECUFFT;
    }
    return PPPM_OK;
}

// Fork the lanes off `s` / join them back (graph branches under capture).
bool fan_out(pppm_batch *b, cudaStream_t s) {
    if (cudaEventRecord(b->fan, s) != cudaSuccess) return false;
    for (auto st : b->lanes)
        if (cudaStreamWaitEvent(st, b->fan, 0) != cudaSuccess) return false;
    return true;
}
bool fan_in(pppm_batch *b, cudaStream_t s) {
    for (size_t i = 0; i < b->lanes.size(); ++i)
        if (cudaEventRecord(b->lane_done[i], b->lanes[i]) != cudaSuccess ||
            cudaStreamWaitEvent(s, b->lane_done[i], 0) != cudaSuccess)
            return false;
    return true;
}

template <typename R>
int batch_enqueue(pppm_batch *b, const R *x, const R *q, R *f, double *ev) {
    cudaStream_t s = b->stream;
    const auto *sys = reinterpret_cast<const BatchSys<R> *>(b->d_sys);
    const size_t rs = sizeof(R);
    const int nl = (int)b->lanes.size();
    for (auto &mc : b->classes)
        if (cudaMemsetAsync(mc.rho, 0, rs * mc.Mtot * mc.members.size(), s) != cudaSuccess) return PPPM_ECUDA;
    launch_batch_sort<R>(sys, b->map_list, x, q, s);
    // make_rho per order, then each class's forward transform: independent
    // systems and meshes, one branch each
    if (!fan_out(b, s)) return PPPM_ECUDA;
    for (int P = 2; P <= MAXP; ++P) {
        const bool pairs = ((b->variants >> (16 + P)) & 1) != 0;
        launch_batch_make_rho<R>(sys, pairs ? b->rho_pair_list[P] : b->rho_list[P], P, b->comp,
                                 ((b->variants >> P) & 1) != 0, pairs, b->lanes[P % nl]);
    }
    if (!fan_in(b, s) || !fan_out(b, s)) return PPPM_ECUDA;
    for (size_t i = 0; i < b->classes.size(); ++i) {
        auto &mc = b->classes[i];
        if (cufftSetStream(mc.r2c, b->lanes[i % nl]) != CUFFT_SUCCESS) return PPPM_ECUFFT;
        cufftResult r = b->fp64 ? cufftExecD2Z(mc.r2c, (cufftDoubleReal *)mc.rho, (cufftDoubleComplex *)mc.rho_hat)
                                : cufftExecR2C(mc.r2c, (cufftReal *)mc.rho, (cufftComplex *)mc.rho_hat);
        if (r != CUFFT_SUCCESS) return PPPM_ECUFFT;
    }
    if (!fan_in(b, s)) return PPPM_ECUDA;
    launch_batch_green<R>(sys, b->green_list, b->ik, s);
    if (cudaEventRecord(b->fork, s) != cudaSuccess || cudaStreamWaitEvent(b->side, b->fork, 0) != cudaSuccess)
        return PPPM_ECUDA;
    launch_batch_energy_final<R>(sys, b->nsys, ev, b->side);
    if (cudaEventRecord(b->join, b->side) != cudaSuccess) return PPPM_ECUDA;
    if (!fan_out(b, s)) return PPPM_ECUDA;
    for (size_t i = 0; i < b->classes.size(); ++i) {
        auto &mc = b->classes[i];
        if (cufftSetStream(mc.c2r, b->lanes[i % nl]) != CUFFT_SUCCESS) return PPPM_ECUFFT;
        cufftResult r = b->fp64 ? cufftExecZ2D(mc.c2r, (cufftDoubleComplex *)mc.spec, (cufftDoubleReal *)mc.field)
                                : cufftExecC2R(mc.c2r, (cufftComplex *)mc.spec, (cufftReal *)mc.field);
        if (r != CUFFT_SUCCESS) return PPPM_ECUFFT;
    }
    if (!fan_in(b, s) || !fan_out(b, s)) return PPPM_ECUDA;
    for (int P = 2; P <= MAXP; ++P) {
        const bool tiled = ((b->variants >> (8 + P)) & 1) != 0;
        launch_batch_fieldforce<R>(sys, tiled ? b->ff_tile_list[P] : b->ff_list[P], P, b->ik, tiled, f, (R)b->C,
                                   b->lanes[P % nl]);
    }
    if (!fan_in(b, s)) return PPPM_ECUDA;
    if (cudaStreamWaitEvent(s, b->join, 0) != cudaSuccess) return PPPM_ECUDA;
    return cudaGetLastError() == cudaSuccess ? PPPM_OK : PPPM_ECUDA;
}

int batch_enqueue_any(pppm_batch *b, const void *x, const void *q, void *f, double *ev) {
    if (b->fp64) return batch_enqueue<double>(b, (const double *)x, (const double *)q, (double *)f, ev);
    return batch_enqueue<float>(b, (const float *)x, (const float *)q, (float *)f, ev);
}

}  // namespace

extern "C" {

int pppm_batch_setup(pppm_batch **out, int nsys, const double *box, const int64_t *n, const int *order,
                     const int *mesh, const double *g_ewald, int diff_mode, int precision, double qqrd2e,
                     void *cuda_stream) {
    if (!out) return PPPM_EINVAL;
    *out = nullptr;
    if (nsys <= 0 || !box || !n || !order || !mesh || !g_ewald) return PPPM_EINVAL;
    if (diff_mode != PPPM_IK && diff_mode != PPPM_AD) return PPPM_EINVAL;
    if (precision != PPPM_FP64 && precision != PPPM_FP32C && precision != PPPM_FP32) return PPPM_EINVAL;
    if (!std::isfinite(qqrd2e)) return PPPM_EINVAL;
    int64_t total = 0;
    for (int s = 0; s < nsys; ++s) {
        if (n[s] < 0 || order[s] < 2 || order[s] > MAXP || !(g_ewald[s] > 0)) return PPPM_EINVAL;
        for (int d = 0; d < 3; ++d) {
            if (!(box[3 * s + d] > 0) || !std::isfinite(box[3 * s + d])) return PPPM_EINVAL;
            if (mesh[3 * s + d] < order[s] || mesh[3 * s + d] > MAX_MESH) return PPPM_EINVAL;
        }
        const int nt = ((mesh[3 * s] + TILE_B - 1) / TILE_B) * ((mesh[3 * s + 1] + TILE_B - 1) / TILE_B) *
                       ((mesh[3 * s + 2] + TILE_B - 1) / TILE_B);
        if (nt > BATCH_SMALL_TILES) return PPPM_EINVAL;
        total += n[s];
    }
    if (total > ((int64_t)1 << 30)) return PPPM_EINVAL;
    pppm_batch *b = new (std::nothrow) pppm_batch();
    if (!b) return PPPM_ENOMEM;
    b->nsys = nsys;
    b->fp64 = precision == PPPM_FP64;
    b->comp = precision == PPPM_FP32C;
    b->ik = diff_mode == PPPM_IK;
    b->prec = precision;
    b->mode = diff_mode;
    b->C = qqrd2e;
    b->stream = (cudaStream_t)cuda_stream;
    int rc = PPPM_OK;
    if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fan, cudaEventDisableTiming) != cudaSuccess)
        rc = PPPM_ECUDA;
    for (int i = 0; i < pppm_batch::kLanes && !rc; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            rc = PPPM_ECUDA;
            break;
        }
        b->lanes.push_back(st);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            rc = PPPM_ECUDA;
            break;
        }
        b->lane_done.push_back(e);
    }
    if (!rc) rc = bmalloc(b, (void **)&b->err, 16);
    if (!rc && cudaMemset(b->err, 0, 16) != cudaSuccess) rc = PPPM_ECUDA;
    for (int P = 2; P <= MAXP && !rc; ++P) {
        bool used = false;
        for (int s = 0; s < nsys; ++s) used |= order[s] == P;
        if (!used) continue;
        cudaError_t e = b->fp64 ? prepare_make_rho<double>(P, false) : prepare_make_rho<float>(P, b->comp);
        if (e == cudaSuccess) e = b->fp64 ? prepare_fieldforce<double>(P) : prepare_fieldforce<float>(P);
        if (e != cudaSuccess) rc = PPPM_ECUDA;
    }
    if (!rc) rc = b->fp64 ? batch_build<double>(b, box, n, order, mesh, g_ewald)
                          : batch_build<float>(b, box, n, order, mesh, g_ewald);
    if (!rc && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = PPPM_ECUDA;
    if (rc) {
        batch_release(b);
        return rc;
    }
    *out = b;
    return PPPM_OK;
}

int pppm_batch_destroy(pppm_batch *b) {
    if (!b) return PPPM_EINVAL;
    batch_release(b);
    return PPPM_OK;
}

int pppm_batch_set_graph(pppm_batch *b, int enable) {
    if (!b) return PPPM_EINVAL;
    b->graph_on = enable != 0;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return PPPM_OK;
}

int pppm_batch_compute(pppm_batch *b, const void *x, const void *q, void *f, double *ev) {
    if (!b) return PPPM_EINVAL;
    if (b->ntot > 0 && (!x || !q || !f)) return PPPM_EINVAL;
    if (!b->graph_on) return batch_enqueue_any(b, x, q, f, ev);
    const void *key[4] = {x, q, f, ev};
    bool same = b->gexec != nullptr;
    for (int i = 0; i < 4 && same; ++i) same = key[i] == b->gkey[i];
    if (!same) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PPPM_ECUDA;
        const int rc = batch_enqueue_any(b, x, q, f, ev);
        const cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ee != cudaSuccess) return PPPM_ECUDA;
        const cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return PPPM_ECUDA;
        for (int i = 0; i < 4; ++i) b->gkey[i] = key[i];
    }
    return cudaGraphLaunch(b->gexec, b->stream) == cudaSuccess ? PPPM_OK : PPPM_ECUDA;
}

int pppm_batch_set_variant(pppm_batch *b, int variants) {
    if (!b || (variants & ~0xFCFCFC)) return PPPM_EINVAL;
    if ((variants & 0xFC) && !b->comp) return PPPM_EINVAL;  // the brick copies are the FP32C accumulator
    if (variants & (variants >> 16) & 0xFC) return PPPM_EINVAL;  // one make_rho brick layout per order
    b->variants = variants;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return PPPM_OK;
}

int pppm_batch_get_variant(const pppm_batch *b, int *variants) {
    if (!b || !variants) return PPPM_EINVAL;
    *variants = b->variants;
    return PPPM_OK;
}

constexpr int BATCH_TUNE_TIMED = 5;  // timed calls per setting, after one warm-up

int pppm_batch_autotune(pppm_batch *b, const void *x, const void *q, void *f, int *choice_out) {
    if (!b) return PPPM_EINVAL;
    if (b->ntot > 0 && (!x || !q || !f)) return PPPM_EINVAL;
    int best = b->variants;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PPPM_ECUDA;
    // each setting is timed the way the batch runs (one graph when graph mode
    // is on), scored by its fastest call
    auto time_calls = [&](int v, float &ms_out) -> int {
        const int rc0 = pppm_batch_set_variant(b, v);
        if (rc0) return rc0;
        float fastest = 1e30f;
        for (int it = 0; it < 1 + BATCH_TUNE_TIMED; ++it) {
            if (cudaEventRecord(e0, b->stream) != cudaSuccess) return PPPM_ECUDA;
            const int rc = pppm_batch_compute(b, x, q, f, nullptr);
            if (rc) return rc;
            if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return PPPM_ECUDA;
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return PPPM_ECUDA;
            if (it > 0) fastest = fminf(fastest, ms);
        }
        ms_out = fastest;
        return PPPM_OK;
    };
    float t_best = 0.0f;
    int rc = time_calls(best, t_best);
    // each order's make_rho and fieldforce are launches of their own: choose
    // each one's kernel on its own, flipping one bit at a time
    for (int P = 2; P <= MAXP && rc == PPPM_OK; ++P) {
        if (b->rho_list[P].nblocks == 0) continue;
        for (int bit : {16 + P, P, 8 + P}) {
            if (bit < 8 && !b->comp) continue;  // the brick copies are the FP32C accumulator
            const int v = best ^ (1 << bit);
            if (v & (v >> 16) & 0xFC) continue;  // tile pairs and brick copies exclude each other
            float t = 0.0f;
            rc = time_calls(v, t);
            if (rc) break;
            if (t < t_best) {
                t_best = t;
                best = v;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rs = pppm_batch_set_variant(b, best);
    if (rc) return rc;
    if (rs) return rs;
    // leave f holding the chosen setting's result
    if ((rc = pppm_batch_compute(b, x, q, f, nullptr))) return rc;
    if (choice_out) *choice_out = best;
    return PPPM_OK;
}

int pppm_batch_sync(pppm_batch *b) {
    if (!b) return PPPM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return PPPM_ECUDA;
    }
    if (err) {
        cudaMemset(b->err, 0, sizeof(int));
        return (err & ERR_INTERNAL) ? PPPM_EINTERNAL : PPPM_ENONFINITE;
    }
    return PPPM_OK;
}

int pppm_batch_info(const pppm_batch *b, int64_t info[4]) {
    if (!b || !info) return PPPM_EINVAL;
    info[0] = b->nsys;
    info[1] = b->ntot;
    info[2] = (int64_t)b->classes.size();
    int orders = 0;
    for (int P = 2; P <= MAXP; ++P) orders += b->rho_list[P].L > 0;
    info[3] = orders;
    return PPPM_OK;
}

}  // extern "C"
