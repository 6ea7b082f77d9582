// C-ABI layer: plan set-up (Sec. 2.1/2.3 parameters: order, mesh, g_ewald,
// differentiation mode), per-step enqueue of the three PPPM steps, CUDA-graph
// capture of a whole step, the host-buffer variant, and read-back of internal
// arrays for stage-by-stage checking.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "pppm_common.cuh"

namespace pppm {
static thread_local cudaError_t last_cuda_err = cudaSuccess;
static thread_local const char *last_cuda_stage = nullptr;
void note_cuda_error(cudaError_t e) {
    if (e != cudaSuccess) last_cuda_err = e;
}
// PPPM_SYNC_CHECK=1 in the environment: synchronise after every stage of a
// step and name the stage that saw a CUDA error (diagnosis; slow).
static bool sync_check_on() {
    static const bool on = [] {
        const char *v = std::getenv("PPPM_SYNC_CHECK");
        return v && v[0] == '1';
    }();
    return on;
}
}  // namespace pppm

using namespace pppm;

struct pppm_plan {
    int device = 0;
    cudaStream_t stream = nullptr;
    int P = 0, mode = 0, prec = 0;
    bool fp64 = false, comp = false, ik = true;
    int M[3] = {0, 0, 0}, Mzh = 0;
    int64_t Mtot = 0, Mhalf = 0;
    int T[3] = {0, 0, 0}, TE[3] = {0, 0, 0}, ntiles = 0;
    int ntiles_alloc = 0;              // tile arrays are sized for 4^3 tiles, the most numerous shape
    double box[3] = {0, 0, 0}, h[3] = {0, 0, 0}, g = 0, C = 0, V = 0, vcell = 0;
    int64_t n_max = 0, n_last = -1;
    Geom<float> gf{};
    Geom<double> gd{};
    SortBufs sb{};
    GreenBufs gb{};
    EnergyConsts ec{};
    void *rho = nullptr, *rho_hat = nullptr, *spec = nullptr, *field = nullptr;
    double *G64 = nullptr;
    void *Gs = nullptr, *kvec = nullptr, *kdiff = nullptr;
    double *green_part = nullptr;
    double *ev = nullptr;              // [8]
    double *d_sf = nullptr;            // [6] setup sums
    double sf[6] = {0, 0, 0, 0, 0, 0};
    cufftHandle r2c = 0, c2r = 0, c2r1 = 0;
    bool have_r2c = false, have_c2r = false, have_c2r1 = false;
    bool field_is_field = false, have_rho = false;
    void *hx = nullptr, *hq = nullptr, *hf = nullptr;  // device staging for the host path
    bool stage_in = false;  // this call's particle_map copies x, q (read over the link) into hx, hq
    double *hev = nullptr;
    int *h_err = nullptr;              // pinned host copy of the device error word (host path)
    cudaStream_t side = nullptr;       // energy/virial reduction branch
    cudaEvent_t fork = nullptr, join = nullptr;
    int prof_mask = 0, prof_valid = 0;  // stages timed; stages timed by the last call
    cudaEvent_t prof[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool graph_on = false;
    // instantiated step graphs, one per (n, pointers, profiled stages): a
    // caller that profiles every k-th step alternates between two of them
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const void *key[4] = {nullptr, nullptr, nullptr, nullptr};
        int64_t n = -1;
        int prof = 0;
        bool stage = false;
        uint64_t used = 0;
    };
    static constexpr int kGraphSlots = 4;
    GraphSlot graphs[kGraphSlots];
    uint64_t graph_clock = 0;
    int variants = 0;  // bit 0: tile-staged fieldforce, 1: long tiles along z, 2: four-copy
                       // make_rho brick, 3: hand-written Poisson solve (k_fft.cu)
    bool fft_own = false;  // the plan's mesh and precision admit variant bit 3
    std::vector<void *> allocs;
};

namespace {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PPPM_OK;
    note_cuda_error(e);
    if (e == cudaErrorMemoryAllocation) return PPPM_ENOMEM;
    return PPPM_ECUDA;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

#define CKF(call)                                  \
    do {                                           \
        cufftResult r_ = (call);                   \
        if (r_ != CUFFT_SUCCESS) return PPPM_ECUFFT; \
    } while (0)

template <typename T>
int dmalloc(pppm_plan *p, T **ptr, size_t bytes) {
    void *v = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PPPM_ENOMEM;
    }
    p->allocs.push_back(v);
    *ptr = reinterpret_cast<T *>(v);
    return PPPM_OK;
}

__global__ void k_scale_green(const double *__restrict__ G, float *__restrict__ out32,
                              double *__restrict__ out64, int64_t n, double s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = G[i] * s;
        if (out32) out32[i] = (float)v;
        if (out64) out64[i] = v;
    }
}

template <typename R>
void fill_geom(pppm_plan *p, Geom<R> &g, const double coef[MAXP][MAXP], const double dcoef[MAXP][MAXP]) {
    for (int d = 0; d < 3; ++d) {
        g.M[d] = p->M[d];
        g.T[d] = p->T[d];
        g.TE[d] = p->TE[d];
        g.L[d] = (R)p->box[d];
        g.iL[d] = (R)(1.0 / p->box[d]);
        const double ih = (double)p->M[d] / p->box[d];
        g.ih[d] = (R)ih;
        g.ih_lo[d] = (R)(ih - (double)(R)ih);
        g.h[d] = (R)p->h[d];
    }
    g.Mzh = p->Mzh;
    g.ntiles = p->ntiles;
    g.P = p->P;
    g.rlo = (p->P - 1) / 2;
    g.ivcell = (R)(1.0 / p->vcell);
    for (int k = 0; k < MAXP; ++k)
        for (int l = 0; l < MAXP; ++l) {
            g.coef[k][l] = (R)coef[k][l];
            g.dcoef[k][l] = (R)dcoef[k][l];
        }
    const double wm = stencil_weight_max(p->P, coef);
    g.wmax3 = (float)(wm * wm * wm * (1.0 + 1e-6));
}

void release(pppm_plan *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    for (auto &g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (p->h_err) cudaFreeHost(p->h_err);
    for (auto &e : p->prof)
        if (e) cudaEventDestroy(e);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->have_r2c) cufftDestroy(p->r2c);
    if (p->have_c2r) cufftDestroy(p->c2r);
    if (p->have_c2r1) cufftDestroy(p->c2r1);
    for (void *v : p->allocs) cudaFree(v);
    delete p;
}

}  // namespace

namespace pppm {

// Per-dimension wavenumber and alias tables over (Mx, My, Mz/2 + 1), laid out
// [x | y | z]: ktab = k (Nyquist negative), kdiff = k with the Nyquist entry
// zeroed, atab[m + 2] = exp(-k_m^2/4g^2) U1^2(k_m) for aliases |m| <= 2,
// dtab = the full alias sum of U1^2 (a finite cosine series), and on request
// btab[n] (ad self-force sums) and etab[m + 2] = exp(-k_m^2/2g^2).
void alias_tables(const int M[3], const double h[3], int P, double g, std::vector<double> &ktab,
                  std::vector<double> &kdiff, std::vector<double> &atab, std::vector<double> &dtab,
                  std::vector<double> *btab, std::vector<double> *etab) {
    const int Mx = M[0], My = M[1], Mzh = M[2] / 2 + 1;
    const int len = Mx + My + Mzh;
    const int dimlen[3] = {Mx, My, Mzh};
    const int off[3] = {0, Mx, Mx + My};
    ktab.assign(len, 0.0);
    kdiff.assign(len, 0.0);
    atab.assign(5 * (size_t)len, 0.0);
    dtab.assign(len, 0.0);
    if (btab) btab->assign(3 * (size_t)len, 0.0);
    if (etab) etab->assign(5 * (size_t)len, 0.0);
    double m2p[MAXP + 1];
    spline2p_at_integers(P, m2p);
    for (int d = 0; d < 3; ++d) {
        for (int i = 0; i < dimlen[d]; ++i) {
            const double kappa = grid_kappa(i, M[d]);  // k h
            const double k = kappa / h[d];
            ktab[off[d] + i] = k;
            kdiff[off[d] + i] = (2 * i == M[d]) ? 0.0 : k;  // Nyquist derivative dropped
            for (int m = -2; m <= 2; ++m) {
                const double km = k + 2.0 * M_PI * m / h[d];
                const double u = alias_cross(kappa + 2.0 * M_PI * m, 0, P, 0);  // U1^2 at this alias
                atab[(size_t)(m + 2) * len + off[d] + i] = std::exp(-km * km / (4.0 * g * g)) * u;
                if (etab) (*etab)[(size_t)(m + 2) * len + off[d] + i] = std::exp(-km * km / (2.0 * g * g));
            }
            double D = m2p[0];
            for (int gg = 1; gg < P; ++gg) D += 2.0 * m2p[gg] * std::cos(kappa * gg);
            dtab[off[d] + i] = D;
            if (btab)
                for (int n = 0; n <= 2; ++n) (*btab)[(size_t)n * len + off[d] + i] = alias_cross(kappa, n, P, 50);
        }
    }
}

// FP64 influence function and ad self-force coefficients of one system
// (used by single plans and by batches).  Temporary device tables are
// allocated and freed here; G64 must hold Mx*My*(Mz/2+1) doubles.
int green_setup_fp64(const int M[3], const double h[3], double V, int P, bool ik, double g, double C,
                     double *G64, double sf_out[6], std::vector<double> &ktab, std::vector<double> &kdiff,
                     cudaStream_t stream) {
    const int Mzh = M[2] / 2 + 1;
    const int len = M[0] + M[1] + Mzh;
    std::vector<double> atab, dtab, btab;
    alias_tables(M, h, P, g, ktab, kdiff, atab, dtab, &btab, nullptr);
    double *tmp = nullptr;  // ktab | atab | dtab | btab | sf sums
    const size_t words = (size_t)len * 10 + 6;
    if (cudaMalloc(&tmp, words * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return PPPM_ENOMEM;
    }
    double *d_ktab = tmp, *d_atab = tmp + len, *d_dtab = d_atab + 5 * (size_t)len, *d_btab = d_dtab + len;
    double *d_sf = d_btab + 3 * (size_t)len;
    int rc = PPPM_OK;
    double sums[6] = {0, 0, 0, 0, 0, 0};
    do {
        if (cudaMemcpy(d_ktab, ktab.data(), sizeof(double) * len, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_atab, atab.data(), sizeof(double) * 5 * len, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_dtab, dtab.data(), sizeof(double) * len, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_btab, btab.data(), sizeof(double) * 3 * len, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = PPPM_ECUDA;
            break;
        }
        GreenSetup gs{};
        for (int d = 0; d < 3; ++d) {
            gs.M[d] = M[d];
            gs.h[d] = h[d];
        }
        gs.Mzh = Mzh;
        gs.P = P;
        gs.ik = ik;
        gs.g = g;
        gs.ktab = d_ktab;
        gs.atab = d_atab;
        gs.dtab = d_dtab;
        gs.btab = d_btab;
        launch_green_setup(gs, G64, d_sf, stream);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(sums, d_sf, sizeof(sums), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            rc = PPPM_ECUDA;
    } while (0);
    cudaFree(tmp);
    if (rc) return rc;
    for (int a = 0; a < 3; ++a)
        for (int n = 1; n <= 2; ++n) sf_out[a * 2 + n - 1] = 2.0 * M_PI * n * C / (h[a] * V) * sums[a * 2 + n - 1];
    return PPPM_OK;
}

// Smallest FFT-friendly edge >= n: kind 0 n itself, 1 prime factors 2, 3, 5, 7,
// 2 a power of two.  -1 for n < 1 or an unknown kind.
int fft_size_host(int n, int kind) {
    if (n < 1 || kind < 0 || kind > 2) return -1;
    if (kind == 0) return n;
    for (int m = n;; ++m) {
        int r = m;
        while (r % 2 == 0) r /= 2;
        if (kind == 1) {
            while (r % 3 == 0) r /= 3;
            while (r % 5 == 0) r /= 5;
            while (r % 7 == 0) r /= 7;
        }
        if (r == 1) return m;
    }
}

// Full alias sum of U1^2(k_m) k_m^2 per dimension (|m| <= 2000), laid out as
// ktab: the ad error functional's S2 factors.
void alias_s2_table(const int M[3], const double h[3], int P, std::vector<double> &s2tab) {
    const int Mzh = M[2] / 2 + 1;
    const int dimlen[3] = {M[0], M[1], Mzh};
    const int off[3] = {0, M[0], M[0] + M[1]};
    s2tab.assign((size_t)M[0] + M[1] + Mzh, 0.0);
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i < dimlen[d]; ++i) {
            const double kappa = grid_kappa(i, M[d]);
            double s = 0.0;
            for (int m = -2000; m <= 2000; ++m) {
                const double km = (kappa + 2.0 * M_PI * m) / h[d];
                s += alias_cross(kappa + 2.0 * M_PI * m, 0, P, 0) * km * km;
            }
            s2tab[off[d] + i] = s;
        }
}

// RMS k-space force error of an ik (ad = false) or ad mesh for n random
// charges with sum q^2 = q2 (units C e^2 / A^2): q2 sqrt(Q / (n V)), Q the
// Hockney-Eastwood functional of k_kspace_error divided by V.  Synchronous,
// on the calling thread's default stream.
int kspace_error_mesh(const int M[3], const double box[3], int P, double g, bool ad, int64_t n, double q2,
                      double *err) {
    double h[3];
    for (int d = 0; d < 3; ++d) h[d] = box[d] / M[d];
    const double V = box[0] * box[1] * box[2];
    const int Mzh = M[2] / 2 + 1;
    const int len = M[0] + M[1] + Mzh;
    std::vector<double> ktab, kdiff, atab, dtab, etab, s2tab;
    alias_tables(M, h, P, g, ktab, kdiff, atab, dtab, nullptr, &etab);
    if (ad) alias_s2_table(M, h, P, s2tab);
    else s2tab.assign(len, 0.0);
    double *tmp = nullptr;  // ktab | atab | dtab | etab | s2tab | partials
    const size_t words = (size_t)len * 13 + KERR_MAX_BLOCKS;
    if (cudaMalloc(&tmp, words * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return PPPM_ENOMEM;
    }
    double *d_ktab = tmp, *d_atab = tmp + len, *d_dtab = d_atab + 5 * (size_t)len, *d_etab = d_dtab + len;
    double *d_s2tab = d_etab + 5 * (size_t)len;
    double *d_part = d_s2tab + len;
    std::vector<double> part(KERR_MAX_BLOCKS, 0.0);
    int rc = PPPM_OK, nb = 0;
    do {
        if (cudaMemcpy(d_ktab, ktab.data(), sizeof(double) * len, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_atab, atab.data(), sizeof(double) * 5 * len, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_dtab, dtab.data(), sizeof(double) * len, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_etab, etab.data(), sizeof(double) * 5 * len, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_s2tab, s2tab.data(), sizeof(double) * len, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = PPPM_ECUDA;
            break;
        }
        KErrSetup ks{};
        for (int d = 0; d < 3; ++d) {
            ks.M[d] = M[d];
            ks.h[d] = h[d];
        }
        ks.Mzh = Mzh;
        ks.ktab = d_ktab;
        ks.atab = d_atab;
        ks.dtab = d_dtab;
        ks.etab = d_etab;
        ks.s2tab = d_s2tab;
        ks.ad = ad ? 1 : 0;
        nb = launch_kspace_error(ks, d_part, 0);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(part.data(), d_part, sizeof(double) * nb, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = PPPM_ECUDA;
    } while (0);
    cudaFree(tmp);
    if (rc) return rc;
    double sum = 0.0;
    for (int b = 0; b < nb; ++b) sum += part[b];  // fixed order
    const double Q = sum / V;
    *err = q2 * std::sqrt(std::max(Q, 0.0) / ((double)n * V));
    return PPPM_OK;
}

}  // namespace pppm

namespace {

int build_tables_and_green(pppm_plan *p) {
    const int len = p->M[0] + p->M[1] + p->Mzh;
    std::vector<double> ktab, kdiff;
    int rc = green_setup_fp64(p->M, p->h, p->V, p->P, p->ik, p->g, p->C, p->G64, p->sf, ktab, kdiff, p->stream);
    if (rc) return rc;
    // step-type copies: G / M, wavenumbers
    const double sc = 1.0 / (double)p->Mtot;
    k_scale_green<<<256, 256, 0, p->stream>>>(p->G64, p->fp64 ? nullptr : (float *)p->Gs,
                                               p->fp64 ? (double *)p->Gs : nullptr, p->Mhalf, sc);
    CK(cudaGetLastError());
    if (p->fp64) {
        CK(cudaMemcpy(p->kvec, ktab.data(), sizeof(double) * len, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->kdiff, kdiff.data(), sizeof(double) * len, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> a(len), b(len);
        for (int i = 0; i < len; ++i) {
            a[i] = (float)ktab[i];
            b[i] = (float)kdiff[i];
        }
        CK(cudaMemcpy(p->kvec, a.data(), sizeof(float) * len, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->kdiff, b.data(), sizeof(float) * len, cudaMemcpyHostToDevice));
    }
    CK(cudaStreamSynchronize(p->stream));
    return PPPM_OK;
}

int make_ffts(pppm_plan *p) {
    const cufftType tr2c = p->fp64 ? CUFFT_D2Z : CUFFT_R2C;
    const cufftType tc2r = p->fp64 ? CUFFT_Z2D : CUFFT_C2R;
    CKF(cufftPlan3d(&p->r2c, p->M[0], p->M[1], p->M[2], tr2c));
    p->have_r2c = true;
    CKF(cufftSetStream(p->r2c, p->stream));
    CKF(cufftPlan3d(&p->c2r1, p->M[0], p->M[1], p->M[2], tc2r));
    p->have_c2r1 = true;
    CKF(cufftSetStream(p->c2r1, p->stream));
    if (p->ik) {
        // three field spectra -> one interleaved (Ex, Ey, Ez, pad) real array
        int n[3] = {p->M[0], p->M[1], p->M[2]};
        int inembed[3] = {p->M[0], p->M[1], p->Mzh};
        int onembed[3] = {p->M[0], p->M[1], p->M[2]};
        CKF(cufftPlanMany(&p->c2r, 3, n, inembed, 1, (int)p->Mhalf, onembed, 4, 1, tc2r, 3));
        p->have_c2r = true;
        CKF(cufftSetStream(p->c2r, p->stream));
    }
    return PPPM_OK;
}

int exec_r2c(pppm_plan *p) {
    if (p->fp64) CKF(cufftExecD2Z(p->r2c, (cufftDoubleReal *)p->rho, (cufftDoubleComplex *)p->rho_hat));
    else CKF(cufftExecR2C(p->r2c, (cufftReal *)p->rho, (cufftComplex *)p->rho_hat));
    return PPPM_OK;
}

int exec_c2r(pppm_plan *p, bool all3) {
    cufftHandle h = (all3 && p->ik) ? p->c2r : p->c2r1;
    if (p->fp64) CKF(cufftExecZ2D(h, (cufftDoubleComplex *)p->spec, (cufftDoubleReal *)p->field));
    else CKF(cufftExecC2R(h, (cufftComplex *)p->spec, (cufftReal *)p->field));
    return PPPM_OK;
}

// kind 0: forces, 1: energy gradient
template <typename R>
int enqueue_t(pppm_plan *p, const Geom<R> &gp, int64_t n, const void *x, const void *q, void *f, void *dq,
              double *ev, int kind) {
    Geom<R> g = gp;  // this step's copy: launch flags below
    cudaStream_t s = p->stream;
    const int pmask = (kind == 0) ? p->prof_mask : 0;
    const bool prof = pmask != 0;
    // External records stay real timing records inside a captured graph
    // (a plain record during capture only becomes a dependency edge).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (prof || sync_check_on()) CK(cudaStreamIsCapturing(s, &cap));
    // boundary i opens stage i and closes stage i - 1
    auto need_mark = [&](int i) { return ((pmask >> i) & 1) || (i > 0 && ((pmask >> (i - 1)) & 1)); };
    auto mark = [&](int i) {
        if (!need_mark(i)) return;
        if (cap == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(p->prof[i], s, cudaEventRecordExternal);
        else
            cudaEventRecord(p->prof[i], s);
    };
    const bool chk = sync_check_on() && cap == cudaStreamCaptureStatusNone;
    auto check = [&](const char *stage) -> int {
        if (!chk) return PPPM_OK;
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->side);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) return PPPM_OK;
        last_cuda_stage = stage;
        return cuda_status(e);
    };
    // green follows the forward transform's last kernel and fieldforce the
    // inverse transform's, unless a stage event node sits in between
    g.launch_flags = 0;
    if (!chk && !need_mark(3)) g.launch_flags |= LF_PDL_GREEN;
    if (!chk && !need_mark(5)) g.launch_flags |= LF_PDL_FF;
    int rc;
    mark(0);
    launch_sort<R>(g, n, (const R *)x, (const R *)q, p->sb, s, (R *)p->rho, p->Mtot,  // also clears rho
                   p->stage_in ? (R *)p->hx : nullptr, p->stage_in ? (R *)p->hq : nullptr);
    if ((rc = check("particle_map/scatter"))) return rc;
    mark(1);
    // programmatic launch straight after the scatter unless a stage event sits between them
    launch_make_rho<R>(g, n, p->sb, (R *)p->rho, p->comp, s, true, !need_mark(1) && !chk);
    if ((rc = check("make_rho"))) return rc;
    const bool ik_spec = (kind == 0) && p->ik;
    const int mn = map_blocks(n);  // k_particle_map blocks, one q, q^2 partial each
    if constexpr (std::is_same<R, float>::value) {
        if (p->variants & 8) {
            // forward plane pass | x pass with G and the energy partials | inverse plane pass
            mark(2);
            launch_custom_fft(0, g, ik_spec, (const float *)p->rho, p->rho_hat, p->spec, (float *)p->field, p->gb,
                              p->ec, !need_mark(2) && !chk, s);
            if ((rc = check("forward FFT"))) return rc;
            mark(3);
            const int gn = launch_custom_fft(1, g, ik_spec, (const float *)p->rho, p->rho_hat, p->spec,
                                             (float *)p->field, p->gb, p->ec, !need_mark(3) && !chk, s);
            if ((rc = check("green"))) return rc;
            mark(4);
            bool pdl_inv = !need_mark(4) && !chk;
            if (kind == 0) {
                // the final energy/virial sum runs beside the inverse pass and fieldforce
                CK(cudaEventRecord(p->fork, s));
                CK(cudaStreamWaitEvent(p->side, p->fork, 0));
                launch_energy_final(p->gb, p->ec, gn, mn, ev, p->side);
                CK(cudaEventRecord(p->join, p->side));
                pdl_inv = false;  // an event record sits between the x pass and the inverse pass
            } else {
                launch_energy_final(p->gb, p->ec, gn, mn, ev, s);  // dE/dq needs sum q first
                pdl_inv = false;
            }
            if ((rc = check("energy_final"))) return rc;
            launch_custom_fft(2, g, ik_spec, (const float *)p->rho, p->rho_hat, p->spec, (float *)p->field, p->gb,
                              p->ec, pdl_inv, s);
            if ((rc = check("inverse FFT"))) return rc;
            mark(5);
            if (kind == 0) {
                launch_fieldforce<R>(g, p->ik, n, p->sb, (const R *)p->field, (R *)f, (R)p->C, p->sf, s);
            } else {
                const double gself = -2.0 * p->C * p->g / std::sqrt(M_PI);
                const double gbg = -p->C * M_PI / (p->g * p->g * p->V);
                launch_energy_grad<R>(g, n, p->sb, (const R *)p->field, (R *)f, (R *)dq, (R)p->C, p->sb.qsum,
                                      gself, gbg, s);
            }
            if ((rc = check("fieldforce"))) return rc;
            mark(6);
            if (kind == 0) CK(cudaStreamWaitEvent(s, p->join, 0));
            p->prof_valid = pmask;
            CK(cudaGetLastError());
            return PPPM_OK;
        }
    }
    mark(2);
    if ((rc = exec_r2c(p))) return rc;
    if ((rc = check("forward FFT"))) return rc;
    mark(3);
    const int gn = launch_green<R>(g, ik_spec, p->rho_hat, p->spec, p->gb, p->ec, s);
    if ((rc = check("green"))) return rc;
    mark(4);
    if (kind == 0) {
        // the final energy/virial sum runs beside the inverse FFTs and fieldforce
        CK(cudaEventRecord(p->fork, s));
        CK(cudaStreamWaitEvent(p->side, p->fork, 0));
        launch_energy_final(p->gb, p->ec, gn, mn, ev, p->side);
        CK(cudaEventRecord(p->join, p->side));
    } else {
        launch_energy_final(p->gb, p->ec, gn, mn, ev, s);  // dE/dq needs sum q first
    }
    if ((rc = check("energy_final"))) return rc;
    if ((rc = exec_c2r(p, ik_spec))) return rc;
    if ((rc = check("inverse FFT"))) return rc;
    mark(5);
    if (kind == 0) {
        launch_fieldforce<R>(g, p->ik, n, p->sb, (const R *)p->field, (R *)f, (R)p->C, p->sf, s);
    } else {
        const double gself = -2.0 * p->C * p->g / std::sqrt(M_PI);
        const double gbg = -p->C * M_PI / (p->g * p->g * p->V);
        launch_energy_grad<R>(g, n, p->sb, (const R *)p->field, (R *)f, (R *)dq, (R)p->C, p->sb.qsum, gself,
                              gbg, s);
    }
    if ((rc = check("fieldforce"))) return rc;
    mark(6);
    if (kind == 0) CK(cudaStreamWaitEvent(s, p->join, 0));
    p->prof_valid = pmask;
    CK(cudaGetLastError());
    return PPPM_OK;
}

int enqueue(pppm_plan *p, int64_t n, const void *x, const void *q, void *f, void *dq, double *ev, int kind) {
    if (n == 0) {
        CK(cudaMemsetAsync(p->ev, 0, 8 * sizeof(double), p->stream));
        if (ev) CK(cudaMemsetAsync(ev, 0, 7 * sizeof(double), p->stream));
        CK(cudaMemsetAsync(p->rho, 0, (p->fp64 ? 8 : 4) * (size_t)p->Mtot, p->stream));
        return PPPM_OK;
    }
    if (p->fp64) return enqueue_t<double>(p, p->gd, n, x, q, f, dq, ev, kind);
    return enqueue_t<float>(p, p->gf, n, x, q, f, dq, ev, kind);
}

bool valid_ptr_arg(int64_t n, const void *ptr) { return n == 0 || ptr != nullptr; }

void drop_graph(pppm_plan *p) {
    for (auto &g : p->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = pppm_plan::GraphSlot{};
    }
}

bool variant_ok(const pppm_plan *p, int v) {
    if (v & ~255) return false;
    // make_rho on z-pairs of tiles: 8^3 tiles (at most), one brick layout
    if ((v & 128) && (v & (2 | 4 | 16))) return false;
    if ((v & 64) && (p->fp64 || (v & 1))) return false;  // the persistent fieldforce: FP32 step types, one variant
    if ((v & 16) && (v & 2)) return false;      // one tile shape at a time
    if ((v & 32) && (v & 4)) return false;      // one make_rho brick layout at a time
    if ((v & 8) && !p->fft_own) return false;  // FP32 plans on meshes the hand-written solve serves
    if ((v & 4) && !p->comp) return false;  // the four-copy brick is the FP32C accumulator
    if ((v & 2) && !long_tiles_allowed(p->P, p->comp)) return false;
    return !((v & 1) && (v & 2));  // the tile-staged fieldforce brick holds 8^3 tiles only
}

// Variant bits: 0 tile-staged fieldforce, 1 long tiles (16 along z), 2
// four-copy make_rho brick, 3 hand-written Poisson solve, 4 small tiles (4^3),
// 5 make_rho brick with compile-time strides, 6 persistent double-buffered
// tile-staged fieldforce, 7 make_rho on z-pairs of tiles.
// The tile shape changes the sort; the histogram is cleared for the new shape.
void set_variants(pppm_plan *p, int v) {
    p->variants = v;
    tile_shape(p->M, (v & 2) != 0, p->T, p->TE, (v & 16) != 0);
    p->ntiles = p->T[0] * p->T[1] * p->T[2];
    for (int d = 0; d < 3; ++d) {
        p->gf.T[d] = p->gd.T[d] = p->T[d];
        p->gf.TE[d] = p->gd.TE[d] = p->TE[d];
    }
    p->gf.ntiles = p->gd.ntiles = p->ntiles;
    p->gf.ff_tiled = p->gd.ff_tiled = (v & 64) ? 2 : ((v & 1) ? 1 : 0);
    p->gf.rho_copies = p->gd.rho_copies = (v & 128) ? 4 : ((v & 4) ? 1 : ((v & 32) ? 2 : 0));
    if (p->sb.tile_count) cudaMemsetAsync(p->sb.tile_count, 0, 4 * (size_t)p->ntiles_alloc, p->stream);
    drop_graph(p);
}

// The device address of a caller's host buffer when the current device can
// dereference it (pinned host memory mapped into the unified address space,
// e.g. from cudaHostAlloc or cudaHostRegister), else nullptr.  Asked on every
// call: a cached answer could outlive the buffer.
// pppm_compute_host copies mapped inputs in bulk from this many particles on
constexpr int64_t DIRECT_IN_MAX_N = 1 << 18;

void *device_alias(const void *host) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

}  // namespace

extern "C" {

const char *pppm_strerror(int s) {
    switch (s) {
        case PPPM_OK: return "ok";
        case PPPM_EINVAL: return "invalid argument";
        case PPPM_ENOMEM: return "device allocation failed";
        case PPPM_ECUDA: return "CUDA runtime error";
        case PPPM_ECUFFT: return "cuFFT error";
        case PPPM_ENONFINITE: return "non-finite position or charge";
        case PPPM_ETIMEOUT: return "device wait timed out";
        case PPPM_ENOTREADY: return "quantity not computed by the last call";
        case PPPM_EINTERNAL: return "device consistency check failed (results invalid)";
        default: return "unknown status";
    }
}


const char *pppm_last_cuda_error(void) {
    static thread_local char buf[256];
    cudaError_t e = pppm::last_cuda_err != cudaSuccess ? pppm::last_cuda_err : cudaPeekAtLastError();
    if (e == cudaSuccess) return "";
    if (pppm::last_cuda_stage)
        snprintf(buf, sizeof(buf), "%s: %s (after %s)", cudaGetErrorName(e), cudaGetErrorString(e),
                 pppm::last_cuda_stage);
    else
        snprintf(buf, sizeof(buf), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return buf;
}

int pppm_estimate_g(double rel_acc, double r_cut, int64_t n, double q2, const double box[3], double *g_out) {
    if (!box || !g_out || !(rel_acc > 0) || !(r_cut > 0) || n <= 0 || !(q2 > 0)) return PPPM_EINVAL;
    if (!(box[0] > 0 && box[1] > 0 && box[2] > 0)) return PPPM_EINVAL;
    const double V = box[0] * box[1] * box[2];
    const double arg = rel_acc * std::sqrt((double)n * r_cut * V) / (2.0 * q2);
    if (!(arg > 0.0 && arg < 1.0)) return PPPM_EINVAL;
    *g_out = std::sqrt(-std::log(arg)) / r_cut;
    return PPPM_OK;
}

int pppm_fft_size(int n, int kind, int *out) {
    if (!out) return PPPM_EINVAL;
    const int m = fft_size_host(n, kind);
    if (m < 0) return PPPM_EINVAL;
    *out = m;
    return PPPM_OK;
}

int pppm_kspace_error(const double box[3], const int mesh[3], int order, double g_ewald, int diff_mode, int64_t n,
                      double q2, double *err_out) {
    if (!box || !mesh || !err_out || n <= 0 || !(q2 > 0) || !(g_ewald > 0) || !std::isfinite(g_ewald))
        return PPPM_EINVAL;
    if (order < 2 || order > MAXP || (diff_mode != PPPM_IK && diff_mode != PPPM_AD)) return PPPM_EINVAL;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0) || !std::isfinite(box[d])) return PPPM_EINVAL;
        if (mesh[d] < order || mesh[d] > MAX_MESH) return PPPM_EINVAL;
    }
    return kspace_error_mesh(mesh, box, order, g_ewald, diff_mode == PPPM_AD, n, q2, err_out);
}

int pppm_choose_mesh(const double box[3], int64_t n, double q2, int order, int diff_mode, double r_cut,
                     double rel_acc, int kind, int mesh_out[3], double *g_out, double *err_out) {
    if (!box || !mesh_out || !g_out || order < 2 || order > MAXP || (diff_mode != PPPM_IK && diff_mode != PPPM_AD) ||
        kind < 0 || kind > 2)
        return PPPM_EINVAL;
    double g = 0.0;
    int rc = pppm_estimate_g(rel_acc, r_cut, n, q2, box, &g);
    if (rc) return rc;
    const double lmax = std::max(box[0], std::max(box[1], box[2]));
    int prev[3] = {0, 0, 0};
    for (int c = order;; ++c) {
        int mesh[3];
        for (int d = 0; d < 3; ++d) {
            const double want = std::ceil(box[d] * c / lmax);
            if (want > MAX_MESH) return PPPM_EINVAL;  // no mesh up to the size limit meets the accuracy
            mesh[d] = std::max(order, fft_size_host((int)want, kind));
            if (mesh[d] > MAX_MESH) return PPPM_EINVAL;
        }
        if (mesh[0] == prev[0] && mesh[1] == prev[1] && mesh[2] == prev[2]) continue;
        double err = 0.0;
        if ((rc = kspace_error_mesh(mesh, box, order, g, diff_mode == PPPM_AD, n, q2, &err))) return rc;
        if (err <= rel_acc) {
            for (int d = 0; d < 3; ++d) mesh_out[d] = mesh[d];
            *g_out = g;
            if (err_out) *err_out = err;
            return PPPM_OK;
        }
        for (int d = 0; d < 3; ++d) prev[d] = mesh[d];
    }
}

int pppm_setup(pppm_plan **out, const double box[3], int64_t n_max, int order, const int mesh[3], double g_ewald,
               int diff_mode, int precision, double qqrd2e, void *cuda_stream) {
    if (!out) return PPPM_EINVAL;
    *out = nullptr;
    if (!box || !mesh || n_max < 0 || n_max > (int64_t)1 << 30) return PPPM_EINVAL;
    if (order < 2 || order > MAXP) return PPPM_EINVAL;
    if (!(g_ewald > 0) || !std::isfinite(g_ewald) || !std::isfinite(qqrd2e)) return PPPM_EINVAL;
    if (diff_mode != PPPM_IK && diff_mode != PPPM_AD) return PPPM_EINVAL;
    if (precision != PPPM_FP64 && precision != PPPM_FP32C && precision != PPPM_FP32) return PPPM_EINVAL;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0) || !std::isfinite(box[d])) return PPPM_EINVAL;
        if (mesh[d] < order || mesh[d] > MAX_MESH) return PPPM_EINVAL;  // stencil must fit the mesh
    }
    pppm_plan *p = new (std::nothrow) pppm_plan();
    if (!p) return PPPM_ENOMEM;
    int rc = PPPM_OK;
    cudaGetDevice(&p->device);
    p->stream = (cudaStream_t)cuda_stream;
    p->P = order;
    p->mode = diff_mode;
    p->ik = diff_mode == PPPM_IK;
    p->prec = precision;
    p->fp64 = precision == PPPM_FP64;
    p->comp = precision == PPPM_FP32C;
    p->g = g_ewald;
    p->C = qqrd2e;
    p->n_max = n_max;
    for (int d = 0; d < 3; ++d) {
        p->M[d] = mesh[d];
        p->box[d] = box[d];
        p->h[d] = box[d] / mesh[d];
    }
    tile_shape(p->M, false, p->T, p->TE);
    int T4[3], TE4[3];
    tile_shape(p->M, false, T4, TE4, true);
    p->Mzh = mesh[2] / 2 + 1;
    p->Mtot = (int64_t)mesh[0] * mesh[1] * mesh[2];
    p->Mhalf = (int64_t)mesh[0] * mesh[1] * p->Mzh;
    p->ntiles = p->T[0] * p->T[1] * p->T[2];
    p->ntiles_alloc = T4[0] * T4[1] * T4[2];
    p->V = box[0] * box[1] * box[2];
    p->vcell = p->h[0] * p->h[1] * p->h[2];

    double coef[MAXP][MAXP], dcoef[MAXP][MAXP];
    stencil_polynomials(order, coef, dcoef);
    fill_geom<float>(p, p->gf, coef, dcoef);
    fill_geom<double>(p, p->gd, coef, dcoef);

    const size_t rs = p->fp64 ? 8 : 4;
    const int64_t nm = std::max<int64_t>(n_max, 1);
    const int nblk_map = (int)((nm + 255) / 256);
    // k_green's partials (at most 152 x 8 CTAs), or the hand-written x pass's
    const int nblk_green = std::max(152 * 8, custom_fft_parts(p->M));
    do {
        if ((rc = dmalloc(p, &p->sb.anchor, 4 * nm))) break;
        if ((rc = dmalloc(p, &p->sb.rank, 4 * nm))) break;
        if ((rc = dmalloc(p, &p->sb.tile_count, 4 * (size_t)p->ntiles_alloc))) break;
        if ((rc = dmalloc(p, &p->sb.tile_start, 4 * ((size_t)p->ntiles_alloc + 1)))) break;
        if ((rc = dmalloc(p, &p->sb.perm, 4 * nm))) break;
        if ((rc = dmalloc(p, &p->sb.rec, 4 * rs * nm))) break;
        if ((rc = dmalloc(p, &p->sb.cell, 4 * nm))) break;
        if ((rc = dmalloc(p, &p->sb.blk, sizeof(double) * 2 * nblk_map))) break;
        if ((rc = dmalloc(p, &p->sb.qsum, 2 * sizeof(double)))) break;
        if ((rc = dmalloc(p, &p->sb.err, 4 * sizeof(int)))) break;
        if ((rc = dmalloc(p, &p->sb.queue, 2 * sizeof(unsigned int)))) break;
        if ((rc = dmalloc(p, &p->rho, rs * p->Mtot))) break;
        if ((rc = dmalloc(p, &p->rho_hat, 2 * rs * p->Mhalf))) break;
        if ((rc = dmalloc(p, &p->spec, 2 * rs * p->Mhalf * (p->ik ? 3 : 1)))) break;
        if ((rc = dmalloc(p, &p->field, rs * p->Mtot * (p->ik ? 4 : 1)))) break;
        if ((rc = dmalloc(p, &p->G64, sizeof(double) * p->Mhalf))) break;
        if ((rc = dmalloc(p, &p->Gs, rs * p->Mhalf))) break;
        const size_t len = (size_t)p->M[0] + p->M[1] + p->Mzh;
        if ((rc = dmalloc(p, &p->kvec, rs * len))) break;
        if ((rc = dmalloc(p, &p->kdiff, rs * len))) break;
        if ((rc = dmalloc(p, &p->green_part, sizeof(double) * 7 * nblk_green))) break;
        if ((rc = dmalloc(p, &p->ev, 8 * sizeof(double)))) break;
        if ((rc = dmalloc(p, &p->d_sf, 6 * sizeof(double)))) break;
        if ((rc = dmalloc(p, &p->hx, 3 * rs * nm))) break;
        if ((rc = dmalloc(p, &p->hq, rs * nm))) break;
        if ((rc = dmalloc(p, &p->hf, 3 * rs * nm))) break;
        if ((rc = dmalloc(p, &p->hev, 8 * sizeof(double)))) break;
        if (cudaHostAlloc((void **)&p->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p->h_err = nullptr;
            rc = PPPM_ENOMEM;
            break;
        }
    } while (0);
    if (rc) {
        release(p);
        return rc;
    }
    p->gb.G64 = p->G64;
    p->gb.Gs = p->Gs;
    p->gb.kvec = p->kvec;
    p->gb.kdiff = p->kdiff;
    p->gb.part = p->green_part;
    p->gb.qsum = p->sb.qsum;
    p->gb.map_part = p->sb.blk;
    p->gb.ev = p->ev;
    p->ec.epref = 0.5 * p->C * p->vcell * p->vcell / p->V * (double)p->Mtot;
    p->ec.inv4g2 = 1.0 / (4.0 * p->g * p->g);
    p->ec.eself = -p->C * p->g / std::sqrt(M_PI);
    p->ec.ebg = -p->C * M_PI / (2.0 * p->g * p->g * p->V);

    auto fail = [&](int code) {
        release(p);
        return code;
    };
    if (cudaMemsetAsync(p->sb.tile_count, 0, 4 * (size_t)p->ntiles_alloc, p->stream) != cudaSuccess ||
        cudaMemsetAsync(p->sb.err, 0, 4 * sizeof(int), p->stream) != cudaSuccess ||
        cudaMemsetAsync(p->sb.queue, 0, 2 * sizeof(unsigned int), p->stream) != cudaSuccess ||
        cudaMemsetAsync(p->ev, 0, 8 * sizeof(double), p->stream) != cudaSuccess)
        return fail(PPPM_ECUDA);
    if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming) != cudaSuccess)
        return fail(PPPM_ECUDA);
    cudaError_t pe = p->fp64 ? prepare_make_rho<double>(order, false) : prepare_make_rho<float>(order, p->comp);
    if (pe == cudaSuccess) pe = p->fp64 ? prepare_fieldforce<double>(order) : prepare_fieldforce<float>(order);
    if (pe == cudaSuccess) pe = p->fp64 ? prepare_green<double>() : prepare_green<float>();
    p->fft_own = !p->fp64 && custom_fft_supported(p->M);
    if (pe == cudaSuccess && p->fft_own) pe = prepare_custom_fft(p->M);
    if (pe != cudaSuccess) return fail(PPPM_ECUDA);
    // default kernel variants (pppm_autotune refines them on real inputs):
    // the ik field (16 bytes a point) is worth staging per tile once tiles
    // hold enough particles; the ad potential (4 bytes) reads best through L1
    // (the four-copy make_rho brick measured level at P = 5 and slower at P = 7)
    // the hand-written Poisson solve replaces seven cuFFT/green launches by three
    // with fewer 8^3 tiles than two per SM, 4^3 tiles give the mesh stages enough CTAs
    const bool small_tiles = p->ntiles < 2 * 152;
    int T0[3], TE0[3];
    tile_shape(p->M, false, T0, TE0, small_tiles);
    const int nt0 = T0[0] * T0[1] * T0[2];
    // compile-time brick strides never measured slower (c3 make_rho 688 -> 665 us); the
    // persistent one-particle-per-thread ad fieldforce halves the 2M-charge gather (545 -> 258 us)
    const bool ad_persist = !p->ik && !p->fp64;
    // make_rho on z-pairs of 8^3 tiles (c3: 358 -> 262 us in FP32)
    const bool pairs = !small_tiles;
    set_variants(p, ((p->ik && (double)n_max >= 16.0 * nt0) ? 1 : 0) | (p->fft_own && custom_fft_default(p->M) ? 8 : 0) |
                        (small_tiles ? 16 : 0) | 32 | (ad_persist ? 64 : 0) | (pairs ? 128 : 0));
    if ((rc = build_tables_and_green(p))) return fail(rc);
    if ((rc = make_ffts(p))) return fail(rc);
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return fail(PPPM_ECUDA);
    *out = p;
    return PPPM_OK;
}

int pppm_destroy(pppm_plan *p) {
    if (!p) return PPPM_EINVAL;
    release(p);
    return PPPM_OK;
}

int pppm_set_stream(pppm_plan *p, void *cuda_stream) {
    if (!p) return PPPM_EINVAL;
    p->stream = (cudaStream_t)cuda_stream;
    drop_graph(p);
    if (p->have_r2c) CKF(cufftSetStream(p->r2c, p->stream));
    if (p->have_c2r) CKF(cufftSetStream(p->c2r, p->stream));
    if (p->have_c2r1) CKF(cufftSetStream(p->c2r1, p->stream));
    return PPPM_OK;
}

int pppm_set_graph(pppm_plan *p, int enable) {
    if (!p) return PPPM_EINVAL;
    p->graph_on = enable != 0;
    if (!p->graph_on) drop_graph(p);
    return PPPM_OK;
}

int pppm_compute(pppm_plan *p, int64_t n, const void *x, const void *q, void *f, double *ev) {
    if (!p || n < 0 || n > p->n_max) return PPPM_EINVAL;
    if (!valid_ptr_arg(n, x) || !valid_ptr_arg(n, q) || !valid_ptr_arg(n, f)) return PPPM_EINVAL;
    p->n_last = n;
    p->field_is_field = true;
    p->have_rho = true;
    if (!p->graph_on) return enqueue(p, n, x, q, f, nullptr, ev, 0);
    const void *key[4] = {x, q, f, ev};
    pppm_plan::GraphSlot *hit = nullptr, *lru = &p->graphs[0];
    for (auto &g : p->graphs) {
        if (g.exec && g.n == n && g.prof == p->prof_mask && g.stage == p->stage_in && g.key[0] == key[0] &&
            g.key[1] == key[1] && g.key[2] == key[2] && g.key[3] == key[3])
            hit = &g;
        if (!g.exec || (lru->exec && g.used < lru->used)) lru = &g;
    }
    if (!hit) {
        hit = lru;
        if (hit->exec) cudaGraphExecDestroy(hit->exec);
        *hit = pppm_plan::GraphSlot{};
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue(p, n, x, q, f, nullptr, ev, 0);
        cudaError_t ee = cudaStreamEndCapture(p->stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        CK(ee);
        cudaError_t ie = cudaGraphInstantiate(&hit->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) hit->exec = nullptr;
        CK(ie);
        for (int i = 0; i < 4; ++i) hit->key[i] = key[i];
        hit->n = n;
        hit->prof = p->prof_mask;
        hit->stage = p->stage_in;
    }
    hit->used = ++p->graph_clock;
    CK(cudaGraphLaunch(hit->exec, p->stream));
    p->prof_valid = p->prof_mask;
    return PPPM_OK;
}

int pppm_sync(pppm_plan *p) {
    if (!p) return PPPM_EINVAL;
    CK(cudaStreamSynchronize(p->stream));
    int err = 0;
    CK(cudaMemcpy(&err, p->sb.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CK(cudaMemset(p->sb.err, 0, sizeof(int)));
        return (err & ERR_INTERNAL) ? PPPM_EINTERNAL : PPPM_ENONFINITE;
    }
    return PPPM_OK;
}

int pppm_compute_host(pppm_plan *p, int64_t n, const void *x_host, const void *q_host, void *f_host,
                      double *ev_host) {
    if (!p || n < 0 || n > p->n_max) return PPPM_EINVAL;
    if (!valid_ptr_arg(n, x_host) || !valid_ptr_arg(n, q_host) || !valid_ptr_arg(n, f_host)) return PPPM_EINVAL;
    const size_t rs = p->fp64 ? 8 : 4;
    // Pinned buffers mapped into the device's address space may be read (x, q,
    // see below) and written (energy/virial) by the kernels themselves over
    // the host-device link; other buffers go through the plan's device staging.
    const void *xa = (n > 0) ? device_alias(x_host) : nullptr;
    const void *qa = (n > 0) ? device_alias(q_host) : nullptr;
    double *eva = (n > 0 && ev_host) ? static_cast<double *>(device_alias(ev_host)) : nullptr;
    // Mapped x and q are read in place by the sort kernels on small systems
    // (no copy launches; 32,001 charges 66 us a call in place vs 70 us
    // copied).  From DIRECT_IN_MAX_N particles on particle_map reads them
    // over the link once and writes device copies that the scatter reads
    // (read twice over the link, 2,048,001 charges took 1.42 ms a call against
    // 1.34 ms after a bulk copy); unmapped inputs are copied in bulk first.
    const bool mapped_in = xa && qa;
    const bool direct_in = mapped_in && n < DIRECT_IN_MAX_N;
    const bool stage_in = mapped_in && !direct_in;
    if (n > 0 && !mapped_in) {
        CK(cudaMemcpyAsync(p->hx, x_host, 3 * rs * n, cudaMemcpyHostToDevice, p->stream));
        CK(cudaMemcpyAsync(p->hq, q_host, rs * n, cudaMemcpyHostToDevice, p->stream));
    }
    // f comes back as one bulk copy: fieldforce's stores are scattered in
    // input order, and writing them straight to host memory measured no faster
    p->stage_in = stage_in;
    int rc = pppm_compute(p, n, mapped_in ? xa : p->hx, mapped_in ? qa : p->hq, p->hf, eva ? eva : p->hev);
    p->stage_in = false;
    if (rc) return rc;
    if (n > 0) CK(cudaMemcpyAsync(f_host, p->hf, 3 * rs * n, cudaMemcpyDeviceToHost, p->stream));
    if (ev_host && !eva) CK(cudaMemcpyAsync(ev_host, p->hev, 7 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    // the error word travels with the results: one stream synchronisation per call
    CK(cudaMemcpyAsync(p->h_err, p->sb.err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    const int err = *p->h_err;
    if (err) {
        CK(cudaMemsetAsync(p->sb.err, 0, sizeof(int), p->stream));
        CK(cudaStreamSynchronize(p->stream));
        return (err & ERR_INTERNAL) ? PPPM_EINTERNAL : PPPM_ENONFINITE;
    }
    return PPPM_OK;
}

int pppm_energy_grad(pppm_plan *p, int64_t n, const void *x, const void *q, void *dEdx, void *dEdq, double *ev) {
    if (!p || n < 0 || n > p->n_max) return PPPM_EINVAL;
    if (!valid_ptr_arg(n, x) || !valid_ptr_arg(n, q)) return PPPM_EINVAL;
    p->n_last = n;
    p->field_is_field = false;
    p->have_rho = true;
    return enqueue(p, n, x, q, dEdx, dEdq, ev, 1);
}

int pppm_potential(pppm_plan *p, int64_t n, const void *x, const void *q, void *phi) {
    if (!p || n < 0 || n > p->n_max) return PPPM_EINVAL;
    if (!valid_ptr_arg(n, x) || !valid_ptr_arg(n, q) || !valid_ptr_arg(n, phi)) return PPPM_EINVAL;
    p->n_last = n;
    p->field_is_field = false;
    p->have_rho = true;
    return enqueue(p, n, x, q, nullptr, phi, nullptr, 1);
}

int pppm_get_array(pppm_plan *p, int which, void *dst, size_t bytes, int to_host) {
    if (!p || !dst) return PPPM_EINVAL;
    const size_t rs = p->fp64 ? 8 : 4;
    const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(cudaStreamSynchronize(p->stream));
    switch (which) {
        case PPPM_ARR_RHO:
            if (bytes != rs * (size_t)p->Mtot) return PPPM_EINVAL;
            if (!p->have_rho) return PPPM_ENOTREADY;
            CK(cudaMemcpy(dst, p->rho, bytes, kind));
            return PPPM_OK;
        case PPPM_ARR_GREEN:
            if (bytes != 8 * (size_t)p->Mhalf) return PPPM_EINVAL;
            CK(cudaMemcpy(dst, p->G64, bytes, kind));
            return PPPM_OK;
        case PPPM_ARR_FIELD: {
            const size_t want = rs * (size_t)p->Mtot * ((p->ik && p->field_is_field) ? 4 : 1);
            if (bytes != want) return PPPM_EINVAL;
            if (p->n_last < 0) return PPPM_ENOTREADY;
            CK(cudaMemcpy(dst, p->field, bytes, kind));
            return PPPM_OK;
        }
        case PPPM_ARR_ANCHOR: {
            if (p->n_last < 0) return PPPM_ENOTREADY;
            const int64_t n = p->n_last;
            if (bytes != 12 * (size_t)n) return PPPM_EINVAL;
            std::vector<uint32_t> packed(n);
            std::vector<int32_t> a(3 * n);
            if (n) CK(cudaMemcpy(packed.data(), p->sb.anchor, 4 * n, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < n; ++i) {
                int u, v, w;
                unpack_anchor(packed[i], u, v, w);
                a[3 * i] = u;
                a[3 * i + 1] = v;
                a[3 * i + 2] = w;
            }
            if (n) CK(cudaMemcpy(dst, a.data(), bytes, to_host ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice));
            return PPPM_OK;
        }
        case PPPM_ARR_TILESTART:
            if (bytes != 4 * ((size_t)p->ntiles + 1)) return PPPM_EINVAL;
            if (p->n_last < 0) return PPPM_ENOTREADY;
            CK(cudaMemcpy(dst, p->sb.tile_start, bytes, kind));
            return PPPM_OK;
        case PPPM_ARR_PERM:
            if (p->n_last < 0) return PPPM_ENOTREADY;
            if (bytes != 4 * (size_t)p->n_last) return PPPM_EINVAL;
            if (bytes) CK(cudaMemcpy(dst, p->sb.perm, bytes, kind));
            return PPPM_OK;
        case PPPM_ARR_SELFFORCE:
            if (bytes != sizeof(p->sf)) return PPPM_EINVAL;
            CK(cudaMemcpy(dst, p->sf, bytes, to_host ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice));
            return PPPM_OK;
        case PPPM_ARR_ENERGY:
            if (bytes != 7 * sizeof(double)) return PPPM_EINVAL;
            CK(cudaMemcpy(dst, p->ev, bytes, kind));
            return PPPM_OK;
        default:
            return PPPM_EINVAL;
    }
}

int pppm_set_profiling(pppm_plan *p, int enable) {
    if (!p) return PPPM_EINVAL;
    if (enable && !p->prof[0]) {
        for (auto &e : p->prof) CK(cudaEventCreate(&e));
    }
    p->prof_mask = enable & 0x3f;
    p->prof_valid = 0;
    return PPPM_OK;
}

int pppm_stage_times(pppm_plan *p, float ms[6]) {
    if (!p || !ms) return PPPM_EINVAL;
    if (!p->prof_valid || !p->prof[0]) return PPPM_ENOTREADY;
    for (int i = 0; i < 6; ++i) {
        ms[i] = -1.0f;
        if ((p->prof_valid >> i) & 1) {
            CK(cudaEventSynchronize(p->prof[i + 1]));
            CK(cudaEventElapsedTime(&ms[i], p->prof[i], p->prof[i + 1]));
        }
    }
    return PPPM_OK;
}

int pppm_set_lut(pppm_plan *p, int entries) {
    if (!p || entries < 0 || entries == 1 || entries > (1 << 24)) return PPPM_EINVAL;
    p->gf.lut_bins = p->gd.lut_bins = entries;
    drop_graph(p);
    return PPPM_OK;
}

int pppm_set_variant(pppm_plan *p, int variants) {
    if (!p || !variant_ok(p, variants)) return PPPM_EINVAL;
    set_variants(p, variants);
    return PPPM_OK;
}

constexpr int AUTOTUNE_TIMED = 10;  // timed steps per variant (after two warm-up steps)

int pppm_autotune(pppm_plan *p, int64_t n, const void *x, const void *q, void *f, int *choice_out) {
    if (!p || n < 0 || n > p->n_max) return PPPM_EINVAL;
    if (!valid_ptr_arg(n, x) || !valid_ptr_arg(n, q) || !valid_ptr_arg(n, f)) return PPPM_EINVAL;
    // variants are timed the way the plan's steps run (as CUDA graphs when
    // the plan uses them), each by its fastest of AUTOTUNE_TIMED steps: the
    // variants of a small system differ by about a microsecond, below the
    // launch jitter of ungraphed steps
    const bool graph = p->graph_on;
    const int pmask = p->prof_mask;
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f;
    int best_v = p->variants;
    int rc = PPPM_OK;
    for (int v = 0; v <= 255 && rc == PPPM_OK; ++v) {
        if (!variant_ok(p, v)) continue;
        set_variants(p, v);
        float vbest = 1e30f;
        // two warm-up steps (the first captures the variant's graph), then timed ones
        for (int it = 0; it < 2 + AUTOTUNE_TIMED && rc == PPPM_OK; ++it) {
            if (cudaEventRecord(a, p->stream) != cudaSuccess) rc = PPPM_ECUDA;
            if (!rc) rc = graph ? pppm_compute(p, n, x, q, f, nullptr) : enqueue(p, n, x, q, f, nullptr, nullptr, 0);
            if (!rc && cudaEventRecord(b, p->stream) != cudaSuccess) rc = PPPM_ECUDA;
            if (!rc && cudaEventSynchronize(b) != cudaSuccess) rc = PPPM_ECUDA;
            float ms = 0.0f;
            if (!rc && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) rc = PPPM_ECUDA;
            if (it >= 2) vbest = fminf(vbest, ms);
        }
        if (!rc && vbest < best) {
            best = vbest;
            best_v = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    set_variants(p, best_v);
    p->graph_on = graph;
    p->prof_mask = pmask;
    p->n_last = n;
    p->field_is_field = true;
    p->have_rho = true;
    if (choice_out) *choice_out = best_v;
    return rc;
}

int pppm_get_variant(const pppm_plan *p, int *variants) {
    if (!p || !variants) return PPPM_EINVAL;
    *variants = p->variants;
    return PPPM_OK;
}

int pppm_plan_info(const pppm_plan *p, int64_t info[10]) {
    if (!p || !info) return PPPM_EINVAL;
    info[0] = p->M[0];
    info[1] = p->M[1];
    info[2] = p->M[2];
    info[3] = p->P;
    info[4] = p->ntiles;
    info[5] = p->TE[2];
    info[6] = p->mode;
    info[7] = p->prec;
    info[8] = p->n_max;
    info[9] = p->n_last;
    return PPPM_OK;
}

}  // extern "C"
