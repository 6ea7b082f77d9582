/*
 * pppm_gb300.h -- C ABI of the GB300 (sm_103a) PPPM k-space particle-mesh path.
 *
 * The path is the long-range half of PPPM electrostatics as McDoniel et al.,
 * "LAMMPS' PPPM Long-Range Solver for the Second Generation Xeon Phi"
 * (arXiv:1702.04250), define it in Sec. 2.1 (three steps: map charges to a
 * grid with a stencil; solve Poisson's equation with a forward 3-D FFT and one
 * (ad) or three (ik) inverse FFTs; map back to the particles with the same
 * stencil) and Sec. 3.1-3.2 (the Map-Charge and Distribute-Force mapping
 * functions, the Poisson solver).
 *
 * Conventions for every call:
 *  - Boxes are orthorhombic with the lower corner at the origin; positions
 *    outside [0, L) are wrapped periodically (not an error).
 *  - "device" pointers are CUDA device (or managed) memory on the plan's
 *    device; "host" pointers are ordinary or pinned host memory.
 *  - Layouts are C order: positions x[n][3], forces f[n][3], charges q[n];
 *    the element type is double for PPPM_FP64 and float for PPPM_FP32 /
 *    PPPM_FP32C.  Meshes are [Mx][My][Mz] with z fastest.
 *  - The caller owns x, q, f and the energy/virial buffer; the plan owns its
 *    mesh, spectra, Green's function, sort scratch and cuFFT plans.
 *  - Every call returns a pppm_status; nothing is thrown across the ABI.
 *    Calls that enqueue GPU work are asynchronous on the plan's stream unless
 *    stated otherwise; device-side problems (non-finite inputs) are recorded
 *    in a device error word and reported by pppm_sync().
 *  - A plan is bound to one device and one stream and is not thread-safe.
 */
#ifndef PPPM_GB300_H
#define PPPM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pppm_plan pppm_plan;

enum pppm_status {
    PPPM_OK = 0,
    PPPM_EINVAL = 1,      /* bad argument (sizes, order, mesh smaller than the stencil, ...) */
    PPPM_ENOMEM = 2,      /* device allocation failed */
    PPPM_ECUDA = 3,       /* a CUDA runtime call failed */
    PPPM_ECUFFT = 4,      /* a cuFFT call failed */
    PPPM_ENONFINITE = 5,  /* a position or charge was NaN/Inf (reported by pppm_sync) */
    PPPM_ETIMEOUT = 6,    /* a bounded device wait gave up */
    PPPM_ENOTREADY = 7,   /* the requested quantity was not computed by the last call */
    PPPM_EINTERNAL = 8    /* a device-side consistency check failed (a particle's stencil
                             anchor outside its tile, a sort slot out of range): the kernel
                             skipped that work, so the call's results are invalid
                             (reported by pppm_sync) */
};

/* Differentiation mode (Sec. 2.1 / Sec. 3.1): ik takes the gradient in
 * k-space (three inverse FFTs, three field components interpolated); ad
 * interpolates the scalar potential with derivative coefficients. */
enum pppm_diff { PPPM_IK = 0, PPPM_AD = 1 };

/* Arithmetic of the per-step path.  FP64: everything in double.  FP32:
 * spreading, FFTs and interpolation in float, the mesh charge of each tile
 * accumulated exactly in one 32-bit fixed-point word per point (every
 * contribution rounded once, to 2^-23 of the tile's largest possible one;
 * two words on tiles whose charge sum would cost that more than two bits).
 * FP32C: as FP32, with the mesh charge accumulated in two words (hi + lo)
 * that carry every contribution's exact product to 2^-37 of the largest.
 * In all three the Green's function, the ad self-force coefficients and the
 * energy/virial reductions are computed in double. */
enum pppm_precision { PPPM_FP64 = 0, PPPM_FP32C = 1, PPPM_FP32 = 2 };

/* Ewald splitting parameter from a target relative force accuracy.
 * Sec. 2.3 lists the accuracy epsilon and the cutoff r_C as the user's
 * parameters; the paper does not print the rule, so this solves the
 * real-space force-error estimate 2 q2 exp(-g^2 rc^2) / sqrt(N rc V) = rel_acc
 * (q2 = sum q_i^2) for g.  Host only, synchronous.
 * Returns PPPM_EINVAL if no positive g satisfies it or an argument is <= 0. */
int pppm_estimate_g(double rel_acc, double r_cut, int64_t n, double q2,
                    const double box[3], double *g_out);

/* FFT-friendly mesh edge (the analogue of Sec. 5's "adjust grid sizes", which
 * works around sizes its FFT library handled badly): *out = the smallest
 * m >= n that is n itself (kind 0), has no prime factor above 7 (kind 1, the
 * sizes cuFFT runs in its fast kernels), or is a power of two (kind 2, the
 * sizes of the hand-written Poisson solve, variant bit 3).  Host only.
 * PPPM_EINVAL for n < 1, an unknown kind or out == NULL. */
int pppm_fft_size(int n, int kind, int *out);

/* RMS k-space force error of a mesh (Sec. 2.3 / Sec. 4: the accuracy a
 * mesh, order and g deliver; the paper leaves the estimate to LAMMPS).
 * Reading: the Hockney-Eastwood functional of the scheme's force error over
 * this mesh's wavevectors k != 0, phi = 4 pi exp(-k^2/4g^2)/k^2,
 * |R(k)|^2 = k^2 phi^2, U = prod sinc^P(k h/2), k_m = k + 2 pi m/h:
 *   PPPM_IK  Q_k = sum_m |R(k_m)|^2 - [sum_m U^2(k_m) (k.k_m) phi(k_m)]^2
 *                  / (k^2 [sum_m U^2(k_m)]^2)   (optimal ik influence function)
 *   PPPM_AD  Q_k = G^2 [sum_m U^2(k_m)] [sum_m U^2(k_m) k_m^2]
 *                  - 2 G sum_m U^2(k_m) k_m^2 phi(k_m) + sum_m |R(k_m)|^2
 *            (each alias carries its own derivative; G = the plan's ad
 *            influence function, sum_m U^2 phi / [sum_m U^2]^2)
 * aliases |m_d| <= 2, the plain U^2 and U^2 k_m^2 sums exact/|m_d| <= 2000;
 * Q = (1/V) sum_k Q_k; *err_out = q2 sqrt(Q / (n V)), the RMS force error
 * of n randomly placed charges with sum q^2 = q2, in units of C e^2 / A^2
 * (the units of pppm_estimate_g's rel_acc).  Computed in FP64 by one kernel
 * on the current device (temporary device memory, synchronous).
 * PPPM_EINVAL for an unknown diff_mode, order outside 2..7, a mesh edge
 * < order or > 1024, or an argument <= 0; PPPM_ENOMEM / PPPM_ECUDA from the
 * device. */
int pppm_kspace_error(const double box[3], const int mesh[3], int order, double g_ewald, int diff_mode,
                      int64_t n, double q2, double *err_out);

/* Mesh and g for a target accuracy (Sec. 2.3, Sec. 4: LAMMPS chooses the mesh
 * from the accuracy; a larger stencil allows a coarser mesh).  g from
 * pppm_estimate_g(rel_acc, r_cut, n, q2, box); then for c = order, order + 1,
 * ... points along the longest edge, mesh_d = max(order,
 * pppm_fft_size(ceil(box_d c / L_max), kind)), skipping repeats, until
 * pppm_kspace_error(...) <= rel_acc.  Writes mesh_out[3], *g_out and
 * (nullable) *err_out.  Synchronous.  PPPM_EINVAL as for the two calls it
 * uses, or when no mesh with edges <= 1024 meets rel_acc. */
int pppm_choose_mesh(const double box[3], int64_t n, double q2, int order, int diff_mode, double r_cut,
                     double rel_acc, int kind, int mesh_out[3], double *g_out, double *err_out);

/* Create a plan (Sec. 2.1 setup before step 1): the order-P assignment
 * polynomials (Sec. 3.1: product of three 1-D polynomials of order S = P),
 * the influence function G(k) on the half spectrum, the ad self-force
 * coefficients, cuFFT plans and all scratch for up to n_max particles.
 *   box[3]      box edges (> 0)
 *   n_max       largest particle count pppm_compute will be given (>= 0)
 *   order       P in 2..7 (stencil of P^3 mesh points)
 *   mesh[3]     mesh points per dimension, each >= order and <= 1024
 *   g_ewald     Ewald splitting parameter (> 0)
 *   diff_mode   PPPM_IK or PPPM_AD
 *   precision   PPPM_FP64, PPPM_FP32C or PPPM_FP32
 *   qqrd2e      Coulomb constant C (energies in C * e^2 / length)
 *   cuda_stream cudaStream_t the plan enqueues on (NULL = legacy default)
 * Setup is synchronous.  On failure *out is NULL and nothing is leaked. */
int pppm_setup(pppm_plan **out, const double box[3], int64_t n_max, int order,
               const int mesh[3], double g_ewald, int diff_mode, int precision,
               double qqrd2e, void *cuda_stream);

/* Release every resource of the plan (synchronises its stream first). */
int pppm_destroy(pppm_plan *p);

/* Change the stream the plan enqueues on (drops any captured graph). */
int pppm_set_stream(pppm_plan *p, void *cuda_stream);

/* One k-space evaluation (Sec. 2.1 steps 1-3; Sec. 3.1 Map-Charge and
 * Distribute-Force ik/ad; Sec. 3.2 Poisson solver):
 *   particle_map (wrap, stencil anchor, sort by mesh tile) -> make_rho ->
 *   forward FFT -> influence-function multiply with energy/virial ->
 *   3 (ik) / 1 (ad) inverse FFTs -> fieldforce.
 *   n        particle count, 0 <= n <= n_max
 *   x        device, [n][3] positions
 *   q        device, [n] charges
 *   f        device, [n][3] k-space forces, overwritten (C q E, minus the ad
 *            self-force correction in ad mode)
 *   ev       device, 7 doubles or NULL: energy (mesh part minus the self and
 *            neutralising-background terms) then virial xx yy zz xy xz yz
 * Asynchronous; inputs must stay valid until the stream reaches the end of
 * the call.  With graph mode on (pppm_set_graph) the whole step is launched
 * as one CUDA graph; the plan keeps up to four instantiated graphs keyed by
 * n, the four pointers and the profiled stages (least recently used one
 * replaced), so alternating profiled and plain steps captures nothing new. */
int pppm_compute(pppm_plan *p, int64_t n, const void *x, const void *q, void *f, double *ev);

/* pppm_compute on HOST buffers: moves x and q to the device, computes, moves
 * f and the 7 energy/virial doubles back, synchronises and returns the device
 * status (PPPM_ENONFINITE if an input was not finite).  ev_host may be NULL.
 * Buffers in pinned host memory that the device can address (cudaHostAlloc,
 * cudaHostRegister) are read (x, q) and written (ev) by the kernels directly
 * over the host-device link: below 262,144 particles the sort's two passes
 * read x and q in place; from 262,144 on the first pass reads them once and
 * leaves device copies for the second.  Other buffers are copied in bulk
 * through device staging.  f always comes back as one device-to-host copy. */
int pppm_compute_host(pppm_plan *p, int64_t n, const void *x_host, const void *q_host,
                      void *f_host, double *ev_host);

/* Synchronise the plan's stream and report (then clear) the device error
 * word: PPPM_EINTERNAL if a device-side consistency check failed,
 * PPPM_ENONFINITE if a non-finite position or charge was seen by any compute
 * since the last sync, else PPPM_OK (or PPPM_ECUDA). */
int pppm_sync(pppm_plan *p);

/* Turn CUDA-graph launch of pppm_compute on (1) or off (0). */
int pppm_set_graph(pppm_plan *p, int enable);

/* Exact gradients of the PPPM energy (the energy reported by pppm_compute):
 *   dEdx[i][a] = C q_i sum_p dW(p - u_i)/dx_a phi(p)   (no self-force term)
 *   dEdq[i]    = C phi(x_i) - 2 C g q_i / sqrt(pi) - C pi Q / (g^2 V)
 * with phi the mesh potential of this plan's influence function (one extra
 * inverse FFT in ik mode).  Same element types and ownership as pppm_compute;
 * dEdx or dEdq may be NULL.  ev as in pppm_compute.  Asynchronous. */
int pppm_energy_grad(pppm_plan *p, int64_t n, const void *x, const void *q,
                     void *dEdx, void *dEdq, double *ev);

/* Electrostatic k-space potential felt by each atom, phi_i = dE/dq_i (the
 * dEdq of pppm_energy_grad: the mesh potential interpolated with the
 * assignment stencil of Sec. 3.1, times C, plus the self and neutralising-
 * background terms), i.e. the vector the backward pass of an energy with
 * respect to the charges needs.  phi: device, n values of the step type,
 * caller-owned, overwritten.  Asynchronous. */
int pppm_potential(pppm_plan *p, int64_t n, const void *x, const void *q, void *phi);

/* Internal arrays, for checking each stage against an independent
 * implementation.  Synchronous device-to-device (or device-to-host when
 * to_host != 0) copy of `bytes` bytes into dst; PPPM_EINVAL if bytes does not
 * equal the array's size, PPPM_ENOTREADY if the last compute did not make it.
 *   PPPM_ARR_RHO        mesh charge density, [Mx][My][Mz] of the step's type
 *   PPPM_ARR_GREEN      G(k), double [Mx][My][Mz/2+1] (unscaled)
 *   PPPM_ARR_FIELD      ik: E as [Mx][My][Mz][4] (x,y,z,unused); ad: phi [Mx][My][Mz]
 *   PPPM_ARR_ANCHOR     int32 [n][3] stencil anchor per particle, input order
 *   PPPM_ARR_TILESTART  int32 [ntiles+1] tile offsets of the sorted order
 *   PPPM_ARR_PERM       int32 [n] input index of each sorted particle
 *   PPPM_ARR_SELFFORCE  double [3][2] ad self-force coefficients c[a][n-1]
 *   PPPM_ARR_ENERGY     double [7] energy and virial of the last call */
enum pppm_array {
    PPPM_ARR_RHO = 0, PPPM_ARR_GREEN = 1, PPPM_ARR_FIELD = 2, PPPM_ARR_ANCHOR = 3,
    PPPM_ARR_TILESTART = 4, PPPM_ARR_PERM = 5, PPPM_ARR_SELFFORCE = 6, PPPM_ARR_ENERGY = 7
};
int pppm_get_array(pppm_plan *p, int which, void *dst, size_t bytes, int to_host);

/* Per-stage device timing of pppm_compute with CUDA events recorded on the
 * plan's stream between stages (also inside a captured graph).  Stages:
 * [0] particle_map + sort, [1] make_rho (incl. mesh clear), [2] forward FFT,
 * [3] influence-function multiply + energy/virial, [4] inverse FFT(s),
 * [5] fieldforce.  `stages` is a bitmask (bit s times stage s; 0 = off,
 * 0x3f = all); each event adds a few microseconds to a graph launch, so
 * time only the stages you need.  pppm_stage_times waits for the last
 * profiled call and writes milliseconds (-1 for stages not timed);
 * PPPM_ENOTREADY if profiling was off for it. */
int pppm_set_profiling(pppm_plan *p, int stages);
int pppm_stage_times(pppm_plan *p, float ms[6]);

/* Kernel variants of a plan (Sec. 3.1's mapping functions have one result
 * and several implementations; the paper picks them by measurement, and so
 * does this).  Bit 0: fieldforce stages the tile's field brick in shared
 * memory (1) or reads the field through L1 per particle (0); it applies to
 * force steps -- pppm_energy_grad and pppm_potential always gather the
 * potential through L1.  Bit 1
 * (mesh tiles 16 points long along z) is reserved: refused with PPPM_EINVAL
 * by every plan of this build.  Bit 2: PPPM_FP32C make_rho accumulates in
 * four interleaved copies of the tile brick (no shared-memory bank
 * conflicts, four times the brick's memory) instead of one (PPPM_EINVAL for
 * other precisions).  Bit 3: the Poisson solve (forward FFT, influence
 * function with the energy/virial sums, inverse FFT(s); Sec. 2.1 step 2) runs
 * as three hand-written kernels instead of cuFFT plus two kernels; allowed
 * for PPPM_FP32 / PPPM_FP32C plans whose three mesh edges are each 16, 32, 64
 * or 128, or cubic meshes of edge 48, 96 or 256 (PPPM_EINVAL otherwise).  Results agree with the cuFFT path to FP32
 * rounding.  Bit 4: mesh tiles of 4 points per edge instead of 8 (eight
 * times the tiles and CTAs of the sort, make_rho and the tile-staged
 * fieldforce, a larger halo share); not with bit 1.  Bit 5: make_rho's brick
 * laid out with the strides of the largest tile (compile-time offsets); not
 * with bit 2.  Bit 6: fieldforce runs as a persistent kernel (a few CTAs per
 * SM walk the tiles) whose CTAs stage the next tile's field brick and
 * particle records into a second shared-memory buffer while they gather the
 * current tile (PPPM_FP32 / PPPM_FP32C only; not with bit 0; force steps
 * only, like bit 0; the ad form runs one particle per thread over units of
 * two z-adjacent tiles).  Bit 7: make_rho takes z-pairs of tiles, one
 * brick and one flush per pair (the last tile of a row of an odd number of z
 * tiles alone; not with bits 1, 2, 4).  Default: bit 4 when the mesh has fewer than 304 tiles
 * of 8^3 (two per SM), bit 0 for ik plans whose n_max is at least 16 per
 * tile, bit 3 where it is allowed except on 256^3 meshes (cuFFT measured
 * faster there), bit 5, bit 6 for PPPM_FP32 / PPPM_FP32C ad plans, bit 7
 * unless bit 4 is set.
 * pppm_set_variant forces a bitmask (PPPM_EINVAL for unknown bits or a
 * combination the plan does not allow).
 * pppm_autotune times every variant on the caller's inputs (two warm-up and
 * ten timed pppm_compute steps each, synchronous, as CUDA graphs when the
 * plan's graph mode is on; a variant scores its fastest step), keeps the
 * fastest, writes its bitmask to choice_out (nullable), and leaves f holding
 * a valid result.  Both drop any captured graph. */
int pppm_set_variant(pppm_plan *p, int variants);
/* The plan's current variant bitmask (the default, the last pppm_set_variant
 * or the autotuner's choice) into *variants; PPPM_EINVAL for NULL. */
int pppm_get_variant(const pppm_plan *p, int *variants);

/* Lookup-table stencil coefficients (Sec. 3.1 "precompute", Table 1's LUT-500
 * and LUT-5000): the coefficients are tabulated at `entries` equally spaced
 * offsets and each particle takes the nearest entry -- every per-particle use
 * of the stencil offset (weights, derivative weights, the ad self-force
 * sines) sees the offset rounded to the centre of its bin.  entries = 0
 * restores the exact polynomials (the default); 2 <= entries <= 2^24, else
 * PPPM_EINVAL.  Drops any captured graph. */
int pppm_set_lut(pppm_plan *p, int entries);
int pppm_autotune(pppm_plan *p, int64_t n, const void *x, const void *q, void *f, int *choice_out);

/* Plan facts: [0..2] mesh, [3] order, [4] ntiles, [5] widest tile along z,
 * [6] diff mode, [7] precision, [8] n_max, [9] last n. */
int pppm_plan_info(const pppm_plan *p, int64_t info[10]);

/* Mesh charge density without any device allocation (particle_map, sort and
 * make_rho as in pppm_compute, FP32 arithmetic).  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc where they
 * need the mesh -- a host engine that owns all device memory through its own
 * pool and budget, or a step loop that must not pay the device-wide
 * synchronisation of cudaMalloc/cudaFree.
 *   box[3], mesh[3], order   as for pppm_setup (order 2..7, mesh >= order;
 *                            box edges finite, and L, 1/L and M/L finite
 *                            normal floats)
 *   precision               PPPM_FP32 or PPPM_FP32C
 *   n                       0 <= n <= 65536
 *   x, q                    device, float [n][3] and [n]
 *   rho                     device, float [Mx][My][Mz], overwritten
 *   cuda_stream             stream to enqueue on (NULL = legacy default)
 * Limits: at most 65536 particles and ceil(Mx/8)*ceil(My/8)*ceil(Mz/8) <= 4096
 * mesh tiles (e.g. up to 128^3); larger sizes return PPPM_EINVAL before any
 * GPU work.  The sort scratch is one fixed ~2.1 MiB device array compiled
 * into the library, held on every device that loads it until exit, and shared
 * by all calls: it keeps the previous call's contents (the call clears what
 * must start at zero), and calls that overlap on the GPU race -- serialise
 * them.  The first call on a device looks the array's address up and sets
 * the kernels' shared-memory limits, and both are cached for the process:
 * make that first call before any stream capture, and do not reset the
 * device (cudaDeviceReset) between calls.  Allocates nothing.  Asynchronous:
 * device-side findings (a non-finite position or charge, which is counted as
 * zero; a failed consistency check, whose work is skipped) are only visible
 * through pppm_make_rho_noalloc_status. */
int pppm_make_rho_noalloc(const double box[3], const int mesh[3], int order, int precision,
                          int64_t n, const float *x, const float *q, float *rho,
                          void *cuda_stream);
/* Status of the last pppm_make_rho_noalloc on this device: synchronises
 * cuda_stream (the stream that call used), then returns PPPM_ENONFINITE if it
 * met a non-finite input, PPPM_EINTERNAL if a device consistency check failed,
 * else PPPM_OK (PPPM_ECUDA on a CUDA error).  Call it after the call and
 * before the next one, which clears the word.  Allocates nothing. */
int pppm_make_rho_noalloc_status(void *cuda_stream);

/* ---- Batched path: many independent systems per call -------------------
 * The same three PPPM steps (Sec. 2.1) for nsys unrelated periodic systems
 * of uneven size, mesh and order, advanced together: each stage is one launch
 * over all systems (the paper's mapping functions of Sec. 3.1 run per system
 * inside it), the 3-D FFTs are one batched transform per mesh size, and with
 * graph mode on the whole step is one CUDA graph launch.
 *   box[nsys][3], n[nsys], order[nsys] (2..7), mesh[nsys][3] (>= order,
 *   at most 4096 tiles of 8^3 points each, e.g. 128^3), g_ewald[nsys]
 *   diff_mode, precision, qqrd2e, cuda_stream  as for pppm_setup (shared)
 * pppm_batch_compute takes the systems' particles concatenated in system
 * order: x [sum n][3], q [sum n], f [sum n][3] (device, step type), and ev
 * (device, [nsys][7] energy + virial per system, or NULL).  Asynchronous;
 * pppm_batch_sync reports non-finite inputs like pppm_sync. */
typedef struct pppm_batch pppm_batch;
int pppm_batch_setup(pppm_batch **out, int nsys, const double *box, const int64_t *n, const int *order,
                     const int *mesh, const double *g_ewald, int diff_mode, int precision, double qqrd2e,
                     void *cuda_stream);
int pppm_batch_compute(pppm_batch *b, const void *x, const void *q, void *f, double *ev);
int pppm_batch_set_graph(pppm_batch *b, int enable);
int pppm_batch_sync(pppm_batch *b);
/* Kernel variants of a batch: bit P (P = 2..7) makes the FP32C make_rho of
 * the order-P systems accumulate in four interleaved brick copies (see
 * pppm_set_variant bit 2; PPPM_EINVAL for other precisions); bit 8 + P runs
 * the order-P fieldforce tile-staged, one CTA per system tile staging its
 * field brick in shared memory (see pppm_set_variant bit 0; any precision);
 * bit 16 + P runs the order-P make_rho over z-pairs of tiles, one CTA per
 * pair (see pppm_set_variant bit 7; any precision; not with bit P).
 * PPPM_EINVAL for other bits or both of bits P and 16 + P.  Default: bits
 * 16 + P of every order (0xFC0000).
 * pppm_batch_autotune times the whole call as the batch runs it (one graph
 * per setting when graph mode is on; one warm-up and five timed calls,
 * scored by the fastest) with each present order's tile-pair bit, brick-copy
 * bit (FP32C only) and fieldforce bit flipped in turn (a flip that would set
 * both make_rho bits is skipped), keeps every flip that is faster, writes
 * the mask to choice_out (nullable) and leaves f holding a valid result.
 * Both drop the captured graph. */
int pppm_batch_set_variant(pppm_batch *b, int variants);
/* The batch's current variant bitmask (the default, the last
 * pppm_batch_set_variant or the autotuner's choice) into *variants;
 * PPPM_EINVAL for NULL. */
int pppm_batch_get_variant(const pppm_batch *b, int *variants);
int pppm_batch_autotune(pppm_batch *b, const void *x, const void *q, void *f, int *choice_out);
/* [0] systems, [1] total particles, [2] mesh-size classes, [3] distinct orders */
int pppm_batch_info(const pppm_batch *b, int64_t info[4]);
int pppm_batch_destroy(pppm_batch *b);

/* ------------------------------------------------------------------------
 * Real-space part of the Ewald split (Sec. 2.1: the short-range erfc(g r)/r
 * interaction, summed directly within the cut-off r_C).  With the k-space
 * result of a plan of the same g_ewald and qqrd2e it gives the total Coulomb
 * energy, forces and virial of the periodic system:
 *   E    = (C/2) sum_i sum_{j != i, r_ij < r_C} q_i q_j erfc(g r_ij)/r_ij
 *   F_i  = C q_i sum_j q_j [erfc(g r)/r + 2g/sqrt(pi) exp(-g^2 r^2)] r_ij/r^2
 *   W_ab = (1/2) sum_i sum_j (F_ij)_a (r_ij)_b       (r_ij = r_i - r_j)
 * over minimum images; r_cut must be below half of every box edge
 * (PPPM_EINVAL otherwise).  Orthorhombic box at the origin, positions
 * wrapped.  precision: PPPM_FP64 (double) or PPPM_FP32 / PPPM_FP32C (float;
 * the same float path).  pppm_real_compute: x [n][3], q [n], f [n][3] device
 * buffers of the step type (caller-owned); f is overwritten, or added to when
 * accumulate != 0 (e.g. onto pppm_compute's k-space forces); ev (device, 7
 * doubles, nullable) receives energy then virial xx yy zz xy xz yz.
 * Asynchronous on the stream given at setup; pppm_real_sync reports the
 * device error word like pppm_sync.  info: cells per dimension, n_max. */
typedef struct pppm_real pppm_real;
int pppm_real_setup(pppm_real **out, const double box[3], int64_t n_max, double r_cut, double g_ewald,
                    int precision, double qqrd2e, void *cuda_stream);
int pppm_real_compute(pppm_real *r, int64_t n, const void *x, const void *q, void *f, int accumulate,
                      double *ev);
int pppm_real_sync(pppm_real *r);
int pppm_real_info(const pppm_real *r, int64_t info[4]);
int pppm_real_destroy(pppm_real *r);

/* Static description of a status code (never NULL). */
const char *pppm_strerror(int status);

/* Name and description of the last CUDA runtime error this library saw on
 * the calling thread, or of the pending (sticky) CUDA error, "" if none.
 * Points to thread-local storage that the next call overwrites. */
const char *pppm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PPPM_GB300_H */
