/*
 * cwthf.h -- C ABI of libcwthf.so, the GB300 (sm_103a) implementation of the
 * single-scale hot path of CWTHF, the continuous-wavelet-transform halo finder
 * of Li, Wang & He (arXiv:2501.10622).
 *
 * The path, in the order of the paper's step list (Sec. 2):
 *   cwthf_deposit    Sec. 2.1, Eq. 1   cloud-in-cell mass grid (int64 fixed point)
 *   cwthf_transform  Sec. 2.1, Eq. 2-4 grid CWT with the 3D Mexican-hat wavelet
 *   cwthf_segment    Sec. 2 steps 4-5, Sec. 2.3  26-neighbour maxima and
 *                                      steepest-ascent segments of the CWT
 *   cwthf_assign     Sec. 2 steps 6-7, Sec. 2.3-2.4, Table 1  particles to
 *                                      segments, per-halo sums, thresholds
 *   cwthf_find       all of the above, for one or more wavelet scales
 *
 * Conventions shared by every entry point
 *   - Grids are row-major [z][y][x] with x fastest; grid node g sits at
 *     g * (L / ng) in a periodic box of side L.  ng must be even with
 *     8 <= ng <= 1152 (cwthf_check_ng tells), otherwise
 *     CWTHF_E_UNSUPPORTED_SIZE.  Pass lengths (ng along y and z, ng / 2 for
 *     the paired real samples along x) whose factors are all radices of
 *     2, 3, 5, 7 run mixed-radix FFTs; any other length (a prime factor above
 *     7, or no tile that fits the kernels) runs a Bluestein (chirp-z) pass
 *     through an inner FFT of length >= 2 n - 1.
 *   - Positions are float [np][3] (x, y, z), in the units of L.  Any finite
 *     value with |x * ng / L| < 2^30 is accepted and wrapped into the box;
 *     others make the call fail with CWTHF_E_BAD_INPUT (reported by
 *     cwthf_sync, see below).
 *   - Positions are quantised to CWTHF_FRAC_BITS fractional bits of a cell:
 *     q = floor(x * s) mod ng*2^10, where s = (ng / L) * 2^10 is formed in
 *     fp64 and rounded to 29 significant bits, so that x * s is exact (the
 *     device forms it as one 32 x 32 -> 64-bit integer product).
 *   - Masses: mass == NULL means every particle has mass mass_unit.
 *     Otherwise particle i has integer mass m_q = rint(mass[i] / mass_unit)
 *     in units of mass_unit; 0 <= m_q < 2^31 is required per particle and
 *     sum m_q < 2^33 in total (CWTHF_E_OVERFLOW), which keeps every int64
 *     grid cell exact.
 *   - Every pointer argument named *device* is device memory owned by the
 *     caller, and must stay valid until the work queued on `stream` is done.
 *     `stream` is a cudaStream_t (NULL = legacy default stream).  All calls
 *     are asynchronous with respect to the host.
 *   - Return values: CWTHF_OK, or an error detected on the host before any
 *     work is queued (nothing was queued then).  Errors that only the GPU can
 *     see (bad positions, int64 budget, capacity, convergence) are recorded
 *     in the context's status word and returned by the next cwthf_sync().
 *   - A context serialises its own scratch memory: calls that share a
 *     context must be issued on one stream (or be otherwise ordered).
 *   - Nothing throws across this ABI; no function calls exit().
 */
#ifndef CWTHF_H
#define CWTHF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CWTHF_API __attribute__((visibility("default")))
#else
#define CWTHF_API
#endif

#define CWTHF_FRAC_BITS 10
#define CWTHF_MAX_NG 1152
#define CWTHF_MIN_NG 8
#define CWTHF_MAX_STENCIL_R 64

enum {
    CWTHF_OK = 0,
    CWTHF_E_INVALID_ARG = 1,      /* NULL pointer, non-positive size or box, ... */
    CWTHF_E_UNSUPPORTED_SIZE = 2, /* ng odd or out of range (see above), or above the context's limits */
    CWTHF_E_OVERFLOW = 3,         /* integer mass budget: m_q >= 2^31 or sum m_q >= 2^33 */
    CWTHF_E_OOM = 4,              /* device allocation failed in cwthf_create */
    CWTHF_E_CUDA = 5,             /* a CUDA runtime call failed */
    CWTHF_E_NOT_CONVERGED = 6,    /* label propagation hit its round limit */
    CWTHF_E_TIMEOUT = 7,          /* a bounded device wait gave up */
    CWTHF_E_CAPACITY = 8,         /* more halos than cat_cap; the count is still reported */
    CWTHF_E_BAD_INPUT = 9,        /* non-finite or out-of-range position / mass / CWT value */
    CWTHF_E_SCRATCH_LIMIT = 10,   /* too large for cwthf_deposit_noalloc's fixed scratch */
    CWTHF_E_TABLE_CACHE = 11,     /* no FFT / wavelet table slot left (see cwthf_create) */
    CWTHF_E_INDEX = 12            /* checked builds only: a data-driven index was out of range; its
                                     access was skipped and the call's results are unspecified */
};

typedef struct cwthf_ctx cwthf_ctx;

/* Per-scale parameters (Table 1 of the paper gives dens_th = 4 and
 * particle_th = 15; Sec. 2.3 seeds halos at positive CWT peaks, cwt_min = 0). */
typedef struct {
    double w;            /* wavelet scale in 1/length (k_w = w * L / 1000, Sec. 2 footnote) */
    float cwt_min;       /* a maximum seeds a halo iff its CWT value > cwt_min */
    float reserved0;
    double dens_th;      /* keep iff segment mass / (n_cells * cell volume) >= dens_th * mean density */
    int64_t particle_th; /* keep iff the halo has >= particle_th particles */
} cwthf_params;

/* One halo of the catalogue (64 bytes).  Halos are sorted by seed. */
typedef struct {
    int64_t seed;      /* linear index (z*ng + y)*ng + x of the maximum that seeds the halo */
    int64_t n_part;    /* particles assigned to the halo */
    int64_t n_cells;   /* grid cells of its segment (the "grid volume" of Sec. 2.4) */
    double mass;       /* sum of particle masses (m_q * mass_unit) */
    double centre[3];  /* centre of mass (Sec. 2.3), minimum image about the seed, in [0, L) */
    float peak;        /* CWT value at the seed */
    int32_t reserved;
} cwthf_halo;

/* One halo of the multi-scale catalogue (64 bytes), in halo-id order. */
typedef struct {
    int64_t seed;      /* linear index of the seed on its scale's ng^3 grid */
    int64_t n_part;    /* particles of the halo (none of which an earlier scale took) */
    int64_t n_cells;   /* cells of its segment on its scale's grid */
    double mass;       /* sum of particle masses */
    double centre[3];  /* centre of mass, minimum image about the seed, in [0, L) */
    float peak;        /* corrected peak (App. B): the value compared across scales */
    int32_t scale;     /* index of the scale that found it */
} cwthf_ms_halo;

/* Fills *p with the defaults above for scale w. */
CWTHF_API void cwthf_default_params(double w, cwthf_params *p);

/* Creates a context on `device` with scratch for grids up to max_ng and up
 * to max_np particles; max_scales (>= 1) is the largest scale count a
 * cwthf_find call will use (scales beyond the first need a second complex
 * workspace).  Allocates all device memory up front (cudaMalloc), so later
 * calls allocate nothing.  Returns CWTHF_E_OOM if that fails (nothing is
 * leaked), CWTHF_E_CUDA if the device cannot be used.
 * The context keeps 48 slots for the FFT twiddles (one per grid size) and the
 * wavelet spectra (one per grid size, box and scale) that the transform
 * needs.  A call that needs a table not yet held computes it on the host in
 * fp64 and queues one copy on its stream; a full cache reuses the least
 * recently used slot (waiting, on the host, for that slot's previous copy).
 * A slot used by work captured into a CUDA graph is kept for the context's
 * lifetime.  A captured call records the host-to-device copy of every table
 * it needs that no uncaptured call has copied yet, so such a graph is self-
 * contained; tables already copied (by cwthf_prepare or an earlier call) are
 * only read by the graph, and those copies must have completed before the
 * graph runs.  During a capture, a call that needs a new table while no slot
 * is free fails with CWTHF_E_TABLE_CACHE (nothing queued). */
CWTHF_API int cwthf_create(int device, int max_ng, int64_t max_np, int max_scales, cwthf_ctx **out);
/* Optional parts of a context, for cwthf_create_ex and cwthf_workspace_bytes_ex. */
#define CWTHF_CREATE_UNBIND 1u /* scratch of the self-boundness check: 36 bytes per particle + 24 per group + 2.2 MB */
/* cwthf_create with optional parts (flags: CWTHF_CREATE_*; unknown bits ->
 * CWTHF_E_INVALID_ARG).  cwthf_create is this with flags 0. */
CWTHF_API int cwthf_create_ex(int device, int max_ng, int64_t max_np, int max_scales, unsigned flags,
                              cwthf_ctx **out);
CWTHF_API void cwthf_destroy(cwthf_ctx *ctx);

/* Device bytes a context created with these limits holds (for admission
 * against a memory budget).  Host-only; needs no GPU. */
CWTHF_API int cwthf_workspace_bytes(int max_ng, int64_t max_np, int max_scales, size_t *out);
CWTHF_API int cwthf_workspace_bytes_ex(int max_ng, int64_t max_np, int max_scales, unsigned flags, size_t *out);

/* Checks a grid size against the supported set (CWTHF_OK or
 * CWTHF_E_UNSUPPORTED_SIZE).  Host-only. */
CWTHF_API int cwthf_check_ng(int ng);

/* Sec. 2.1, Eq. 1.  CIC deposit of np particles onto the periodic ng^3 grid.
 *   pos   device, float [np][3]
 *   mass  device, float [np], or NULL (all masses equal mass_unit)
 *   grid  device, int64 [ng][ng][ng]; fully overwritten with the CIC mass in
 *         units of mass_unit * 2^-30 (each particle spreads m_q * 2^30 over
 *         at most 8 nodes with integer weights); bit-exact and independent
 *         of particle order.
 *   mtot  device, int64 [1] or NULL: receives sum_i m_q. */
CWTHF_API int cwthf_deposit(cwthf_ctx *ctx, const float *pos, const float *mass, double mass_unit, int64_t np,
                  double L, int ng, int64_t *grid, int64_t *mtot, void *stream);

/* Fills the context's table slots (see cwthf_create) with the FFT twiddles
 * of grid size ng and the wavelet spectra of the n_scales scales w[] (host,
 * double [n_scales]) for a box of side L, so that later calls with these
 * parameters do no host-side table work.  Queues one small copy per new table
 * on `stream`.  Errors: as cwthf_transform, and CWTHF_E_TABLE_CACHE. */
CWTHF_API int cwthf_prepare(cwthf_ctx *ctx, int ng, double L, const double *w, int n_scales, void *stream);

/* Sec. 2.1, Eq. 2-4.  Grid CWT at scale w of the CIC mass grid: the circular
 * convolution C(x_g) = sum_g' m_g' Psi(w, x_g - x_g') with the Mexican hat
 * Psi(w, r) = w^1.5 (6 - w^2 r^2) exp(-w^2 r^2 / 4) sampled at minimum-image
 * node offsets, computed as a forward 3D real FFT, a multiply by the exact
 * DFT of the sampled wavelet, and an inverse FFT, in fp32.
 *   grid  device, int64 [ng^3] as written by cwthf_deposit (units mass_unit*2^-30)
 *   cwt   device, float [ng][ng][ng]; overwritten.  Must not alias grid. */
CWTHF_API int cwthf_transform(cwthf_ctx *ctx, const int64_t *grid, int ng, double L, double mass_unit, double w,
                    float *cwt, void *stream);

/* Sec. 2.1 as the paper evaluates the grid CWT: every node adds its mass
 * times the wavelet sampled on the grid around it, over the cube of offsets
 * |d_x|, |d_y|, |d_z| <= R (Table 1's gdw_resolution = Int(1.5 / k_w + 5),
 * read as the cube's radius), periodic:
 *   C(x_g) = sum_{|d| <= R per axis} m_{g - d} Psi(w, (L / ng) |d|).
 * Computed exactly separably (the Mexican hat restricted to a cube is a sum
 * of products of 1D factors) as seven 1D convolutions in three passes, fp32.
 * For R large enough that the wavelet vanishes beyond the cube this equals
 * cwthf_transform.
 *   grid  device, int64 [ng^3] as written by cwthf_deposit
 *   R     0 <= R <= CWTHF_MAX_STENCIL_R and 2R + 1 <= ng (CWTHF_E_INVALID_ARG)
 *   cwt   device, float [ng][ng][ng]; overwritten.  Must not alias grid.
 * Uses the context's grid, CWT and label scratch. */
CWTHF_API int cwthf_transform_stencil(cwthf_ctx *ctx, const int64_t *grid, int ng, double L, double mass_unit,
                                      double w, int R, float *cwt, void *stream);

/* Sec. 2 steps 4-5, Sec. 2.3.  Every cell points at the best of itself and
 * its 26 periodic neighbours under the strict order (C[a] > C[b]) or
 * (C[a] == C[b] and a < b); chains end at local maxima.  A maximum with
 * C > cwt_min seeds a segment; every cell gets the linear index of the seed
 * its chain reaches, or -1.
 *   cwt         device, float [ng^3] (NaN -> CWTHF_E_BAD_INPUT)
 *   cell_label  device, int32 [ng^3]; overwritten. */
CWTHF_API int cwthf_segment(cwthf_ctx *ctx, const float *cwt, int ng, float cwt_min, int32_t *cell_label,
                  void *stream);

/* Sec. 2.4 (the "grid volume" of a segment).  The seeds found by the last
 * cwthf_segment call on this context, in increasing cell order, and the
 * number of cells labelled with each.  Valid until the next call on the
 * context; queue it on the segmentation's stream.
 *   seeds    device, int32 [cap]: linear index of each seed
 *   n_cells  device, int64 [cap]: cells of its segment
 *   n_seeds  device, int64 [1]: the number of seeds (may exceed cap; only
 *            the first cap are written). */
CWTHF_API int cwthf_segment_sizes(cwthf_ctx *ctx, int32_t *seeds, int64_t *n_cells, int64_t cap, int64_t *n_seeds,
                                  void *stream);

/* Sec. 2 steps 6-7, Sec. 2.3-2.4, Table 1.  Each particle takes the label of
 * its nearest node ((q + 2^9) >> 10 per axis, wrapped).  Per seed: particle
 * count, integer mass, integer first moment about the seed node (minimum
 * image) and the number of cells with its label.  A seed is kept iff
 * n_part >= particle_th and (double)M_halo * ng^3 >= (dens_th * (double)M_tot)
 * * n_cells in integer mass units (M_tot = all particles).  Kept halos are
 * written to cat in increasing seed order; halo_id[i] is the particle's seed
 * or -1.
 *   pos, mass, mass_unit, np, L, ng  as for cwthf_deposit (same quantisation)
 *   cell_label  device, int32 [ng^3] from cwthf_segment
 *   cwt         device, float [ng^3] or NULL (then cat[].peak = 0)
 *   params      host; w is ignored here
 *   halo_id     device, int32 [np]; overwritten (unspecified when the call fails)
 *   cat         device, cwthf_halo [cat_cap]
 *   n_halo      device, int64 [1]: the number of kept halos (even when it
 *               exceeds cat_cap, which also records CWTHF_E_CAPACITY). */
CWTHF_API int cwthf_assign(cwthf_ctx *ctx, const float *pos, const float *mass, double mass_unit, int64_t np, double L,
                 int ng, const int32_t *cell_label, const float *cwt, const cwthf_params *params,
                 int32_t *halo_id, cwthf_halo *cat, int64_t cat_cap, int64_t *n_halo, void *stream);

/* The whole path for n_scales wavelet scales on one particle set: one
 * deposit and one forward transform shared by all scales, then per scale the
 * wavelet multiply, inverse transform, segmentation and assignment.
 *   params   host, cwthf_params [n_scales]
 *   halo_id  device, int32 [n_scales][np]
 *   cat      device, cwthf_halo [n_scales][cat_cap]
 *   n_halo   device, int64 [n_scales]
 * Intermediate grids live in the context (n_scales <= max_scales). */
CWTHF_API int cwthf_find(cwthf_ctx *ctx, const float *pos, const float *mass, double mass_unit, int64_t np, double L,
               int ng, const cwthf_params *params, int n_scales, int32_t *halo_id, cwthf_halo *cat,
               int64_t cat_cap, int64_t *n_halo, void *stream);

/* Sec. 2 (step list 1-10), Fig. 1, Sec. 2.2 with App. B, Sec. 2.3, Sec. 2.4: the multi-scale
 * identification loop.  Scales are given from the largest physical scale
 * (smallest k_w) to the smallest: w[j] (1/length) on an ng[j]^3 grid (each a
 * supported size <= the context's max_ng; the paper's Int(400 k_w + 150)
 * rounded to an even size is the caller's choice).  For every scale all
 * particles are deposited and the CWT computed; scale j is then decided with
 * scale j + 1's field as its comparison field (a zero field after the last):
 *   - segments of scale j's field (seeds: maxima above cwt_min);
 *   - groups: the particles that hold no halo id yet, by the label of their
 *     nearest node; per group count, mass, first moment; n_cells of the segment;
 *   - a group is kept iff n_part >= particle_th, its mass over its segment's
 *     volume is >= dens_th times the mean density of all particles, and its
 *     seed is a maximum across scales: the seed's corrected peak (App. B:
 *     the node value plus l1^2 / (16 l2 - 8 l1) per axis, plus
 *     (5/16)(2 mean l2 - mean l1)(1 - (ng[j]/ng[j+1])^2)) exceeds the 2x2x2
 *     nodes of scale j+1's field enclosing the seed's position (exceeds 0
 *     after the last scale);
 *   - with vel given (step 9), the particles of every kept group pass the
 *     self-boundness check of cwthf_unbind (G, at most max_iter rounds): a
 *     group that loses more than 40 % of them is dropped, and a kept group's
 *     n_part, mass and centre are summed again over the members that stay
 *     (the thresholds above are not applied again);
 *   - kept groups, in seed order, take the next halo ids; their particles
 *     (with vel: the members that stayed) keep them for good; the others
 *     remain free for the later scales.
 *   vel       device, float [np][3] (velocities, the units of G), or NULL:
 *             no self-boundness check; needs a context created with
 *             CWTHF_CREATE_UNBIND
 *   w, ng     host, [n_scales], n_scales >= 1
 *   halo_id   device, int32 [np]: the particle's halo id, or -1
 *   cat       device, cwthf_ms_halo [cat_cap], halos in id order
 *   n_halo    device, int64 [1]: halos found (CWTHF_E_CAPACITY beyond cat_cap)
 * Needs a context created with max_scales >= 2 (two fields are kept). */
CWTHF_API int cwthf_find_multiscale(cwthf_ctx *ctx, const float *pos, const float *mass, double mass_unit,
                                    int64_t np, double L, int n_scales, const double *w, const int *ng,
                                    float cwt_min, double dens_th, int64_t particle_th, const float *vel, double G,
                                    int max_iter, int32_t *halo_id, cwthf_ms_halo *cat, int64_t cat_cap,
                                    int64_t *n_halo, void *stream);

/* Sec. 2.3 (step 9 of the Sec. 2 step list): the self-boundness check of
 * every group, each on its own:
 *   1. centre = the centre of mass of the group's current members (mass-weighted
 *      minimum-image offsets from the group's first member in particle order);
 *   2. spherical symmetry: the potential at member i is that of the other
 *      members' shells about the centre, Phi_i = -G sum_{j != i} m_j / max(r_i,
 *      r_j) (shell theorem), the local escape speed sqrt(-2 Phi_i);
 *   3. members whose speed relative to the group's mass-weighted mean velocity
 *      exceeds it are excluded, all at once, and the centre is recomputed;
 *   4. repeated until nothing is excluded, at most max_iter rounds;
 *   5. a group that lost more than 40 % of its particles is discarded.
 * Masses are the deposit's integer quanta times mass_unit (mass_unit each when
 * mass is NULL).  A group whose extent reaches half the box is not supported
 * (offsets are minimum images).
 *   pos, vel    device, float [np][3]: positions (units of L), velocities
 *   mass        device, float [np] or NULL
 *   G           the gravitational constant in the caller's units (e.g.
 *               4.30091727e-9 for Mpc/h, km/s and Msun/h)
 *   group       device, int32 [np]: the particle's group, or -1 (ignored)
 *   n_groups    groups 0 .. n_groups-1 (at most max_ng^3 / 8 + 8)
 *   group_out   device, int32 [np]: the group after the check, or -1
 *   n_kept      device, int64 [n_groups]: members kept (0 when discarded)
 *   iters       device, int32 [n_groups]: rounds run
 * Each group's sums run in a fixed order, so results repeat exactly; a member
 * exactly at its escape speed within fp64 rounding may fall either way.
 * Invalid masses are reported as in cwthf_deposit.  Needs a context created
 * with CWTHF_CREATE_UNBIND (else CWTHF_E_INVALID_ARG). */
CWTHF_API int cwthf_unbind(cwthf_ctx *ctx, const float *pos, const float *vel, const float *mass, double mass_unit,
                           int64_t np, double L, double G, const int32_t *group, int64_t n_groups, int max_iter,
                           int32_t *group_out, int64_t *n_kept, int32_t *iters, void *stream);

/* Waits for `stream`, then returns (and clears) the first error the device
 * recorded since the last cwthf_sync, or CWTHF_E_CUDA if the stream failed.
 * After CWTHF_E_TIMEOUT or CWTHF_E_NOT_CONVERGED every output of the calls
 * since the previous cwthf_sync is unspecified. */
CWTHF_API int cwthf_sync(cwthf_ctx *ctx, void *stream);

/* Static English text for a status code. */
CWTHF_API const char *cwthf_error_string(int code);

/* Number of kernel launches queued by this context since it was created
 * (instrumentation for launch accounting). */
CWTHF_API int64_t cwthf_launch_count(const cwthf_ctx *ctx);

/* The CIC deposit of cwthf_deposit without a context and without any device
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- for example code recorded
 * into a CUDA graph while a stream is being captured (allocation calls are
 * not capturable), or hosts whose device memory belongs to another allocator
 * or pool, or loops that must not pay the device synchronisation of
 * cudaMalloc / cudaFree.  The caller passes inputs and outputs as for
 * cwthf_deposit (same arguments, same bit-exact grid); the binning scratch is
 * a fixed array inside the library (about 3.3 MB, held on every GPU that
 * uses the library until the process exits).
 *   ng <= 128 and np <= 262144, else CWTHF_E_SCRATCH_LIMIT (nothing queued).
 *   status  device, int [1] or NULL: receives the device-detected status of
 *           this call (CWTHF_OK, CWTHF_E_BAD_INPUT, CWTHF_E_OVERFLOW) once the
 *           stream reaches it.
 * Runs on the current device.  Every call shares the one scratch array, so
 * calls whose GPU work overlaps (other streams, other host threads) race and
 * corrupt each other's result: keep them ordered on one stream.  A call made
 * outside a stream capture looks up the array's device address; a call made
 * while its stream is being captured reuses the last address found on that
 * device, so make one call on each device before any stream capture. */
CWTHF_API int cwthf_deposit_noalloc(const float *pos, const float *mass, double mass_unit, int64_t np, double L,
                                    int ng, int64_t *grid, int64_t *mtot, int *status, void *stream);

/* Tuning: the FFT plan this context uses for grid size ng instead of its
 * built-in rule (the paper has no counterpart; an autotuner picks plans by
 * timing them).
 *   which      0: the y/z passes (length ng), 1: the x passes (length ng / 2)
 *   C          sequences per tile: 2, 4, 8 or 16
 *   radices    host, int [n_radices]: 1-3 radices from {2, 3, 4, 5, 6, 7, 8, 9,
 *              10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 30, 32} whose
 *              product is the length, applied in this order
 *   n_radices  0 returns the pass to the built-in rule
 * A plan the kernels cannot run (product, tile over 64 KB, over 512 threads, no
 * TMA box for the y/z tile) is refused with CWTHF_E_INVALID_ARG, so a pass
 * whose length has a prime factor above 7 keeps its Bluestein plan.  Results
 * change only by fp32 rounding; set plans between calls, not while work of
 * this context is being enqueued. */
CWTHF_API int cwthf_set_fft_plan(cwthf_ctx *ctx, int ng, int which, int C, const int *radices, int n_radices);

/* Test and fault-injection settings of a context (instrumentation; the paper
 * has no counterpart).  They let a test reach the library's error paths
 * without faulting the GPU.  Keys and values:
 *   CWTHF_DEBUG_JUMP_ROUNDS  0..31 (default 31): pointer-doubling rounds the
 *       segmentation may run after its bounded chain walks; a chain still
 *       unfinished after them is reported as CWTHF_E_NOT_CONVERGED.
 *   CWTHF_DEBUG_CHASE_LIMIT  1..64 (default 64): steps of the bounded chain
 *       walks across segmentation tiles before the doubling rounds take over.
 *   CWTHF_DEBUG_TMA_NO_COPY  nonzero: in the next y/z FFT pass of this
 *       context, one CTA arms its transfer barrier but issues no copy, so its
 *       bounded wait runs out (nothing is in flight) and the call reports
 *       CWTHF_E_TIMEOUT.  One-shot.
 *   CWTHF_DEBUG_FALLBACK_RAN (get only): 1 if the last segmentation needed
 *       the doubling rounds (a chain outlived the bounded walks), else 0;
 *       waits for `stream`.
 *   CWTHF_DEBUG_TABLE_FILLS (get only): table slots filled since the context
 *       was created (each a host-side table computation and one copy).
 *   CWTHF_DEBUG_CHECKED (get only): 1 if this library is the range-checked
 *       build (compiled with CWTHF_CHECKED: every data-driven index -- record
 *       slots, label and chain targets, seed slots, group members -- is tested
 *       before use, and one out of range is skipped and reported as
 *       CWTHF_E_INDEX), else 0.
 *   CWTHF_DEBUG_UNBIND_GRID_MIN  1..2^31-1 (default 65536): groups of the
 *       self-boundness check with more members than this are processed by
 *       the whole grid (one cooperative launch, one group at a time), smaller
 *       ones by one CTA each; both give the same decisions up to rounding.
 * cwthf_debug_set returns CWTHF_E_INVALID_ARG for an unknown key or a value
 * out of range; settings persist for the context's lifetime. */
#define CWTHF_DEBUG_JUMP_ROUNDS 1
#define CWTHF_DEBUG_CHASE_LIMIT 2
#define CWTHF_DEBUG_TMA_NO_COPY 3
#define CWTHF_DEBUG_FALLBACK_RAN 4
#define CWTHF_DEBUG_TABLE_FILLS 5
#define CWTHF_DEBUG_UNBIND_GRID_MIN 6
#define CWTHF_DEBUG_CHECKED 7
CWTHF_API int cwthf_debug_set(cwthf_ctx *ctx, int key, int64_t value);
CWTHF_API int cwthf_debug_get(cwthf_ctx *ctx, int key, int64_t *value, void *stream);

/* Per-kernel timing (instrumentation).  With enable != 0 every later kernel
 * launch of this context is bracketed by two CUDA events recorded on its own
 * stream; any call clears the totals.  Do not enable it while a stream is
 * being captured into a CUDA graph.
 * cwthf_profile_count waits for the recorded events, folds them into the
 * per-kernel totals and returns the number of distinct kernels seen (or a
 * negative CWTHF_E_* code); cwthf_profile_read then returns kernel i's name
 * (a static string), summed device time in ms and launch count. */
CWTHF_API int cwthf_profile(cwthf_ctx *ctx, int enable);
CWTHF_API int cwthf_profile_count(cwthf_ctx *ctx);
CWTHF_API int cwthf_profile_read(const cwthf_ctx *ctx, int i, const char **name, double *total_ms,
                                 int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* CWTHF_H */
