/*
 * rt.h -- C ABI of the B300 column radiative-transfer library.
 *
 * The library solves, for every atmospheric column, every k-table bin and
 * every Gauss point (one "system"), the improved two-stream equations with
 * multiple scattering of Deitrick et al., "The THOR+HELIOS general
 * circulation model" (arXiv 2203.02293), Sec. 2.2 and App. B, by a
 * tridiagonal (Thomas) elimination over the layer interfaces (Sec. 2.2.2,
 * Eqs. 12-15), then sums the systems over Gauss points and bins (Sec. 2.2.6)
 * into interface fluxes, net flux (stellar beam added to the downward flux,
 * Sec. 2.2.1) and a heating rate per layer (App. A: Q depends on the
 * vertical gradient of the net flux).
 *
 * Conventions
 *   - Every call returns an rt_status (0 = RT_OK); rt_last_error() gives a
 *     one-line reason for the last failure on that handle.
 *   - Layer 0 and interface 0 are at the top of the atmosphere (TOA);
 *     interface L is the bottom (BOA).  Optical depth grows with the index.
 *   - Device pointers are CUDA device memory owned by the caller and must
 *     stay valid until the work enqueued on the stream has finished.  Host
 *     pointers are read before the call returns.
 *   - Work is asynchronous on the caller's CUDA stream (cudaStream_t passed
 *     as void*; NULL = the legacy default stream).  Only rt_stats(),
 *     rt_kernel_times() and rt_set_ktable() synchronise.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - Nothing in the library calls back into the host or waits on the
 *     device inside a kernel; no kernel spins.
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_handle rt_handle;

typedef enum {
    RT_OK = 0,
    RT_EINVAL = -1,       /* malformed argument: shape, pointer, range */
    RT_ENOMEM = -2,       /* device or pinned-host allocation failed */
    RT_ECUDA = -3,        /* a CUDA call failed (message in rt_last_error) */
    RT_ENOTSOLVED = -4,   /* rt_fluxes / rt_heating before a successful solve */
    RT_EBUDGET = -5,      /* workspace would exceed hbm_budget_bytes */
    RT_ETIMEOUT = -6      /* reserved for bounded device waits (none today) */
} rt_status;

/* Two-stream closure (Sec. 2.2.4, Eq. 19): improved = E from the fit for
 * w0 > 0.1 and E = 1 otherwise; regular = E = 1 everywhere. */
enum { RT_IMPROVED = 0, RT_REGULAR = 1 };
/* Layer model (Sec. 2.2.1): non-isothermal layers are split into two
 * sub-layers with a linear Planck function in optical depth; isothermal
 * layers carry one Planck value at the layer centre. */
enum { RT_NONISOTHERMAL = 0, RT_ISOTHERMAL = 1 };
/* Arithmetic of the solve: FP32 cancellation-free form (FP64 only for the
 * resonance test near |D| = 1e-5), or FP64 with the paper's literal
 * formulas. */
enum { RT_FP32_FORM = 0, RT_FP64_PLAIN = 1 };
/* Where the FP32 solve gets the bin-integrated Planck values (no effect on
 * results, which are bitwise the same every way). */
enum { RT_STAGE_AUTO = 0, RT_STAGE_SHARED = 1, RT_STAGE_DIRECT = 2, RT_STAGE_INLINE = 3 };
/* Beam singularity of Eq. B8 at D = 4 E mu*^2 (E - w0)(1 - w0 g0) - 1 = 0
 * (Eq. 11): PAPER switches D to 2 mu* when |D| < 1e-5 (text after Eq. 11);
 * LIMIT uses the exact (finite) solution at every mu*. */
enum { RT_RESONANCE_PAPER = 0, RT_RESONANCE_LIMIT = 1 };

typedef struct {
    int32_t n_g;                 /* Gauss points per bin, 1..64 */
    const double *g_weights;     /* HOST [n_g], copied by rt_create; should sum to 1 */
    double wn_min, wn_max;       /* bin range in cm^-1; a column with NB bins uses NB
                                    bins of equal width in wavenumber (Sec. 2.1.3) */
    int32_t two_stream;          /* RT_IMPROVED | RT_REGULAR */
    int32_t layers;              /* RT_NONISOTHERMAL | RT_ISOTHERMAL */
    int32_t precision;           /* RT_FP32_FORM | RT_FP64_PLAIN */
    int32_t resonance;           /* RT_RESONANCE_PAPER | RT_RESONANCE_LIMIT */
    int32_t e_clamp;             /* 1: E := max(E_fit, 1); 0: raw fit (may give NaN) */
    double eps2;                 /* second Eddington coefficient, Table 3: 2/3 (App. B) */
    double grav, cp;             /* m s^-2 and J kg^-1 K^-1 for the heating rate (Table 3) */
    double T_int;                /* K; F_BOA = pi B(T_int) per bin (Eq. 10); 0 gives 0 */
    double F_toa_diffuse;        /* W m^-2 diffuse downward flux imposed at the TOA of
                                    every (bin, g) system (caption of the matrix-form
                                    figure of Sec. 2.2); normally 0 */
    int32_t max_layers;          /* largest L of any column, 1..1024 */
    int32_t max_bins;            /* largest NB of any column, >= 1 */
    size_t hbm_budget_bytes;     /* workspace cap; 0 = no cap */
    int32_t block_threads;       /* threads per CTA (multiple of 32; 64..256 for the FP32
                                    form, 64..512 for FP64); 0 = default (128 for the
                                    FP32 form, 256 for FP64) */
    int32_t ctas_per_sm;         /* cap on resident CTAs per SM of the persistent grid;
                                    0 = as many as fit */
    int32_t planck_staging;      /* FP32 form, where the solve gets B(T) per bin:
                                    RT_STAGE_AUTO, RT_STAGE_SHARED (a pre-kernel
                                    tabulates B per column and level; staged per
                                    warp in shared memory; pays off when many
                                    g-points share a bin), RT_STAGE_DIRECT (read
                                    from that table in device memory) or
                                    RT_STAGE_INLINE (no table: the solve kernel
                                    evaluates B for each system at each level;
                                    for one g-point on narrow bins, where the
                                    table's write and reads cost more than the
                                    sums).  AUTO: INLINE for n_g = 1 with
                                    explicit edges all at most 1% of their lower
                                    edge apart, else DIRECT for n_g < 4, else
                                    SHARED */
    int32_t systems_per_lane;    /* FP32 form: systems each GPU lane carries, 1 or 2
                                    (0 = 2: two systems share the paired FP32
                                    instructions of sm_100+); results differ only
                                    in rounding */
    int32_t kernel_timing;       /* 1: record CUDA events around each kernel of a
                                    solve (read with rt_kernel_times) */
    int32_t n_edges;             /* 0: NB bins of equal width on [wn_min, wn_max];
                                    > 1: explicit bin edges, every column then has
                                    n_edges - 1 bins (e.g. the R = 500 sampling of
                                    the post-processing step, Sec. 2.1.3) */
    const double *wn_edges;      /* HOST [n_edges], cm^-1, increasing; copied by rt_create */
    int32_t n_sweeps;            /* multiple scattering (Sec. 2.2.2).  0: Thomas's
                                    algorithm on the block system (Eqs. 12-15).  N > 0:
                                    the iterative method the paper replaces with it --
                                    N sweeps of the sub-layers' pairwise two-stream
                                    relations through the column (a downward pass from
                                    the TOA condition, the BOA condition of Eq. 10, an
                                    upward pass), starting from zero diffuse flux; the
                                    result converges to Thomas's as N grows.  FP32 form,
                                    cube optics, every column L <= RT_SWEEP_MAX_LAYERS;
                                    RT_EINVAL otherwise.  At most 1 << 20 */
    int32_t staging_depth;       /* FP32 form, Thomas: levels of elimination scratch
                                    (and, with RT_STAGE_INLINE, of B) that the
                                    back-substitution (Eq. 15) has in flight ahead of
                                    their use, copied into a shared-memory ring
                                    (cp.async): RT_STAGING_DEPTH_MIN ..
                                    RT_STAGING_DEPTH_MAX, 0 = RT_STAGING_DEPTH_MIN;
                                    RT_EINVAL otherwise.  More hides more L2 latency
                                    and costs shared memory (resident CTAs); results
                                    are the same bits */
} rt_config;
#define RT_STAGING_DEPTH_MIN 2
#define RT_STAGING_DEPTH_MAX 3

/* Largest layer count of a column solved with n_sweeps > 0 (each GPU lane
 * holds its system's per-layer transmission, reflection and level fluxes in
 * registers). */
#define RT_SWEEP_MAX_LAYERS 40

/* A packed batch of columns.  Column c has L_c layers, NB_c bins and
 * S_c = NB_c * n_g systems.  Data of consecutive columns follow each other
 * with no gaps:
 *   dtau, w0, g0   DEVICE float  [sum_c L_c*NB_c*n_g], per column
 *                  [layer][bin][g] with g fastest (layer 0 = TOA):
 *                  layer optical depth (>= 0), single-scattering albedo
 *                  ([0, 1]), asymmetry parameter ((-1, 1)).  In
 *                  non-isothermal mode each sub-layer gets half the optical
 *                  depth and the layer's w0, g0 (Sec. 2.2.1).
 *   T_center       DEVICE double [sum_c L_c]      K, layer centres
 *   T_iface        DEVICE double [sum_c (L_c+1)]  K, interfaces
 *   p_iface        DEVICE double [sum_c (L_c+1)]  Pa, interfaces, increasing
 *   mu_star        DEVICE double [n_cols]         cos(zenith angle); <= 0: no beam
 *   F_star         DEVICE double [sum_c NB_c]     W m^-2 stellar flux per bin,
 *                                                  normal to the beam, at the TOA
 * Shapes are HOST arrays (or NULL with the uniform L, NB given). */
typedef struct {
    int32_t n_cols;
    const int32_t *n_layers;     /* HOST [n_cols] or NULL -> every column has L layers */
    const int32_t *n_bins;       /* HOST [n_cols] or NULL -> every column has NB bins */
    int32_t L, NB;
    const float *dtau, *w0, *g0;
    const double *T_center, *T_iface, *p_iface;
    const double *mu_star, *F_star;
    /* Optional gather (HOST [n_cols] each, or NULL for the packed layout
     * above): where column c's inputs start, in elements of each array.
     * Columns may then live anywhere in the input arrays, be shared by
     * several batch entries, or skip data -- e.g. requests that slice a
     * device-resident pool.  Outputs stay packed in batch order. */
    const int64_t *cube_offset;    /* into dtau, w0, g0 (block of L_c*NB_c*n_g) */
    const int64_t *center_offset;  /* into T_center (L_c values) */
    const int64_t *iface_offset;   /* into T_iface and p_iface (L_c+1 values) */
    const int64_t *bin_offset;     /* into F_star (NB_c values) */
    const int64_t *col_index;      /* into mu_star (1 value) */
    /* Element counts of the device arrays (0 = not given).  The library
     * cannot see device allocations, so these bound every read: each
     * column's block [offset, offset + span) must lie inside its array's
     * count, or the call returns RT_EINVAL before anything is enqueued.  A
     * gather offset array requires the counts of the arrays it indexes; in
     * the packed layout a given count is checked against the packed
     * extent. */
    int64_t n_cube;                /* elements of each of dtau, w0, g0 */
    int64_t n_center;              /* elements of T_center */
    int64_t n_iface;               /* elements of each of T_iface, p_iface */
    int64_t n_fstar;               /* elements of F_star */
    int64_t n_mu;                  /* elements of mu_star */
} rt_columns;

typedef struct {
    int64_t systems;             /* (column, bin, g) systems in the last solve */
    int64_t resonance_hits;      /* layer-systems with |D| < 1e-5 (Eq. 11) */
    int64_t etau_hits;           /* sub-layer-systems below e_tau = 1e-4 (Sec. 2.2.1) */
    int64_t eclamp_hits;         /* layer-systems where the E fit fell below 1 */
    int64_t invalid_inputs;      /* layer-systems with dtau < 0, w0 outside [0,1], |g0| >= 1, NaN */
    int64_t nonfinite_outputs;   /* systems whose fluxes came out non-finite */
    int64_t fp64_evals;          /* FP32 form: layer-systems whose resonance test ran in FP64 */
    int64_t bounds_violations;   /* bounds-check build of the library (built with
                                    RT_BOUNDS_CHECK): device accesses found outside
                                    their array and skipped; always 0 otherwise */
} rt_stats_t;

/* Create a handle for the problem statement of Sec. 2.2 (the layer model,
 * two-stream closure and constants of rt_config: Sec. 2.2.1, Eq. 19, Table
 * 3).  Copies cfg (and g_weights).  RT_EINVAL on a bad field, RT_ECUDA if no
 * device is usable.  The handle holds device workspace that grows on demand
 * and is freed by rt_destroy. */
int rt_create(const rt_config *cfg, rt_handle **out);

/* Device workspace (bytes) that a solve of cols needs, outputs included:
 * the per-system elimination state of Eqs. 13-15 and the spectral sums of
 * Sec. 2.2.6 for the batch.  Validates cols as rt_solve_columns does. */
int rt_query_bytes(const rt_handle *h, const rt_columns *cols, size_t *bytes);

/* Validate cfg and cols on the host alone -- no device, no handle: every
 * check rt_solve_columns makes before it enqueues work (shapes, pointers,
 * gather offsets against the element counts).  A descriptor with NULL
 * dtau, w0 and g0 is checked as for rt_solve_ktable.  Writes a one-line
 * reason into msg (msg_len bytes, may be NULL).  Returns RT_OK or
 * RT_EINVAL. */
int rt_check_columns(const rt_config *cfg, const rt_columns *cols, char *msg, size_t msg_len);

/* Enqueue the whole path for cols on stream: Planck per bin, layer
 * coefficients (App. B), beam (Eq. B6), sources, Thomas elimination,
 * spectral sum, net flux and heating.  Results stay in the handle until the
 * next solve.  Validates shapes and pointers synchronously (RT_EINVAL);
 * RT_EBUDGET if the workspace would pass hbm_budget_bytes.  May grow the
 * workspace (cudaMalloc) when cols is larger than anything seen before; a
 * solve inside CUDA-graph capture must therefore follow one of the same
 * shape outside it.  A captured solve completes when its graph is replayed:
 * order later rt_fluxes / rt_heating / rt_stats after the replay (same
 * stream, or a synchronisation). */
int rt_solve_columns(rt_handle *h, const rt_columns *cols, void *stream);

/* Copy the last solve's interface fluxes, W m^-2, [sum_c (L_c+1)] each,
 * interface 0 = TOA, to F_up, F_down (diffuse + beam), F_net (= F_up -
 * F_down): the Gauss-weighted sums over g-points and bins (Sec. 2.2.6), the
 * beam added to the downward flux before the net flux is formed (Sec.
 * 2.2.1).  Pointers may be host or device memory, or NULL to skip.
 * RT_ENOTSOLVED before a solve. */
int rt_fluxes(rt_handle *h, double *F_up, double *F_down, double *F_net, void *stream);

/* Copy the last solve's heating rates, K s^-1, [sum_c L_c], layer 0 = TOA:
 * Q_l = (g / c_P) (F_net[l+1] - F_net[l]) / (p[l+1] - p[l]). */
int rt_heating(rt_handle *h, double *Q, void *stream);

/* Copy the last solve's upward flux at the top of the atmosphere per bin, W
 * m^-2 per bin, [sum_c NB_c] (column c's bins at the sum of the earlier
 * columns' NB): the Gauss-weighted sum over the bin's g-points -- the
 * emission plus reflected-light spectrum that post-processing turns into
 * synthetic spectra (Sec. 2.1.3, R = 500 with one point per bin).  Host or
 * device pointer.  Bit-reproducible for n_g <= 32. */
int rt_toa_spectrum(rt_handle *h, double *F_up_toa, void *stream);

/* ---------------------------------------------------------------------
 * Input front end (Sec. 2.1.3): the optics of every layer, bin and g-point
 * derived from the column state and a premixed k-table, instead of being
 * passed in as cubes.
 *
 *   kappa   = 10^(bilinear interpolation of log10 kappa in (T, log10 p))
 *             at the layer's centre temperature T_center and pressure
 *             sqrt(p_top p_bot); T and log10 p are clamped to the grid;
 *   sigma_g = x_H2 sigma_H2 + x_He sigma_He, the Rayleigh cross sections of
 *             App. C averaged over the bin in wavenumber;
 *   w0      = (sigma_g + f_cloud sigma_scat,cloud) / E,                (Eq. 17)
 *   g0      = f_cloud sigma_scat,cloud g0_cloud / (sigma_g + f_cloud sigma_scat,cloud),   (Eq. 18)
 *             with E = sigma_g + kappa mbar + f_cloud (sigma_abs,cloud +
 *             sigma_scat,cloud) the extinction per gas particle (g0 = 0
 *             where nothing scatters); kappa is the premixed opacity of
 *             Eq. 16, summed over species when the table was built;
 *   dtau    = E / mbar * (p_bot - p_top) / g.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t n_T, n_P;              /* grid sizes (the paper's tables: 60 x 28), >= 2 each */
    const double *T_grid;          /* HOST [n_T] K, strictly increasing */
    const double *log10p_grid;     /* HOST [n_P] log10(p / Pa), strictly increasing */
    int32_t n_bins;                /* NB of the table; columns solved with it have NB = n_bins */
    int32_t n_g;                   /* Gauss points of the table; must equal the handle's n_g */
    const float *log10_kappa;      /* HOST [n_T][n_P][n_bins][n_g] log10(kappa / m^2 kg^-1) */
    const double *sigma_scat_cloud;  /* HOST [n_bins] m^2 per cloud particle, bin averages */
    const double *sigma_abs_cloud;   /* HOST [n_bins] m^2 per cloud particle */
    const double *g0_cloud;          /* HOST [n_bins] asymmetry factor of the cloud */
    double f_cloud;                /* cloud-to-gas number ratio (the paper's runs: 1e-17) */
    double x_H2, x_He;             /* number fractions for Rayleigh scattering, >= 0 */
    double mbar_amu;               /* mean molecular mass, amu (Table 3: 2.34) */
} rt_ktable;

/* Copy a k-table into the handle (device memory) and precompute the per-bin
 * scattering data from the handle's bins (uniform or explicit edges).  The
 * device copy holds each node's value beside its next T-neighbour's,
 * 2 (n_T - 1) / n_T times the caller's table; the caller's arrays may be
 * freed on return.
 * RT_EINVAL on a bad field or when the table's n_g differs from the
 * handle's; replaces any earlier table (synchronises the device). */
int rt_set_ktable(rt_handle *h, const rt_ktable *kt);

/* Write the front end's FP32 optics for cols (whose dtau, w0, g0 must be
 * NULL and whose columns all have NB = the table's n_bins) into DEVICE cubes
 * dtau, w0, g0 in the packed layout of rt_columns.  Gather offsets other than
 * cube_offset are honoured.  RT_ENOTSOLVED without a table. */
int rt_ktable_optics(rt_handle *h, const rt_columns *cols, float *dtau, float *w0, float *g0,
                     void *stream);

/* rt_solve_columns with the optics from the front end (cols->dtau, w0, g0
 * and cube_offset NULL).  The FP32 form evaluates the front end inside the
 * solve kernel, so no cube is written or read; the FP64 path first writes
 * the FP32 optics of rt_ktable_optics into handle workspace.  Outputs are
 * read as after rt_solve_columns. */
int rt_solve_ktable(rt_handle *h, const rt_columns *cols, void *stream);

/* Device durations (ms, CUDA events on the solve's stream) of the last
 * solve's kernels: the Planck/front-end pre-kernel and the solve kernel (for
 * the FP64 path: 0 and the solve).  Needs cfg->kernel_timing; synchronises
 * on the last solve.  RT_ENOTSOLVED before a timed solve. */
int rt_kernel_times(rt_handle *h, float *prep_ms, float *solve_ms);

/* Branch and error counters of the last solve (synchronises the stream of
 * that solve). */
int rt_stats(rt_handle *h, rt_stats_t *out);

/* Last error message of this handle ("" if none).  Valid until the next call. */
const char *rt_last_error(const rt_handle *h);

/* Free the handle and its workspace (synchronises the device). */
void rt_destroy(rt_handle *h);

/* Failure injection, for tests of the callers' error handling: the next n
 * device workspace allocations (any handle's, when a solve must grow its
 * workspace) fail as an out-of-memory device would, and the call that needed
 * them returns RT_ENOMEM ("injected" in rt_last_error).  The handle stays
 * usable: its next call allocates again.  n = 0 clears; n < 0 is RT_EINVAL.
 * Nothing is launched or allocated by this call.  Returns RT_OK. */
int rt_inject_alloc_failures(int n);

/* ---------------------------------------------------------------------
 * Solve without allocating.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- programs whose device
 * memory belongs to their own pool or to a framework that forbids raw
 * allocations, and loops that cannot take the device-wide synchronisation
 * an allocation may bring.
 *
 * It runs the FP32 form (cfg->precision must be RT_FP32_FORM, uniform bins:
 * cfg->n_edges = 0) on a packed batch in which every column has the same shape (cols->n_layers, cols->n_bins
 * and the gather offsets NULL; cols->L and cols->NB set), with no handle: the caller passes the inputs
 * (same layout as rt_solve_columns) and DEVICE output arrays F_up, F_down,
 * F_net [n_cols (L+1)] and Q [n_cols L], written in place (same meaning as
 * rt_fluxes / rt_heating).  Every intermediate lives in one file-scope device
 * array of RT_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the
 * library keeps reserved until the process exits.  It needs about
 *   8 n_cols NB (L + 2) + 8 n_cols ceil(NB n_g / 32) (L + 1) + 16 L per
 *   resident thread (at least 64 threads)
 * bytes; a batch that does not fit returns RT_EBUDGET and nothing runs.
 * Element counts given in cols must cover the packed batch (RT_EINVAL).
 * No cudaMalloc, cudaFree or allocating library routine is called.
 *
 * Fixed launch choices: one system per GPU lane (the regular entry point
 * defaults to two), the Planck values tabulated by the pre-kernel and staged
 * per warp in shared memory, Thomas's algorithm (n_sweeps must be 0), the
 * default staging depth.  cfg->block_threads caps the CTA size;
 * systems_per_lane, planck_staging, staging_depth, ctas_per_sm,
 * hbm_budget_bytes, kernel_timing, max_layers and max_bins are ignored.  The elimination scratch shares the fixed array with the
 * per-column tables, so it caps the resident threads: at the 2562-column GCM
 * shape (2562 x 40 x 30 x 20) about one 256-thread CTA per SM runs, roughly
 * a third of the warps rt_solve_columns keeps resident, and the solve takes
 * several times longer than rt_solve_columns.
 *
 * The first call on a device looks up the array's device address and sets the
 * kernels' shared-memory limits; make that first call before any stream
 * capture.  All calls share the one array and each call overwrites what the
 * previous one left there: calls whose work overlaps on the GPU (different
 * streams, or several host threads) race and give wrong results -- order
 * them.  Returns RT_OK, RT_EINVAL (bad argument), RT_EBUDGET (too large) or
 * RT_ECUDA. */
#define RT_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int rt_solve_uniform_noalloc(const rt_config *cfg, const rt_columns *cols, double *F_up,
                             double *F_down, double *F_net, double *Q, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_H */
