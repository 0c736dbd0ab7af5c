// rt_internal.h -- kernel parameter block shared by the API and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rt {

// Device counters, in this order (see rt_stats_t).
enum StatIdx {
    ST_RESONANCE = 0,
    ST_ETAU = 1,
    ST_ECLAMP = 2,
    ST_INVALID = 3,
    ST_NONFINITE = 4,
    ST_FP64 = 5,
    ST_BOUNDS = 6,   // bounds-check builds: accesses found outside their array (and skipped)
    ST_COUNT = 8
};

// Element counts of every array the kernels index, for the bounds-check
// build (RT_BOUNDS_CHECK); unused otherwise.
struct Extents {
    long long cube, center, iface, fstar, mu;   // caller inputs
    long long scr32, scr64, scrB;               // elimination scratch (float4, double2, float units)
    long long part, planck, bins, cols;         // unit partials, Planck table, per-bin and per-column staging
    long long out_if, out_lay;                  // outputs
};

struct KParams {
    // inputs (caller-owned device memory)
    const float *dtau, *w0, *g0;
    const double *T_center, *T_iface, *p_iface, *mu_star, *F_star;
    // per-column layout (handle workspace)
    const int32_t *n_layers, *n_bins;
    const int64_t *cube_off;     // input: element offset of the column's cube block
    const int64_t *tc_off;       // input: offset into T_center
    const int64_t *if_off;       // input: offset into T_iface and p_iface
    const int64_t *fs_off;       // input: offset into F_star
    const int64_t *mu_idx;       // input: index into mu_star
    const int64_t *lay_off;      // packed: offset into Q (sum of L); F_up etc. at lay_off + c
    const int64_t *bin_off;      // packed: offset into the per-bin staging (sum of NB)
    const int32_t *order;        // columns in processing order (largest first)
    int32_t n_cols;
    // Gauss points
    int32_t n_g;
    const double *g_w;           // [n_g]
    // outputs (handle workspace); interface arrays use lay_off[c] + c
    double *F_up, *F_dn, *F_net, *Q;
    // per-level elimination scratch, layout [level][slot]; one slot per
    // resident thread of the persistent grid (slot = global thread index)
    float4 *scr32;               // FP32 form: (P, Q, alpha', e) per interface
    double2 *scr64;              // FP64 path: 2 x double2 = (P, Q), (a, e) per level
    int64_t n_slots;
    // FP32 form: warp-sized work units (32 consecutive systems of a column)
    const int32_t *unit_col;     // [n_units] column of each unit, largest column first
    const int32_t *unit_k;       // [n_units] index of the unit within its column
    const int32_t *col_units;    // [n_cols] units per column
    const int64_t *part_off;     // [n_cols] offset of the column's partial sums
    float *partial;              // per unit and interface: (sum w F_up, sum w F_net)
    int32_t n_units;
    int32_t warp_floats;         // shared-memory floats per warp
    int32_t group_shift;         // FP32 form: log2 of the interfaces per transposed sum (3 or 4)
    int32_t back_depth;          // FP32 form: back-substitution levels in flight (kBackDepthMin..kBackDepthMax)
    // FP32 form: per-column staging written by fp32_prep
    float *planck32;             // B per column [2L+1][NB] (levels: 2i interface, 2i+1 centre)
    const int64_t *planck_off;   // [n_cols]
    float *fs32, *fboa32;        // [sum NB] F* and F_BOA per bin
    float4 *colf;                // [n_cols] (mu, 1/mu, beam?, coldest level T or 0)
    const float *g_w32;          // [n_g] Gauss weights in FP32
    int32_t nbw;                 // bins one warp's 32 systems can touch
    int32_t direct;              // 1: read B from planck32 directly (no staging)
    int32_t inline_b;            // 1: the solve kernel evaluates B per system (no planck32 levels)
    void *scrB;                  // inline_b: B per interface, [level][thread slot] x systems per lane
    int32_t ns;                  // systems per lane (1 or 2; 0 counts as 1)
    // scheduling and counters
    int32_t *counter;
    unsigned long long *stats;
    // method switches and constants
    int32_t improved, isothermal, resonance_paper, e_clamp;
    double eps2, grav, cp, T_int, F_toa, wn_min, wn_max;
    const double *edges;         // [NB+1] explicit bin edges (cm^-1) or nullptr (uniform)
    const float *edges32;        // the same edges rounded to FP32 (FP32 form)
    const float *dnu32;          // [NB] bin widths formed in FP64, rounded to FP32
    double *toa;                 // [sum NB] TOA upward flux per bin (zeroed before the solve)
    // k-table front end (set when the optics come from the table)
    const float *kt_lk;          // [nT - 1][nP][NB * n_g][2] log10 kappa at (iT, iP) and (iT + 1, iP)
    const float4 *kt_bin;        // [NB] (scattering, cloud absorption per unit mass, g0, 0)
    const double *kt_T, *kt_lp;  // grids [nT] K, [nP] log10(p / Pa)
    int32_t kt_nT, kt_nP;
    float4 *kt_lay;              // [sum L] per layer: (corner offset bits, wT, wP, dp / g)
    float inv_eps2;
    int32_t n_sweeps;            // 0: Thomas elimination; N > 0: N sweeps of the iterative method
    int32_t Lmax;                // largest L in this batch
    int32_t nb_chunk;            // bins covered by one chunk of systems (smem sizing)
    int32_t staged;              // staged Planck values per warp (FP32) or CTA (FP64): the
                                 // largest (2 L_c + 1) x (bins a chunk of column c covers)
    Extents ext;                 // array extents (checked in bounds-check builds)
};

// Shared memory needed per CTA for a given block size (bytes).
// `staged`: the staged Planck values of one warp (shared staging).
size_t fp32_smem_bytes(int block, int Lmax, int nbw, int direct, int ns, int group_shift, int inline_b, int depth,
                       int staged);
int fp32_warp_floats(int Lmax, int nbw, int direct, int ns, int group_shift, int inline_b, int depth, int staged);
// Back-substitution prefetch depths with a kernel instance (kp.back_depth).
constexpr int kBackDepthMin = 2, kBackDepthMax = 3;
size_t fp64_smem_bytes(int block, int Lmax, int nb_chunk, int staged);
// Scratch bytes per thread slot.
size_t fp32_scratch_per_slot(int Lmax);
size_t fp64_scratch_per_slot(int Lmax, int isothermal);
// Bins that one chunk of `block` consecutive systems can touch.
int bins_per_chunk(int block, int n_g, int max_bins);

// One-time per-device set-up (dynamic shared-memory limits).
cudaError_t init_kernels();
// Resident CTAs per SM for a launch shape (0 if it does not fit).
int occupancy(int precision_fp64, int block, size_t smem, int ns = 1, int sweeps = 0);
// Launch the fused column kernels.  Return cudaGetLastError().
// ev (optional): three events recorded before the pre-kernel, between the
// two kernels and after the solve kernel.
cudaError_t launch_fp32(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s,
                        cudaEvent_t const *ev = nullptr);
cudaError_t launch_fp64(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s);
// The iterative method (kp.n_sweeps > 0): the Planck pre-kernel, then the
// sweep kernel; ev as for launch_fp32.
cudaError_t launch_sweeps(const KParams &kp, int grid, int block, size_t smem, cudaStream_t s,
                          cudaEvent_t const *ev = nullptr);
// Front end alone: FP32 optics of every (column, layer, bin, g) into packed
// cubes (cube offsets of the packed layout in pcube_off).
cudaError_t launch_kt_optics(const KParams &kp, const int64_t *pcube_off, float *dtau, float *w0,
                             float *g0, cudaStream_t s);

// Largest L the kernels support.
constexpr int kMaxLayers = 1024;
// Largest L of the iterative method's kernel (each lane holds its system's
// per-layer t, r and the level fluxes in registers).
constexpr int kSweepMaxLayers = 40;
// Shared memory of the iterative method's kernel: floats per warp, bytes per CTA.
int sweep_warp_floats(int Lmax, int nbw, int direct, int isothermal);
size_t sweep_smem_bytes(int block, int Lmax, int nbw, int direct, int isothermal);
// Largest CTA size (launch bounds): FP64 kernel, FP32 kernel.
constexpr int kMaxBlock = 512;
constexpr int kMaxBlock32 = 256;

}  // namespace rt
