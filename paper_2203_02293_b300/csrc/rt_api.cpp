// rt_api.cpp -- host side of the C ABI declared in include/rt.h.
//
// A handle owns: a copy of the configuration, the Gauss weights on the
// device, a per-batch plan (column shapes, offsets and processing order),
// the output arrays, the per-thread-slot elimination scratch, a work counter
// and the branch counters.  Device buffers grow on demand and are reused.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rt.h"
#include "rt_internal.h"

static_assert(rt::kSweepMaxLayers == RT_SWEEP_MAX_LAYERS, "sweep layer limit differs between rt.h and the kernels");
static_assert(rt::kBackDepthMin == RT_STAGING_DEPTH_MIN && rt::kBackDepthMax == RT_STAGING_DEPTH_MAX,
              "staging depths differ between rt.h and the kernels");

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// An NVTX range over a host call (shows the enqueue of each solve in a
// profiler timeline; a near no-op when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

struct rt_handle {
    rt_config cfg{};
    std::vector<double> gw;
    int device = 0;
    int sm_count = 0;
    double *d_gw = nullptr;
    float *d_gw32 = nullptr;
    std::vector<double> edges;
    double *d_edges = nullptr;
    float *d_edges32 = nullptr;   // [n_edges] edges, then [n_edges - 1] widths, FP32
    bool narrow_edges = false;    // every explicit bin at most 1% of its lower edge wide
    // k-table front end
    bool kt_set = false;
    int kt_nT = 0, kt_nP = 0, kt_NB = 0;
    float *d_klk = nullptr;
    float4 *d_kbin = nullptr;
    double *d_kT = nullptr, *d_klp = nullptr;
    DevBuf kcube;                  // FP64 path: front-end optics cubes
    // plan
    DevBuf plan;                  // n_layers, n_bins, order (int32) + offsets (int64)
    std::vector<int32_t> plan_nl, plan_nb;
    std::vector<int64_t> plan_cube, plan_tc, plan_if, plan_fs, plan_mu;
    bool plan_valid = false;
    int plan_prec = -1;
    void *h_stage = nullptr;      // pinned staging for plan uploads
    size_t stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    bool stage_pending = false;
    // outputs and scratch
    DevBuf out, scr, aux;          // aux: FP32 unit partials, Planck table, per-bin and per-column data
    int32_t *d_counter = nullptr;
    unsigned long long *d_stats = nullptr;
    cudaEvent_t done_ev = nullptr;
    cudaEvent_t kev[3] = {nullptr, nullptr, nullptr};   // kernel timing (cfg.kernel_timing)
    bool kev_valid = false, kev_fp64 = false;
    bool done_valid = false;       // done_ev marks the last solve (false when it was captured)
    cudaStream_t last_stream = nullptr;
    bool solved = false;
    int64_t n_cols = 0, n_if = 0, n_lay = 0, n_sys = 0, n_bins = 0;
    std::string err;
};

namespace {

int fail(rt_handle *h, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return code;
}

int cuda_fail(rt_handle *h, cudaError_t e, const char *what) {
    return fail(h, RT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Sizes derived from one batch.
struct Plan {
    std::vector<int32_t> nl, nb, order, col_units, unit_col, unit_k;
    std::vector<int64_t> cube_off, lay_off, bin_off, part_off, planck_off;
    std::vector<int64_t> tc_off, if_off, fs_off, mu_idx;   // input offsets (gather or packed)
    int64_t n_if = 0, n_lay = 0, n_sys = 0, n_cube = 0, n_bins = 0, n_part = 0, n_planck = 0;
    int64_t n_units = 0;
    int Lmax = 0, NBmax = 0;
    // launch
    int block = 0, grid = 0, nb_chunk = 0, nbw = 0, warp_floats = 0, direct = 0, inline_b = 0, ns = 1;
    int staged = 0;               // staged Planck values per warp (FP32) / CTA (FP64), see staged_capacity
    int group_shift = 4;          // FP32 form: log2 of the interfaces per transposed sum
    int depth = 2;                // FP32 form: back-substitution levels in flight (cfg.staging_depth)
    bool sweeps = false;          // the iterative method (cfg.n_sweeps > 0) instead of Thomas
    size_t smem = 0;
    int64_t n_slots = 0;
    // workspace layout (bytes); the plan blob is int32 arrays then int64 arrays
    size_t i32_count = 0, plan_bytes = 0, out_bytes = 0, scr_bytes = 0, aux_bytes = 0, kcube_bytes = 0;
    bool kt = false;              // optics from the k-table front end
};

// Shared memory for the staged Planck values: a chunk of systems covers at
// most `chunk` bins of its column, so column c stages (2 L_c + 1) x
// min(NB_c, chunk) values; the largest over the batch (not the product of
// the batch's largest L and NB, which may belong to different columns).
int staged_capacity(const std::vector<int32_t> &nl, const std::vector<int32_t> &nb, int chunk) {
    int64_t m = 0;
    for (size_t i = 0; i < nl.size(); ++i)
        m = std::max<int64_t>(m, (int64_t)(2 * nl[i] + 1) * std::min<int32_t>(nb[i], chunk));
    return (int)std::min<int64_t>(m, 1 << 30);
}

// Element counts of the input arrays: a column's block [off, off + span) of
// an array must lie inside its count.  Gather offsets need the counts of
// the arrays they index; in the packed layout a given count is checked too.
int check_span(rt_handle *h, int col, const char *what, int64_t off, int64_t span, int64_t count, bool gathered) {
    if (count < 0) return fail(h, RT_EINVAL, "%s: negative element count %lld", what, (long long)count);
    if (count == 0) {
        if (gathered) return fail(h, RT_EINVAL, "%s: gather offsets need the array's element count", what);
        return RT_OK;
    }
    if (off > count || span > count - off)
        return fail(h, RT_EINVAL, "column %d: %s elements [%lld, %lld) outside the array's %lld", col, what,
                    (long long)off, (long long)(off + span), (long long)count);
    return RT_OK;
}

// The FP32 work units, largest column first: unit u is unit k of column c.
void fill_units(Plan &P) {
    P.unit_col.resize((size_t)P.n_units);
    P.unit_k.resize((size_t)P.n_units);
    int64_t u = 0;
    for (size_t oi = 0; oi < P.order.size(); ++oi) {
        const int col = P.order[oi];
        for (int k = 0; k < P.col_units[col]; ++k, ++u) {
            P.unit_col[u] = col;
            P.unit_k[u] = k;
        }
    }
}

// The host-side part of a plan: shapes, offsets (gather or packed), their
// bounds, processing order and work units (the per-unit lists only when
// `units`: sizes need their count alone).  No device call.
int validate_plan(rt_handle *h, const rt_columns *c, Plan &P, bool kt, bool units = true) {
    const rt_config &cfg = h->cfg;
    const int n = c->n_cols;
    const bool fp64 = cfg.precision == RT_FP64_PLAIN;
    P.sweeps = cfg.n_sweeps > 0;
    if (P.sweeps && fp64) return fail(h, RT_EINVAL, "the iterative method (n_sweeps > 0) runs in the FP32 form only");
    if (P.sweeps && kt) return fail(h, RT_EINVAL, "the iterative method (n_sweeps > 0) takes optics cubes, not the k-table");
    P.nl.resize(n);
    P.nb.resize(n);
    for (int i = 0; i < n; ++i) {
        P.nl[i] = c->n_layers ? c->n_layers[i] : c->L;
        P.nb[i] = c->n_bins ? c->n_bins[i] : c->NB;
        if (P.nl[i] < 1 || P.nl[i] > cfg.max_layers)
            return fail(h, RT_EINVAL, "column %d: n_layers %d outside [1, %d]", i, P.nl[i], cfg.max_layers);
        if (P.nb[i] < 1 || P.nb[i] > cfg.max_bins)
            return fail(h, RT_EINVAL, "column %d: n_bins %d outside [1, %d]", i, P.nb[i], cfg.max_bins);
        if (cfg.n_edges > 1 && P.nb[i] != cfg.n_edges - 1)
            return fail(h, RT_EINVAL, "column %d: n_bins %d but %d explicit bin edges", i, P.nb[i], cfg.n_edges);
        if (kt && h->kt_NB >= 0 && P.nb[i] != h->kt_NB)
            return fail(h, RT_EINVAL, "column %d: n_bins %d but the k-table has %d", i, P.nb[i], h->kt_NB);
        if (P.sweeps && P.nl[i] > rt::kSweepMaxLayers)
            return fail(h, RT_EINVAL, "column %d: n_layers %d above %d, the iterative method's limit", i, P.nl[i],
                        rt::kSweepMaxLayers);
    }
    P.kt = kt;
    P.ns = (fp64 || P.sweeps) ? 1 : (cfg.systems_per_lane == 1 ? 1 : 2);
    P.depth = cfg.staging_depth > 0 ? cfg.staging_depth : 2;
    const int spu = 32 * P.ns;                    // systems per FP32 work unit
    const int64_t *gath[5] = {c->cube_offset, c->center_offset, c->iface_offset, c->bin_offset, c->col_index};
    for (int g = 0; g < 5; ++g)
        if (gath[g])
            for (int i = 0; i < n; ++i)
                if (gath[g][i] < 0) return fail(h, RT_EINVAL, "column %d: negative gather offset", i);
    P.tc_off.resize(n);
    P.if_off.resize(n);
    P.fs_off.resize(n);
    P.mu_idx.resize(n);
    P.cube_off.resize(n);
    P.lay_off.resize(n);
    P.bin_off.resize(n);
    P.part_off.resize(n);
    P.planck_off.resize(n);
    P.col_units.resize(n);
    int64_t cube = 0, lay = 0, bins = 0, part = 0, planck = 0;
    for (int i = 0; i < n; ++i) {
        P.cube_off[i] = c->cube_offset ? c->cube_offset[i] : cube;
        P.tc_off[i] = c->center_offset ? c->center_offset[i] : lay;
        P.if_off[i] = c->iface_offset ? c->iface_offset[i] : lay + i;
        P.fs_off[i] = c->bin_offset ? c->bin_offset[i] : bins;
        P.mu_idx[i] = c->col_index ? c->col_index[i] : i;
        P.lay_off[i] = lay;
        P.bin_off[i] = bins;
        P.part_off[i] = part;
        P.planck_off[i] = planck;
        planck += (int64_t)(2 * P.nl[i] + 1) * P.nb[i];
        const int64_t S = (int64_t)P.nb[i] * cfg.n_g;
        P.col_units[i] = (int32_t)((S + spu - 1) / spu);
        cube += (int64_t)P.nl[i] * S;
        lay += P.nl[i];
        bins += P.nb[i];
        part += (int64_t)P.col_units[i] * 2 * (P.nl[i] + 1);
        P.Lmax = std::max(P.Lmax, (int)P.nl[i]);
        P.NBmax = std::max(P.NBmax, (int)P.nb[i]);
    }
    for (int i = 0; i < n; ++i) {
        const int64_t S = (int64_t)P.nb[i] * cfg.n_g;
        int rc = RT_OK;
        if (!kt) rc = check_span(h, i, "dtau/w0/g0", P.cube_off[i], (int64_t)P.nl[i] * S, c->n_cube, c->cube_offset);
        if (!rc) rc = check_span(h, i, "T_center", P.tc_off[i], P.nl[i], c->n_center, c->center_offset);
        if (!rc) rc = check_span(h, i, "T_iface/p_iface", P.if_off[i], P.nl[i] + 1, c->n_iface, c->iface_offset);
        if (!rc) rc = check_span(h, i, "F_star", P.fs_off[i], P.nb[i], c->n_fstar, c->bin_offset);
        if (!rc) rc = check_span(h, i, "mu_star", P.mu_idx[i], 1, c->n_mu, c->col_index);
        if (rc) return rc;
    }
    P.n_cube = cube;
    P.n_lay = lay;
    P.n_if = lay + n;
    P.n_bins = bins;
    P.n_sys = bins * cfg.n_g;
    P.n_part = part;
    P.n_planck = planck;
    // largest work first (longest-processing-time order), ties by index
    P.order.resize(n);
    std::iota(P.order.begin(), P.order.end(), 0);
    std::stable_sort(P.order.begin(), P.order.end(), [&](int a, int b) {
        return (int64_t)P.nl[a] * P.nb[a] > (int64_t)P.nl[b] * P.nb[b];
    });
    if (!fp64) {
        int64_t nu = 0;
        for (int i = 0; i < n; ++i) nu += P.col_units[i];
        if (nu > INT32_MAX) return fail(h, RT_EINVAL, "too many work units");
        P.n_units = nu;
        if (units) fill_units(P);
    }
    return RT_OK;
}

int build_plan(rt_handle *h, const rt_columns *c, Plan &P, bool kt, bool units = true) {
    int rc = validate_plan(h, c, P, kt, units);
    if (rc) return rc;
    const rt_config &cfg = h->cfg;
    const int n = c->n_cols;
    const bool fp64 = cfg.precision == RT_FP64_PLAIN;
    const int spu = 32 * P.ns;
    // launch shape (the FP32 kernel is compiled for at most 256 threads)
    P.block = fp64 ? cfg.block_threads : std::min(cfg.block_threads, rt::kMaxBlock32);
    if (n > 0 && P.sweeps) {
        // the sweep kernel: each warp needs ~8 KB of shared memory per 10
        // layers, so take the CTA size that keeps the most warps resident
        P.nbw = rt::bins_per_chunk(spu, cfg.n_g, P.NBmax);
        P.direct = cfg.planck_staging == RT_STAGE_DIRECT || cfg.planck_staging == RT_STAGE_INLINE ||
                   (cfg.planck_staging == RT_STAGE_AUTO && cfg.n_g < 4);
        P.warp_floats = rt::sweep_warp_floats(P.Lmax, P.nbw, P.direct, cfg.layers == RT_ISOTHERMAL);
        int best = 0;
        for (int b = 32; b <= rt::kMaxBlock32; b += 32) {
            const size_t sm = rt::sweep_smem_bytes(b, P.Lmax, P.nbw, P.direct, cfg.layers == RT_ISOTHERMAL);
            const int occ = rt::occupancy(0, b, sm, 1, 1);
            if (occ * b > best) {
                best = occ * b;
                P.block = b;
                P.smem = sm;
                P.grid = occ;
            }
        }
        if (best == 0) return fail(h, RT_EINVAL, "no launch shape of the sweep kernel fits (L=%d)", P.Lmax);
        int occ = P.grid;
        if (cfg.ctas_per_sm > 0 && occ > cfg.ctas_per_sm) occ = cfg.ctas_per_sm;
        const int64_t wpb = P.block / 32;
        P.grid = (int)std::min<int64_t>((P.n_units + wpb - 1) / wpb, (int64_t)occ * h->sm_count);
        P.n_slots = (int64_t)P.grid * P.block;
    } else if (n > 0) {
        for (;;) {
            int occ;
            if (fp64) {
                P.nb_chunk = rt::bins_per_chunk(P.block, cfg.n_g, P.NBmax);
                P.staged = staged_capacity(P.nl, P.nb, P.nb_chunk);
                P.smem = rt::fp64_smem_bytes(P.block, P.Lmax, P.nb_chunk, P.staged);
                occ = rt::occupancy(1, P.block, P.smem);
                if (occ > 0) P.grid = (int)std::min<int64_t>(n, (int64_t)occ * h->sm_count);
            } else {
                P.nbw = rt::bins_per_chunk(spu, cfg.n_g, P.NBmax);
                // staging B per warp pays off when several lanes share a bin;
                // with few g-points per bin it only costs shared memory
                // (occupancy), so the lanes read the table directly.  With
                // one g-point on narrow bins (the R = 500 shape) the solve
                // kernel evaluates B itself, each value once, instead of a
                // table written and read back through HBM (wide bins need
                // edge series, which the pre-kernel shares between bins).
                P.inline_b = cfg.planck_staging == RT_STAGE_INLINE ||
                             (cfg.planck_staging == RT_STAGE_AUTO && cfg.n_g == 1 && h->narrow_edges);
                P.direct = P.inline_b || cfg.planck_staging == RT_STAGE_DIRECT ||
                           (cfg.planck_staging == RT_STAGE_AUTO && cfg.n_g < 4);
                // 16 interfaces per transposed sum of the back-substitution,
                // unless 8 (half the transpose buffer) keep more CTAs
                // resident: tall columns' staged B fills shared memory
                P.group_shift = 4;
                P.staged = P.direct ? 0 : staged_capacity(P.nl, P.nb, P.nbw);
                P.smem = rt::fp32_smem_bytes(P.block, P.Lmax, P.nbw, P.direct, P.ns, 4, P.inline_b, P.depth, P.staged);
                occ = rt::occupancy(0, P.block, P.smem, P.ns);
                {
                    const size_t sm8 = rt::fp32_smem_bytes(P.block, P.Lmax, P.nbw, P.direct, P.ns, 3, P.inline_b, P.depth,
                                                           P.staged);
                    const int occ8 = rt::occupancy(0, P.block, sm8, P.ns);
                    const int cap = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : 1 << 20;
                    if (std::min(occ8, cap) > std::min(occ, cap)) {
                        P.group_shift = 3;
                        P.smem = sm8;
                        occ = occ8;
                    }
                }
                P.warp_floats = rt::fp32_warp_floats(P.Lmax, P.nbw, P.direct, P.ns, P.group_shift, P.inline_b, P.depth,
                                                     P.staged);
                const int64_t wpb = P.block / 32;
                if (occ > 0) P.grid = (int)std::min<int64_t>((P.n_units + wpb - 1) / wpb, (int64_t)occ * h->sm_count);
            }
            if (occ > 0) {
                if (cfg.ctas_per_sm > 0 && occ > cfg.ctas_per_sm) {
                    occ = cfg.ctas_per_sm;
                    const int64_t cap = (int64_t)occ * h->sm_count;
                    if (P.grid > cap) P.grid = (int)cap;
                }
                break;
            }
            if (P.block <= 64)
                return fail(h, RT_EINVAL, "no launch shape fits shared memory (L=%d, NB=%d)", P.Lmax, P.NBmax);
            P.block -= 32;
        }
        P.n_slots = (int64_t)P.grid * P.block * P.ns;
        if (P.inline_b) P.n_planck = 0;           // no B table: the solve kernel evaluates B
    }
    P.i32_count = 4 * (size_t)n + 2 * (size_t)P.n_units;
    P.plan_bytes = align_up(sizeof(int32_t) * P.i32_count, 256) + align_up(sizeof(int64_t) * 9 * (size_t)n, 256);
    P.out_bytes = align_up(sizeof(double) * 3 * (size_t)P.n_if, 256) + align_up(sizeof(double) * (size_t)P.n_lay, 256) +
                  align_up(sizeof(double) * (size_t)P.n_bins, 256);
    P.scr_bytes = P.sweeps ? sizeof(float2) * (size_t)P.n_slots * rt::kSweepMaxLayers   // (t, r) transfer
                           : (size_t)P.n_slots * (fp64 ? rt::fp64_scratch_per_slot(P.Lmax, cfg.layers == RT_ISOTHERMAL)
                                                       : rt::fp32_scratch_per_slot(P.Lmax));
    // inline B: the interfaces' B for the back-substitution, after the elimination scratch
    if (P.inline_b) P.scr_bytes = align_up(P.scr_bytes, 256) + sizeof(float) * (size_t)P.n_slots * P.Lmax;
    // FP32 aux: partial | planck32 | fs32 | fboa32 | colf [| kt_lay]
    P.aux_bytes = fp64 ? 0
                       : align_up(sizeof(float) * (size_t)P.n_part, 256) +
                             align_up(sizeof(float) * (size_t)P.n_planck, 256) +
                             2 * align_up(sizeof(float) * (size_t)P.n_bins, 256) + align_up(sizeof(float4) * (size_t)n, 256) +
                             (kt ? align_up(sizeof(float4) * (size_t)P.n_lay, 256) : 0);
    // FP64 path with the front end: the optics cubes
    P.kcube_bytes = (kt && fp64) ? 3 * align_up(sizeof(float) * (size_t)P.n_cube, 256) : 0;
    return RT_OK;
}

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// Pending injected allocation failures (rt_inject_alloc_failures).
std::atomic<int> g_inject_allocs{0};

int grow(rt_handle *h, DevBuf &b, size_t need, bool capturing, const char *what) {
    if (b.cap >= need) return RT_OK;
    if (capturing)
        return fail(h, RT_EINVAL, "%s workspace must grow (%zu bytes) during stream capture; "
                    "run one solve of this shape outside capture first", what, need);
    if (b.p) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    if (g_inject_allocs.load() > 0 && g_inject_allocs.fetch_sub(1) > 0)
        return fail(h, RT_ENOMEM, "cudaMalloc(%zu) for %s: injected failure", need, what);
    cudaError_t e = cudaMalloc(&b.p, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, RT_ENOMEM, "cudaMalloc(%zu) for %s: %s", need, what, cudaGetErrorString(e));
    }
    b.cap = need;
    return RT_OK;
}

int check_columns(rt_handle *h, const rt_columns *c, bool kt = false) {
    if (!c) return fail(h, RT_EINVAL, "columns descriptor is NULL");
    if (kt && !h->kt_set) return fail(h, RT_ENOTSOLVED, "no k-table set (rt_set_ktable)");
    if (c->n_cols < 0) return fail(h, RT_EINVAL, "n_cols %d < 0", c->n_cols);
    if (c->n_cols == 0) return RT_OK;
    if (!c->n_layers && c->L < 1) return fail(h, RT_EINVAL, "uniform L %d < 1", c->L);
    if (!c->n_bins && c->NB < 1) return fail(h, RT_EINVAL, "uniform NB %d < 1", c->NB);
    const void *ptrs[] = {c->dtau, c->w0, c->g0, c->T_center, c->T_iface, c->p_iface, c->mu_star, c->F_star};
    const char *names[] = {"dtau", "w0", "g0", "T_center", "T_iface", "p_iface", "mu_star", "F_star"};
    for (int i = kt ? 3 : 0; i < 8; ++i)
        if (!ptrs[i]) return fail(h, RT_EINVAL, "%s is NULL", names[i]);
    if (kt && (c->dtau || c->w0 || c->g0 || c->cube_offset))
        return fail(h, RT_EINVAL, "the k-table front end takes no dtau, w0, g0 or cube_offset");
    return RT_OK;
}

// Optics descriptor for a k-table solve: NULL cubes select the front end.
bool wants_kt(const rt_handle *h, const rt_columns *c) {
    return c && h->kt_set && !c->dtau && !c->w0 && !c->g0;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// The configuration fields rt_create accepts.
int check_config(const rt_config *cfg) {
    if (!cfg) return RT_EINVAL;
    if (cfg->n_g < 1 || cfg->n_g > 64 || !cfg->g_weights) return RT_EINVAL;
    if (!(cfg->wn_max > cfg->wn_min) || !(cfg->wn_min >= 0.0)) return RT_EINVAL;
    if (cfg->two_stream != RT_IMPROVED && cfg->two_stream != RT_REGULAR) return RT_EINVAL;
    if (cfg->layers != RT_NONISOTHERMAL && cfg->layers != RT_ISOTHERMAL) return RT_EINVAL;
    if (cfg->precision != RT_FP32_FORM && cfg->precision != RT_FP64_PLAIN) return RT_EINVAL;
    if (cfg->resonance != RT_RESONANCE_PAPER && cfg->resonance != RT_RESONANCE_LIMIT) return RT_EINVAL;
    if (!(cfg->eps2 > 0.0) || !(cfg->cp > 0.0) || !(cfg->T_int >= 0.0)) return RT_EINVAL;
    if (cfg->max_layers < 1 || cfg->max_layers > rt::kMaxLayers || cfg->max_bins < 1) return RT_EINVAL;
    if (cfg->block_threads != 0 &&
        (cfg->block_threads % 32 || cfg->block_threads < 64 || cfg->block_threads > rt::kMaxBlock))
        return RT_EINVAL;
    if (cfg->ctas_per_sm < 0) return RT_EINVAL;
    if (cfg->planck_staging < RT_STAGE_AUTO || cfg->planck_staging > RT_STAGE_INLINE) return RT_EINVAL;
    if (cfg->systems_per_lane < 0 || cfg->systems_per_lane > 2) return RT_EINVAL;
    if (cfg->staging_depth != 0 &&
        (cfg->staging_depth < RT_STAGING_DEPTH_MIN || cfg->staging_depth > RT_STAGING_DEPTH_MAX))
        return RT_EINVAL;
    if (cfg->n_edges < 0 || cfg->n_edges == 1 || (cfg->n_edges > 1 && !cfg->wn_edges)) return RT_EINVAL;
    if (cfg->n_sweeps < 0 || cfg->n_sweeps > (1 << 20)) return RT_EINVAL;
    for (int i = 0; i < cfg->n_edges; ++i) {
        if (!(cfg->wn_edges[i] >= 0.0)) return RT_EINVAL;
        if (i > 0 && !(cfg->wn_edges[i] > cfg->wn_edges[i - 1])) return RT_EINVAL;
    }
    for (int i = 0; i < cfg->n_g; ++i)
        if (!(cfg->g_weights[i] >= 0.0)) return RT_EINVAL;
    return RT_OK;
}

}  // namespace

extern "C" {

int rt_create(const rt_config *cfg, rt_handle **out) {
    if (!out) return RT_EINVAL;
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc) return rc;

    rt_handle *h = new rt_handle();
    h->cfg = *cfg;
    // default CTA: 4 warps for the FP32 form (4 CTAs of 128 per SM measured 1% faster than
    // 2 of 256 at the same 16 warps), 8 for the FP64 path
    if (h->cfg.block_threads == 0) h->cfg.block_threads = cfg->precision == RT_FP64_PLAIN ? 256 : 128;
    h->gw.assign(cfg->g_weights, cfg->g_weights + cfg->n_g);
    h->cfg.g_weights = h->gw.data();
    if (cfg->n_edges > 1) h->edges.assign(cfg->wn_edges, cfg->wn_edges + cfg->n_edges);
    h->cfg.wn_edges = h->edges.empty() ? nullptr : h->edges.data();
    h->narrow_edges = !h->edges.empty();
    for (size_t i = 0; i + 1 < h->edges.size(); ++i)
        h->narrow_edges = h->narrow_edges && h->edges[i + 1] - h->edges[i] <= 0.01 * h->edges[i];
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = rt::init_kernels();
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_gw, sizeof(double) * cfg->n_g);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_gw, h->gw.data(), sizeof(double) * cfg->n_g, cudaMemcpyHostToDevice);
    std::vector<float> gw32(h->gw.begin(), h->gw.end());
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_gw32, sizeof(float) * cfg->n_g);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_gw32, gw32.data(), sizeof(float) * cfg->n_g, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h->edges.empty()) {
        const size_t ne = h->edges.size();
        e = cudaMalloc((void **)&h->d_edges, sizeof(double) * ne);
        if (e == cudaSuccess)
            e = cudaMemcpy(h->d_edges, h->edges.data(), sizeof(double) * ne, cudaMemcpyHostToDevice);
        // FP32 copies for the FP32 form (the width is formed before rounding)
        std::vector<float> e32(2 * ne - 1);
        for (size_t i = 0; i < ne; ++i) e32[i] = (float)h->edges[i];
        for (size_t i = 0; i + 1 < ne; ++i) e32[ne + i] = (float)(h->edges[i + 1] - h->edges[i]);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_edges32, sizeof(float) * e32.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(h->d_edges32, e32.data(), sizeof(float) * e32.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_counter, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_stats, sizeof(unsigned long long) * rt::ST_COUNT);
    if (e == cudaSuccess) e = cudaMemset(h->d_stats, 0, sizeof(unsigned long long) * rt::ST_COUNT);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->done_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming);
    for (int i = 0; i < 3 && e == cudaSuccess && cfg->kernel_timing; ++i) e = cudaEventCreate(&h->kev[i]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rt_destroy(h);
        return RT_ECUDA;
    }
    *out = h;
    return RT_OK;
}

int rt_query_bytes(const rt_handle *hc, const rt_columns *cols, size_t *bytes) {
    rt_handle *h = const_cast<rt_handle *>(hc);
    if (!h || !bytes) return RT_EINVAL;
    const bool kt = wants_kt(h, cols);
    int rc = check_columns(h, cols, kt);
    if (rc) return rc;
    Plan P;
    rc = build_plan(h, cols, P, kt, false);
    if (rc) return rc;
    *bytes = P.plan_bytes + P.out_bytes + P.scr_bytes + P.aux_bytes + P.kcube_bytes;
    return RT_OK;
}

int rt_check_columns(const rt_config *cfg, const rt_columns *cols, char *msg, size_t msg_len) {
    if (msg && msg_len) msg[0] = '\0';
    int rc = check_config(cfg);
    if (rc) {
        if (msg && msg_len) snprintf(msg, msg_len, "invalid configuration");
        return rc;
    }
    rt_handle tmp;                 // host state only: no device is touched
    tmp.cfg = *cfg;
    if (tmp.cfg.block_threads == 0) tmp.cfg.block_threads = cfg->precision == RT_FP64_PLAIN ? 256 : 128;
    const bool kt = cols && !cols->dtau && !cols->w0 && !cols->g0;
    tmp.kt_set = kt;               // a state-only descriptor is checked as for rt_solve_ktable
    tmp.kt_NB = -1;                // (with no table, its bin count is not known)
    rc = check_columns(&tmp, cols, kt);
    Plan P;
    if (!rc && cols->n_cols > 0) rc = validate_plan(&tmp, cols, P, kt, false);
    if (rc && msg && msg_len) snprintf(msg, msg_len, "%s", tmp.err.c_str());
    return rc;
}

}  // extern "C"

namespace {

// The whole path for one batch.  kt: optics from the front end.  With
// optics_out set (three device cubes) only the front end runs and writes
// them; the handle's outputs are left alone.
int solve_impl(rt_handle *h, const rt_columns *cols, void *stream, bool kt, float *const *optics_out) {
    if (!h) return RT_EINVAL;
    NvtxRange range(optics_out ? "rt_ktable_optics" : kt ? "rt_solve_ktable"
                    : h->cfg.n_sweeps > 0 ? "rt_solve_columns (sweeps)" : "rt_solve_columns");
    h->err.clear();
    int rc = check_columns(h, cols, kt);
    if (rc) return rc;
    Plan P;
    rc = build_plan(h, cols, P, kt, false);     // unit lists only if the plan is new (below)
    if (rc) return rc;
    const rt_config &cfg = h->cfg;
    const size_t ws_bytes = P.plan_bytes + P.out_bytes + P.scr_bytes + P.aux_bytes + P.kcube_bytes;
    if (cfg.hbm_budget_bytes && ws_bytes > cfg.hbm_budget_bytes)
        return fail(h, RT_EBUDGET, "workspace %zu bytes exceeds budget %zu", ws_bytes, cfg.hbm_budget_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    const bool cap = stream_capturing(s);
    // order after the previous solve of this handle when it ran on another stream
    if (h->solved && h->done_valid && s != h->last_stream && !cap) {
        cudaError_t e = cudaStreamWaitEvent(s, h->done_ev, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamWaitEvent");
    }
    const int n = cols->n_cols;
    void *old_plan = h->plan.p;
    if ((rc = grow(h, h->plan, std::max<size_t>(P.plan_bytes, 256), cap, "plan"))) return rc;
    if (h->plan.p != old_plan) h->plan_valid = false;
    if ((rc = grow(h, h->out, std::max<size_t>(P.out_bytes, 256), cap, "output"))) return rc;
    if ((rc = grow(h, h->scr, std::max<size_t>(P.scr_bytes, 256), cap, "scratch"))) return rc;
    if ((rc = grow(h, h->aux, std::max<size_t>(P.aux_bytes, 256), cap, "partial-sum"))) return rc;
    if (P.kcube_bytes && (rc = grow(h, h->kcube, P.kcube_bytes, cap, "optics"))) return rc;

    char *pb = (char *)h->plan.p;
    int32_t *d_nl = (int32_t *)pb;
    int32_t *d_nb = d_nl + n;
    int32_t *d_order = d_nb + n;
    int32_t *d_cu = d_order + n;
    int32_t *d_ucol = d_cu + n;
    int32_t *d_uk = d_ucol + P.n_units;
    int64_t *d_cube = (int64_t *)(pb + align_up(sizeof(int32_t) * P.i32_count, 256));
    int64_t *d_lay = d_cube + n;
    int64_t *d_bin = d_lay + n;
    int64_t *d_poff = d_bin + n;
    int64_t *d_pkoff = d_poff + n;
    int64_t *d_tc = d_pkoff + n;
    int64_t *d_ifin = d_tc + n;
    int64_t *d_fsin = d_ifin + n;
    int64_t *d_mu = d_fsin + n;

    const bool same_plan = h->plan_valid && h->plan_nl == P.nl && h->plan_nb == P.nb &&
                           h->plan_prec == cfg.precision && h->plan_cube == P.cube_off &&
                           h->plan_tc == P.tc_off && h->plan_if == P.if_off && h->plan_fs == P.fs_off &&
                           h->plan_mu == P.mu_idx;
    if (n > 0 && !same_plan) {
        if (cap) return fail(h, RT_EINVAL, "a new batch shape cannot be planned during stream capture");
        if (cfg.precision != RT_FP64_PLAIN) fill_units(P);
        const size_t need = P.plan_bytes;
        if (h->stage_pending) {
            cudaError_t e = cudaEventSynchronize(h->stage_ev);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
            h->stage_pending = false;
        }
        if (h->stage_cap < need) {
            if (h->h_stage) cudaFreeHost(h->h_stage);
            h->h_stage = nullptr;
            h->stage_cap = 0;
            cudaError_t e = cudaMallocHost(&h->h_stage, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(h, RT_ENOMEM, "cudaMallocHost(%zu): %s", need, cudaGetErrorString(e));
            }
            h->stage_cap = need;
        }
        char *hs = (char *)h->h_stage;
        int32_t *h32 = (int32_t *)hs;
        memcpy(h32, P.nl.data(), sizeof(int32_t) * n);
        memcpy(h32 + n, P.nb.data(), sizeof(int32_t) * n);
        memcpy(h32 + 2 * n, P.order.data(), sizeof(int32_t) * n);
        memcpy(h32 + 3 * n, P.col_units.data(), sizeof(int32_t) * n);
        if (P.n_units) {
            memcpy(h32 + 4 * n, P.unit_col.data(), sizeof(int32_t) * P.n_units);
            memcpy(h32 + 4 * n + P.n_units, P.unit_k.data(), sizeof(int32_t) * P.n_units);
        }
        int64_t *h64 = (int64_t *)(hs + align_up(sizeof(int32_t) * P.i32_count, 256));
        memcpy(h64, P.cube_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + n, P.lay_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + 2 * n, P.bin_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + 3 * n, P.part_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + 4 * n, P.planck_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + 5 * n, P.tc_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + 6 * n, P.if_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + 7 * n, P.fs_off.data(), sizeof(int64_t) * n);
        memcpy(h64 + 8 * n, P.mu_idx.data(), sizeof(int64_t) * n);
        cudaError_t e = cudaMemcpyAsync(h->plan.p, h->h_stage, need, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(h->stage_ev, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "plan upload");
        h->stage_pending = true;
        h->plan_nl = P.nl;
        h->plan_nb = P.nb;
        h->plan_prec = cfg.precision;
        h->plan_cube = P.cube_off;
        h->plan_tc = P.tc_off;
        h->plan_if = P.if_off;
        h->plan_fs = P.fs_off;
        h->plan_mu = P.mu_idx;
        h->plan_valid = true;
    }

    char *ob = (char *)h->out.p;
    double *F_up = (double *)ob;
    double *F_dn = F_up + P.n_if;
    double *F_net = F_dn + P.n_if;
    double *Q = (double *)(ob + align_up(sizeof(double) * 3 * (size_t)P.n_if, 256));
    double *toa = (double *)((char *)Q + align_up(sizeof(double) * (size_t)P.n_lay, 256));

    cudaError_t e = cudaSuccess;
    if (!optics_out) {
        e = cudaMemsetAsync(h->d_stats, 0, sizeof(unsigned long long) * rt::ST_COUNT, s);
        if (e == cudaSuccess && P.n_bins) e = cudaMemsetAsync(toa, 0, sizeof(double) * (size_t)P.n_bins, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_counter, 0, sizeof(int32_t), s);
    float *d_part = nullptr, *d_planck = nullptr, *d_fs = nullptr, *d_fboa = nullptr;
    float4 *d_colf = nullptr, *d_klay = nullptr;
    if (P.aux_bytes) {
        char *a = (char *)h->aux.p;
        d_part = (float *)a;
        a += align_up(sizeof(float) * (size_t)P.n_part, 256);
        d_planck = (float *)a;
        a += align_up(sizeof(float) * (size_t)P.n_planck, 256);
        d_fs = (float *)a;
        a += align_up(sizeof(float) * (size_t)P.n_bins, 256);
        d_fboa = (float *)a;
        a += align_up(sizeof(float) * (size_t)P.n_bins, 256);
        d_colf = (float4 *)a;
        a += align_up(sizeof(float4) * (size_t)n, 256);
        if (P.kt) d_klay = (float4 *)a;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");

    if (n > 0) {
        rt::KParams kp{};
        kp.dtau = cols->dtau;
        kp.w0 = cols->w0;
        kp.g0 = cols->g0;
        kp.T_center = cols->T_center;
        kp.T_iface = cols->T_iface;
        kp.p_iface = cols->p_iface;
        kp.mu_star = cols->mu_star;
        kp.F_star = cols->F_star;
        kp.n_layers = d_nl;
        kp.n_bins = d_nb;
        kp.cube_off = d_cube;
        kp.lay_off = d_lay;
        kp.bin_off = d_bin;
        kp.tc_off = d_tc;
        kp.if_off = d_ifin;
        kp.fs_off = d_fsin;
        kp.mu_idx = d_mu;
        kp.order = d_order;
        kp.n_cols = n;
        kp.n_g = cfg.n_g;
        kp.g_w = h->d_gw;
        kp.F_up = F_up;
        kp.F_dn = F_dn;
        kp.F_net = F_net;
        kp.Q = Q;
        kp.scr32 = (float4 *)h->scr.p;
        kp.scr64 = (double2 *)h->scr.p;
        kp.n_slots = P.n_slots;
        kp.counter = h->d_counter;
        kp.stats = h->d_stats;
        kp.improved = cfg.two_stream == RT_IMPROVED;
        kp.isothermal = cfg.layers == RT_ISOTHERMAL;
        kp.resonance_paper = cfg.resonance == RT_RESONANCE_PAPER;
        kp.e_clamp = cfg.e_clamp;
        kp.eps2 = cfg.eps2;
        kp.inv_eps2 = (float)(1.0 / cfg.eps2);
        kp.n_sweeps = P.sweeps ? cfg.n_sweeps : 0;
        kp.grav = cfg.grav;
        kp.cp = cfg.cp;
        kp.T_int = cfg.T_int;
        kp.F_toa = cfg.F_toa_diffuse;
        kp.wn_min = cfg.wn_min;
        kp.wn_max = cfg.wn_max;
        kp.edges = h->d_edges;
        kp.edges32 = h->d_edges32;
        kp.dnu32 = h->d_edges32 ? h->d_edges32 + h->edges.size() : nullptr;
        kp.toa = toa;
        kp.Lmax = P.Lmax;
        kp.nb_chunk = P.nb_chunk;
        kp.staged = P.staged;
        kp.unit_col = d_ucol;
        kp.unit_k = d_uk;
        kp.col_units = d_cu;
        kp.part_off = d_poff;
        kp.partial = d_part;
        kp.n_units = (int32_t)P.n_units;
        kp.warp_floats = P.warp_floats;
        kp.group_shift = P.group_shift;
        kp.back_depth = P.depth;
        kp.nbw = P.nbw;
        kp.direct = P.direct;
        kp.inline_b = P.inline_b;
        if (P.inline_b)
            kp.scrB = (char *)h->scr.p + align_up((size_t)P.n_slots * rt::fp32_scratch_per_slot(P.Lmax), 256);
        kp.ns = P.ns;
        kp.planck32 = d_planck;
        kp.planck_off = d_pkoff;
        kp.fs32 = d_fs;
        kp.fboa32 = d_fboa;
        kp.colf = d_colf;
        kp.g_w32 = h->d_gw32;
        if (P.kt) {
            kp.kt_lk = h->d_klk;
            kp.kt_bin = h->d_kbin;
            kp.kt_T = h->d_kT;
            kp.kt_lp = h->d_klp;
            kp.kt_nT = h->kt_nT;
            kp.kt_nP = h->kt_nP;
            kp.kt_lay = d_klay;
        }
        // array extents (read by bounds-check builds only)
        kp.ext.cube = cols->n_cube > 0 ? cols->n_cube : P.n_cube;
        kp.ext.center = cols->n_center > 0 ? cols->n_center : P.n_lay;
        kp.ext.iface = cols->n_iface > 0 ? cols->n_iface : P.n_if;
        kp.ext.fstar = cols->n_fstar > 0 ? cols->n_fstar : P.n_bins;
        kp.ext.mu = cols->n_mu > 0 ? cols->n_mu : n;
        kp.ext.scr32 = cfg.precision == RT_FP64_PLAIN ? 0
                       : P.sweeps ? P.n_slots * (long long)rt::kSweepMaxLayers / 2      // float2 (t, r) per layer
                                  : P.n_slots * (long long)P.Lmax;
        kp.ext.scr64 = cfg.precision == RT_FP64_PLAIN
                           ? (long long)(P.scr_bytes / sizeof(double2)) : 0;
        kp.ext.scrB = P.inline_b ? P.n_slots * (long long)P.Lmax : 0;
        kp.ext.part = P.n_part;
        kp.ext.planck = P.n_planck;
        kp.ext.bins = P.n_bins;
        kp.ext.cols = n;
        kp.ext.out_if = P.n_if;
        kp.ext.out_lay = P.n_lay;
#ifdef RT_BOUNDS_CHECK
        // test hook of the checking build: a smaller declared cube extent
        // (the reads past it stay inside the real arrays and are skipped)
        if (const char *sh = getenv("RT_BOUNDS_TEST_CUBE_EXTENT")) kp.ext.cube = atoll(sh);
#endif
        if (optics_out) {
            kp.ext.cube = P.n_cube;                  // the packed output cubes
            e = rt::launch_kt_optics(kp, d_cube, optics_out[0], optics_out[1], optics_out[2], s);
            if (e != cudaSuccess) return cuda_fail(h, e, "front-end launch");
            return RT_OK;
        }
        if (P.kt && cfg.precision == RT_FP64_PLAIN) {
            // the FP64 path solves from cubes: write the front end's optics first
            char *kc = (char *)h->kcube.p;
            const size_t cb = align_up(sizeof(float) * (size_t)P.n_cube, 256);
            float *cd = (float *)kc, *cw = (float *)(kc + cb), *cg = (float *)(kc + 2 * cb);
            e = rt::launch_kt_optics(kp, d_cube, cd, cw, cg, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "front-end launch");
            kp.dtau = cd;
            kp.w0 = cw;
            kp.g0 = cg;
            kp.ext.cube = P.n_cube;
            kp.kt_lk = nullptr;
        }
        const bool timing = cfg.kernel_timing && !cap;
        if (timing && cfg.precision == RT_FP64_PLAIN) cudaEventRecord(h->kev[1], s);
        e = cfg.precision == RT_FP64_PLAIN ? rt::launch_fp64(kp, P.grid, P.block, P.smem, s)
            : P.sweeps ? rt::launch_sweeps(kp, P.grid, P.block, P.smem, s, timing ? h->kev : nullptr)
                       : rt::launch_fp32(kp, P.grid, P.block, P.smem, s, timing ? h->kev : nullptr);
        if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
        if (timing && cfg.precision == RT_FP64_PLAIN) cudaEventRecord(h->kev[2], s);
        h->kev_valid = timing;
        h->kev_fp64 = cfg.precision == RT_FP64_PLAIN;
    }
    if (optics_out) return RT_OK;
    // A solve captured into a graph completes when the graph is replayed; the
    // caller orders later reads after the replay (same stream or a sync).
    if (!cap) {
        e = cudaEventRecord(h->done_ev, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventRecord");
    }
    h->done_valid = !cap;
    h->last_stream = s;
    h->solved = true;
    h->n_cols = n;
    h->n_if = P.n_if;
    h->n_lay = P.n_lay;
    h->n_sys = P.n_sys;
    h->n_bins = P.n_bins;
    return RT_OK;
}

// ---- k-table set-up on the host -------------------------------------------------

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n).
void gauss_nodes(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Rayleigh cross section per molecule, m^2 (App. C): 24 pi^3 / (N^2 lambda^4)
// ((n^2 - 1) / (n^2 + 2))^2 with King factor 1; the index is passed as n - 1.
double rayleigh(double lam_m, double n_minus_1, double n_ref) {
    const double pi = 3.14159265358979323846;
    const double d = n_minus_1 * (2.0 + n_minus_1);           // n^2 - 1
    const double f = d / (3.0 + d);                           // (n^2 - 1) / (n^2 + 2)
    const double l2 = lam_m * lam_m;
    return 24.0 * pi * pi * pi / (n_ref * n_ref * l2 * l2) * f * f;
}

// H2 + He mixture at wavenumber nu (cm^-1), App. C indices and reference densities.
double sigma_h2_he(double nu, double x_h2, double x_he) {
    const double lam_um = 1.0e4 / nu, lam_m = 1.0e-2 / nu;
    const double il2 = 1.0 / (lam_um * lam_um);
    const double n_h2 = 1.358e-4 * (1.0 + 7.52e-3 * il2);
    const double n_he = 1.0e-8 * (2283.0 + 1.8102e13 / (1.5342e10 - il2));
    return x_h2 * rayleigh(lam_m, n_h2, 2.68678e25) + x_he * rayleigh(lam_m, n_he, 2.546899e25);
}

}  // namespace

extern "C" {

int rt_solve_columns(rt_handle *h, const rt_columns *cols, void *stream) {
    return solve_impl(h, cols, stream, false, nullptr);
}

int rt_solve_ktable(rt_handle *h, const rt_columns *cols, void *stream) {
    if (!h) return RT_EINVAL;
    return solve_impl(h, cols, stream, true, nullptr);
}

int rt_ktable_optics(rt_handle *h, const rt_columns *cols, float *dtau, float *w0, float *g0, void *stream) {
    if (!h) return RT_EINVAL;
    if (!dtau || !w0 || !g0) return fail(h, RT_EINVAL, "optics outputs are NULL");
    float *const outs[3] = {dtau, w0, g0};
    return solve_impl(h, cols, stream, true, outs);
}

int rt_set_ktable(rt_handle *h, const rt_ktable *kt) {
    if (!h) return RT_EINVAL;
    h->err.clear();
    if (!kt) return fail(h, RT_EINVAL, "k-table is NULL");
    const rt_config &cfg = h->cfg;
    if (kt->n_T < 2 || kt->n_P < 2) return fail(h, RT_EINVAL, "k-table grid needs >= 2 points per axis");
    if (!kt->T_grid || !kt->log10p_grid || !kt->log10_kappa || !kt->sigma_scat_cloud || !kt->sigma_abs_cloud ||
        !kt->g0_cloud)
        return fail(h, RT_EINVAL, "k-table array is NULL");
    if (kt->n_bins < 1 || kt->n_bins > cfg.max_bins) return fail(h, RT_EINVAL, "k-table n_bins %d", kt->n_bins);
    if (kt->n_g != cfg.n_g) return fail(h, RT_EINVAL, "k-table n_g %d but the handle has %d", kt->n_g, cfg.n_g);
    if (cfg.n_edges > 1 && kt->n_bins != cfg.n_edges - 1)
        return fail(h, RT_EINVAL, "k-table n_bins %d but %d bin edges", kt->n_bins, cfg.n_edges);
    for (int i = 1; i < kt->n_T; ++i)
        if (!(kt->T_grid[i] > kt->T_grid[i - 1])) return fail(h, RT_EINVAL, "T grid not increasing");
    for (int i = 1; i < kt->n_P; ++i)
        if (!(kt->log10p_grid[i] > kt->log10p_grid[i - 1])) return fail(h, RT_EINVAL, "log10 p grid not increasing");
    if (!std::isfinite(kt->T_grid[0]) || !std::isfinite(kt->T_grid[kt->n_T - 1]) ||
        !std::isfinite(kt->log10p_grid[0]) || !std::isfinite(kt->log10p_grid[kt->n_P - 1]))
        return fail(h, RT_EINVAL, "k-table grid not finite");
    if (!(kt->f_cloud >= 0.0) || !(kt->x_H2 >= 0.0) || !(kt->x_He >= 0.0) || !(kt->mbar_amu > 0.0))
        return fail(h, RT_EINVAL, "f_cloud, x_H2, x_He must be >= 0 and mbar > 0");
    const int64_t S = (int64_t)kt->n_bins * cfg.n_g;
    const int64_t n_tab = (int64_t)kt->n_T * kt->n_P * S;
    // device layout: the T-neighbours side by side, [n_T - 1][n_P][S][2] =
    // (log10 kappa at iT, at iT + 1), so that a system's four cell corners
    // are two 8-byte loads and its two interpolations along log p one paired
    // operation
    const int64_t n_pair = (int64_t)(kt->n_T - 1) * kt->n_P * S * 2;
    if (n_pair >= INT32_MAX) return fail(h, RT_EINVAL, "k-table too large (%lld entries)", (long long)n_tab);
    for (int b = 0; b < kt->n_bins; ++b)
        if (!(kt->sigma_scat_cloud[b] >= 0.0) || !(kt->sigma_abs_cloud[b] >= 0.0) || !(fabs(kt->g0_cloud[b]) < 1.0))
            return fail(h, RT_EINVAL, "bin %d: cloud data out of range", b);

    // per-bin scattering and cloud absorption per unit mass, and g0
    std::vector<double> gx, gwt;
    gauss_nodes(8, gx, gwt);
    const double mbar = kt->mbar_amu * 1.66053906660e-27;
    std::vector<float4> bin(kt->n_bins);
    for (int b = 0; b < kt->n_bins; ++b) {
        const double lo = cfg.wn_edges ? cfg.wn_edges[b] : cfg.wn_min + b * (cfg.wn_max - cfg.wn_min) / kt->n_bins;
        const double hi = cfg.wn_edges ? cfg.wn_edges[b + 1]
                                       : cfg.wn_min + (b + 1) * (cfg.wn_max - cfg.wn_min) / kt->n_bins;
        // bin mean of the gas cross section: 8 sub-intervals x 8-point Gauss-Legendre
        const int nsub = 8;
        const double h_sub = (hi - lo) / nsub;
        double acc = 0.0;
        for (int k = 0; k < nsub; ++k) {
            const double mid = lo + (k + 0.5) * h_sub;
            for (int j = 0; j < 8; ++j) {
                const double nu = mid + 0.5 * h_sub * gx[j];
                if (nu > 0.0) acc += 0.5 * h_sub * gwt[j] * sigma_h2_he(nu, kt->x_H2, kt->x_He);
            }
        }
        const double sg = acc / (hi - lo);
        const double scat = sg + kt->f_cloud * kt->sigma_scat_cloud[b];
        const double g0 = scat > 0.0 ? kt->f_cloud * kt->sigma_scat_cloud[b] / scat * kt->g0_cloud[b] : 0.0;
        bin[b] = make_float4((float)(scat / mbar), (float)(kt->f_cloud * kt->sigma_abs_cloud[b] / mbar), (float)g0, 0.f);
    }

    cudaError_t e = cudaDeviceSynchronize();      // earlier solves may still read the old table
    cudaFree(h->d_klk);
    cudaFree(h->d_kbin);
    cudaFree(h->d_kT);
    cudaFree(h->d_klp);
    h->d_klk = nullptr;
    h->d_kbin = nullptr;
    h->d_kT = h->d_klp = nullptr;
    h->kt_set = false;
    std::vector<float> pairs((size_t)n_pair);
    for (int64_t iT = 0; iT + 1 < kt->n_T; ++iT)
        for (int64_t iP = 0; iP < kt->n_P; ++iP) {
            const float *lo = kt->log10_kappa + (iT * kt->n_P + iP) * S, *hi = lo + kt->n_P * S;
            float *d = pairs.data() + (iT * kt->n_P + iP) * S * 2;
            for (int64_t s = 0; s < S; ++s) {
                d[2 * s] = lo[s];
                d[2 * s + 1] = hi[s];
            }
        }
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_klk, sizeof(float) * (size_t)n_pair);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_klk, pairs.data(), sizeof(float) * (size_t)n_pair, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_kbin, sizeof(float4) * bin.size());
    if (e == cudaSuccess) e = cudaMemcpy(h->d_kbin, bin.data(), sizeof(float4) * bin.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_kT, sizeof(double) * kt->n_T);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_kT, kt->T_grid, sizeof(double) * kt->n_T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_klp, sizeof(double) * kt->n_P);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_klp, kt->log10p_grid, sizeof(double) * kt->n_P, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(h, e, "k-table upload");
    }
    h->kt_nT = kt->n_T;
    h->kt_nP = kt->n_P;
    h->kt_NB = kt->n_bins;
    h->kt_set = true;
    return RT_OK;
}

static int copy_out(rt_handle *h, void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (!dst || bytes == 0) return RT_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync");
    return RT_OK;
}

int rt_fluxes(rt_handle *h, double *F_up, double *F_down, double *F_net, void *stream) {
    if (!h) return RT_EINVAL;
    if (!h->solved) return fail(h, RT_ENOTSOLVED, "rt_fluxes before rt_solve_columns");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->done_valid && s != h->last_stream && !stream_capturing(s)) {
        cudaError_t e = cudaStreamWaitEvent(s, h->done_ev, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamWaitEvent");
    }
    const double *base = (const double *)h->out.p;
    const size_t b = sizeof(double) * (size_t)h->n_if;
    int rc = copy_out(h, F_up, base, b, s);
    if (!rc) rc = copy_out(h, F_down, base + h->n_if, b, s);
    if (!rc) rc = copy_out(h, F_net, base + 2 * h->n_if, b, s);
    return rc;
}

int rt_heating(rt_handle *h, double *Q, void *stream) {
    if (!h) return RT_EINVAL;
    if (!h->solved) return fail(h, RT_ENOTSOLVED, "rt_heating before rt_solve_columns");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->done_valid && s != h->last_stream && !stream_capturing(s)) {
        cudaError_t e = cudaStreamWaitEvent(s, h->done_ev, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamWaitEvent");
    }
    const char *ob = (const char *)h->out.p;
    const double *q = (const double *)(ob + align_up(sizeof(double) * 3 * (size_t)h->n_if, 256));
    return copy_out(h, Q, q, sizeof(double) * (size_t)h->n_lay, s);
}

int rt_toa_spectrum(rt_handle *h, double *F_up_toa, void *stream) {
    if (!h) return RT_EINVAL;
    if (!h->solved) return fail(h, RT_ENOTSOLVED, "rt_toa_spectrum before rt_solve_columns");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->done_valid && s != h->last_stream && !stream_capturing(s)) {
        cudaError_t e = cudaStreamWaitEvent(s, h->done_ev, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamWaitEvent");
    }
    const char *ob = (const char *)h->out.p;
    const char *q = ob + align_up(sizeof(double) * 3 * (size_t)h->n_if, 256);
    const double *toa = (const double *)(q + align_up(sizeof(double) * (size_t)h->n_lay, 256));
    return copy_out(h, F_up_toa, toa, sizeof(double) * (size_t)h->n_bins, s);
}

int rt_kernel_times(rt_handle *h, float *prep_ms, float *solve_ms) {
    if (!h) return RT_EINVAL;
    if (!h->kev_valid) return fail(h, RT_ENOTSOLVED, "no timed solve (cfg.kernel_timing)");
    cudaError_t e = cudaEventSynchronize(h->kev[2]);
    float a = 0.f, b = 0.f;
    if (e == cudaSuccess && !h->kev_fp64) e = cudaEventElapsedTime(&a, h->kev[0], h->kev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, h->kev[1], h->kev[2]);
    if (e != cudaSuccess) return cuda_fail(h, e, "rt_kernel_times");
    if (prep_ms) *prep_ms = a;
    if (solve_ms) *solve_ms = b;
    return RT_OK;
}

int rt_stats(rt_handle *h, rt_stats_t *out) {
    if (!h || !out) return RT_EINVAL;
    if (!h->solved) return fail(h, RT_ENOTSOLVED, "rt_stats before rt_solve_columns");
    cudaError_t e = h->done_valid ? cudaEventSynchronize(h->done_ev) : cudaDeviceSynchronize();
    unsigned long long v[rt::ST_COUNT] = {0};
    if (e == cudaSuccess) e = cudaMemcpy(v, h->d_stats, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "rt_stats");
    out->systems = h->n_sys;
    out->resonance_hits = (int64_t)v[rt::ST_RESONANCE];
    out->etau_hits = (int64_t)v[rt::ST_ETAU];
    out->eclamp_hits = (int64_t)v[rt::ST_ECLAMP];
    out->invalid_inputs = (int64_t)v[rt::ST_INVALID];
    out->nonfinite_outputs = (int64_t)v[rt::ST_NONFINITE];
    out->fp64_evals = (int64_t)v[rt::ST_FP64];
    out->bounds_violations = (int64_t)v[rt::ST_BOUNDS];
    return RT_OK;
}

const char *rt_last_error(const rt_handle *h) { return h ? h->err.c_str() : "null handle"; }

int rt_inject_alloc_failures(int n) {
    if (n < 0) return RT_EINVAL;
    g_inject_allocs.store(n);
    return RT_OK;
}

void rt_destroy(rt_handle *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->d_gw);
    cudaFree(h->d_gw32);
    cudaFree(h->d_edges);
    cudaFree(h->d_edges32);
    cudaFree(h->d_klk);
    cudaFree(h->d_kbin);
    cudaFree(h->d_kT);
    cudaFree(h->d_klp);
    cudaFree(h->kcube.p);
    cudaFree(h->plan.p);
    cudaFree(h->out.p);
    cudaFree(h->scr.p);
    cudaFree(h->aux.p);
    cudaFree(h->d_counter);
    cudaFree(h->d_stats);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    if (h->done_ev) cudaEventDestroy(h->done_ev);
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    for (int i = 0; i < 3; ++i)
        if (h->kev[i]) cudaEventDestroy(h->kev[i]);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
