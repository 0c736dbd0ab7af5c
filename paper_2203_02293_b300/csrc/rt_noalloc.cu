// rt_noalloc.cu -- a solve entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: host programs whose device memory is
// handed out by their own pool or by a framework that forbids raw
// allocations, and loops that cannot afford the device-wide synchronisation
// an allocation may cause.  rt_solve_uniform_noalloc serves them.  It runs the same FP32 kernels
// as rt_solve_columns on a batch whose columns all have the same shape, and
// keeps every intermediate in one file-scope device array of fixed size
// (RT_NOALLOC_SCRATCH_BYTES).  That array is reserved on every GPU that loads
// this library and stays reserved until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "rt.h"
#include "rt_internal.h"

namespace {

// The scratch of every no-alloc call.  In host code its name only stands in
// for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];   // device address of g_noalloc_scratch, per device
std::mutex g_setup_mu;

constexpr int kMaxG = 64;

struct UniformPlan {
    int32_t n_cols, L, NB, n_g, upc;
    int32_t *nl, *nb, *order, *cu, *ucol, *uk;
    int64_t *cube, *lay, *bin, *part, *pk, *tc, *ifo, *fs, *mu;
    float *gw32;
    float gw[kMaxG];
};

// Per-column and per-unit tables of a uniform batch, written in place of the
// host-built plan that rt_solve_columns uploads.
__global__ void uniform_plan(UniformPlan a) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t S = (int64_t)a.NB * a.n_g;
    for (int64_t c = tid; c < a.n_cols; c += nth) {
        a.nl[c] = a.L;
        a.nb[c] = a.NB;
        a.order[c] = (int32_t)c;
        a.cu[c] = a.upc;
        a.cube[c] = c * a.L * S;
        a.lay[c] = c * a.L;
        a.bin[c] = c * a.NB;
        a.part[c] = c * a.upc * 2 * (int64_t)(a.L + 1);
        a.pk[c] = c * (int64_t)(2 * a.L + 1) * a.NB;
        a.tc[c] = c * a.L;
        a.ifo[c] = c * (a.L + 1);
        a.fs[c] = c * a.NB;
        a.mu[c] = c;
    }
    const int64_t nu = (int64_t)a.n_cols * a.upc;
    for (int64_t u = tid; u < nu; u += nth) {
        a.ucol[u] = (int32_t)(u / a.upc);
        a.uk[u] = (int32_t)(u % a.upc);
    }
    if (tid < a.n_g) a.gw32[tid] = a.gw[tid];
}

size_t up(size_t x) { return (x + 255) / 256 * 256; }

// Once per device, with that device current: look up the array's address.
int scratch_address(int dev, char **out) {
    if (dev < 0 || dev >= kMaxDevices) return RT_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return RT_ECUDA;
        }
        e = rt::init_kernels();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return RT_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = (char *)g_scratch_addr[dev];
    return RT_OK;
}

}  // namespace

extern "C" int rt_solve_uniform_noalloc(const rt_config *cfg, const rt_columns *cols, double *F_up,
                                        double *F_down, double *F_net, double *Q, void *stream) {
    if (!cfg || !cols || !F_up || !F_down || !F_net || !Q) return RT_EINVAL;
    if (cfg->precision != RT_FP32_FORM) return RT_EINVAL;
    if (cfg->n_edges != 0) return RT_EINVAL;                   // uniform bins only
    if (cfg->n_g < 1 || cfg->n_g > kMaxG || !cfg->g_weights) return RT_EINVAL;
    for (int i = 0; i < cfg->n_g; ++i)
        if (!(cfg->g_weights[i] >= 0.0)) return RT_EINVAL;     // as rt_create: no negative or NaN weight
    if (cfg->n_sweeps != 0) return RT_EINVAL;                  // Thomas's algorithm only
    if (!(cfg->wn_max > cfg->wn_min) || !(cfg->wn_min >= 0.0) || !(cfg->eps2 > 0.0) || !(cfg->cp > 0.0) ||
        !(cfg->T_int >= 0.0))
        return RT_EINVAL;
    if (cfg->two_stream != RT_IMPROVED && cfg->two_stream != RT_REGULAR) return RT_EINVAL;
    if (cfg->layers != RT_NONISOTHERMAL && cfg->layers != RT_ISOTHERMAL) return RT_EINVAL;
    if (cfg->resonance != RT_RESONANCE_PAPER && cfg->resonance != RT_RESONANCE_LIMIT) return RT_EINVAL;
    if (cols->n_layers || cols->n_bins) return RT_EINVAL;      // uniform shape only
    if (cols->cube_offset || cols->center_offset || cols->iface_offset || cols->bin_offset || cols->col_index)
        return RT_EINVAL;                                       // packed layout only
    const int64_t n = cols->n_cols, L = cols->L, NB = cols->NB, NG = cfg->n_g;
    if (n < 1 || L < 1 || L > rt::kMaxLayers || NB < 1) return RT_EINVAL;
    if (!cols->dtau || !cols->w0 || !cols->g0 || !cols->T_center || !cols->T_iface || !cols->p_iface ||
        !cols->mu_star || !cols->F_star)
        return RT_EINVAL;
    // element counts, where given, must cover the packed batch
    const int64_t need_cnt[5] = {n * L * NB * NG, n * L, n * (L + 1), n * NB, n};
    const int64_t have_cnt[5] = {cols->n_cube, cols->n_center, cols->n_iface, cols->n_fstar, cols->n_mu};
    for (int i = 0; i < 5; ++i)
        if (have_cnt[i] < 0 || (have_cnt[i] > 0 && have_cnt[i] < need_cnt[i])) return RT_EINVAL;

    // carve the fixed scratch; refuse batches that do not fit
    const int64_t upc = (NB * NG + 31) / 32, nu = n * upc;
    if (nu > INT32_MAX) return RT_EBUDGET;
    const int nbw = rt::bins_per_chunk(32, (int)NG, (int)NB);
    const int staged = (2 * (int)L + 1) * nbw;    // staged Planck values per warp (nbw <= NB already)
    size_t off = 0;
    const size_t o_cnt = off;     off += up(sizeof(int32_t));
    const size_t o_stats = off;   off += up(sizeof(unsigned long long) * rt::ST_COUNT);
    const size_t o_part = off;    off += up(sizeof(float) * nu * 2 * (L + 1));
    const size_t o_planck = off;  off += up(sizeof(float) * n * (2 * L + 1) * NB);
    const size_t o_fs = off;      off += up(sizeof(float) * n * NB);
    const size_t o_fboa = off;    off += up(sizeof(float) * n * NB);
    const size_t o_colf = off;    off += up(sizeof(float4) * n);
    const size_t o_gw = off;      off += up(sizeof(float) * kMaxG);
    const size_t o_i32 = off;     off += up(sizeof(int32_t) * (4 * n + 2 * nu));
    const size_t o_i64 = off;     off += up(sizeof(int64_t) * 9 * n);
    const size_t o_scr = off;
    if (off >= (size_t)RT_NOALLOC_SCRATCH_BYTES) return RT_EBUDGET;
    const int64_t slots_fit = (int64_t)(((size_t)RT_NOALLOC_SCRATCH_BYTES - off) / (sizeof(float4) * (size_t)L));

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return RT_ECUDA;
    }
    char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return RT_ECUDA;
    }

    // launch shape: the CTA size (at most cfg->block_threads) that keeps the
    // most threads resident within the slots the scratch holds, preferring
    // a grid that reaches every SM
    int bmax = cfg->block_threads ? cfg->block_threads : rt::kMaxBlock32;
    if (bmax > rt::kMaxBlock32) bmax = rt::kMaxBlock32;
    if (bmax % 32 || bmax < 64) return RT_EINVAL;
    size_t smem = 0;
    int grid = 0, block = 0;
    int64_t best = 0;
    for (int b = bmax; b >= 64; b -= 32) {
        const size_t sm = rt::fp32_smem_bytes(b, (int)L, nbw, 0, 1, 4, 0, 2, staged);
        const int occ = rt::occupancy(0, b, sm);
        int64_t g = (int64_t)occ * sms;
        const int64_t by_scr = slots_fit / b;
        if (g > by_scr) g = by_scr;
        const int64_t by_work = (nu + b / 32 - 1) / (b / 32);
        if (g > by_work) g = by_work;
        if (occ <= 0 || g <= 0) continue;
        const int64_t score = g * b + (g >= sms ? (int64_t)1 << 40 : 0);
        if (score > best) {
            best = score;
            grid = (int)g;
            block = b;
            smem = sm;
        }
    }
    if (!grid) return RT_EBUDGET;

    cudaStream_t s = (cudaStream_t)stream;
    int32_t *counter = (int32_t *)(base + o_cnt);
    unsigned long long *stats = (unsigned long long *)(base + o_stats);
    int32_t *i32 = (int32_t *)(base + o_i32);
    int64_t *i64 = (int64_t *)(base + o_i64);

    // everything that must start at zero: work counter and branch counters
    // (the array keeps the last call's data)
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * rt::ST_COUNT, s);
    if (e != cudaSuccess) return RT_ECUDA;

    UniformPlan a{};
    a.n_cols = (int32_t)n;
    a.L = (int32_t)L;
    a.NB = (int32_t)NB;
    a.n_g = (int32_t)NG;
    a.upc = (int32_t)upc;
    a.nl = i32;
    a.nb = i32 + n;
    a.order = i32 + 2 * n;
    a.cu = i32 + 3 * n;
    a.ucol = i32 + 4 * n;
    a.uk = i32 + 4 * n + nu;
    a.cube = i64;
    a.lay = i64 + n;
    a.bin = i64 + 2 * n;
    a.part = i64 + 3 * n;
    a.pk = i64 + 4 * n;
    a.tc = i64 + 5 * n;
    a.ifo = i64 + 6 * n;
    a.fs = i64 + 7 * n;
    a.mu = i64 + 8 * n;
    a.gw32 = (float *)(base + o_gw);
    for (int i = 0; i < NG; ++i) a.gw[i] = (float)cfg->g_weights[i];
    int pgrid = (int)((std::max<int64_t>(n, nu) + 255) / 256);
    if (pgrid > 4 * sms) pgrid = 4 * sms;
    uniform_plan<<<pgrid, 256, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return RT_ECUDA;

    rt::KParams kp{};
    kp.dtau = cols->dtau;
    kp.w0 = cols->w0;
    kp.g0 = cols->g0;
    kp.T_center = cols->T_center;
    kp.T_iface = cols->T_iface;
    kp.p_iface = cols->p_iface;
    kp.mu_star = cols->mu_star;
    kp.F_star = cols->F_star;
    kp.n_layers = a.nl;
    kp.n_bins = a.nb;
    kp.cube_off = a.cube;
    kp.lay_off = a.lay;
    kp.bin_off = a.bin;
    kp.tc_off = a.tc;
    kp.if_off = a.ifo;
    kp.fs_off = a.fs;
    kp.mu_idx = a.mu;
    kp.order = a.order;
    kp.n_cols = (int32_t)n;
    kp.n_g = (int32_t)NG;
    kp.g_w = nullptr;
    kp.F_up = F_up;
    kp.F_dn = F_down;
    kp.F_net = F_net;
    kp.Q = Q;
    kp.scr32 = (float4 *)(base + o_scr);
    kp.n_slots = (int64_t)grid * block;
    kp.counter = counter;
    kp.stats = stats;
    kp.improved = cfg->two_stream == RT_IMPROVED;
    kp.isothermal = cfg->layers == RT_ISOTHERMAL;
    kp.resonance_paper = cfg->resonance == RT_RESONANCE_PAPER;
    kp.e_clamp = cfg->e_clamp;
    kp.eps2 = cfg->eps2;
    kp.inv_eps2 = (float)(1.0 / cfg->eps2);
    kp.grav = cfg->grav;
    kp.cp = cfg->cp;
    kp.T_int = cfg->T_int;
    kp.F_toa = cfg->F_toa_diffuse;
    kp.wn_min = cfg->wn_min;
    kp.wn_max = cfg->wn_max;
    kp.Lmax = (int32_t)L;
    kp.unit_col = a.ucol;
    kp.unit_k = a.uk;
    kp.col_units = a.cu;
    kp.part_off = a.part;
    kp.partial = (float *)(base + o_part);
    kp.n_units = (int32_t)nu;
    kp.warp_floats = rt::fp32_warp_floats((int)L, nbw, 0, 1, 4, 0, 2, staged);
    kp.staged = staged;
    kp.group_shift = 4;
    kp.back_depth = 2;
    kp.nbw = nbw;
    kp.planck32 = (float *)(base + o_planck);
    kp.planck_off = a.pk;
    kp.fs32 = (float *)(base + o_fs);
    kp.fboa32 = (float *)(base + o_fboa);
    kp.colf = (float4 *)(base + o_colf);
    kp.g_w32 = a.gw32;
    kp.ext.cube = n * L * NB * NG;
    kp.ext.center = n * L;
    kp.ext.iface = n * (L + 1);
    kp.ext.fstar = n * NB;
    kp.ext.mu = n;
    kp.ext.scr32 = (long long)(((size_t)RT_NOALLOC_SCRATCH_BYTES - o_scr) / sizeof(float4));
    kp.ext.part = nu * 2 * (L + 1);
    kp.ext.planck = n * (2 * L + 1) * NB;
    kp.ext.bins = n * NB;
    kp.ext.cols = n;
    kp.ext.out_if = n * (L + 1);
    kp.ext.out_lay = n * L;
    e = rt::launch_fp32(kp, grid, block, smem, s);
    return e == cudaSuccess ? RT_OK : RT_ECUDA;
}
