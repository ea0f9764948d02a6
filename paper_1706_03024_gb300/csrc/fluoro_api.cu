// fluoro_api.cu -- host side of the C ABI declared in include/fluoro.h.
//
// Validates inputs, builds the per-medium spectral tables (absorption per unit concentration,
// emission CDFs of Eq. 10, per-bin majorant), lays the dye grids out interleaved in HBM, and
// launches the sm_103a kernels of fluoro_kernels.cu. No compute runs on the host beyond these
// small tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fluoro.h"
#include "fluoro_internal.cuh"

namespace {
// An NVTX range over one C-ABI call, so that a whole-program trace shows the library's calls
// around their kernels (a no-op unless a profiling tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

using namespace flr;

struct flr_ctx {
    int device = 0;
    std::string err;
    int B = 0;
    double lambda0 = 0.0, dlambda = 0.0;
    int n_dyes = 0;
    std::vector<float> abs_shape, emit_spec, eps, qy;
    std::vector<flr_source> sources;
    bool medium_set = false;
    flr_medium medium{};
    float cmax[MAXD] = {0, 0, 0, 0};
    float smax = 1.0f;
    float4 *d_grid = nullptr;
    size_t grid_cap = 0;
    bool sensor_set = false;
    flr_sensor sensor{};
    bool tables_dirty = true;
    float *d_tables = nullptr;
    unsigned long long *d_tallies = nullptr;
    unsigned long long *d_counters = nullptr;
    int *d_error = nullptr;
    unsigned long long *d_work = nullptr;
    unsigned int *d_scratch = nullptr;  // medium upload: [0..MAXD) dye maxima (bits), [MAXD] bad-value flag, [MAXD+1] solvent present
    // two-pass adjoint replay (warp-regrouped form): per-path contributions of one path chunk
    float *d_adj_ak = nullptr;
    size_t adj_ak_cap = 0;
    float *d_adj_ovf = nullptr;
    size_t adj_ovf_cap = 0;
    unsigned long long *d_adj_tal = nullptr;  // the replays' tallies (written, never read)
    size_t adj_tal_cap = 0;
    unsigned long long *d_film_fx = nullptr;  // a launch's film sums in fixed point (film-sized)
    size_t film_fx_cap = 0;
    uint64_t paths_since_clear = 0;
    std::vector<float> h_tables;
    // local majorants of the current medium (built on demand for one cell size)
    float4 *d_mc_c = nullptr;
    float *d_mc_s = nullptr;
    uint8_t *d_mc_dist = nullptr;
    uint8_t *d_mc_tmp = nullptr;
    size_t mc_tmp_cap = 0;
    size_t mc_cap = 0;
    int mc_cell = 0;
    int mc_dims[3] = {0, 0, 0};
    double tables_margin = 0.0;  // majorant margin the uploaded tables were built with
    // batched form
    struct Batch {
        int n_media = 0;
        std::vector<uint64_t> n_paths;
        std::vector<int> n_dyes;
        float4 *d_arena = nullptr;
        size_t arena_cap = 0;
        flr::MediumDev *d_media = nullptr;
        size_t media_cap = 0;
        flr::ChunkDev *d_chunks = nullptr;
        size_t chunks_cap = 0;
        float *d_tables = nullptr;
        size_t tables_cap = 0;
        unsigned long long *d_tallies = nullptr;
        size_t tallies_cap = 0;
        unsigned long long *d_counters = nullptr;
        unsigned long long *d_head = nullptr;
        unsigned int *d_max = nullptr;
        size_t max_cap = 0;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        bool ready = false;
    } batch;
    cudaStream_t cap_stream = nullptr;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int fail(flr_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

// Every library-owned device buffer is allocated here. A test hook (flr_debug_fail_alloc) can make
// the k-th following allocation fail as out of memory, so that each caller's error path runs on
// the host without a real exhaustion; 0 (the default) leaves allocation alone.
static std::atomic<long long> g_fail_alloc{0};

cudaError_t dev_alloc(void **p, size_t bytes)
{
    if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}


template <class T>
cudaError_t dev_alloc(T **p, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}

int cuda_fail(flr_ctx *ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? FLR_ERR_OOM : FLR_ERR_CUDA, m);
}

bool finite3(const float *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Nearest bin centre, ties to the lower bin.
int snap_bin(double lambda_nm, double l0, double dl, int B)
{
    const double b = (lambda_nm - l0) / dl;
    int k = (int)std::ceil(b - 0.5);
    return std::min(std::max(k, 0), B - 1);
}

float round_up_f32(double v)
{
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

long long nvox(const flr_medium &m) { return (long long)m.dims[0] * m.dims[1] * m.dims[2]; }

bool medium_has_grid(const flr_medium &m)
{
    for (int d = 0; d < m.n_dyes; ++d)
        if (m.conc[d]) return true;
    return false;
}

// Per-medium spectral tables (host fp64, stored fp32): absorption per unit concentration, the
// emission CDF of Eq. 10 (running sum over the total, rounded to fp32, last entry 1), the per-bin
// majorant max_x sigma_t(x, lambda) (rounded up, with a 1e-6 relative margin for the kernels' fp32
// sums) and QY.
void build_medium_tables(const flr_ctx *ctx, const flr_medium &m, const float *cmax, float smax,
                         float *out, double margin = 0.0)
{
    const int B = ctx->B;
    std::fill(out, out + tab_size(B), 0.0f);
    float *sig = out + tab_sig_a(B);
    float *cdf = out + tab_cdf(B);
    float *maj = out + tab_majorant(B);
    float *imaj = out + tab_inv_majorant(B);
    float *qy = out + tab_qy(B);
    for (int b = 0; b < B; ++b) {
        double mj = (double)smax * ((double)m.sigma_s + (double)m.sigma_a0);
        for (int d = 0; d < m.n_dyes; ++d) {
            const int id = m.dye_ids[d];
            const double s = (double)ctx->eps[id] * (double)ctx->abs_shape[(size_t)id * B + b];
            sig[tab_sig_a_at(B, d, b)] = (float)s;
            mj += s * (double)cmax[d];
        }
        maj[b] = mj > 0.0 ? round_up_f32(mj * (1.0 + 1e-6) * (1.0 + margin)) : 0.0f;
        imaj[b] = maj[b] > 0.0f ? (float)(1.0 / (double)maj[b]) : 0.0f;
    }
    for (int d = 0; d < m.n_dyes; ++d) {
        const int id = m.dye_ids[d];
        const float *f = ctx->emit_spec.data() + (size_t)id * B;
        double tot = 0.0;
        for (int b = 0; b < B; ++b) tot += (double)f[b];
        double run = 0.0;
        for (int b = 0; b < B; ++b) {
            run += (double)f[b];
            cdf[d * B + b] = (float)(run / tot);
        }
        cdf[d * B + B - 1] = 1.0f;
        qy[d] = ctx->qy[id];
    }
}

void build_tables(flr_ctx *ctx)
{
    ctx->h_tables.assign(tab_size(ctx->B), 0.0f);
    build_medium_tables(ctx, ctx->medium, ctx->cmax, ctx->smax, ctx->h_tables.data(),
                        ctx->tables_margin);
}

// The spectral lines of a medium's sources, chosen in proportion to power (p(lambda_x), Eq. 12).
int build_emitters(flr_ctx *ctx, const flr_medium &m, int max_lines, EmitterDev *em, float *em_cdf,
                   int *n_out, int *group_first = nullptr, int *group_n = nullptr)
{
    int first = m.source_first, count = m.source_count;
    if (count == 0) { first = 0; count = (int)ctx->sources.size(); }
    if (first < 0 || count < 0 || first + count > (int)ctx->sources.size() || count == 0)
        return fail(ctx, FLR_ERR_STATE, "medium references sources that are not set");
    std::vector<double> pw;
    int n = 0;
    for (int s = first; s < first + count; ++s) {
        const flr_source &src = ctx->sources[s];
        const int g0 = n;
        for (int l = 0; l < src.n_lines; ++l) {
            if (n >= max_lines) return fail(ctx, FLR_ERR_ARG, "too many source lines for one medium");
            if (group_first) group_first[n] = g0;
            if (group_n) group_n[n] = src.n_lines;
            EmitterDev &e = em[n];
            for (int k = 0; k < 3; ++k) {
                e.origin[k] = src.origin[k];
                e.eu[k] = src.eu[k];
                e.ev[k] = src.ev[k];
                e.dir[k] = src.dir[k];
            }
            e.kind = src.kind;
            e.bin = snap_bin(src.lambda_nm[l], ctx->lambda0, ctx->dlambda, ctx->B);
            int ax = 0;
            for (int k = 1; k < 3; ++k)
                if (std::fabs(src.dir[k]) > std::fabs(src.dir[ax])) ax = k;
            e.axis = ax;
            e.sign = src.dir[ax] > 0.0f ? 1.0f : -1.0f;
            // entry through a dielectric face: the source's parallelogram lies in an open face's
            // plane and its direction (or normal) points into the box
            e.entry = -1;
            if (m.ior > 1.0f)
                for (int a = 0; a < 3 && e.entry < 0; ++a) {
                    if (src.eu[a] != 0.0f || src.ev[a] != 0.0f) continue;
                    int f = -1;
                    if (src.origin[a] == m.lo[a] && src.dir[a] > 0.0f) f = 2 * a;
                    if (src.origin[a] == m.hi[a] && src.dir[a] < 0.0f) f = 2 * a + 1;
                    if (f >= 0 && !(m.wall_mask & (1 << f))) e.entry = f;
                }
            pw.push_back((double)src.power[l]);
            ++n;
        }
    }
    double tot = 0.0;
    for (double v : pw) tot += v;
    if (!(tot > 0.0)) return fail(ctx, FLR_ERR_ARG, "total source power must be positive");
    double run = 0.0;
    for (int k = 0; k < n; ++k) {
        run += pw[k];
        em_cdf[k] = (float)(run / tot);
    }
    em_cdf[n - 1] = 1.0f;
    *n_out = n;
    return FLR_OK;
}

int fill_scene(flr_ctx *ctx, SceneDev &S, bool with_film, int macro_cell = 0, int skip_cell = 0)
{
    const flr_medium &m = ctx->medium;
    std::memset(&S, 0, sizeof(S));
    S.B = ctx->B;
    S.D = m.n_dyes;
    for (int k = 0; k < 3; ++k) {
        S.lo[k] = m.lo[k];
        S.hi[k] = m.hi[k];
        S.dims[k] = std::max(m.dims[k], 1);
        S.bdims[k] = grid_bricks(S.dims[k]);
        S.vox_scale[k] = (float)((double)S.dims[k] / ((double)m.hi[k] - (double)m.lo[k]));
    }
    S.grid = medium_has_grid(m) ? ctx->d_grid : nullptr;
    S.solvent = m.solvent;
    S.homogeneous = (S.grid == nullptr && S.solvent == nullptr) ? 1 : 0;
    for (int d = 0; d < MAXD; ++d) S.conc_uniform[d] = d < m.n_dyes ? m.conc_uniform[d] : 0.0f;
    S.sigma_s = m.sigma_s;
    S.sigma_a0 = m.sigma_a0;
    S.wall_mask = m.wall_mask;
    S.wall_albedo = m.wall_albedo;
    S.tables = ctx->d_tables;
    int ne = 0;
    const int rc = build_emitters(ctx, m, FLR_MAX_EMITTERS, S.em, S.em_cdf, &ne, S.em_group_first,
                                  S.em_group_n);
    if (rc != FLR_OK) return rc;
    S.n_emitters = ne;
    const int cell = macro_cell > 0 ? macro_cell : skip_cell;
    if (cell > 0 && !S.homogeneous && ctx->mc_cell == cell) {
        if (macro_cell > 0) S.mc = macro_cell; else S.sk = skip_cell;
        for (int k = 0; k < 3; ++k) {
            S.mc_dims[k] = ctx->mc_dims[k];
            const double cs = (double)cell * ((double)m.hi[k] - (double)m.lo[k]) / (double)S.dims[k];
            S.mc_size[k] = (float)cs;
            S.mc_inv[k] = (float)(1.0 / cs);
        }
        S.mc_c = ctx->d_mc_c;
        S.mc_s = ctx->d_mc_s;
        S.mc_dist = ctx->d_mc_dist;
    }
    S.maj_margin = (float)(1.0 + ctx->tables_margin);
    // interfaces and glossy walls
    S.dielectric = m.ior > 1.0f ? 1 : 0;
    S.iface = (S.dielectric || m.wall_gloss > 0.0f) ? 1 : 0;
    S.ior = S.dielectric ? m.ior : 1.0f;
    S.inv_ior = (float)(1.0 / (double)S.ior);
    {
        // Fresnel reflectance at normal incidence, ((n - 1)/(n + 1))^2, and the radiance factor
        const double n = (double)S.ior, f0 = ((n - 1.0) / (n + 1.0)) * ((n - 1.0) / (n + 1.0));
        S.iface_exit = (float)((1.0 - f0) / (n * n));
    }
    S.wall_gloss = m.wall_gloss;
    S.wall_exp = m.wall_exponent;
    // the instances that settle decisions without a grid read pay where the bounds decide most
    // steps: sigma_s + sigma_a0 (the minorant without a solvent mask) at least 0.9 of the
    // majorant of every bin that has one (measured: the light sheet at 0.99 gains 8 %, the
    // adjoint and paper-model media at lower albedo lose 13-16 % to the extra code)
    S.lazy = 0;
    if (S.grid && !S.solvent && ctx->h_tables.size() >= (size_t)tab_size(S.B)) {
        const float *maj = ctx->h_tables.data() + tab_majorant(S.B);
        const double smin = (double)m.sigma_s + (double)m.sigma_a0;
        bool ok = true;
        for (int b = 0; b < S.B && ok; ++b)
            if (maj[b] > 0.0f && smin < 0.9 * (double)maj[b]) ok = false;
        S.lazy = ok ? 1 : 0;
    }
    // sensor
    const flr_sensor &c = ctx->sensor;
    S.sensor_kind = (ctx->sensor_set && with_film) ? c.kind : FLR_SENSOR_NONE;
    if (S.sensor_kind != FLR_SENSOR_NONE) {
        S.W = c.width;
        S.H = c.height;
        for (int k = 0; k < 3; ++k) {
            S.s_origin[k] = c.origin[k];
            S.s_view[k] = c.view[k];
        }
        if (c.kind == FLR_SENSOR_ORTHO) {
            double uu = 0, vv = 0;
            for (int k = 0; k < 3; ++k) {
                uu += (double)c.U[k] * c.U[k];
                vv += (double)c.V[k] * c.V[k];
            }
            for (int k = 0; k < 3; ++k) {
                S.s_U[k] = (float)(c.U[k] / uu);
                S.s_V[k] = (float)(c.V[k] / vv);
                S.cam_U[k] = c.U[k];
                S.cam_V[k] = c.V[k];
            }
            S.inv_A_pix = (float)((double)c.width * c.height / (std::sqrt(uu) * std::sqrt(vv)));
        } else {
            for (int k = 0; k < 3; ++k) {
                S.s_U[k] = c.U[k];
                S.s_V[k] = c.V[k];
            }
            const double ty = std::tan(0.5 * (double)c.fov_y_deg * M_PI / 180.0);
            const double tx = ty * (double)c.width / (double)c.height;
            S.tan_x = (float)tx;
            S.tan_y = (float)ty;
            S.inv_tan_x = (float)(1.0 / tx);
            S.inv_tan_y = (float)(1.0 / ty);
            S.inv_A_pix = (float)((double)c.width * c.height / ((2.0 * tx) * (2.0 * ty)));
        }
    }
    return FLR_OK;
}

// Local-majorant grid of the current medium for cells of `cell`^3 voxels (built on `st` when the
// cell size differs from the one built last; the medium's packed grid must be current).
int prepare_macro(flr_ctx *ctx, int cell, cudaStream_t st)
{
    const flr_medium &m = ctx->medium;
    const bool grids = medium_has_grid(m) || m.solvent;
    if (cell <= 0 || !grids || ctx->mc_cell == cell) return FLR_OK;
    int md[3];
    size_t n = 1;
    for (int k = 0; k < 3; ++k) {
        md[k] = (m.dims[k] + cell - 1) / cell;
        n *= (size_t)md[k];
    }
    if (n > ctx->mc_cap) {
        cudaFree(ctx->d_mc_c);
        cudaFree(ctx->d_mc_s);
        cudaFree(ctx->d_mc_dist);
        ctx->d_mc_c = nullptr;
        ctx->d_mc_s = nullptr;
        ctx->d_mc_dist = nullptr;
        ctx->mc_cap = 0;
        cudaError_t e = dev_alloc(&ctx->d_mc_c, sizeof(float4) * n);
        if (e == cudaSuccess) e = dev_alloc(&ctx->d_mc_s, sizeof(float) * n);
        if (e == cudaSuccess) e = dev_alloc(&ctx->d_mc_dist, n);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "allocate the local-majorant grid");
        ctx->mc_cap = n;
    }
    float4 uni = make_float4(0.f, 0.f, 0.f, 0.f);
    float u[4] = {0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < m.n_dyes; ++d) u[d] = m.conc_uniform[d];
    uni = make_float4(u[0], u[1], u[2], u[3]);
    cudaError_t e = launch_build_macro(medium_has_grid(m) ? ctx->d_grid : nullptr, uni, m.solvent,
                                       m.dims, cell, md, ctx->d_mc_c, ctx->d_mc_s, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "build the local-majorant grid");
    // Chebyshev distance (in cells, capped at 31) from every empty cell to the nearest cell that
    // may hold matter, by repeated 26-neighbour relaxation on the device
    const int solvent_matter = ((double)m.sigma_s + (double)m.sigma_a0) > 0.0 ? 1 : 0;
    if (n > ctx->mc_tmp_cap) {
        cudaFree(ctx->d_mc_tmp);
        ctx->d_mc_tmp = nullptr;
        ctx->mc_tmp_cap = 0;
        e = dev_alloc(&ctx->d_mc_tmp, n);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "allocate the distance scratch");
        ctx->mc_tmp_cap = n;
    }
    e = launch_empty_distance(ctx->d_mc_c, ctx->d_mc_s, md, solvent_matter, 31, ctx->d_mc_dist,
                              ctx->d_mc_tmp, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "empty-space distances");
    ctx->mc_cell = cell;
    for (int k = 0; k < 3; ++k) ctx->mc_dims[k] = md[k];
    return FLR_OK;
}

int prepare_tables(flr_ctx *ctx, double margin, cudaStream_t st)
{
    if (margin != ctx->tables_margin) {
        ctx->tables_margin = margin;
        ctx->tables_dirty = true;
    }
    if (!ctx->tables_dirty) return FLR_OK;
    build_tables(ctx);
    // ordered on the caller's stream (pageable source: staged before the call returns)
    cudaError_t e = cudaMemcpyAsync(ctx->d_tables, ctx->h_tables.data(), sizeof(float) * ctx->h_tables.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload spectral tables");
    ctx->tables_dirty = false;
    return FLR_OK;
}

// Dielectric faces need an orthographic sensor looking along a face normal (or none); hero paths
// and the paper's model take index-matched faces and Lambertian walls only.
int check_interfaces(flr_ctx *ctx, const flr_medium &m, bool sensor_set, const flr_sensor &c, int hero,
                     int paper_mode)
{
    const bool dielectric = m.ior > 1.0f, special = dielectric || m.wall_gloss > 0.0f;
    if (special && (hero != 0 || paper_mode != 0))
        return fail(ctx, FLR_ERR_ARG, "interfaces: hero paths and the paper's model need index-matched faces and Lambertian walls");
    if (dielectric && sensor_set && c.kind != FLR_SENSOR_NONE) {
        if (c.kind != FLR_SENSOR_ORTHO)
            return fail(ctx, FLR_ERR_ARG, "interfaces: dielectric faces need an orthographic sensor");
        const int zeros = (c.view[0] == 0.0f) + (c.view[1] == 0.0f) + (c.view[2] == 0.0f);
        if (zeros != 2)
            return fail(ctx, FLR_ERR_ARG, "interfaces: the orthographic sensor must look along a face normal");
    }
    return FLR_OK;
}

// Checks one medium against the context's spectrum and dye table (no device work).
int validate_medium(flr_ctx *ctx, const flr_medium *m)
{
    if (!m) return fail(ctx, FLR_ERR_ARG, "medium: NULL");
    if (ctx->B <= 0) return fail(ctx, FLR_ERR_STATE, "set the spectrum before the medium");
    if (m->n_dyes < 0 || m->n_dyes > MAXD) return fail(ctx, FLR_ERR_ARG, "medium: 0..4 dyes");
    for (int k = 0; k < 3; ++k)
        if (!(std::isfinite(m->lo[k]) && std::isfinite(m->hi[k]) && m->hi[k] > m->lo[k]))
            return fail(ctx, FLR_ERR_ARG, "medium: box must have hi > lo");
    for (int d = 0; d < m->n_dyes; ++d) {
        if (m->dye_ids[d] < 0 || m->dye_ids[d] >= ctx->n_dyes)
            return fail(ctx, FLR_ERR_ARG, "medium: dye id outside the dye table");
        if (!m->conc[d] && !(std::isfinite(m->conc_uniform[d]) && m->conc_uniform[d] >= 0.0f))
            return fail(ctx, FLR_ERR_ARG, "medium: uniform concentration must be finite and >= 0");
    }
    if (!(std::isfinite(m->sigma_s) && m->sigma_s >= 0.0f && std::isfinite(m->sigma_a0) && m->sigma_a0 >= 0.0f))
        return fail(ctx, FLR_ERR_ARG, "medium: sigma_s and sigma_a0 must be finite and >= 0");
    if (m->wall_mask < 0 || m->wall_mask > 63 || !(m->wall_albedo >= 0.0f && m->wall_albedo <= 1.0f))
        return fail(ctx, FLR_ERR_ARG, "medium: wall mask 0..63 and albedo in [0,1]");
    if (!((m->ior == 0.0f || (m->ior >= 1.0f && m->ior <= 10.0f)) &&
          (m->wall_gloss >= 0.0f && m->wall_gloss <= 1.0f) &&
          (m->wall_exponent >= 0.0f && m->wall_exponent <= 10000.0f)))
        return fail(ctx, FLR_ERR_ARG, "medium: ior 0 or in [1, 10], wall_gloss in [0, 1], wall_exponent in [0, 1e4]");
    const bool grids = medium_has_grid(*m) || m->solvent;
    if (grids) {
        for (int k = 0; k < 3; ++k)
            if (m->dims[k] < 1 || m->dims[k] > 4096) return fail(ctx, FLR_ERR_ARG, "medium: dims 1..4096");
        // the kernels index voxels with 32-bit integers
        if ((long long)m->dims[0] * m->dims[1] * m->dims[2] > 2147483647LL ||
            packed_voxels(m->dims) > 2147483647LL)
            return fail(ctx, FLR_ERR_ARG, "medium: at most 2^31 - 1 voxels (also once padded to whole 4^3 bricks)");
        for (int d = 0; d < m->n_dyes; ++d)
            if (m->conc[d] && !is_device_pointer(m->conc[d]))
                return fail(ctx, FLR_ERR_ARG, "medium: concentration grids must be device memory");
        if (m->solvent && !is_device_pointer(m->solvent))
            return fail(ctx, FLR_ERR_ARG, "medium: solvent mask must be device memory");
    }
    return FLR_OK;
}

}  // namespace

extern "C" {

int flr_create(flr_ctx **out, int cuda_device)
{
    if (!out) return FLR_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
        cudaGetLastError();
        return FLR_ERR_ARG;
    }
    flr_ctx *ctx = new flr_ctx();
    ctx->device = cuda_device;
    DeviceGuard g(cuda_device);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dev_alloc(&ctx->d_tables, sizeof(float) * tab_size(FLR_MAX_BINS));
    if (e == cudaSuccess) e = dev_alloc(&ctx->d_tallies, sizeof(unsigned long long) * tal_size(FLR_MAX_BINS));
    if (e == cudaSuccess) e = dev_alloc(&ctx->d_counters, sizeof(unsigned long long) * FLR_NCOUNTERS);
    if (e == cudaSuccess) e = dev_alloc(&ctx->d_error, sizeof(int));
    if (e == cudaSuccess) e = dev_alloc(&ctx->d_work, sizeof(unsigned long long));
    if (e == cudaSuccess) e = dev_alloc(&ctx->d_scratch, sizeof(unsigned int) * 8);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_tallies, 0, sizeof(unsigned long long) * tal_size(FLR_MAX_BINS));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * FLR_NCOUNTERS);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_error, 0, sizeof(int));
    if (e != cudaSuccess) {
        flr_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? FLR_ERR_OOM : FLR_ERR_CUDA;
    }
    *out = ctx;
    return FLR_OK;
}

void flr_destroy(flr_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaFree(ctx->d_tables);
    cudaFree(ctx->d_tallies);
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_error);
    cudaFree(ctx->d_work);
    cudaFree(ctx->d_scratch);
    cudaFree(ctx->d_adj_ak);
    cudaFree(ctx->d_adj_ovf);
    cudaFree(ctx->d_adj_tal);
    cudaFree(ctx->d_film_fx);
    cudaFree(ctx->d_grid);
    cudaFree(ctx->d_mc_c);
    cudaFree(ctx->d_mc_s);
    cudaFree(ctx->d_mc_dist);
    cudaFree(ctx->d_mc_tmp);
    auto &bt = ctx->batch;
    if (bt.exec) cudaGraphExecDestroy(bt.exec);
    if (bt.graph) cudaGraphDestroy(bt.graph);
    cudaFree(bt.d_arena);
    cudaFree(bt.d_media);
    cudaFree(bt.d_chunks);
    cudaFree(bt.d_tables);
    cudaFree(bt.d_tallies);
    cudaFree(bt.d_counters);
    cudaFree(bt.d_head);
    cudaFree(bt.d_max);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

int flr_set_spectrum(flr_ctx *ctx, float lambda0_nm, float dlambda_nm, int n_bins)
{
    if (!ctx) return FLR_ERR_ARG;
    if (!(std::isfinite(lambda0_nm) && std::isfinite(dlambda_nm) && dlambda_nm > 0.0f) ||
        n_bins < 1 || n_bins > FLR_MAX_BINS)
        return fail(ctx, FLR_ERR_ARG, "spectrum: need finite lambda0, dlambda > 0, 1..128 bins");
    ctx->B = n_bins;
    ctx->lambda0 = lambda0_nm;
    ctx->dlambda = dlambda_nm;
    ctx->n_dyes = 0;
    ctx->abs_shape.clear();
    ctx->emit_spec.clear();
    ctx->eps.clear();
    ctx->qy.clear();
    ctx->medium_set = false;
    ctx->tables_dirty = true;
    return FLR_OK;
}

int flr_set_dyes(flr_ctx *ctx, int n, const float *abs_shape, const float *emit_spec,
                 const float *eps, const float *qy)
{
    if (!ctx) return FLR_ERR_ARG;
    if (ctx->B <= 0) return fail(ctx, FLR_ERR_STATE, "set the spectrum before the dyes");
    if (n < 1 || n > FLR_MAX_DYES || !abs_shape || !emit_spec || !eps || !qy)
        return fail(ctx, FLR_ERR_ARG, "dyes: need 1..1024 dyes and four host arrays");
    const int B = ctx->B;
    for (int d = 0; d < n; ++d) {
        double tot = 0.0;
        for (int b = 0; b < B; ++b) {
            const float a = abs_shape[(size_t)d * B + b], e = emit_spec[(size_t)d * B + b];
            if (!(std::isfinite(a) && a >= 0.0f && std::isfinite(e) && e >= 0.0f))
                return fail(ctx, FLR_ERR_ARG, "dyes: spectra must be finite and non-negative");
            tot += e;
        }
        if (!(tot > 0.0)) return fail(ctx, FLR_ERR_ARG, "dyes: an emission spectrum sums to zero");
        if (!(std::isfinite(eps[d]) && eps[d] >= 0.0f))
            return fail(ctx, FLR_ERR_ARG, "dyes: eps must be finite and non-negative");
        if (!(qy[d] >= 0.0f && qy[d] <= 1.0f)) return fail(ctx, FLR_ERR_ARG, "dyes: QY outside [0,1]");
    }
    ctx->n_dyes = n;
    ctx->abs_shape.assign(abs_shape, abs_shape + (size_t)n * B);
    ctx->emit_spec.assign(emit_spec, emit_spec + (size_t)n * B);
    ctx->eps.assign(eps, eps + n);
    ctx->qy.assign(qy, qy + n);
    if (ctx->medium_set) {
        for (int d = 0; d < ctx->medium.n_dyes; ++d)
            if (ctx->medium.dye_ids[d] >= n) ctx->medium_set = false;
    }
    ctx->tables_dirty = true;
    return FLR_OK;
}

int flr_set_sources(flr_ctx *ctx, int n, const flr_source *s)
{
    if (!ctx) return FLR_ERR_ARG;
    if (n < 1 || n > FLR_MAX_SOURCES || !s) return fail(ctx, FLR_ERR_ARG, "sources: need 1..65536");
    for (int i = 0; i < n; ++i) {
        const flr_source &q = s[i];
        if (q.kind != FLR_SOURCE_COLLIMATED && q.kind != FLR_SOURCE_LAMBERTIAN)
            return fail(ctx, FLR_ERR_ARG, "sources: unknown kind");
        if (!(finite3(q.origin) && finite3(q.eu) && finite3(q.ev) && finite3(q.dir)))
            return fail(ctx, FLR_ERR_ARG, "sources: non-finite geometry");
        const double len = std::sqrt((double)q.dir[0] * q.dir[0] + (double)q.dir[1] * q.dir[1] +
                                     (double)q.dir[2] * q.dir[2]);
        if (std::fabs(len - 1.0) > 1e-5) return fail(ctx, FLR_ERR_ARG, "sources: dir must be a unit vector");
        if (q.kind == FLR_SOURCE_LAMBERTIAN) {
            int nz = 0;
            for (int k = 0; k < 3; ++k) nz += q.dir[k] != 0.0f;
            if (nz != 1) return fail(ctx, FLR_ERR_ARG, "sources: Lambertian normals must be axis-aligned");
        }
        if (q.n_lines < 1 || q.n_lines > FLR_MAX_LINES)
            return fail(ctx, FLR_ERR_ARG, "sources: 1..8 lines per source");
        for (int l = 0; l < q.n_lines; ++l)
            if (!(std::isfinite(q.lambda_nm[l]) && std::isfinite(q.power[l]) && q.power[l] >= 0.0f))
                return fail(ctx, FLR_ERR_ARG, "sources: bad line");
    }
    ctx->sources.assign(s, s + n);
    return FLR_OK;
}

// The medium upload on `st`: the grids are packed, and their maxima (and a bad-value flag and the
// solvent mask's presence) are read back with one copy, synchronising `st`; `device_sync` keeps
// flr_set_medium's contract of a synchronised device.
static int set_medium_on(flr_ctx *ctx, const flr_medium *m, cudaStream_t st, bool device_sync)
{
    if (!ctx) return FLR_ERR_ARG;
    int vrc = validate_medium(ctx, m);
    if (vrc != FLR_OK) return vrc;
    const bool grids = medium_has_grid(*m) || m->solvent;
    DeviceGuard g(ctx->device);
    flr_medium mm = *m;
    if (!grids) mm.dims[0] = mm.dims[1] = mm.dims[2] = 1;
    const long long n = nvox(mm);
    float cmax[MAXD] = {0, 0, 0, 0};
    float smax = 1.0f;
    cudaError_t e;
    if (medium_has_grid(mm)) {
        const size_t np = (size_t)packed_voxels(mm.dims);
        if (np > ctx->grid_cap) {
            cudaFree(ctx->d_grid);
            ctx->d_grid = nullptr;
            ctx->grid_cap = 0;
            e = dev_alloc(&ctx->d_grid, sizeof(float4) * np);
            if (e != cudaSuccess) {
                ctx->medium_set = false;   // the previous medium's grid is gone: renders need a new upload
                return cuda_fail(ctx, e, "allocate the interleaved grid");
            }
            ctx->grid_cap = np;
        }
        e = launch_pack_grid(mm.conc, mm.conc_uniform, mm.n_dyes, mm.dims, ctx->d_grid, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "pack grids");
    }
    bool any_grid = false;
    for (int d = 0; d < mm.n_dyes; ++d) any_grid = any_grid || mm.conc[d];
    if (any_grid || mm.solvent) {
        unsigned int h[MAXD + 2] = {0, 0, 0, 0, 0, 0};
        e = cudaMemsetAsync(ctx->d_scratch, 0, sizeof(h), st);
        for (int d = 0; d < mm.n_dyes && e == cudaSuccess; ++d)
            if (mm.conc[d])
                e = launch_grid_max(mm.conc[d], n, ctx->d_scratch + d, (int *)(ctx->d_scratch + MAXD), st);
        if (e == cudaSuccess && mm.solvent) e = launch_solvent_any(mm.solvent, n, ctx->d_scratch + MAXD + 1, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, ctx->d_scratch, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "grid maxima");
        if (h[MAXD]) return fail(ctx, FLR_ERR_ARG, "medium: concentration grid has negative or non-finite values");
        for (int d = 0; d < mm.n_dyes; ++d)
            if (mm.conc[d]) std::memcpy(&cmax[d], &h[d], sizeof(float));
        if (mm.solvent) smax = h[MAXD + 1] ? 1.0f : 0.0f;
    }
    for (int d = 0; d < mm.n_dyes; ++d)
        if (!mm.conc[d]) cmax[d] = mm.conc_uniform[d];
    if (device_sync) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "set medium");
    }
    ctx->medium = mm;
    std::memcpy(ctx->cmax, cmax, sizeof(cmax));
    ctx->smax = smax;
    ctx->medium_set = true;
    ctx->tables_dirty = true;
    ctx->mc_cell = 0;
    return FLR_OK;
}

int flr_set_medium(flr_ctx *ctx, const flr_medium *m)
{
    const NvtxRange nvtx_range("flr_set_medium");
    return set_medium_on(ctx, m, 0, true);
}

int flr_set_medium_async(flr_ctx *ctx, const flr_medium *m, void *stream)
{
    const NvtxRange nvtx_range("flr_set_medium_async");
    return set_medium_on(ctx, m, (cudaStream_t)stream, false);
}

int flr_set_sensor(flr_ctx *ctx, const flr_sensor *c)
{
    if (!ctx) return FLR_ERR_ARG;
    if (!c) return fail(ctx, FLR_ERR_ARG, "sensor: NULL");
    if (c->kind == FLR_SENSOR_NONE) {
        ctx->sensor = *c;
        ctx->sensor_set = false;
        return FLR_OK;
    }
    if (c->kind != FLR_SENSOR_ORTHO && c->kind != FLR_SENSOR_PINHOLE)
        return fail(ctx, FLR_ERR_ARG, "sensor: unknown kind");
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return fail(ctx, FLR_ERR_ARG, "sensor: width and height 1..16384");
    if (!(finite3(c->origin) && finite3(c->U) && finite3(c->V) && finite3(c->view)))
        return fail(ctx, FLR_ERR_ARG, "sensor: non-finite geometry");
    if (c->kind == FLR_SENSOR_PINHOLE && !(c->fov_y_deg > 0.0f && c->fov_y_deg < 179.0f))
        return fail(ctx, FLR_ERR_ARG, "sensor: pinhole field of view in (0, 179) degrees");
    if (c->kind == FLR_SENSOR_ORTHO) {
        const double uu = (double)c->U[0] * c->U[0] + (double)c->U[1] * c->U[1] + (double)c->U[2] * c->U[2];
        const double vv = (double)c->V[0] * c->V[0] + (double)c->V[1] * c->V[1] + (double)c->V[2] * c->V[2];
        if (!(uu > 0.0 && vv > 0.0)) return fail(ctx, FLR_ERR_ARG, "sensor: film edges must be non-zero");
    }
    ctx->sensor = *c;
    ctx->sensor_set = true;
    return FLR_OK;
}

static int grow(flr_ctx *ctx, void **ptr, size_t *cap, size_t need, size_t elem, const char *what);

// Zeroes the context's film accumulator for a launch over n film values (grown on demand).
static int film_accumulator(flr_ctx *ctx, size_t n, cudaStream_t st);

int flr_render(flr_ctx *ctx, const flr_params *p, void *stream)
{
    const NvtxRange nvtx_range("flr_render");
    if (!ctx) return FLR_ERR_ARG;
    if (!p) return fail(ctx, FLR_ERR_ARG, "params: NULL");
    if (ctx->B <= 0 || !ctx->medium_set) return fail(ctx, FLR_ERR_STATE, "render: spectrum, dyes and medium must be set");
    if (ctx->sources.empty()) return fail(ctx, FLR_ERR_STATE, "render: no sources");
    if (p->form != FLR_FORM_PLAIN && p->form != FLR_FORM_WAVEFRONT && p->form != FLR_FORM_WAVEFRONT_WARP &&
        p->form != FLR_FORM_WAVEFRONT_POOL)
        return fail(ctx, FLR_ERR_ARG, "params: unknown form");
    if (p->form == FLR_FORM_WAVEFRONT_POOL && (p->macro_cell > 0 || p->hero > 0))
        return fail(ctx, FLR_ERR_ARG, "params: the pool form takes one majorant per bin and one wavelength per path");
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 256 || (p->block_size & 31)))
        return fail(ctx, FLR_ERR_ARG, "params: block_size must be 32..256, a multiple of 32");
    if (p->n_rr < 0 || p->max_events < 0 || p->max_steps < 1 || p->max_events > 2000000000LL)
        return fail(ctx, FLR_ERR_ARG, "params: n_rr, max_events >= 0, max_steps >= 1");
    if (p->macro_cell < 0 || p->macro_cell > 4096 || p->skip_cell < 0 || p->skip_cell > 4096)
        return fail(ctx, FLR_ERR_ARG, "params: macro_cell and skip_cell 0..4096");
    if (!(p->majorant_margin >= 0.0f && p->majorant_margin <= 100.0f))
        return fail(ctx, FLR_ERR_ARG, "params: majorant_margin in [0, 100]");
    if (p->hero < 0 || p->hero > 4) return fail(ctx, FLR_ERR_ARG, "params: hero must be 0..4");
    if (p->hero > 0 && (p->form == FLR_FORM_WAVEFRONT || p->macro_cell > 0 || p->paper_mode))
        return fail(ctx, FLR_ERR_ARG, "params: hero paths need the plain or warp form, no macro cells and no paper mode");
    if (p->film && !is_device_pointer(p->film)) return fail(ctx, FLR_ERR_ARG, "params: film must be device memory");
    if (p->path_events && !is_device_pointer(p->path_events))
        return fail(ctx, FLR_ERR_ARG, "params: path_events must be device memory");
    if (ctx->sensor_set && ctx->sensor.kind == FLR_SENSOR_PINHOLE) {
        const float *o = ctx->sensor.origin;
        bool inside = true;
        for (int k = 0; k < 3; ++k) inside = inside && o[k] >= ctx->medium.lo[k] && o[k] <= ctx->medium.hi[k];
        if (inside) return fail(ctx, FLR_ERR_ARG, "sensor: the pinhole must lie outside the medium box");
    }
    {
        const int irc = check_interfaces(ctx, ctx->medium, ctx->sensor_set && p->film, ctx->sensor, p->hero,
                                         p->paper_mode);
        if (irc != FLR_OK) return irc;
    }
    DeviceGuard g(ctx->device);
    int rc = prepare_tables(ctx, p->majorant_margin, (cudaStream_t)stream);
    if (rc != FLR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = prepare_macro(ctx, p->macro_cell > 0 ? p->macro_cell : p->skip_cell, st);
    if (rc != FLR_OK) return rc;
    SceneDev S;
    rc = fill_scene(ctx, S, p->film != nullptr, p->macro_cell, p->skip_cell);
    if (rc != FLR_OK) return rc;
    cudaError_t e = cudaSuccess;
    const bool film_on = p->film && S.sensor_kind != FLR_SENSOR_NONE;
    const size_t n_film = film_on ? (size_t)S.W * S.H * S.B : 0;
    if (!p->accumulate) {
        e = cudaMemsetAsync(ctx->d_tallies, 0, sizeof(unsigned long long) * tal_size(FLR_MAX_BINS), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_counters, 0, sizeof(unsigned long long) * FLR_NCOUNTERS, st);
        // a launch with paths writes every film value when it folds its sums
        if (e == cudaSuccess && film_on && p->n_paths == 0)
            e = cudaMemsetAsync(p->film, 0, sizeof(float) * n_film, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clear tallies");
        ctx->paths_since_clear = 0;
    }
    if (p->n_paths == 0) return FLR_OK;
    if (film_on) {
        rc = film_accumulator(ctx, n_film, st);
        if (rc != FLR_OK) return rc;
    }
    e = cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reset work counter");
    RunDev R;
    std::memset(&R, 0, sizeof(R));
    R.n_paths = p->n_paths;
    R.path_offset = p->path_offset;
    R.seed = p->seed;
    R.medium_id = p->medium_id;
    set_round_keys(R);
    R.n_rr = p->n_rr;
    R.max_inelastic = p->max_inelastic;
    R.analog = p->analog;
    R.max_events = p->max_events;
    R.max_steps = p->max_steps;
    R.film_scale = (float)(1.0 / (double)p->n_paths);
    R.film = film_on ? p->film : nullptr;
    R.film_fx = film_on ? ctx->d_film_fx : nullptr;
    R.path_events = p->path_events;
    R.tallies = ctx->d_tallies;
    R.counters = ctx->d_counters;
    R.error_word = ctx->d_error;
    R.work_counter = ctx->d_work;
    R.regroup = p->regroup_interval;
    R.paper_mode = p->paper_mode ? 1 : 0;
    R.hero = p->hero;
    e = launch_trace(S, R, p->form, p->block_size, p->blocks_per_sm, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch trace kernel");
    if (film_on) {
        e = launch_film_fold(p->film, ctx->d_film_fx, n_film, p->accumulate ? 1 : 0, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "fold film sums");
    }
    ctx->paths_since_clear += p->n_paths;
    return FLR_OK;
}

int flr_render_camera(flr_ctx *ctx, const flr_params *p, void *stream)
{
    const NvtxRange nvtx_range("flr_render_camera");
    if (!ctx) return FLR_ERR_ARG;
    if (!p) return fail(ctx, FLR_ERR_ARG, "params: NULL");
    if (ctx->B <= 0 || !ctx->medium_set) return fail(ctx, FLR_ERR_STATE, "camera: spectrum, dyes and medium must be set");
    if (ctx->sources.empty()) return fail(ctx, FLR_ERR_STATE, "camera: no sources");
    if (!ctx->sensor_set || ctx->sensor.kind == FLR_SENSOR_NONE) return fail(ctx, FLR_ERR_STATE, "camera: needs a sensor");
    if (ctx->medium.n_dyes < 1) return fail(ctx, FLR_ERR_ARG, "camera: the medium has no dyes");
    if (!p->film || !is_device_pointer(p->film)) return fail(ctx, FLR_ERR_ARG, "camera: p->film must be device memory");
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 256 || (p->block_size & 31)))
        return fail(ctx, FLR_ERR_ARG, "params: block_size must be 32..256, a multiple of 32");
    if (p->form != FLR_FORM_PLAIN && p->form != FLR_FORM_WAVEFRONT && p->form != FLR_FORM_WAVEFRONT_WARP)
        return fail(ctx, FLR_ERR_ARG, "params: unknown form");
    if (p->n_rr < 0 || p->max_events < 0 || p->max_steps < 1 || p->max_events > 2000000000LL)
        return fail(ctx, FLR_ERR_ARG, "params: n_rr, max_events >= 0, max_steps >= 1");
    if (p->hero != 0) return fail(ctx, FLR_ERR_ARG, "params: hero paths are for flr_render only");
    if (ctx->medium.ior > 1.0f || ctx->medium.wall_gloss > 0.0f)
        return fail(ctx, FLR_ERR_ARG, "camera: index-matched faces and Lambertian walls only");
    const uint64_t npix = (uint64_t)ctx->sensor.width * (uint64_t)ctx->sensor.height;
    if (p->n_paths % npix != 0 || p->path_offset % npix != 0)
        return fail(ctx, FLR_ERR_ARG, "camera: n_paths and path_offset must be multiples of the pixel count");
    if (ctx->sensor.kind == FLR_SENSOR_PINHOLE) {
        const float *o = ctx->sensor.origin;
        bool inside = true;
        for (int k = 0; k < 3; ++k) inside = inside && o[k] >= ctx->medium.lo[k] && o[k] <= ctx->medium.hi[k];
        if (inside) return fail(ctx, FLR_ERR_ARG, "sensor: the pinhole must lie outside the medium box");
    }
    {
        const flr_medium &m = ctx->medium;
        int first = m.source_first, count = m.source_count;
        if (count == 0) { first = 0; count = (int)ctx->sources.size(); }
        for (int k = first; k < first + count && k < (int)ctx->sources.size(); ++k) {
            const flr_source &src = ctx->sources[k];
            const double n0 = (double)src.eu[1] * src.ev[2] - (double)src.eu[2] * src.ev[1];
            const double n1 = (double)src.eu[2] * src.ev[0] - (double)src.eu[0] * src.ev[2];
            const double n2 = (double)src.eu[0] * src.ev[1] - (double)src.eu[1] * src.ev[0];
            if (!(n0 * n0 + n1 * n1 + n2 * n2 > 0.0))
                return fail(ctx, FLR_ERR_ARG, "camera: every source needs a non-zero area (no pencil beams)");
        }
    }
    DeviceGuard g(ctx->device);
    int rc = prepare_tables(ctx, 0.0, (cudaStream_t)stream);
    if (rc != FLR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    SceneDev S;
    rc = fill_scene(ctx, S, true, 0, 0);
    if (rc != FLR_OK) return rc;
    cudaError_t e = cudaSuccess;
    const size_t n_film = (size_t)S.W * S.H * S.B;
    if (!p->accumulate) {
        e = cudaMemsetAsync(ctx->d_counters, 0, sizeof(unsigned long long) * FLR_NCOUNTERS, st);
        // a launch with paths writes every film value when it folds its sums
        if (e == cudaSuccess && p->n_paths == 0) e = cudaMemsetAsync(p->film, 0, sizeof(float) * n_film, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clear film");
    }
    if (p->n_paths == 0) return FLR_OK;
    rc = film_accumulator(ctx, n_film, st);
    if (rc != FLR_OK) return rc;
    // the kernel's block tallies are flushed into a scratch copy: the camera estimator has none
    rc = grow(ctx, (void **)&ctx->d_adj_tal, &ctx->adj_tal_cap, (size_t)tal_size(FLR_MAX_BINS),
              sizeof(unsigned long long), "camera tallies");
    if (rc != FLR_OK) return rc;
    RunDev R;
    std::memset(&R, 0, sizeof(R));
    R.n_paths = p->n_paths;
    R.path_offset = p->path_offset;
    R.seed = p->seed;
    R.medium_id = p->medium_id;
    set_round_keys(R);
    R.n_rr = p->n_rr;
    R.analog = p->analog;
    R.max_events = p->max_events;
    R.max_steps = p->max_steps;
    R.film_scale = (float)((double)npix / (double)p->n_paths);
    R.film = p->film;
    R.film_fx = ctx->d_film_fx;
    R.tallies = ctx->d_adj_tal;
    R.counters = ctx->d_counters;
    R.error_word = ctx->d_error;
    R.work_counter = ctx->d_work;
    e = cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_camera(S, R, p->form, p->block_size, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch camera kernel");
    e = launch_film_fold(p->film, ctx->d_film_fx, n_film, p->accumulate ? 1 : 0, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fold film sums");
    return FLR_OK;
}

int flr_read_tallies(flr_ctx *ctx, double *face, double *absorbed, double *emitted,
                     uint64_t *counters, void *stream)
{
    const NvtxRange nvtx_range("flr_read_tallies");
    if (!ctx) return FLR_ERR_ARG;
    if (ctx->B <= 0) return fail(ctx, FLR_ERR_STATE, "read: no spectrum");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before reading tallies");
    const int B = ctx->B;
    std::vector<unsigned long long> t(tal_size(FLR_MAX_BINS));
    unsigned long long c[FLR_NCOUNTERS];
    e = cudaMemcpy(t.data(), ctx->d_tallies, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read tallies");
    const double inv = ctx->paths_since_clear ? 1.0 / ((double)ctx->paths_since_clear * TALLY_ONE) : 0.0;
    const int D = ctx->medium_set ? ctx->medium.n_dyes : 0;
    if (face)
        for (int i = 0; i < 12 * B; ++i) face[i] = (double)t[tal_face(B) + i] * inv;
    if (absorbed) {
        for (int d = 0; d < D; ++d)
            for (int b = 0; b < B; ++b) absorbed[d * B + b] = (double)t[tal_absorbed(B) + d * B + b] * inv;
        for (int b = 0; b < B; ++b) absorbed[D * B + b] = (double)t[tal_absorbed(B) + D * B + b] * inv;
    }
    if (emitted)
        for (int d = 0; d < D; ++d)
            for (int b = 0; b < B; ++b) emitted[d * B + b] = (double)t[tal_emitted(B) + d * B + b] * inv;
    if (counters)
        for (int k = 0; k < FLR_NCOUNTERS; ++k) counters[k] = c[k];
    return FLR_OK;
}

int flr_status(flr_ctx *ctx)
{
    if (!ctx) return FLR_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device status");
    int w = 0;
    e = cudaMemcpy(&w, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read error word");
    if (w) {
        // reported once: the word covers the launches since the previous flr_status
        e = cudaMemset(ctx->d_error, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clear error word");
        return fail(ctx, FLR_ERR_BUDGET, "a path or a sensor connection ran out of its step budget "
                                         "(counters step_budget / connect_budget)");
    }
    unsigned long long cw = 0ull;
    e = check_word_take(&cw);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read check word");
    if (cw) {
        const int site = (int)((cw >> 56) & 0x7F);
        const long long idx = (long long)(cw & 0x00FFFFFFFFFFFFFFull);
        return fail(ctx, FLR_ERR_CHECK, "checked build: index " + std::to_string(idx) +
                                            " out of range at access site " + std::to_string(site));
    }
    return FLR_OK;
}

int flr_checked_build(void) { return checked_build(); }

int flr_debug_check(int64_t index, int64_t bound, void *stream)
{
    const cudaError_t e = launch_debug_check((long long)index, (long long)bound, (cudaStream_t)stream);
    return e == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

const char *flr_last_error(flr_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int flr_debug_philox(uint32_t seed, uint32_t medium, const uint32_t *ctr, int64_t n, uint32_t *out,
                     void *stream)
{
    if (n < 0 || (n > 0 && (!ctr || !out))) return FLR_ERR_ARG;
    if (n == 0) return FLR_OK;
    if (!is_device_pointer(ctr) || !is_device_pointer(out)) return FLR_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) & 15u) return FLR_ERR_ARG;
    return launch_philox(seed, medium, ctr, n, out, (cudaStream_t)stream) == cudaSuccess ? FLR_OK : FLR_ERR_CUDA;
}

int flr_debug_sample_emission(flr_ctx *ctx, int dye, const float *u, int64_t n, int32_t *out, void *stream)
{
    if (!ctx) return FLR_ERR_ARG;
    if (!ctx->medium_set) return fail(ctx, FLR_ERR_STATE, "sample: no medium");
    if (dye < 0 || dye >= ctx->medium.n_dyes || n < 0) return fail(ctx, FLR_ERR_ARG, "sample: bad dye or n");
    if (n == 0) return FLR_OK;
    if (!is_device_pointer(u) || !is_device_pointer(out)) return fail(ctx, FLR_ERR_ARG, "sample: device buffers");
    DeviceGuard g(ctx->device);
    int rc = prepare_tables(ctx, 0.0, (cudaStream_t)stream);
    if (rc != FLR_OK) return rc;
    SceneDev S;
    std::memset(&S, 0, sizeof(S));
    S.B = ctx->B;
    S.tables = ctx->d_tables;
    cudaError_t e = launch_sample_emission(S, dye, u, n, out, (cudaStream_t)stream);
    return e == cudaSuccess ? FLR_OK : cuda_fail(ctx, e, "sample emission");
}

int flr_debug_fail_alloc(int64_t k)
{
    if (k < 0) return FLR_ERR_ARG;
    g_fail_alloc.store(k);
    return FLR_OK;
}


int flr_debug_sigma_t(flr_ctx *ctx, const float *points, int64_t n, int bin, float *sigma_t,
                      int32_t *voxel, void *stream)
{
    if (!ctx) return FLR_ERR_ARG;
    if (ctx->B <= 0 || !ctx->medium_set) return fail(ctx, FLR_ERR_STATE, "sigma_t: spectrum, dyes and medium must be set");
    if (bin < 0 || bin >= ctx->B || n < 0) return fail(ctx, FLR_ERR_ARG, "sigma_t: bin in [0, n_bins), n >= 0");
    if (n == 0) return FLR_OK;
    if (!points || !sigma_t || !is_device_pointer(points) || !is_device_pointer(sigma_t) ||
        (voxel && !is_device_pointer(voxel)))
        return fail(ctx, FLR_ERR_ARG, "sigma_t: points and outputs must be device memory");
    DeviceGuard g(ctx->device);
    int rc = prepare_tables(ctx, 0.0, (cudaStream_t)stream);
    if (rc != FLR_OK) return rc;
    SceneDev S;
    rc = fill_scene(ctx, S, false);
    if (rc != FLR_OK) return rc;
    cudaError_t e = launch_debug_sigma_t(S, points, n, bin, sigma_t, voxel, (cudaStream_t)stream);
    return e == cudaSuccess ? FLR_OK : cuda_fail(ctx, e, "sigma_t lookup");
}

// ---------------------------------------------------------------------------------------------
// Adjoint by path replay.

int flr_debug_frozen_sums(flr_ctx *ctx, const flr_params *p, const float *adj_film, int pert_dye,
                          int64_t pert_voxel, float pert_delta, float pert_sigma_s, double *out,
                          void *stream)
{
    const NvtxRange nvtx_range("flr_debug_frozen_sums");
    if (!ctx) return FLR_ERR_ARG;
    if (!p || !adj_film || !out) return fail(ctx, FLR_ERR_ARG, "frozen sums: params, adj_film and out are required");
    if (ctx->B <= 0 || !ctx->medium_set || ctx->sources.empty())
        return fail(ctx, FLR_ERR_STATE, "frozen sums: spectrum, dyes, medium and sources must be set");
    if (!ctx->sensor_set) return fail(ctx, FLR_ERR_STATE, "frozen sums: needs a sensor");
    if (p->n_rr < 0 || p->max_events < 0 || p->max_steps < 1 || p->max_events > 2000000000LL)
        return fail(ctx, FLR_ERR_ARG, "params: n_rr, max_events >= 0, max_steps >= 1");
    if (p->hero != 0 || p->paper_mode != 0 || p->macro_cell != 0 || p->skip_cell != 0)
        return fail(ctx, FLR_ERR_ARG, "frozen sums: one majorant per bin, no hero paths, no paper mode");
    if (!(p->majorant_margin >= 0.0f && p->majorant_margin <= 100.0f))
        return fail(ctx, FLR_ERR_ARG, "params: majorant_margin in [0, 100]");
    if (!is_device_pointer(adj_film) || !is_device_pointer(out))
        return fail(ctx, FLR_ERR_ARG, "frozen sums: adj_film and out must be device memory");
    const long long nv = nvox(ctx->medium);
    if (pert_dye >= ctx->medium.n_dyes || pert_dye < -1)
        return fail(ctx, FLR_ERR_ARG, "frozen sums: pert_dye must be -1 or a dye slot of the medium");
    if (pert_dye >= 0 && (!medium_has_grid(ctx->medium) || pert_voxel < 0 || pert_voxel >= nv))
        return fail(ctx, FLR_ERR_ARG, "frozen sums: a concentration perturbation needs grids and a voxel inside them");
    if (!std::isfinite(pert_delta) || !std::isfinite(pert_sigma_s))
        return fail(ctx, FLR_ERR_ARG, "frozen sums: finite perturbations");
    DeviceGuard g(ctx->device);
    int rc = prepare_tables(ctx, p->majorant_margin, (cudaStream_t)stream);
    if (rc != FLR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    SceneDev S;
    rc = fill_scene(ctx, S, true, 0, 0);
    if (rc != FLR_OK) return rc;
    if (p->n_paths == 0) return FLR_OK;
    RunDev R;
    std::memset(&R, 0, sizeof(R));
    R.n_paths = p->n_paths;
    R.path_offset = p->path_offset;
    R.seed = p->seed;
    R.medium_id = p->medium_id;
    set_round_keys(R);
    R.n_rr = p->n_rr;
    R.max_inelastic = p->max_inelastic;
    R.analog = p->analog;
    R.max_events = p->max_events;
    R.max_steps = p->max_steps;
    R.film_scale = (float)(1.0 / (double)p->n_paths);
    R.error_word = ctx->d_error;
    cudaError_t e = launch_frozen_sums(S, R, pert_dye, (long long)pert_voxel, pert_delta, pert_sigma_s,
                                       adj_film, out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch frozen-sum kernel");
    return FLR_OK;
}

// Contributions kept per path between the two adjoint passes, and paths replayed per pass pair.
constexpr int ADJ_K = 32;
constexpr uint64_t ADJ_CHUNK = 1ull << 21;

int flr_adjoint(flr_ctx *ctx, const flr_params *p, const float *adj_film, float *grad_conc,
                float *grad_sigma_s, void *stream)
{
    const NvtxRange nvtx_range("flr_adjoint");
    if (!ctx) return FLR_ERR_ARG;
    if (!p || !adj_film) return fail(ctx, FLR_ERR_ARG, "adjoint: params and adj_film are required");
    if (ctx->B <= 0 || !ctx->medium_set || ctx->sources.empty())
        return fail(ctx, FLR_ERR_STATE, "adjoint: spectrum, dyes, medium and sources must be set");
    if (!ctx->sensor_set) return fail(ctx, FLR_ERR_STATE, "adjoint: needs a sensor");
    if (p->form != FLR_FORM_PLAIN && p->form != FLR_FORM_WAVEFRONT && p->form != FLR_FORM_WAVEFRONT_WARP)
        return fail(ctx, FLR_ERR_ARG, "params: unknown form");
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 256 || (p->block_size & 31)))
        return fail(ctx, FLR_ERR_ARG, "params: block_size must be 32..256, a multiple of 32");
    if (p->n_rr < 0 || p->max_events < 0 || p->max_steps < 1 || p->max_events > 2000000000LL)
        return fail(ctx, FLR_ERR_ARG, "params: n_rr, max_events >= 0, max_steps >= 1");
    if (p->hero != 0) return fail(ctx, FLR_ERR_ARG, "params: hero paths are for flr_render only");
    {
        const int irc = check_interfaces(ctx, ctx->medium, true, ctx->sensor, 0, p->paper_mode);
        if (irc != FLR_OK) return irc;
    }
    if (!is_device_pointer(adj_film)) return fail(ctx, FLR_ERR_ARG, "adjoint: adj_film must be device memory");
    if (grad_conc && !medium_has_grid(ctx->medium))
        return fail(ctx, FLR_ERR_ARG, "adjoint: grad_conc needs a medium with concentration grids");
    if (grad_conc && !is_device_pointer(grad_conc)) return fail(ctx, FLR_ERR_ARG, "adjoint: grad_conc must be device memory");
    if (grad_sigma_s && !is_device_pointer(grad_sigma_s))
        return fail(ctx, FLR_ERR_ARG, "adjoint: grad_sigma_s must be device memory");
    if (p->macro_cell < 0 || p->macro_cell > 4096 || p->skip_cell < 0 || p->skip_cell > 4096)
        return fail(ctx, FLR_ERR_ARG, "params: macro_cell and skip_cell 0..4096");
    if (!(p->majorant_margin >= 0.0f && p->majorant_margin <= 100.0f))
        return fail(ctx, FLR_ERR_ARG, "params: majorant_margin in [0, 100]");
    DeviceGuard g(ctx->device);
    int rc = prepare_tables(ctx, p->majorant_margin, (cudaStream_t)stream);
    if (rc != FLR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = prepare_macro(ctx, p->macro_cell > 0 ? p->macro_cell : p->skip_cell, st);
    if (rc != FLR_OK) return rc;
    SceneDev S;
    rc = fill_scene(ctx, S, true, p->macro_cell, p->skip_cell);
    if (rc != FLR_OK) return rc;
    const long long nv = nvox(ctx->medium);
    cudaError_t e = cudaSuccess;
    if (!p->accumulate) {
        if (grad_conc) e = cudaMemsetAsync(grad_conc, 0, sizeof(float) * (size_t)ctx->medium.n_dyes * nv, st);
        if (e == cudaSuccess && grad_sigma_s) e = cudaMemsetAsync(grad_sigma_s, 0, sizeof(float), st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clear gradients");
    }
    if (p->n_paths == 0) return FLR_OK;
    RunDev R;
    std::memset(&R, 0, sizeof(R));
    R.n_paths = p->n_paths;
    R.path_offset = p->path_offset;
    R.seed = p->seed;
    R.medium_id = p->medium_id;
    set_round_keys(R);
    R.n_rr = p->n_rr;
    R.max_inelastic = p->max_inelastic;
    R.analog = p->analog;
    R.max_events = p->max_events;
    R.max_steps = p->max_steps;
    R.film_scale = (float)(1.0 / (double)p->n_paths);
    R.error_word = ctx->d_error;
    AdjDev A;
    std::memset(&A, 0, sizeof(A));
    A.adj = adj_film;
    A.grad_c = grad_conc;
    A.nvox = nv;
    A.grad_sigma_s = grad_sigma_s;
    if (p->form == FLR_FORM_PLAIN) {
        e = launch_adjoint(S, R, A, p->block_size, p->blocks_per_sm, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "launch adjoint kernel");
        return FLR_OK;
    }
    // warp-regrouped two-pass replay over chunks of at most ADJ_CHUNK paths
    const uint64_t chunk = std::min<uint64_t>(ADJ_CHUNK, p->n_paths);
    rc = grow(ctx, (void **)&ctx->d_adj_ak, &ctx->adj_ak_cap, (size_t)chunk * ADJ_K, sizeof(float),
              "adjoint contributions");
    if (rc != FLR_OK) return rc;
    rc = grow(ctx, (void **)&ctx->d_adj_ovf, &ctx->adj_ovf_cap, (size_t)chunk, sizeof(float),
              "adjoint contributions");
    if (rc != FLR_OK) return rc;
    rc = grow(ctx, (void **)&ctx->d_adj_tal, &ctx->adj_tal_cap, (size_t)tal_size(FLR_MAX_BINS),
              sizeof(unsigned long long), "adjoint tallies");
    if (rc != FLR_OK) return rc;
    R.tallies = ctx->d_adj_tal;
    A.ak = ctx->d_adj_ak;
    A.ovf = ctx->d_adj_ovf;
    A.K = ADJ_K;
    R.work_counter = ctx->d_work;
    R.regroup = p->regroup_interval;
    for (uint64_t off = 0; off < p->n_paths; off += chunk) {
        const uint64_t n = std::min<uint64_t>(chunk, p->n_paths - off);
        R.n_paths = n;
        R.path_offset = p->path_offset + off;
        e = cudaMemsetAsync(A.ak, 0, sizeof(float) * (size_t)n * ADJ_K, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(A.ovf, 0, sizeof(float) * (size_t)n, st);
        for (int pass = 1; pass <= 2 && e == cudaSuccess; ++pass) {
            e = cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), st);
            if (e == cudaSuccess) e = launch_adjoint_warp(S, R, A, pass, p->block_size, p->blocks_per_sm, st);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "launch adjoint kernels");
    }
    return FLR_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched persistent form.

static int grow(flr_ctx *ctx, void **ptr, size_t *cap, size_t need, size_t elem, const char *what)
{
    if (need <= *cap && *ptr) return FLR_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = dev_alloc(ptr, std::max<size_t>(need, 1) * elem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    *cap = std::max<size_t>(need, 1);
    return FLR_OK;
}

static int film_accumulator(flr_ctx *ctx, size_t n, cudaStream_t st)
{
    const int rc = grow(ctx, (void **)&ctx->d_film_fx, &ctx->film_fx_cap, n, sizeof(unsigned long long),
                        "film accumulator");
    if (rc != FLR_OK) return rc;
    const cudaError_t e = cudaMemsetAsync(ctx->d_film_fx, 0, sizeof(unsigned long long) * n, st);
    return e == cudaSuccess ? FLR_OK : cuda_fail(ctx, e, "clear film accumulator");
}

int flr_batch_prepare(flr_ctx *ctx, int n_media, const flr_medium *media, const uint64_t *n_paths,
                      const flr_params *p)
{
    const NvtxRange nvtx_range("flr_batch_prepare");
    if (!ctx) return FLR_ERR_ARG;
    if (n_media < 1 || n_media > 65536 || !media || !n_paths || !p)
        return fail(ctx, FLR_ERR_ARG, "batch: need 1..65536 media, path counts and params");
    if (ctx->sources.empty()) return fail(ctx, FLR_ERR_STATE, "batch: no sources");
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 256 || (p->block_size & 31)))
        return fail(ctx, FLR_ERR_ARG, "params: block_size must be 32..256, a multiple of 32");
    if (p->n_rr < 0 || p->max_events < 0 || p->max_steps < 1 || p->max_events > 2000000000LL)
        return fail(ctx, FLR_ERR_ARG, "params: n_rr, max_events >= 0, max_steps >= 1");
    if (p->hero != 0) return fail(ctx, FLR_ERR_ARG, "params: hero paths are for flr_render only");
    if (!(p->majorant_margin >= 0.0f && p->majorant_margin <= 100.0f))
        return fail(ctx, FLR_ERR_ARG, "params: majorant_margin in [0, 100]");
    const int B = ctx->B;
    std::vector<long long> off(n_media, -1), nv(n_media, 0), npk(n_media, 0);
    long long arena = 0;
    for (int m = 0; m < n_media; ++m) {
        const int rc = validate_medium(ctx, &media[m]);
        if (rc != FLR_OK) return rc;
        if (media[m].ior > 1.0f || media[m].wall_gloss > 0.0f)
            return fail(ctx, FLR_ERR_ARG, "batch: index-matched faces and Lambertian walls only");
        if (n_paths[m] > 0xFFFFFFFFull * 64ull) return fail(ctx, FLR_ERR_ARG, "batch: too many paths");
        const bool grids = medium_has_grid(media[m]) || media[m].solvent;
        nv[m] = grids ? nvox(media[m]) : 1;
        if (medium_has_grid(media[m])) {
            npk[m] = packed_voxels(media[m].dims);
            off[m] = arena;
            arena += npk[m];
        }
    }
    DeviceGuard g(ctx->device);
    auto &bt = ctx->batch;
    bt.ready = false;
    int rc = grow(ctx, (void **)&bt.d_arena, &bt.arena_cap, (size_t)arena, sizeof(float4), "batch arena");
    if (rc == FLR_OK) rc = grow(ctx, (void **)&bt.d_max, &bt.max_cap, (size_t)n_media * 8, sizeof(unsigned), "batch maxima");
    if (rc == FLR_OK) rc = grow(ctx, (void **)&bt.d_tables, &bt.tables_cap, (size_t)n_media * tab_size(B), sizeof(float), "batch tables");
    if (rc == FLR_OK) rc = grow(ctx, (void **)&bt.d_tallies, &bt.tallies_cap, (size_t)n_media * tal_size(B), sizeof(unsigned long long), "batch tallies");
    if (rc == FLR_OK) rc = grow(ctx, (void **)&bt.d_media, &bt.media_cap, (size_t)n_media, sizeof(MediumDev), "batch media");
    if (rc != FLR_OK) return rc;
    if (!bt.d_counters || !bt.d_head) {
        // allocated as a pair: after a failure part-way, the next prepare starts the pair again
        cudaFree(bt.d_counters);
        cudaFree(bt.d_head);
        bt.d_counters = nullptr;
        bt.d_head = nullptr;
        cudaError_t e = dev_alloc(&bt.d_counters, sizeof(unsigned long long) * FLR_NCOUNTERS);
        if (e == cudaSuccess) e = dev_alloc(&bt.d_head, sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch counters");
    }
    // pack grids, reduce maxima (slots [m][0..3] dyes, [m][4] bad-value flag, [m][5] solvent any)
    cudaError_t e = cudaMemset(bt.d_max, 0, sizeof(unsigned) * (size_t)n_media * 8);
    for (int m = 0; m < n_media && e == cudaSuccess; ++m) {
        const flr_medium &md = media[m];
        if (off[m] >= 0) e = launch_pack_grid(md.conc, md.conc_uniform, md.n_dyes, md.dims, bt.d_arena + off[m], 0);
        for (int d = 0; d < md.n_dyes && e == cudaSuccess; ++d)
            if (md.conc[d])
                e = launch_grid_max(md.conc[d], nv[m], bt.d_max + (size_t)m * 8 + d, (int *)(bt.d_max + (size_t)m * 8 + 4), 0);
        if (e == cudaSuccess && md.solvent) e = launch_solvent_any(md.solvent, nv[m], bt.d_max + (size_t)m * 8 + 5, 0);
    }
    std::vector<unsigned> hmax((size_t)n_media * 8);
    if (e == cudaSuccess) e = cudaMemcpy(hmax.data(), bt.d_max, sizeof(unsigned) * hmax.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch grid preparation");
    // tables, media descriptors, chunk queue
    std::vector<float> htab((size_t)n_media * tab_size(B));
    std::vector<MediumDev> hmed(n_media);
    struct Item { double cost; ChunkDev c; };
    std::vector<Item> items;
    // Small chunks keep the media in flight few: every resident warp holds one chunk, and the
    // queue runs medium by medium, so 256-path chunks put the whole GPU on a handful of media at a
    // time whose grids share the L2 (measured on the 256-medium workload: 51.0 ms with about 2,900
    // paths per chunk, 44.1 ms with 256; 64, 128 and 1,024 were slower).
    const uint64_t chunk = 256;
    uint64_t total = 0;
    for (int m = 0; m < n_media; ++m) total += n_paths[m];
    bt.n_paths.assign(n_paths, n_paths + n_media);
    bt.n_dyes.resize(n_media);
    for (int m = 0; m < n_media; ++m) {
        const flr_medium &md = media[m];
        if (hmax[(size_t)m * 8 + 4]) return fail(ctx, FLR_ERR_ARG, "batch: a grid has negative or non-finite values");
        float cmax[MAXD] = {0, 0, 0, 0};
        for (int d = 0; d < md.n_dyes; ++d) {
            if (md.conc[d]) std::memcpy(&cmax[d], &hmax[(size_t)m * 8 + d], sizeof(float));
            else cmax[d] = md.conc_uniform[d];
        }
        const float smax = md.solvent ? (hmax[(size_t)m * 8 + 5] ? 1.0f : 0.0f) : 1.0f;
        float *tab = htab.data() + (size_t)m * tab_size(B);
        build_medium_tables(ctx, md, cmax, smax, tab, p->majorant_margin);
        MediumDev &o = hmed[m];
        std::memset(&o, 0, sizeof(o));
        for (int k = 0; k < 3; ++k) {
            o.lo[k] = md.lo[k];
            o.hi[k] = md.hi[k];
            o.dims[k] = (medium_has_grid(md) || md.solvent) ? md.dims[k] : 1;
            o.bdims[k] = grid_bricks(o.dims[k]);
            o.vox_scale[k] = (float)((double)o.dims[k] / ((double)md.hi[k] - (double)md.lo[k]));
        }
        o.grid = off[m] >= 0 ? bt.d_arena + off[m] : nullptr;
        o.solvent = md.solvent;
        o.homogeneous = (o.grid == nullptr && o.solvent == nullptr) ? 1 : 0;
        o.D = md.n_dyes;
        for (int d = 0; d < MAXD; ++d) o.conc_uniform[d] = d < md.n_dyes ? md.conc_uniform[d] : 0.0f;
        o.sigma_s = md.sigma_s;
        o.sigma_a0 = md.sigma_a0;
        o.wall_mask = md.wall_mask;
        o.wall_albedo = md.wall_albedo;
        o.tables = bt.d_tables + (size_t)m * tab_size(B);
        o.tallies = bt.d_tallies + (size_t)m * tal_size(B);
        o.key1 = p->medium_id + (uint32_t)m;
        int ne = 0;
        rc = build_emitters(ctx, md, BATCH_MAX_LINES, o.em, o.em_cdf, &ne);
        if (rc != FLR_OK) return rc;
        o.n_emitters = ne;
        bt.n_dyes[m] = md.n_dyes;
        // expected real events per path at the first line: albedo-limited or diffusion-limited
        const int b0 = o.em[0].bin;
        const double maj = tab[tab_majorant(B) + b0];
        const double a = maj > 0.0 ? std::min(0.9999, (double)md.sigma_s / maj) : 0.0;
        double L = 1e30;
        for (int k = 0; k < 3; ++k) L = std::min(L, (double)md.hi[k] - md.lo[k]);
        const double cost = std::min(1.0 / (1.0 - a), 1.0 + maj * L * maj * L) * (1.0 + 0.02 * maj * L);
        for (uint64_t s0 = 0; s0 < n_paths[m]; s0 += chunk) {
            ChunkDev c;
            c.medium = m;
            c.start = p->path_offset + s0;
            c.count = (uint32_t)std::min<uint64_t>(chunk, n_paths[m] - s0);
            items.push_back({cost, c});
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
    std::vector<ChunkDev> hch(items.size());
    for (size_t i = 0; i < items.size(); ++i) hch[i] = items[i].c;
    rc = grow(ctx, (void **)&bt.d_chunks, &bt.chunks_cap, hch.size(), sizeof(ChunkDev), "batch queue");
    if (rc != FLR_OK) return rc;
    e = cudaMemcpy(bt.d_tables, htab.data(), sizeof(float) * htab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt.d_media, hmed.data(), sizeof(MediumDev) * hmed.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hch.empty()) e = cudaMemcpy(bt.d_chunks, hch.data(), sizeof(ChunkDev) * hch.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
    // capture tally reset + persistent kernel in a CUDA graph (replayed by flr_batch_launch)
    if (!ctx->cap_stream) {
        e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
    }
    if (bt.exec) { cudaGraphExecDestroy(bt.exec); bt.exec = nullptr; }
    if (bt.graph) { cudaGraphDestroy(bt.graph); bt.graph = nullptr; }
    BatchDev Bt;
    Bt.B = B;
    Bt.n_chunks = (int)hch.size();
    Bt.media = bt.d_media;
    Bt.chunks = bt.d_chunks;
    Bt.head = bt.d_head;
    RunDev R;
    std::memset(&R, 0, sizeof(R));
    R.n_paths = total;
    R.path_offset = p->path_offset;
    R.seed = p->seed;
    R.medium_id = p->medium_id;
    set_round_keys(R);
    R.n_rr = p->n_rr;
    R.max_inelastic = p->max_inelastic;
    R.analog = p->analog;
    R.max_events = p->max_events;
    R.max_steps = p->max_steps;
    R.paper_mode = p->paper_mode ? 1 : 0;
    R.counters = bt.d_counters;
    R.error_word = ctx->d_error;
    cudaStream_t cs = ctx->cap_stream;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(bt.d_tallies, 0, sizeof(unsigned long long) * (size_t)n_media * tal_size(B), cs);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(bt.d_counters, 0, sizeof(unsigned long long) * FLR_NCOUNTERS, cs);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(bt.d_head, 0, sizeof(unsigned long long), cs);
        if (e1 == cudaSuccess && !hch.empty()) e1 = launch_batch(Bt, R, p->block_size, p->blocks_per_sm, cs);
        e = cudaStreamEndCapture(cs, &bt.graph);
        if (e1 != cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bt.exec, bt.graph, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "capture the batched launch");
    bt.n_media = n_media;
    bt.ready = true;
    return FLR_OK;
}

int flr_batch_launch(flr_ctx *ctx, void *stream)
{
    const NvtxRange nvtx_range("flr_batch_launch");
    if (!ctx) return FLR_ERR_ARG;
    if (!ctx->batch.ready) return fail(ctx, FLR_ERR_STATE, "batch: prepare it first");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaGraphLaunch(ctx->batch.exec, (cudaStream_t)stream);
    return e == cudaSuccess ? FLR_OK : cuda_fail(ctx, e, "launch the batch graph");
}

int flr_batch_read(flr_ctx *ctx, double *face, double *absorbed, double *emitted, uint64_t *counters,
                   void *stream)
{
    if (!ctx) return FLR_ERR_ARG;
    auto &bt = ctx->batch;
    if (!bt.ready) return fail(ctx, FLR_ERR_STATE, "batch: prepare it first");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before reading batch tallies");
    const int B = ctx->B, M = bt.n_media;
    std::vector<unsigned long long> t((size_t)M * tal_size(B));
    unsigned long long c[FLR_NCOUNTERS];
    e = cudaMemcpy(t.data(), bt.d_tallies, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(c, bt.d_counters, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "read batch tallies");
    for (int m = 0; m < M; ++m) {
        const unsigned long long *tm = t.data() + (size_t)m * tal_size(B);
        const double inv = bt.n_paths[m] ? 1.0 / ((double)bt.n_paths[m] * TALLY_ONE) : 0.0;
        if (face)
            for (int i = 0; i < 12 * B; ++i) face[(size_t)m * 12 * B + i] = (double)tm[tal_face(B) + i] * inv;
        if (absorbed)
            for (int i = 0; i < (MAXD + 1) * B; ++i)
                absorbed[(size_t)m * (MAXD + 1) * B + i] = (double)tm[tal_absorbed(B) + i] * inv;
        if (emitted)
            for (int i = 0; i < MAXD * B; ++i) emitted[(size_t)m * MAXD * B + i] = (double)tm[tal_emitted(B) + i] * inv;
    }
    if (counters)
        for (int k = 0; k < FLR_NCOUNTERS; ++k) counters[k] = c[k];
    return FLR_OK;
}

int flr_render_batch(flr_ctx *ctx, int n_media, const flr_medium *media, const uint64_t *n_paths,
                     const flr_params *p, void *stream)
{
    const NvtxRange nvtx_range("flr_render_batch");
    int rc = flr_batch_prepare(ctx, n_media, media, n_paths, p);
    if (rc != FLR_OK) return rc;
    return flr_batch_launch(ctx, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Render without device allocation. Everything the render needs beyond the caller's inputs and
// outputs sits in one file-scope device array: the small scratch (spectral tables, fixed-point
// tallies, counters, work counter, grid maxima) in its first 64 KiB, then room for the
// interleaved copy of up to FLR_NOALLOC_MAX_VOXELS voxels.
namespace {
constexpr size_t NA_SMALL = 64 * 1024;
constexpr size_t NA_TABLES = 0;
constexpr size_t NA_TALLIES = 8192;
constexpr size_t NA_COUNTERS = 32768;
constexpr size_t NA_WORK = 33024;
constexpr size_t NA_ERROR = 33088;
constexpr size_t NA_MAXIMA = 33280;
constexpr size_t NA_BYTES = NA_SMALL + (size_t)FLR_NOALLOC_MAX_VOXELS * sizeof(float4);
static_assert(NA_TABLES + sizeof(float) * tab_size(FLR_MAX_BINS) <= NA_TALLIES, "tables fit");
static_assert(NA_TALLIES + sizeof(unsigned long long) * tal_size(FLR_MAX_BINS) <= NA_COUNTERS, "tallies fit");
static_assert(NA_COUNTERS + sizeof(unsigned long long) * FLR_NCOUNTERS <= NA_WORK, "counters fit");
static_assert(NA_MAXIMA + 8 * sizeof(unsigned) <= NA_SMALL, "maxima fit");

std::mutex g_na_mutex;
void *g_na_address[256] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t noalloc_address(int dev, unsigned char **out);
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {
cudaError_t noalloc_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_address[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_address[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_na_address[dev]);
    return cudaSuccess;
}
}  // namespace

extern "C" int flr_render_noalloc(float lambda0_nm, float dlambda_nm, int n_bins, int n_dyes,
                                  const float *abs_shape, const float *emit_spec, const float *eps,
                                  const float *qy, const flr_medium *medium, int n_sources,
                                  const flr_source *sources, const flr_sensor *sensor,
                                  const flr_params *p, double *face, double *absorbed,
                                  double *emitted, uint64_t *counters, void *stream)
{
    flr_ctx c;  // host-side bookkeeping only: no device buffer of its own
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return FLR_ERR_CUDA;
    }
    c.device = dev;
    int rc = flr_set_spectrum(&c, lambda0_nm, dlambda_nm, n_bins);
    if (rc == FLR_OK) rc = flr_set_dyes(&c, n_dyes, abs_shape, emit_spec, eps, qy);
    if (rc == FLR_OK) rc = flr_set_sources(&c, n_sources, sources);
    if (rc == FLR_OK && sensor && sensor->kind != FLR_SENSOR_NONE) rc = flr_set_sensor(&c, sensor);
    if (rc == FLR_OK) rc = validate_medium(&c, medium);
    if (rc != FLR_OK) return rc;
    if (!p || (p->form != FLR_FORM_PLAIN && p->form != FLR_FORM_WAVEFRONT &&
               p->form != FLR_FORM_WAVEFRONT_WARP))
        return FLR_ERR_ARG;
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 256 || (p->block_size & 31)))
        return FLR_ERR_ARG;
    if (p->n_rr < 0 || p->max_events < 0 || p->max_steps < 1 || p->max_events > 2000000000LL)
        return FLR_ERR_ARG;
    if (p->hero != 0) return FLR_ERR_ARG;   /* hero paths: flr_render only */
    // one majorant per bin and the full RTE only: the static scratch holds no local-majorant or
    // empty-space cell grid, and the other settings would change the tallies flr_render gives
    if (p->paper_mode != 0 || p->skip_cell != 0 || p->macro_cell != 0 || p->majorant_margin != 0.0f)
        return FLR_ERR_ARG;
    if (p->film && !is_device_pointer(p->film)) return FLR_ERR_ARG;
    if (p->path_events && !is_device_pointer(p->path_events)) return FLR_ERR_ARG;
    if (c.sensor_set && c.sensor.kind == FLR_SENSOR_PINHOLE) {
        bool inside = true;
        for (int k = 0; k < 3; ++k)
            inside = inside && c.sensor.origin[k] >= medium->lo[k] && c.sensor.origin[k] <= medium->hi[k];
        if (inside) return FLR_ERR_ARG;
    }
    if (check_interfaces(&c, *medium, c.sensor_set && p->film, c.sensor, p->hero, p->paper_mode) != FLR_OK)
        return FLR_ERR_ARG;
    flr_medium mm = *medium;
    const bool grids = medium_has_grid(mm) || mm.solvent;
    if (!grids) mm.dims[0] = mm.dims[1] = mm.dims[2] = 1;
    const long long n = nvox(mm);
    // beyond the static scratch (which holds the grid padded to whole 4^3-voxel bricks)
    if (n > FLR_NOALLOC_MAX_VOXELS || (medium_has_grid(mm) && packed_voxels(mm.dims) > FLR_NOALLOC_MAX_VOXELS))
        return FLR_ERR_ARG;
    unsigned char *base = nullptr;
    cudaError_t e = noalloc_address(dev, &base);
    if (e != cudaSuccess) return FLR_ERR_CUDA;
    float *tables = reinterpret_cast<float *>(base + NA_TABLES);
    unsigned long long *tallies = reinterpret_cast<unsigned long long *>(base + NA_TALLIES);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(base + NA_COUNTERS);
    unsigned long long *work = reinterpret_cast<unsigned long long *>(base + NA_WORK);
    int *err_word = reinterpret_cast<int *>(base + NA_ERROR);
    unsigned *maxima = reinterpret_cast<unsigned *>(base + NA_MAXIMA);
    float4 *grid = reinterpret_cast<float4 *>(base + NA_SMALL);
    cudaStream_t st = (cudaStream_t)stream;
    // grid maxima for the majorant ([0..3] dyes, [4] bad-value flag, [5] solvent present)
    e = cudaMemsetAsync(maxima, 0, 8 * sizeof(unsigned), st);
    if (e == cudaSuccess && medium_has_grid(mm)) e = launch_pack_grid(mm.conc, mm.conc_uniform, mm.n_dyes, mm.dims, grid, st);
    for (int d = 0; d < mm.n_dyes && e == cudaSuccess; ++d)
        if (mm.conc[d]) e = launch_grid_max(mm.conc[d], n, maxima + d, reinterpret_cast<int *>(maxima + 4), st);
    if (e == cudaSuccess && mm.solvent) e = launch_solvent_any(mm.solvent, n, maxima + 5, st);
    unsigned hmax[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmax, maxima, sizeof(hmax), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return FLR_ERR_CUDA;
    if (hmax[4]) return FLR_ERR_ARG;
    for (int d = 0; d < mm.n_dyes; ++d) {
        if (mm.conc[d]) std::memcpy(&c.cmax[d], &hmax[d], sizeof(float));
        else c.cmax[d] = mm.conc_uniform[d];
    }
    c.smax = mm.solvent ? (hmax[5] ? 1.0f : 0.0f) : 1.0f;
    c.medium = mm;
    c.medium_set = true;
    c.d_grid = medium_has_grid(mm) ? grid : nullptr;
    c.d_tables = tables;
    build_tables(&c);
    SceneDev S;
    rc = fill_scene(&c, S, p->film != nullptr);
    if (rc != FLR_OK) return rc;
    e = cudaMemcpyAsync(tables, c.h_tables.data(), sizeof(float) * c.h_tables.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tallies, 0, sizeof(unsigned long long) * tal_size(FLR_MAX_BINS), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * FLR_NCOUNTERS, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err_word, 0, sizeof(int), st);
    if (e == cudaSuccess && p->film && S.sensor_kind != FLR_SENSOR_NONE && !p->accumulate)
        e = cudaMemsetAsync(p->film, 0, sizeof(float) * (size_t)S.W * S.H * S.B, st);
    if (e != cudaSuccess) return FLR_ERR_CUDA;
    if (p->n_paths > 0) {
        RunDev R;
        std::memset(&R, 0, sizeof(R));
        R.n_paths = p->n_paths;
        R.path_offset = p->path_offset;
        R.seed = p->seed;
        R.medium_id = p->medium_id;
        set_round_keys(R);
        R.n_rr = p->n_rr;
        R.max_inelastic = p->max_inelastic;
        R.analog = p->analog;
        R.max_events = p->max_events;
        R.max_steps = p->max_steps;
        R.film_scale = (float)(1.0 / (double)p->n_paths);
        R.film = S.sensor_kind != FLR_SENSOR_NONE ? p->film : nullptr;
        R.path_events = p->path_events;
        R.tallies = tallies;
        R.counters = cnt;
        R.error_word = err_word;
        R.work_counter = work;
        R.regroup = p->regroup_interval;
        e = launch_trace(S, R, p->form, p->block_size, p->blocks_per_sm, st);
        if (e != cudaSuccess) return FLR_ERR_CUDA;
    }
    std::vector<unsigned long long> t(tal_size(FLR_MAX_BINS));
    unsigned long long hc[FLR_NCOUNTERS];
    int herr = 0;
    e = cudaMemcpyAsync(t.data(), tallies, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err_word, sizeof(herr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return FLR_ERR_CUDA;
    // checked build: an index found out of range during this call (the access was skipped)
    unsigned long long cw = 0ull;
    if (check_word_take(&cw) != cudaSuccess) return FLR_ERR_CUDA;
    const int B = c.B, D = mm.n_dyes;
    const double inv = p->n_paths ? 1.0 / ((double)p->n_paths * TALLY_ONE) : 0.0;
    if (face)
        for (int i = 0; i < 12 * B; ++i) face[i] = (double)t[tal_face(B) + i] * inv;
    if (absorbed)
        for (int i = 0; i < (D + 1) * B; ++i) absorbed[i] = (double)t[tal_absorbed(B) + i] * inv;
    if (emitted)
        for (int i = 0; i < D * B; ++i) emitted[i] = (double)t[tal_emitted(B) + i] * inv;
    if (counters)
        for (int k = 0; k < FLR_NCOUNTERS; ++k) counters[k] = hc[k];
    if (cw) return FLR_ERR_CHECK;
    return herr ? FLR_ERR_BUDGET : FLR_OK;
}
