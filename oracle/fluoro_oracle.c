/*
 * fluoro_oracle.c -- CPU oracle for the fluorescent participating-media light tracer.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
 * reference leg may load this library. It shares no code, header, table or constant generator
 * with the CUDA path; both sides implement the same published definitions independently.
 *
 * Plain, scalar, fp64, one path at a time (OpenMP only splits the path-id range).
 * Paper: Abdellah et al., "A Physically Plausible Model for Rendering Highly Scattering
 * Fluorescent Participating Media" (arXiv 1706.03024).
 *
 * What it computes (an unbiased Monte Carlo estimate of the steady, per-wavelength fluorescent
 * RTE of Sec. 4.2, Eq. 9 and Eq. 11, by light (photon) tracing, Sec. 3):
 *   - a photon of unit power leaves a source at one spectral line (p(x_n), p(lambda_x) of Eq. 12);
 *   - free flight by delta tracking against a per-wavelength majorant (transmittance, Eq. 6);
 *   - at a real collision the particle type is chosen in proportion to its coefficient
 *     (Sec. 4.1: scatterer, or dye d with share eps_d * a_d(lambda) * c_d);
 *   - scattering and fluorescent re-emission are isotropic (Sec. 2.1);
 *   - a dye absorption re-emits with probability QY (Sec. 4.1) at a wavelength drawn from the
 *     normalised emission spectrum, independent of the exciting wavelength (Eq. 10, Sec. 2.1);
 *   - photons escaping the medium are tallied per face; every scattering, emission, wall and
 *     Lambertian-light vertex is connected to the sensor with the three-point form (Eq. 3-6):
 *     vertex intensity x transmittance x sensor importance.
 * The transmittance of a connection is the exact line integral of the piecewise-constant
 * extinction (Eq. 6), not an estimate.
 * paper_mode restricts the light tracer to the paper's single-inelastic model (Sec. 4.1), and
 * or_render_camera evaluates that model with the paper's camera-side estimator (Eq. 12), so the
 * two can be checked against each other.
 *
 * Pinned by tests/test_oracle_pins.py against closed forms (Beer-Lambert, uncollided
 * transmission, Chandrasekhar H-function reflectance, thin-dye emission spectrum, slab
 * fluorescence yield with analytic solid angles, single-scattering film), conservation identities
 * and brute-force statistics. Adjoint reference: see or_adjoint below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_DYES 4
#define OR_MAX_EMITTERS 32
#define OR_MAX_BINS 128
#define OR_NCOUNTERS 17
#define OR_PI 3.14159265358979323846

/* counters (same meaning as the GPU library's, defined independently) */
enum {
    OC_PATHS = 0, OC_EVENTS, OC_NULLS, OC_ESCAPES, OC_ABSORBED_DEAD, OC_RR_KILLS, OC_CAP_HITS,
    OC_STEP_BUDGET, OC_CONNECTIONS, OC_VF_REJECTED, OC_WALL_BOUNCES, OC_EMISSIONS, OC_SCATTERS,
    OC_DYE_ABSORPTIONS, OC_STEPS, OC_MAJORANT_VIOLATIONS, OC_IFACE_REFLECTIONS
};

typedef struct {
    int kind;           /* 0 collimated, 1 Lambertian (cosine-weighted about dir, axis-aligned) */
    double origin[3];   /* emitting parallelogram origin + a*eu + b*ev, a, b uniform in [0,1) */
    double eu[3], ev[3];
    double dir[3];      /* propagation direction (collimated) or surface normal (Lambertian) */
    double lambda_nm;   /* spectral line */
    double power;       /* relative power; lines are chosen in proportion (p(lambda_x), Eq. 12) */
    int group;          /* lines of one source (the same geometry) share a group id             */
} or_emitter;

typedef struct {
    int kind;           /* 0 none, 1 orthographic, 2 pinhole */
    int width, height;
    double origin[3];   /* ortho: film corner; pinhole: eye */
    double U[3], V[3];  /* ortho: full film edges; pinhole: right / up unit vectors */
    double view[3];     /* ortho: direction from the scene to the camera; pinhole: forward axis */
    double fov_y_deg;   /* pinhole vertical field of view */
} or_sensor;

typedef struct {
    /* spectrum */
    int n_bins;
    double lambda0, dlambda;
    /* dyes */
    int n_dyes;
    const float *abs_shape;   /* [n_dyes][n_bins] peak-normalised absorption spectrum a_d */
    const float *emit_spec;   /* [n_dyes][n_bins] emission spectrum f_m (any scale)        */
    const float *eps;         /* [n_dyes] napierian cm^-1 per unit concentration at peak    */
    const float *qy;          /* [n_dyes] quantum yield                                      */
    /* medium */
    double lo[3], hi[3];
    int dims[3];              /* grid resolution; all zero => homogeneous                    */
    const float *conc;        /* [n_dyes][nz][ny][nx] or NULL                                */
    const float *conc_uniform;/* [n_dyes] used when conc == NULL                             */
    const uint8_t *solvent;   /* [nz][ny][nx] 0/1 or NULL (solvent everywhere)               */
    double sigma_s, sigma_a0; /* solvent scattering and flat background absorption, cm^-1   */
    int wall_mask;            /* bit f: face f is a Lambertian wall                          */
    double wall_albedo;
    /* sources */
    int n_emitters;
    const or_emitter *emitters;
    /* sensor */
    or_sensor sensor;
    /* Interfaces and glossy walls (the glass vials and the glossy Cornell box of Sec. 5; the
     * paper specifies neither, these are the physically standard choices):
     *   ior > 1: every open face is a smooth dielectric interface between the solution (index
     *   ior) and the outside (index 1): Fresnel reflection for unpolarised light, Snell
     *   refraction, total internal reflection beyond the critical angle. 0 or 1: index-matched.
     *   wall BRDF: wall_albedo [(1 - g)/pi + g (e + 2)/(2 pi) cos^e alpha], g = wall_gloss,
     *   e = wall_exponent, alpha the angle between the outgoing direction and the mirror
     *   direction of the incoming one (a diffuse lobe plus a normalised Phong lobe). */
    double ior;
    double wall_gloss, wall_exponent;
} or_scene;

typedef struct {
    uint64_t n_paths;
    uint64_t path_offset;
    uint32_t seed;
    uint32_t medium_id;
    int n_rr;                 /* Russian roulette once n_events >= n_rr                      */
    int max_inelastic;        /* <0 unlimited; k >= 0: the (k+1)-th dye absorption kills     */
    int analog;               /* 0 weighted QY / albedo, 1 analog coins                      */
    int n_threads;
    int64_t max_events;       /* a real collision with n_events == max_events ends the path */
    int64_t max_steps;        /* tracking-step budget per path                               */
    /* frozen-sampling evaluation (for finite differences with common random numbers): the
     * evaluation medium is the scene plus one perturbation (pert_delta added to dye pert_dye's
     * concentration in voxel pert_voxel, pert_sigma_s added to sigma_s). With frozen = 1 every
     * decision is still sampled in the unperturbed medium and each tally is weighted by the
     * likelihood ratio p_eval / p_sample of the decisions before it; with frozen = 0 the perturbed
     * medium is simply rendered. */
    double majorant_scale;    /* sigma_bar multiplier (>= 1; 0 means 1)                       */
    int frozen;
    int pert_dye;             /* < 0: no concentration perturbation                         */
    int64_t pert_voxel;
    double pert_delta;
    double pert_sigma_s;
    /* free flights against a grid of local majorants: cells of macro_cell^3 voxels, each the
     * maximum of sigma_t over its voxels and a one-voxel halo; 0 = one majorant per bin */
    int macro_cell;
    /* > 0 (with macro_cell = 0): after a null collision where sigma_t = 0, leave the largest cube
     * of skip_cell^3-voxel cells around it that holds no matter and restart the free flight at its
     * boundary (memoryless: every tentative collision inside would be a null) */
    int skip_cell;
    /* 1: the paper's single-inelastic model (Sec. 4.1): excitation light reaches a dye only
     * uncollided (a scattering or wall bounce before the first emission ends the path), a second
     * dye absorption ends the path (V_f of Eq. 9), and only vertices after the emission connect
     * to the sensor (the film holds fluorescence only). */
    int paper_mode;
    /* > 0: hero-wavelength paths carrying up to `hero` wavelengths (1..4), combined by spectral
     * multiple importance sampling; see trace_path_hero. 0: one wavelength per path. */
    int hero;
} or_params;

typedef struct {
    double *face;             /* [2][6][n_bins]   escaped weight: [fluoresced][face][bin]    */
    double *absorbed;         /* [n_dyes+1][n_bins] weight absorbed (last row: background)   */
    double *emitted;          /* [n_dyes][n_bins] weight re-emitted                          */
    double *film;             /* [H][W][n_bins] or NULL                                      */
    uint64_t *counters;       /* [OR_NCOUNTERS]                                              */
    uint32_t *path_events;    /* [n_paths] real events per path, or NULL                     */
} or_result;

/* ---------------------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11): ten rounds of two 32x32->64 multiplies on a 4-word counter, the key bumped by the
 * Weyl constants between rounds. */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24-bit uniform in [0,1): exact in fp32 and fp64 */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

#define STEP_SPAWN 0xFFFFFFFFu

typedef struct { double u[4]; } block4;

static block4 rng_block(uint32_t seed, uint32_t medium, uint64_t path, uint32_t step, uint32_t slot)
{
    uint32_t ctr[4] = { (uint32_t)path, step, slot, (uint32_t)(path >> 32) };
    uint32_t key[2] = { seed, medium };
    uint32_t o[4];
    philox4x32_10(ctr, key, o);
    block4 b;
    for (int i = 0; i < 4; ++i) b.u[i] = u24(o[i]);
    return b;
}

/* ---------------------------------------------------------------------------------------- */
/* Spectral tables built from the scene (Eq. 10 and Sec. 4.1). */
typedef struct {
    int B, D;
    double sig_a[OR_MAX_DYES][OR_MAX_BINS];  /* eps_d * a_d(lambda_i), per unit concentration */
    double cdf[OR_MAX_DYES][OR_MAX_BINS];    /* emission CDF, fp64                           */
    float cdf32[OR_MAX_DYES][OR_MAX_BINS];   /* the same CDF rounded to fp32 (decision)      */
    double qy[OR_MAX_DYES];
    double cmax[OR_MAX_DYES];                /* max concentration over the grid              */
    double smax;                             /* max solvent indicator                        */
    double majorant[OR_MAX_BINS];            /* sigma_bar(lambda)                            */
    int homogeneous;
    int em_bin[OR_MAX_EMITTERS];
    float em_cdf32[OR_MAX_EMITTERS];
    double A_pix, tan_half, aspect;
    int frozen, pert_dye;
    int64_t pert_voxel;
    double pert_delta, pert_sigma_s;
    double maj_scale;
    /* local majorants (macro cells) */
    int mc, mdims[3];
    double *mc_cmax;                         /* [cells][n_dyes] */
    double *mc_smax;                         /* [cells]         */
    int sk, sdims[3];
    /* interfaces: dielectric open faces, the entry face of each emitter (-1: none) */
    int dielectric;
    double ior;
    int entry_face[OR_MAX_EMITTERS];
    unsigned char *sk_dist;                  /* Chebyshev distance to a cell with matter */
} tables;

static int nvox(const or_scene *s);

/* Maxima of each dye's concentration and of the solvent mask over every macro cell (its
 * macro_cell^3 voxels plus a one-voxel halo). */
static void build_macro(const or_scene *s, tables *t, int cell)
{
    t->mc = 0;
    if (cell <= 0 || t->homogeneous) return;
    int64_t nc = 1;
    for (int k = 0; k < 3; ++k) {
        t->mdims[k] = (s->dims[k] + cell - 1) / cell;
        nc *= t->mdims[k];
    }
    t->mc = cell;
    t->mc_cmax = (double *)calloc((size_t)nc * (s->n_dyes > 0 ? s->n_dyes : 1), sizeof(double));
    t->mc_smax = (double *)calloc((size_t)nc, sizeof(double));
    for (int cz = 0; cz < t->mdims[2]; ++cz)
        for (int cy = 0; cy < t->mdims[1]; ++cy)
            for (int cx = 0; cx < t->mdims[0]; ++cx) {
                int64_t c = ((int64_t)cz * t->mdims[1] + cy) * t->mdims[0] + cx;
                int lo[3] = { cx * cell - 1, cy * cell - 1, cz * cell - 1 };
                int hi[3] = { (cx + 1) * cell, (cy + 1) * cell, (cz + 1) * cell };
                for (int k = 0; k < 3; ++k) {
                    if (lo[k] < 0) lo[k] = 0;
                    if (hi[k] > s->dims[k] - 1) hi[k] = s->dims[k] - 1;
                }
                double sm = s->solvent ? 0.0 : 1.0;
                for (int z = lo[2]; z <= hi[2]; ++z)
                    for (int y = lo[1]; y <= hi[1]; ++y)
                        for (int x = lo[0]; x <= hi[0]; ++x) {
                            int v = (z * s->dims[1] + y) * s->dims[0] + x;
                            if (s->solvent && s->solvent[v]) sm = 1.0;
                            for (int d = 0; d < s->n_dyes; ++d) {
                                double cv = s->conc ? (double)s->conc[(size_t)d * nvox(s) + v]
                                                    : (double)s->conc_uniform[d];
                                if (cv > t->mc_cmax[c * s->n_dyes + d]) t->mc_cmax[c * s->n_dyes + d] = cv;
                            }
                        }
                t->mc_smax[c] = sm;
            }
}

static void free_macro(tables *t)
{
    free(t->mc_cmax);
    free(t->mc_smax);
    free(t->sk_dist);
    t->mc_cmax = t->mc_smax = NULL;
    t->sk_dist = NULL;
}

/* Empty-space distances over cells of `cell`^3 voxels: a cell holds matter if any voxel of it or
 * of its one-voxel halo has solvent (with sigma_s + sigma_a0 > 0) or a positive concentration;
 * every other cell stores its Chebyshev distance (in cells) to the nearest such cell, found by
 * breadth-first search over the 26 neighbours and capped at 31. */
static void build_skip(const or_scene *s, tables *t, int cell)
{
    t->sk = 0;
    if (cell <= 0 || t->homogeneous) return;
    int64_t nc = 1;
    for (int k = 0; k < 3; ++k) {
        t->sdims[k] = (s->dims[k] + cell - 1) / cell;
        nc *= t->sdims[k];
    }
    t->sk = cell;
    t->sk_dist = (unsigned char *)malloc((size_t)nc);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
    int64_t head = 0, tail = 0;
    const int solvent_matter = (s->sigma_s + s->sigma_a0) > 0.0;
    for (int cz = 0; cz < t->sdims[2]; ++cz)
        for (int cy = 0; cy < t->sdims[1]; ++cy)
            for (int cx = 0; cx < t->sdims[0]; ++cx) {
                int64_t c = ((int64_t)cz * t->sdims[1] + cy) * t->sdims[0] + cx;
                int lo[3] = { cx * cell - 1, cy * cell - 1, cz * cell - 1 };
                int hi[3] = { (cx + 1) * cell, (cy + 1) * cell, (cz + 1) * cell };
                for (int k = 0; k < 3; ++k) {
                    if (lo[k] < 0) lo[k] = 0;
                    if (hi[k] > s->dims[k] - 1) hi[k] = s->dims[k] - 1;
                }
                int matter = 0;
                for (int z = lo[2]; z <= hi[2] && !matter; ++z)
                    for (int y = lo[1]; y <= hi[1] && !matter; ++y)
                        for (int x = lo[0]; x <= hi[0] && !matter; ++x) {
                            int v = (z * s->dims[1] + y) * s->dims[0] + x;
                            if ((s->solvent ? s->solvent[v] != 0 : 1) && solvent_matter) matter = 1;
                            for (int d = 0; d < s->n_dyes && !matter; ++d) {
                                double cv = s->conc ? (double)s->conc[(size_t)d * nvox(s) + v]
                                                    : (double)s->conc_uniform[d];
                                if (cv > 0.0) matter = 1;
                            }
                        }
                t->sk_dist[c] = matter ? 0 : 255;
                if (matter) queue[tail++] = c;
            }
    while (head < tail) {
        int64_t c = queue[head++];
        int cx = (int)(c % t->sdims[0]), cy = (int)((c / t->sdims[0]) % t->sdims[1]);
        int cz = (int)(c / ((int64_t)t->sdims[0] * t->sdims[1]));
        int next = t->sk_dist[c] + 1;
        if (next >= 255) continue;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int x = cx + dx, y = cy + dy, z = cz + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= t->sdims[0] || y >= t->sdims[1] || z >= t->sdims[2])
                        continue;
                    int64_t j = ((int64_t)z * t->sdims[1] + y) * t->sdims[0] + x;
                    if (t->sk_dist[j] == 255) {
                        t->sk_dist[j] = (unsigned char)next;
                        queue[tail++] = j;
                    }
                }
    }
    free(queue);
    for (int64_t c = 0; c < nc; ++c)
        if (t->sk_dist[c] > 31) t->sk_dist[c] = 31;
}

/* Distance along (x, w) to leave the empty cube around x (0 if x's cell may hold matter). */
static double empty_cube_exit(const or_scene *s, const tables *t, const double x[3], const double w[3])
{
    int c[3];
    for (int k = 0; k < 3; ++k) {
        double cs = t->sk * (s->hi[k] - s->lo[k]) / (double)s->dims[k];
        int ck = (int)floor((x[k] - s->lo[k]) / cs);
        if (ck < 0) ck = 0;
        if (ck > t->sdims[k] - 1) ck = t->sdims[k] - 1;
        c[k] = ck;
    }
    int kd = t->sk_dist[((int64_t)c[2] * t->sdims[1] + c[1]) * t->sdims[0] + c[0]];
    if (kd == 0) return 0.0;
    double best = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double cs = t->sk * (s->hi[k] - s->lo[k]) / (double)s->dims[k];
        double tk;
        if (w[k] > 0.0) tk = (s->lo[k] + (c[k] + kd) * cs - x[k]) / w[k];
        else if (w[k] < 0.0) tk = (s->lo[k] + (c[k] - kd + 1) * cs - x[k]) / w[k];
        else continue;
        if (tk < best) best = tk;
    }
    return best > 0.0 ? best : 0.0;
}

/* Copy the per-render evaluation settings into the tables (majorant scale and perturbation). */
static void apply_params_macro(const or_scene *s, tables *t, const or_params *p);

static void apply_params(tables *t, const or_params *p)
{
    double ms = p->majorant_scale > 0.0 ? p->majorant_scale : 1.0;
    t->maj_scale = ms;
    for (int i = 0; i < t->B; ++i) t->majorant[i] *= ms;
    t->frozen = p->frozen;
    t->pert_dye = p->pert_dye;
    t->pert_voxel = p->pert_voxel;
    t->pert_delta = p->pert_delta;
    t->pert_sigma_s = p->pert_sigma_s;
}

/* Emission pmf p_i = f_m(lambda_i) / sum_j f_m(lambda_j) (Eq. 10 with the bin as delta-lambda);
 * CDF_i = (sum_{j<=i} f_j) / (sum_j f_j), summed left to right in fp64, last entry forced to 1. */
static void build_cdf(const float *f, int B, double *cdf, float *cdf32)
{
    double tot = 0.0;
    for (int i = 0; i < B; ++i) tot += (double)f[i];
    double run = 0.0;
    for (int i = 0; i < B; ++i) {
        run += (double)f[i];
        cdf[i] = run / tot;
        cdf32[i] = (float)cdf[i];
    }
    cdf[B - 1] = 1.0;
    cdf32[B - 1] = 1.0f;
}

/* Nearest bin centre, ties to the lower bin. */
static int snap_bin(double lambda_nm, double l0, double dl, int B)
{
    double b = (lambda_nm - l0) / dl;
    int k = (int)ceil(b - 0.5);
    if (k < 0) k = 0;
    if (k > B - 1) k = B - 1;
    return k;
}

static int nvox(const or_scene *s) { return s->dims[0] * s->dims[1] * s->dims[2]; }

static void build_tables(const or_scene *s, tables *t)
{
    memset(t, 0, sizeof(*t));
    t->pert_dye = -1;
    t->B = s->n_bins;
    t->D = s->n_dyes;
    t->homogeneous = (s->conc == NULL && s->solvent == NULL);
    for (int d = 0; d < s->n_dyes; ++d) {
        for (int i = 0; i < s->n_bins; ++i)
            t->sig_a[d][i] = (double)s->eps[d] * (double)s->abs_shape[d * s->n_bins + i];
        build_cdf(s->emit_spec + (size_t)d * s->n_bins, s->n_bins, t->cdf[d], t->cdf32[d]);
        t->qy[d] = (double)s->qy[d];
        if (s->conc) {
            double m = 0.0;
            const float *g = s->conc + (size_t)d * nvox(s);
            for (int v = 0; v < nvox(s); ++v) if ((double)g[v] > m) m = (double)g[v];
            t->cmax[d] = m;
        } else {
            t->cmax[d] = (double)s->conc_uniform[d];
        }
    }
    t->smax = 1.0;
    if (s->solvent) {
        t->smax = 0.0;
        for (int v = 0; v < nvox(s); ++v) if (s->solvent[v]) { t->smax = 1.0; break; }
    }
    for (int i = 0; i < s->n_bins; ++i) {
        double m = t->smax * (s->sigma_s + s->sigma_a0);
        for (int d = 0; d < s->n_dyes; ++d) m += t->sig_a[d][i] * t->cmax[d];
        t->majorant[i] = m;
    }
    double ptot = 0.0;
    for (int k = 0; k < s->n_emitters; ++k) ptot += s->emitters[k].power;
    double run = 0.0;
    for (int k = 0; k < s->n_emitters; ++k) {
        run += s->emitters[k].power;
        t->em_cdf32[k] = (float)(run / ptot);
        t->em_bin[k] = snap_bin(s->emitters[k].lambda_nm, s->lambda0, s->dlambda, s->n_bins);
    }
    if (s->n_emitters > 0) t->em_cdf32[s->n_emitters - 1] = 1.0f;
    /* dielectric open faces; an emitter enters through face f when its parallelogram lies in
     * that face's plane and its direction (or normal) points into the box */
    t->dielectric = s->ior > 1.0;
    t->ior = t->dielectric ? s->ior : 1.0;
    for (int k = 0; k < s->n_emitters; ++k) {
        const or_emitter *e = &s->emitters[k];
        t->entry_face[k] = -1;
        if (!t->dielectric) continue;
        for (int a = 0; a < 3 && t->entry_face[k] < 0; ++a) {
            if (e->eu[a] != 0.0 || e->ev[a] != 0.0) continue;
            int f = -1;
            if (e->origin[a] == s->lo[a] && e->dir[a] > 0.0) f = 2 * a;
            if (e->origin[a] == s->hi[a] && e->dir[a] < 0.0) f = 2 * a + 1;
            if (f >= 0 && !(s->wall_mask & (1 << f))) t->entry_face[k] = f;
        }
    }
    const or_sensor *c = &s->sensor;
    if (c->kind == 1) {
        double lu = sqrt(c->U[0] * c->U[0] + c->U[1] * c->U[1] + c->U[2] * c->U[2]);
        double lv = sqrt(c->V[0] * c->V[0] + c->V[1] * c->V[1] + c->V[2] * c->V[2]);
        t->A_pix = lu * lv / ((double)c->width * (double)c->height);
    } else if (c->kind == 2) {
        t->tan_half = tan(0.5 * c->fov_y_deg * OR_PI / 180.0);
        t->aspect = (double)c->width / (double)c->height;
        t->A_pix = (2.0 * t->tan_half * t->aspect) * (2.0 * t->tan_half) /
                   ((double)c->width * (double)c->height);
    }
}

/* ---------------------------------------------------------------------------------------- */
/* Medium: nearest-voxel (piecewise-constant) fields over a grid that spans the AABB. */
static int voxel_index(const or_scene *s, const double x[3])
{
    int idx[3];
    for (int k = 0; k < 3; ++k) {
        double f = (x[k] - s->lo[k]) / (s->hi[k] - s->lo[k]) * (double)s->dims[k];
        int i = (int)floor(f);
        if (i < 0) i = 0;
        if (i > s->dims[k] - 1) i = s->dims[k] - 1;
        idx[k] = i;
    }
    return (idx[2] * s->dims[1] + idx[1]) * s->dims[0] + idx[0];
}

/* Coefficients at a point: solvent part and each dye's absorption (Sec. 4.1):
 * sigma_t = s(x) (sigma_s + sigma_a0) + sum_d eps_d a_d(lambda) c_d(x). */
typedef struct { double scat, dye[OR_MAX_DYES], bg, total; } coeffs;

/* `perturbed` selects the evaluation medium (the scene plus the render's perturbation). */
static coeffs coeffs_at_p(const or_scene *s, const tables *t, const double x[3], int bin,
                          int perturbed)
{
    coeffs c;
    double sv = 1.0;
    int v = -1;
    if (!t->homogeneous) v = voxel_index(s, x);
    if (s->solvent) sv = s->solvent[v] ? 1.0 : 0.0;
    double sig_s = s->sigma_s + (perturbed ? t->pert_sigma_s : 0.0);
    c.scat = sv * sig_s;
    c.bg = sv * s->sigma_a0;
    c.total = c.scat + c.bg;
    for (int d = 0; d < s->n_dyes; ++d) {
        double conc = s->conc ? (double)s->conc[(size_t)d * nvox(s) + v] : (double)s->conc_uniform[d];
        if (perturbed && d == t->pert_dye && (int64_t)v == t->pert_voxel) conc += t->pert_delta;
        c.dye[d] = t->sig_a[d][bin] * conc;
        c.total += c.dye[d];
    }
    return c;
}


/* Distance to leave the AABB along (x, w), and the face: faces (-x,+x,-y,+y,-z,+z) = 0..5;
 * ties go to the lowest face index. */
static double exit_distance(const or_scene *s, const double x[3], const double w[3], int *face)
{
    double best = INFINITY;
    int bf = -1;
    for (int k = 0; k < 3; ++k) {
        double tk;
        int f;
        if (w[k] > 0.0)      { tk = (s->hi[k] - x[k]) / w[k]; f = 2 * k + 1; }
        else if (w[k] < 0.0) { tk = (s->lo[k] - x[k]) / w[k]; f = 2 * k; }
        else continue;
        if (tk < 0.0) tk = 0.0;
        if (tk < best) { best = tk; bf = f; }
    }
    *face = bf;
    return best;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Exact optical depth int_0^L sigma_t(x0 + t w) dt of the piecewise-constant field (Eq. 6):
 * the segment is cut at every voxel-plane crossing and sigma_t is evaluated at each piece's
 * midpoint. */
/* Derivative sink of an optical depth: d tau / d c_d[v] = sig_a[d][bin] * (length in v) and
 * d tau / d sigma_s = s(x) * length, each times `scale`, added into grad_c / grad_sigma_s. */
typedef struct { double *grad_c; double *grad_sigma_s; double scale; } tau_grad;

static double optical_depth_g(const or_scene *s, const tables *t, const double x0[3],
                              const double w[3], double L, int bin, int perturbed,
                              const tau_grad *g);

static double optical_depth(const or_scene *s, const tables *t, const double x0[3],
                            const double w[3], double L, int bin)
{
    return optical_depth_g(s, t, x0, w, L, bin, t->frozen || t->pert_dye >= 0 ||
                           t->pert_sigma_s != 0.0, NULL);
}

static double optical_depth_g(const or_scene *s, const tables *t, const double x0[3],
                              const double w[3], double L, int bin, int perturbed,
                              const tau_grad *g)
{
    if (L <= 0.0) return 0.0;
    if (t->homogeneous) {
        coeffs c = coeffs_at_p(s, t, x0, bin, perturbed);
        if (g && g->grad_sigma_s) {
#pragma omp atomic
            *g->grad_sigma_s += g->scale * L;
        }
        return c.total * L;
    }
    int cap = 2 + s->dims[0] + s->dims[1] + s->dims[2] + 8;
    double *cuts = (double *)malloc(sizeof(double) * (size_t)cap);
    int n = 0;
    cuts[n++] = 0.0;
    cuts[n++] = L;
    for (int k = 0; k < 3; ++k) {
        if (w[k] == 0.0) continue;
        double h = (s->hi[k] - s->lo[k]) / (double)s->dims[k];
        for (int j = 1; j < s->dims[k]; ++j) {
            double tk = (s->lo[k] + j * h - x0[k]) / w[k];
            if (tk > 0.0 && tk < L) cuts[n++] = tk;
        }
    }
    qsort(cuts, (size_t)n, sizeof(double), cmp_double);
    double tau = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        double a = cuts[i], b = cuts[i + 1];
        if (b <= a) continue;
        double m = 0.5 * (a + b);
        double xm[3] = { x0[0] + m * w[0], x0[1] + m * w[1], x0[2] + m * w[2] };
        coeffs c = coeffs_at_p(s, t, xm, bin, perturbed);
        tau += c.total * (b - a);
        if (g) {
            int v = voxel_index(s, xm);
            double sv = s->solvent ? (s->solvent[v] ? 1.0 : 0.0) : 1.0;
            if (g->grad_sigma_s && sv != 0.0) {
#pragma omp atomic
                *g->grad_sigma_s += g->scale * sv * (b - a);
            }
            if (g->grad_c && s->conc)
                for (int d = 0; d < s->n_dyes; ++d) {
                    double dv = g->scale * t->sig_a[d][bin] * (b - a);
                    if (dv != 0.0) {
#pragma omp atomic
                        g->grad_c[(size_t)d * nvox(s) + v] += dv;
                    }
                }
        }
    }
    free(cuts);
    return tau;
}

/* ---------------------------------------------------------------------------------------- */
/* Directions. */
static void iso_dir(double u1, double u2, double w[3])
{
    double z = 1.0 - 2.0 * u1;
    double phi = 2.0 * OR_PI * u2;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    w[0] = r * cos(phi);
    w[1] = r * sin(phi);
    w[2] = z;
}

/* Cosine-weighted direction about the axis-aligned normal sign*e_k; tangents e_{k+1}, e_{k+2}. */
static void cosine_dir(double u1, double u2, int k, double sign, double w[3])
{
    double r = sqrt(u1);
    double phi = 2.0 * OR_PI * u2;
    double zl = sqrt(fmax(0.0, 1.0 - u1));
    w[k] = sign * zl;
    w[(k + 1) % 3] = r * cos(phi);
    w[(k + 2) % 3] = r * sin(phi);
}

static void normal_axis(const double n[3], int *k, double *sign)
{
    int best = 0;
    for (int i = 1; i < 3; ++i) if (fabs(n[i]) > fabs(n[best])) best = i;
    *k = best;
    *sign = n[best] > 0.0 ? 1.0 : -1.0;
}

/* Fresnel equations for unpolarised light at a smooth interface from index n1 into n2: the
 * reflected fraction (r_s^2 + r_p^2) / 2 for a ray meeting it at cos_i, and the refracted ray's
 * cosine in cos_t (Snell: n1 sin_i = n2 sin_t); beyond the critical angle everything is reflected
 * (total internal reflection, cos_t = 0). */
static double fresnel(double cos_i, double n1, double n2, double *cos_t)
{
    double sin_t2 = (n1 / n2) * (n1 / n2) * fmax(0.0, 1.0 - cos_i * cos_i);
    if (sin_t2 >= 1.0) { *cos_t = 0.0; return 1.0; }
    double ct = sqrt(1.0 - sin_t2);
    *cos_t = ct;
    double rs = (n1 * cos_i - n2 * ct) / (n1 * cos_i + n2 * ct);
    double rp = (n2 * cos_i - n1 * ct) / (n2 * cos_i + n1 * ct);
    return 0.5 * (rs * rs + rp * rp);
}

/* A photon meets the plane of box face `face` (axis k = face / 2) moving along w, from index n1
 * into n2. Returns 1 if it is reflected (w mirrored in the plane), 0 if refracted (w bent by
 * Snell's law: tangential components scaled by n1 / n2, normal component cos_t with its sign). */
static int interface_event(int face, double w[3], double n1, double n2, double u)
{
    int k = face / 2;
    double ct;
    double F = fresnel(fabs(w[k]), n1, n2, &ct);
    if (u < F) {
        w[k] = -w[k];
        return 1;
    }
    double sg = w[k] > 0.0 ? 1.0 : -1.0;
    for (int a = 0; a < 3; ++a) if (a != k) w[a] *= n1 / n2;
    w[k] = sg * ct;
    return 0;
}

/* Orthonormal tangents t1, t2 of a unit vector n (Duff, Burgess, Christensen, Hery, Kensler,
 * Liani, Villemin, "Building an orthonormal basis, revisited", JCGT 2017). */
static void tangent_frame(const double n[3], double t1[3], double t2[3])
{
    double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n[2]);
    double b = n[0] * n[1] * a;
    t1[0] = 1.0 + sg * n[0] * n[0] * a; t1[1] = sg * b; t1[2] = -sg * n[0];
    t2[0] = b; t2[1] = sg + n[1] * n[1] * a; t2[2] = -n[1];
}

/* Direction of the normalised Phong lobe about the unit vector r: density (e + 1)/(2 pi) cos^e
 * alpha over the sphere around r, cos alpha = u1^(1/(e+1)), azimuth 2 pi u2 in r's tangent frame. */
static void phong_dir(double u1, double u2, const double r[3], double e, double w[3])
{
    double ca = pow(u1, 1.0 / (e + 1.0));
    double sa = sqrt(fmax(0.0, 1.0 - ca * ca));
    double phi = 2.0 * OR_PI * u2;
    double t1[3], t2[3];
    tangent_frame(r, t1, t2);
    for (int k = 0; k < 3; ++k) w[k] = sa * cos(phi) * t1[k] + sa * sin(phi) * t2[k] + ca * r[k];
}

/* Wall BRDF divided by the albedo, times the outgoing cosine cos_o, toward direction o for a
 * photon whose mirror direction is r: (1 - g) cos_o / pi + g (e + 2)/(2 pi) cos^e alpha cos_o. */
static double wall_brdf_cos(const or_scene *s, const double r[3], const double o[3], double cos_o)
{
    double g = s->wall_gloss, e = s->wall_exponent;
    double ca = r[0] * o[0] + r[1] * o[1] + r[2] * o[2];
    double lobe = ca > 0.0 ? (e + 2.0) / (2.0 * OR_PI) * pow(ca, e) : 0.0;
    return ((1.0 - g) / OR_PI + g * lobe) * cos_o;
}

/* ---------------------------------------------------------------------------------------- */
/* Sensor connection (Eq. 3-6): contribution = vertex intensity toward the sensor
 * x transmittance x sensor importance.
 *   vertex intensity per unit photon weight: 1/(4 pi) for isotropic medium vertices (Sec. 2.1),
 *   cos(theta_o)/pi for Lambertian wall and light vertices.
 *   ortho importance: 1/A_pix (film = radiance averaged over the pixel's area);
 *   pinhole importance x geometry: 1/(A_pix r^2 cos^3 theta), A_pix the pixel area on the
 *   image plane at unit distance (film = radiance averaged over image-plane area).
 * The connecting segment must leave the box through an open (non-wall) face. */
typedef struct {
    int lambertian;         /* 1: wall or light vertex with normal sign * e_axis              */
    int axis;
    double sign;
    int glossy;             /* 1: wall vertex of a glossy wall; r is the incoming photon's mirror
                               direction, and the intensity follows the whole wall BRDF          */
    double r[3];
} vtx_kind;

/* Adjoint bookkeeping of one path: its tracking decisions and sensor connections in order. */
typedef struct {
    int64_t step;
    int kind;               /* 0 null, 1 scatter, 2 dye absorption, 3 background absorption */
    int voxel, bin, dye;
    double sigma_t, sigma_bar, solvent, conc;
} dec_rec;

typedef struct {
    int64_t step;
    double a;               /* adjoint-weighted contribution: A[pixel][bin] * value / N       */
    double x[3], dir[3], L;
    int bin;
} con_rec;

typedef struct {
    const double *adj;      /* [H][W][B] dL/dI                                                */
    double inv_n;
    int64_t cur_step;       /* step of the decision or vertex being processed                 */
    dec_rec *dec;
    int64_t n_dec, cap_dec;
    con_rec *con;
    int64_t n_con, cap_con;
} adj_path;

static void adj_push_dec(adj_path *A, dec_rec r)
{
    if (A->n_dec == A->cap_dec) {
        A->cap_dec = A->cap_dec ? 2 * A->cap_dec : 64;
        A->dec = (dec_rec *)realloc(A->dec, sizeof(dec_rec) * (size_t)A->cap_dec);
    }
    A->dec[A->n_dec++] = r;
}

static void adj_push_con(adj_path *A, con_rec r)
{
    if (A->n_con == A->cap_con) {
        A->cap_con = A->cap_con ? 2 * A->cap_con : 64;
        A->con = (con_rec *)realloc(A->con, sizeof(con_rec) * (size_t)A->cap_con);
    }
    A->con[A->n_con++] = r;
}

static void connect_sensor(const or_scene *s, const tables *t, const double x[3], int bin,
                           double w, vtx_kind vk, double *film, uint64_t *cnt, adj_path *A)
{
    const or_sensor *c = &s->sensor;
    if (c->kind == 0 || (film == NULL && A == NULL)) return;
    double dir[3], geom, r2 = 0.0;
    int px, py;
    if (c->kind == 1) {
        for (int k = 0; k < 3; ++k) dir[k] = c->view[k];
        double d[3] = { x[0] - c->origin[0], x[1] - c->origin[1], x[2] - c->origin[2] };
        double uu = c->U[0] * c->U[0] + c->U[1] * c->U[1] + c->U[2] * c->U[2];
        double vv = c->V[0] * c->V[0] + c->V[1] * c->V[1] + c->V[2] * c->V[2];
        double su = (d[0] * c->U[0] + d[1] * c->U[1] + d[2] * c->U[2]) / uu;
        double sv = (d[0] * c->V[0] + d[1] * c->V[1] + d[2] * c->V[2]) / vv;
        if (!(su >= 0.0 && su < 1.0 && sv >= 0.0 && sv < 1.0)) return;
        px = (int)floor(su * c->width);
        py = (int)floor(sv * c->height);
        if (px >= c->width || py >= c->height) return;
        geom = 1.0 / t->A_pix;
    } else {
        double v[3] = { x[0] - c->origin[0], x[1] - c->origin[1], x[2] - c->origin[2] };
        r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double r = sqrt(r2);
        double zf = v[0] * c->view[0] + v[1] * c->view[1] + v[2] * c->view[2];
        if (!(zf > 0.0)) return;
        double X = (v[0] * c->U[0] + v[1] * c->U[1] + v[2] * c->U[2]) / zf;
        double Y = (v[0] * c->V[0] + v[1] * c->V[1] + v[2] * c->V[2]) / zf;
        double sx = 0.5 * (X / (t->tan_half * t->aspect) + 1.0);
        double sy = 0.5 * (Y / t->tan_half + 1.0);
        if (!(sx >= 0.0 && sx < 1.0 && sy >= 0.0 && sy < 1.0)) return;
        px = (int)floor(sx * c->width);
        py = (int)floor(sy * c->height);
        if (px >= c->width || py >= c->height) return;
        for (int k = 0; k < 3; ++k) dir[k] = -v[k] / r;
        double cos_t = zf / r;
        geom = 1.0 / (t->A_pix * r2 * cos_t * cos_t * cos_t);
    }
    double f;
    if (vk.lambertian) {
        double co = vk.sign * dir[vk.axis];
        if (!(co > 0.0)) return;
        f = vk.glossy ? wall_brdf_cos(s, vk.r, dir, co) : co / OR_PI;
    } else {
        f = 1.0 / (4.0 * OR_PI);
    }
    int face;
    double tl = exit_distance(s, x, dir, &face);
    if (face < 0) return;
    if (s->wall_mask & (1 << face)) return;
    if (t->dielectric) {
        /* the connection leaves through a dielectric face at normal incidence (the sensor is
         * orthographic and looks along a face normal): the transmitted fraction 1 - F, and the
         * radiance changes by 1 / ior^2 from the solution into the outside (L / n^2 is invariant
         * along a refracted ray) */
        double ct;
        double F = fresnel(fabs(dir[face / 2]), t->ior, 1.0, &ct);
        f *= (1.0 - F) / (t->ior * t->ior);
    }
    if (c->kind == 2 && tl * tl > r2) return; /* eye inside the box: not supported, skip */
    double T = exp(-optical_depth(s, t, x, dir, tl, bin));
    double val = w * f * T * geom;
    size_t idx = ((size_t)py * c->width + px) * t->B + bin;
    if (film) {
#pragma omp atomic
        film[idx] += val;
    }
    if (A) {
        con_rec r;
        r.step = A->cur_step;
        r.a = A->adj[idx] * val * A->inv_n;
        for (int k = 0; k < 3; ++k) { r.x[k] = x[k]; r.dir[k] = dir[k]; }
        r.L = tl;
        r.bin = bin;
        if (r.a != 0.0) adj_push_con(A, r);
    }
    cnt[OC_CONNECTIONS]++;
}

/* ---------------------------------------------------------------------------------------- */
/* One photon path. */
typedef struct {
    double face[2][6][OR_MAX_BINS];
    double absorbed[OR_MAX_DYES + 1][OR_MAX_BINS];
    double emitted[OR_MAX_DYES][OR_MAX_BINS];
    uint64_t cnt[OR_NCOUNTERS];
} local_tally;

static int sample_emitter(const tables *t, int n, double u)
{
    for (int k = 0; k < n; ++k) if ((double)t->em_cdf32[k] > u) return k;
    return n - 1;
}

/* lambda' = min{ i : CDF_d[i] > u }, decided on the fp32-rounded CDF. */
static int sample_emission_bin(const tables *t, int d, double u)
{
    for (int i = 0; i < t->B; ++i) if ((double)t->cdf32[d][i] > u) return i;
    return t->B - 1;
}

static void apply_params_macro(const or_scene *s, tables *t, const or_params *p)
{
    build_macro(s, t, p->macro_cell);
    if (p->macro_cell <= 0) build_skip(s, t, p->skip_cell);
}

/* Local majorant of macro cell c: the maximum of sigma_t over the cell (Sec. 4.1 coefficients). */
static double cell_majorant(const or_scene *s, const tables *t, int64_t c, int bin)
{
    double m = t->mc_smax[c] * (s->sigma_s + s->sigma_a0);
    for (int d = 0; d < s->n_dyes; ++d) m += t->sig_a[d][bin] * t->mc_cmax[c * s->n_dyes + d];
    return m * t->maj_scale;
}

/* Free flight against local majorants: the optical budget tau = -ln(1 - u) is spent cell by cell
 * along the ray (each cell at its own majorant); returns the tentative collision distance, or
 * INFINITY when the budget outlasts the distance te to the box boundary, and the local majorant
 * at the tentative point. */
static double macro_flight(const or_scene *s, const tables *t, const double x[3], const double w[3],
                           int bin, double tau, double te, double *sb_out)
{
    int c[3], stp[3];
    double tmax[3], tdel[3];
    for (int k = 0; k < 3; ++k) {
        double cs = t->mc * (s->hi[k] - s->lo[k]) / (double)s->dims[k];
        int ck = (int)floor((x[k] - s->lo[k]) / cs);
        if (ck < 0) ck = 0;
        if (ck > t->mdims[k] - 1) ck = t->mdims[k] - 1;
        c[k] = ck;
        if (w[k] > 0.0) {
            stp[k] = 1;
            tmax[k] = (s->lo[k] + (ck + 1) * cs - x[k]) / w[k];
            tdel[k] = cs / w[k];
        } else if (w[k] < 0.0) {
            stp[k] = -1;
            tmax[k] = (s->lo[k] + ck * cs - x[k]) / w[k];
            tdel[k] = -cs / w[k];
        } else {
            stp[k] = 0;
            tmax[k] = INFINITY;
            tdel[k] = INFINITY;
        }
    }
    double t0 = 0.0;
    for (;;) {
        int64_t cell = ((int64_t)c[2] * t->mdims[1] + c[1]) * t->mdims[0] + c[0];
        double sbc = cell_majorant(s, t, cell, bin);
        int ax = 0;
        for (int k = 1; k < 3; ++k) if (tmax[k] < tmax[ax]) ax = k;
        double t1 = tmax[ax] < te ? tmax[ax] : te;
        if (t1 < t0) t1 = t0;
        if (sbc > 0.0 && tau < sbc * (t1 - t0)) {
            *sb_out = sbc;
            return t0 + tau / sbc;
        }
        tau -= sbc * (t1 - t0);
        t0 = t1;
        if (t1 >= te) { *sb_out = sbc; return INFINITY; }
        c[ax] += stp[ax];
        if (c[ax] < 0 || c[ax] >= t->mdims[ax]) { *sb_out = sbc; return INFINITY; }
        tmax[ax] += tdel[ax];
    }
}

static uint32_t trace_path(const or_scene *s, const tables *t, const or_params *p, uint64_t pid,
                           local_tally *lt, double *film, adj_path *A)
{
    uint64_t *cnt = lt->cnt;
    cnt[OC_PATHS]++;
    /* frozen sampling: decisions in the base medium, tallies times W = p_eval / p_sample */
    const int has_pert = t->pert_dye >= 0 || t->pert_sigma_s != 0.0;
    const int samp_pert = has_pert && !t->frozen;
    const int weigh = has_pert && t->frozen;
    double W = 1.0;
    if (A) A->cur_step = -1;
    /* spawn (Eq. 12: p(x_n), p(lambda_x)) */
    block4 S0 = rng_block(p->seed, p->medium_id, pid, STEP_SPAWN, 0);
    int ek = sample_emitter(t, s->n_emitters, S0.u[0]);
    const or_emitter *em = &s->emitters[ek];
    double x[3], w[3];
    for (int k = 0; k < 3; ++k) x[k] = em->origin[k] + S0.u[1] * em->eu[k] + S0.u[2] * em->ev[k];
    int bin = t->em_bin[ek];
    double wt = 1.0;
    if (em->kind == 1) {
        block4 S1 = rng_block(p->seed, p->medium_id, pid, STEP_SPAWN, 1);
        int ax; double sg;
        normal_axis(em->dir, &ax, &sg);
        cosine_dir(S0.u[3], S1.u[0], ax, sg, w);
        vtx_kind vk = { 1, ax, sg, 0, { 0, 0, 0 } };
        if (!p->paper_mode) connect_sensor(s, t, x, bin, wt, vk, film, cnt, A);
    } else {
        for (int k = 0; k < 3; ++k) w[k] = em->dir[k];
    }
    if (t->entry_face[ek] >= 0) {
        /* entering the solution through a dielectric face: Fresnel reflection sends the photon
         * back out through that face, else Snell refraction bends it in (coin: slot 1, word 1) */
        block4 S1 = rng_block(p->seed, p->medium_id, pid, STEP_SPAWN, 1);
        int f = t->entry_face[ek];
        if (interface_event(f, w, 1.0, t->ior, S1.u[1])) {
            cnt[OC_IFACE_REFLECTIONS]++;
            lt->face[0][f][bin] += wt * W;
            cnt[OC_ESCAPES]++;
            return 0;
        }
    }
    int64_t n_events = 0;
    int n_inel = 0;
    int fl = 0;
    for (int64_t step = 0;; ++step) {
        if (step >= p->max_steps) { cnt[OC_STEP_BUDGET]++; break; }
        if (A) A->cur_step = step;
        cnt[OC_STEPS]++;
        block4 B0 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 0);
        int face;
        double te = exit_distance(s, x, w, &face);
        double sb, tf;
        if (t->mc) {
            tf = macro_flight(s, t, x, w, bin, -log(1.0 - B0.u[0]), te, &sb);
        } else {
            sb = t->majorant[bin];
            tf = sb > 0.0 ? -log(1.0 - B0.u[0]) / sb : INFINITY;
        }
        if (tf >= te) {
            for (int k = 0; k < 3; ++k) x[k] += te * w[k];
            if (t->dielectric && !(s->wall_mask & (1 << face))) {
                /* a dielectric face from inside: Fresnel reflection (an event; the coin is the
                 * step's unused u_real) or refraction out of the solution (an escape) */
                double wr[3] = { w[0], w[1], w[2] };
                if (interface_event(face, wr, t->ior, 1.0, B0.u[1])) {
                    if (n_events == p->max_events) { cnt[OC_CAP_HITS]++; break; }
                    n_events++;
                    cnt[OC_EVENTS]++;
                    cnt[OC_IFACE_REFLECTIONS]++;
                    for (int k = 0; k < 3; ++k) w[k] = wr[k];
                    x[face / 2] = (face & 1) ? s->hi[face / 2] : s->lo[face / 2];
                    if (n_events >= p->n_rr) {
                        block4 B1 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 1);
                        double q = wt < 1.0 ? wt : 1.0;
                        if (!(B1.u[2] < q)) { cnt[OC_RR_KILLS]++; break; }
                        wt /= q;
                    }
                    continue;
                }
                lt->face[fl][face][bin] += wt * W;
                cnt[OC_ESCAPES]++;
                break;
            }
            if (s->wall_mask & (1 << face)) {
                /* Lambertian wall: a real event (in paper mode, excitation light reflected by a
                 * wall before any emission is dropped) */
                if (p->paper_mode && !fl) { cnt[OC_VF_REJECTED]++; break; }
                if (n_events == p->max_events) { cnt[OC_CAP_HITS]++; break; }
                n_events++;
                cnt[OC_EVENTS]++;
                cnt[OC_WALL_BOUNCES]++;
                block4 B1 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 1);
                if (p->analog) {
                    if (!(B1.u[3] < s->wall_albedo)) { cnt[OC_ABSORBED_DEAD]++; break; }
                } else {
                    wt *= s->wall_albedo;
                    if (wt == 0.0) { cnt[OC_ABSORBED_DEAD]++; break; }
                }
                int ax = face / 2;
                double sg = (face & 1) ? -1.0 : 1.0;   /* inward normal */
                /* snap onto the wall plane */
                x[ax] = (face & 1) ? s->hi[ax] : s->lo[ax];
                if (s->wall_gloss > 0.0) {
                    /* glossy wall: the sensor sees the whole BRDF; the path continues in the
                     * Phong lobe about the mirror direction with probability g (lobe weight
                     * (e + 2)/(e + 1) cos_o; below the wall it ends), else in the diffuse lobe */
                    vtx_kind vk = { 1, ax, sg, 1, { w[0], w[1], w[2] } };
                    vk.r[ax] = -w[ax];
                    connect_sensor(s, t, x, bin, wt * W, vk, film, cnt, A);
                    if (B1.u[0] < s->wall_gloss) {
                        phong_dir(B0.u[2], B0.u[3], vk.r, s->wall_exponent, w);
                        double co = sg * w[ax];
                        if (!(co > 0.0)) { cnt[OC_ABSORBED_DEAD]++; break; }
                        wt *= (s->wall_exponent + 2.0) / (s->wall_exponent + 1.0) * co;
                    } else {
                        cosine_dir(B0.u[2], B0.u[3], ax, sg, w);
                    }
                } else {
                    cosine_dir(B0.u[2], B0.u[3], ax, sg, w);
                    vtx_kind vk = { 1, ax, sg, 0, { 0, 0, 0 } };
                    connect_sensor(s, t, x, bin, wt * W, vk, film, cnt, A);
                }
                if (n_events >= p->n_rr) {
                    double q = wt < 1.0 ? wt : 1.0;
                    if (!(B1.u[2] < q)) { cnt[OC_RR_KILLS]++; break; }
                    wt /= q;
                }
                continue;
            }
            lt->face[fl][face][bin] += wt * W;
            cnt[OC_ESCAPES]++;
            break;
        }
        for (int k = 0; k < 3; ++k) x[k] += tf * w[k];
        coeffs c = coeffs_at_p(s, t, x, bin, samp_pert);
        coeffs ce = c;
        if (weigh) ce = coeffs_at_p(s, t, x, bin, 1);
        if (c.total > sb) cnt[OC_MAJORANT_VIOLATIONS]++;
        int vox = t->homogeneous ? -1 : voxel_index(s, x);
        double solv = s->solvent ? (s->solvent[vox] ? 1.0 : 0.0) : 1.0;
        if (!(B0.u[1] * sb < c.total)) {
            cnt[OC_NULLS]++;
            if (weigh) W *= (1.0 - ce.total / sb) / (1.0 - c.total / sb);
            if (A) {
                dec_rec r = { step, 0, vox, bin, -1, c.total, sb, solv, 0.0 };
                adj_push_dec(A, r);
            }
            if (t->sk && c.total == 0.0) {
                /* leave the empty cube: every tentative collision inside it would be a null */
                int f2;
                double te2 = exit_distance(s, x, w, &f2);
                double tl = empty_cube_exit(s, t, x, w);
                if (tl > te2) tl = te2;
                for (int k = 0; k < 3; ++k) x[k] += tl * w[k];
            }
            continue;
        }
        /* real collision */
        if (n_events == p->max_events) { cnt[OC_CAP_HITS]++; break; }
        n_events++;
        cnt[OC_EVENTS]++;
        block4 B1 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 1);
        /* particle type in proportion to its coefficient (Sec. 4.1) */
        double ue = B0.u[2] * c.total;
        double acc = c.scat;
        int ev = -1;          /* -1 scatter, 0..D-1 dye, D background */
        if (!(ue < acc)) {
            ev = s->n_dyes;
            for (int d = 0; d < s->n_dyes; ++d) {
                acc += c.dye[d];
                if (ue < acc) { ev = d; break; }
            }
        }
        if (weigh) {
            /* probability of "real collision, then this particle" is sigma_e / sigma_bar */
            double pe = ev < 0 ? ce.scat / c.scat : (ev < s->n_dyes ? ce.dye[ev] / c.dye[ev] : ce.bg / c.bg);
            W *= pe;
        }
        if (A) {
            double conc = 0.0;
            if (ev >= 0 && ev < s->n_dyes)
                conc = s->conc ? (double)s->conc[(size_t)ev * nvox(s) + vox] : (double)s->conc_uniform[ev];
            dec_rec r = { step, ev < 0 ? 1 : (ev < s->n_dyes ? 2 : 3), vox, bin, ev, c.total, sb, solv,
                          conc };
            adj_push_dec(A, r);
        }
        if (ev < 0) {
            cnt[OC_SCATTERS]++;
            if (p->paper_mode && !fl) { cnt[OC_VF_REJECTED]++; break; }  /* excitation scattering */
            iso_dir(B0.u[3], B1.u[0], w);
            vtx_kind vk = { 0, 0, 0.0, 0, { 0, 0, 0 } };
            connect_sensor(s, t, x, bin, wt * W, vk, film, cnt, A);
        } else if (ev < s->n_dyes) {
            cnt[OC_DYE_ABSORPTIONS]++;
            lt->absorbed[ev][bin] += wt * W;
            if ((p->max_inelastic >= 0 && n_inel >= p->max_inelastic) || (p->paper_mode && n_inel >= 1)) {
                cnt[OC_VF_REJECTED]++;
                break;
            }
            if (p->analog) {
                if (!(B1.u[3] < t->qy[ev])) { cnt[OC_ABSORBED_DEAD]++; break; }
            } else {
                wt *= t->qy[ev];
                if (wt == 0.0) { cnt[OC_ABSORBED_DEAD]++; break; }
            }
            bin = sample_emission_bin(t, ev, B1.u[1]);
            lt->emitted[ev][bin] += wt * W;
            cnt[OC_EMISSIONS]++;
            n_inel++;
            fl = 1;
            iso_dir(B0.u[3], B1.u[0], w);
            vtx_kind vk = { 0, 0, 0.0, 0, { 0, 0, 0 } };
            connect_sensor(s, t, x, bin, wt * W, vk, film, cnt, A);
        } else {
            lt->absorbed[s->n_dyes][bin] += wt * W;
            cnt[OC_ABSORBED_DEAD]++;
            break;
        }
        if (n_events >= p->n_rr) {
            double q = wt < 1.0 ? wt : 1.0;
            if (!(B1.u[2] < q)) { cnt[OC_RR_KILLS]++; break; }
            wt /= q;
        }
    }
    return (uint32_t)n_events;
}


/* ---------------------------------------------------------------------------------------- */
/* Hero-wavelength paths (Wilkie et al., "Hero wavelength spectral sampling", EGSR 2014, cited in
 * the paper's Sec. 3 as a way to cut the cost of per-wavelength transport).
 *
 * A path carries a set of up to C wavelengths. One of them, the hero, drives every sampling
 * decision exactly as a single-wavelength path would; the others ride along, and every tally is
 * split among the members by the balance heuristic of spectral MIS. The set is a block of a fixed
 * partition of the wavelengths that holds the hero, so that any member, had it been drawn as the
 * hero, would have carried the same set:
 *   - at the source, the lines of the hero's source (same geometry) in index order, cut into
 *     blocks of C lines; line k is drawn with probability P_k (its power share);
 *   - after a re-emission by dye d, the bins [C floor(b/C), C floor(b/C) + C) around the drawn bin
 *     b; bin k is drawn with probability p_d(k), the emission pmf realised by the fp32 CDF.
 * With P(k) the probability that member k is drawn as the hero and p(path | k) the probability
 * density of the decisions taken since the set was drawn, evaluated at member k's wavelength,
 * the balance-heuristic estimate for member j is W * q_j with
 *     q_j = P(j) p(path | j) / sum_k P(k) p(path | k),
 * W the hero's ordinary path weight. Free flights are drawn against the set's majorant
 * sigma_bar = max_k sigma_bar(lambda_k), so distances and directions have the same density for all
 * members; a null collision at x has probability (sigma_bar - sigma_t(x, lambda_k)) / sigma_bar,
 * a scattering sigma_s / sigma_bar (the same for all: scattering is grey), a dye absorption
 * sigma_a,d(x, lambda_k) / sigma_bar, a background absorption sigma_a0 / sigma_bar and a wall
 * bounce the flat albedo. Hence q changes only at null collisions (and, for the absorbed tally,
 * at a dye absorption). A re-emission's outcome does not depend on which member was absorbed
 * (QY_d and the emission spectrum belong to the dye), so the path goes on with weight W QY_d and
 * a fresh set. With C = 1 the estimator is the single-wavelength one, decision for decision. */
static double emission_pmf(const tables *t, int d, int b);

typedef struct {
    int n;                  /* members                                                         */
    int hero;               /* index of the hero among them                                    */
    int bin[4];
    double q[4];            /* balance-heuristic weights, sum 1                                */
    double sb;              /* the set's majorant                                              */
} hero_set;

static void hero_majorant(const tables *t, hero_set *h)
{
    h->sb = 0.0;
    for (int k = 0; k < h->n; ++k) if (t->majorant[h->bin[k]] > h->sb) h->sb = t->majorant[h->bin[k]];
}

static void hero_normalise(hero_set *h)
{
    double z = 0.0;
    for (int k = 0; k < h->n; ++k) z += h->q[k];
    for (int k = 0; k < h->n; ++k) h->q[k] /= z;
}

static double line_pmf(const tables *t, int k)
{
    return (double)t->em_cdf32[k] - (k > 0 ? (double)t->em_cdf32[k - 1] : 0.0);
}

/* The hero's source lines, blocks of C in index order. */
static void hero_lines(const or_scene *s, const tables *t, int ek, int C, hero_set *h)
{
    int idx[OR_MAX_EMITTERS], m = 0, pos = 0;
    for (int k = 0; k < s->n_emitters; ++k)
        if (s->emitters[k].group == s->emitters[ek].group) {
            if (k == ek) pos = m;
            idx[m++] = k;
        }
    int first = (pos / C) * C;
    h->n = 0;
    for (int k = first; k < m && k < first + C; ++k) {
        if (idx[k] == ek) h->hero = h->n;
        h->bin[h->n] = t->em_bin[idx[k]];
        h->q[h->n] = line_pmf(t, idx[k]);
        h->n++;
    }
    hero_normalise(h);
    hero_majorant(t, h);
}

/* The emission block around bin b of dye d. */
static void hero_emission(const tables *t, int d, int b, int C, hero_set *h)
{
    int first = (b / C) * C;
    h->n = 0;
    for (int k = first; k < t->B && k < first + C; ++k) {
        if (k == b) h->hero = h->n;
        h->bin[h->n] = k;
        h->q[h->n] = emission_pmf(t, d, k);
        h->n++;
    }
    hero_normalise(h);
    hero_majorant(t, h);
}

/* Sensor connection of a vertex for every member: the geometry is shared, the transmittance is
 * each member's (exact optical depth, Eq. 6); member k adds w q_k f T_k geom. */
static void connect_sensor_hero(const or_scene *s, const tables *t, const double x[3],
                                const hero_set *h, double w, vtx_kind vk, double *film, uint64_t *cnt)
{
    const or_sensor *c = &s->sensor;
    if (c->kind == 0 || film == NULL) return;
    double dir[3], geom, r2 = 0.0;
    int px, py;
    if (c->kind == 1) {
        for (int k = 0; k < 3; ++k) dir[k] = c->view[k];
        double d[3] = { x[0] - c->origin[0], x[1] - c->origin[1], x[2] - c->origin[2] };
        double uu = c->U[0] * c->U[0] + c->U[1] * c->U[1] + c->U[2] * c->U[2];
        double vv = c->V[0] * c->V[0] + c->V[1] * c->V[1] + c->V[2] * c->V[2];
        double su = (d[0] * c->U[0] + d[1] * c->U[1] + d[2] * c->U[2]) / uu;
        double sv = (d[0] * c->V[0] + d[1] * c->V[1] + d[2] * c->V[2]) / vv;
        if (!(su >= 0.0 && su < 1.0 && sv >= 0.0 && sv < 1.0)) return;
        px = (int)floor(su * c->width);
        py = (int)floor(sv * c->height);
        if (px >= c->width || py >= c->height) return;
        geom = 1.0 / t->A_pix;
    } else {
        double v[3] = { x[0] - c->origin[0], x[1] - c->origin[1], x[2] - c->origin[2] };
        r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double r = sqrt(r2);
        double zf = v[0] * c->view[0] + v[1] * c->view[1] + v[2] * c->view[2];
        if (!(zf > 0.0)) return;
        double X = (v[0] * c->U[0] + v[1] * c->U[1] + v[2] * c->U[2]) / zf;
        double Y = (v[0] * c->V[0] + v[1] * c->V[1] + v[2] * c->V[2]) / zf;
        double sx = 0.5 * (X / (t->tan_half * t->aspect) + 1.0);
        double sy = 0.5 * (Y / t->tan_half + 1.0);
        if (!(sx >= 0.0 && sx < 1.0 && sy >= 0.0 && sy < 1.0)) return;
        px = (int)floor(sx * c->width);
        py = (int)floor(sy * c->height);
        if (px >= c->width || py >= c->height) return;
        for (int k = 0; k < 3; ++k) dir[k] = -v[k] / r;
        double cos_t = zf / r;
        geom = 1.0 / (t->A_pix * r2 * cos_t * cos_t * cos_t);
    }
    double f;
    if (vk.lambertian) {
        double co = vk.sign * dir[vk.axis];
        if (!(co > 0.0)) return;
        f = co / OR_PI;
    } else {
        f = 1.0 / (4.0 * OR_PI);
    }
    int face;
    double tl = exit_distance(s, x, dir, &face);
    if (face < 0) return;
    if (s->wall_mask & (1 << face)) return;
    if (c->kind == 2 && tl * tl > r2) return;
    for (int k = 0; k < h->n; ++k) {
        if (h->q[k] == 0.0) continue;
        double T = exp(-optical_depth(s, t, x, dir, tl, h->bin[k]));
        size_t idx = ((size_t)py * c->width + px) * t->B + h->bin[k];
#pragma omp atomic
        film[idx] += w * h->q[k] * f * T * geom;
    }
    cnt[OC_CONNECTIONS]++;
}

static uint32_t trace_path_hero(const or_scene *s, const tables *t, const or_params *p,
                                uint64_t pid, local_tally *lt, double *film)
{
    uint64_t *cnt = lt->cnt;
    cnt[OC_PATHS]++;
    const int C = p->hero;
    block4 S0 = rng_block(p->seed, p->medium_id, pid, STEP_SPAWN, 0);
    int ek = sample_emitter(t, s->n_emitters, S0.u[0]);
    const or_emitter *em = &s->emitters[ek];
    hero_set h;
    hero_lines(s, t, ek, C, &h);
    double x[3], w[3];
    for (int k = 0; k < 3; ++k) x[k] = em->origin[k] + S0.u[1] * em->eu[k] + S0.u[2] * em->ev[k];
    double wt = 1.0;
    if (em->kind == 1) {
        block4 S1 = rng_block(p->seed, p->medium_id, pid, STEP_SPAWN, 1);
        int ax; double sg;
        normal_axis(em->dir, &ax, &sg);
        cosine_dir(S0.u[3], S1.u[0], ax, sg, w);
        vtx_kind vk = { 1, ax, sg };
        connect_sensor_hero(s, t, x, &h, wt, vk, film, cnt);
    } else {
        for (int k = 0; k < 3; ++k) w[k] = em->dir[k];
    }
    int64_t n_events = 0;
    int n_inel = 0;
    int fl = 0;
    for (int64_t step = 0;; ++step) {
        if (step >= p->max_steps) { cnt[OC_STEP_BUDGET]++; break; }
        cnt[OC_STEPS]++;
        block4 B0 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 0);
        const int hb = h.bin[h.hero];
        int face;
        double te = exit_distance(s, x, w, &face);
        double sb = h.sb;
        double tf = sb > 0.0 ? -log(1.0 - B0.u[0]) / sb : INFINITY;
        if (tf >= te) {
            for (int k = 0; k < 3; ++k) x[k] += te * w[k];
            if (s->wall_mask & (1 << face)) {
                if (n_events == p->max_events) { cnt[OC_CAP_HITS]++; break; }
                n_events++;
                cnt[OC_EVENTS]++;
                cnt[OC_WALL_BOUNCES]++;
                block4 B1 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 1);
                if (p->analog) {
                    if (!(B1.u[3] < s->wall_albedo)) { cnt[OC_ABSORBED_DEAD]++; break; }
                } else {
                    wt *= s->wall_albedo;
                    if (wt == 0.0) { cnt[OC_ABSORBED_DEAD]++; break; }
                }
                int ax = face / 2;
                double sg = (face & 1) ? -1.0 : 1.0;
                x[ax] = (face & 1) ? s->hi[ax] : s->lo[ax];
                cosine_dir(B0.u[2], B0.u[3], ax, sg, w);
                vtx_kind vk = { 1, ax, sg };
                connect_sensor_hero(s, t, x, &h, wt, vk, film, cnt);
                if (n_events >= p->n_rr) {
                    double q = wt < 1.0 ? wt : 1.0;
                    if (!(B1.u[2] < q)) { cnt[OC_RR_KILLS]++; break; }
                    wt /= q;
                }
                continue;
            }
            for (int k = 0; k < h.n; ++k) lt->face[fl][face][h.bin[k]] += wt * h.q[k];
            cnt[OC_ESCAPES]++;
            break;
        }
        for (int k = 0; k < 3; ++k) x[k] += tf * w[k];
        coeffs c = coeffs_at_p(s, t, x, hb, 0);
        if (c.total > sb) cnt[OC_MAJORANT_VIOLATIONS]++;
        if (!(B0.u[1] * sb < c.total)) {
            cnt[OC_NULLS]++;
            /* member k's null probability over the hero's */
            for (int k = 0; k < h.n; ++k) {
                if (k == h.hero) continue;
                double ck = coeffs_at_p(s, t, x, h.bin[k], 0).total;
                if (ck > sb) cnt[OC_MAJORANT_VIOLATIONS]++;
                h.q[k] *= (sb - ck) / (sb - c.total);
            }
            hero_normalise(&h);
            if (t->sk && c.total == 0.0) {
                int f2;
                double te2 = exit_distance(s, x, w, &f2);
                double tl = empty_cube_exit(s, t, x, w);
                if (tl > te2) tl = te2;
                for (int k = 0; k < 3; ++k) x[k] += tl * w[k];
            }
            continue;
        }
        if (n_events == p->max_events) { cnt[OC_CAP_HITS]++; break; }
        n_events++;
        cnt[OC_EVENTS]++;
        block4 B1 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 1);
        double ue = B0.u[2] * c.total;
        double acc = c.scat;
        int ev = -1;
        if (!(ue < acc)) {
            ev = s->n_dyes;
            for (int d = 0; d < s->n_dyes; ++d) {
                acc += c.dye[d];
                if (ue < acc) { ev = d; break; }
            }
        }
        if (ev < 0) {
            cnt[OC_SCATTERS]++;
            iso_dir(B0.u[3], B1.u[0], w);
            vtx_kind vk = { 0, 0, 0.0, 0, { 0, 0, 0 } };
            connect_sensor_hero(s, t, x, &h, wt, vk, film, cnt);
        } else if (ev < s->n_dyes) {
            cnt[OC_DYE_ABSORPTIONS]++;
            /* the absorbed tally: member k's probability of this dye absorption over the hero's */
            hero_set ha = h;
            for (int k = 0; k < h.n; ++k)
                if (k != h.hero) ha.q[k] *= coeffs_at_p(s, t, x, h.bin[k], 0).dye[ev] / c.dye[ev];
            hero_normalise(&ha);
            for (int k = 0; k < h.n; ++k) lt->absorbed[ev][h.bin[k]] += wt * ha.q[k];
            if (p->max_inelastic >= 0 && n_inel >= p->max_inelastic) { cnt[OC_VF_REJECTED]++; break; }
            if (p->analog) {
                if (!(B1.u[3] < t->qy[ev])) { cnt[OC_ABSORBED_DEAD]++; break; }
            } else {
                wt *= t->qy[ev];
                if (wt == 0.0) { cnt[OC_ABSORBED_DEAD]++; break; }
            }
            int b = sample_emission_bin(t, ev, B1.u[1]);
            hero_emission(t, ev, b, C, &h);
            for (int k = 0; k < h.n; ++k) lt->emitted[ev][h.bin[k]] += wt * h.q[k];
            cnt[OC_EMISSIONS]++;
            n_inel++;
            fl = 1;
            iso_dir(B0.u[3], B1.u[0], w);
            vtx_kind vk = { 0, 0, 0.0, 0, { 0, 0, 0 } };
            connect_sensor_hero(s, t, x, &h, wt, vk, film, cnt);
        } else {
            /* grey background absorption: the weights stay */
            for (int k = 0; k < h.n; ++k) lt->absorbed[s->n_dyes][h.bin[k]] += wt * h.q[k];
            cnt[OC_ABSORBED_DEAD]++;
            break;
        }
        if (n_events >= p->n_rr) {
            double q = wt < 1.0 ? wt : 1.0;
            if (!(B1.u[2] < q)) { cnt[OC_RR_KILLS]++; break; }
            wt /= q;
        }
    }
    return (uint32_t)n_events;
}

/* ---------------------------------------------------------------------------------------- */
/* Exported API (ctypes). Return 0 on success, negative on invalid input. */

/* Interfaces and glossy walls: ior 0 or >= 1, gloss in [0, 1], exponent >= 0. With dielectric
 * faces the sensor must be orthographic and look along a face normal (a connection through a
 * flat interface to a pinhole needs the refraction point, which is not solved here); hero paths
 * and the paper's model are index-matched and Lambertian only. */
static int interfaces_supported(const or_scene *s, const or_params *p)
{
    if (!(s->ior == 0.0 || s->ior >= 1.0) || !(s->wall_gloss >= 0.0 && s->wall_gloss <= 1.0) ||
        !(s->wall_exponent >= 0.0))
        return 0;
    int special = s->ior > 1.0 || s->wall_gloss > 0.0;
    if (special && p && (p->hero > 0 || p->paper_mode)) return 0;
    if (s->ior > 1.0) {
        if (s->sensor.kind == 2) return 0;
        if (s->sensor.kind == 1) {
            int zeros = 0;
            for (int k = 0; k < 3; ++k) zeros += s->sensor.view[k] == 0.0;
            if (zeros != 2) return 0;
        }
    }
    return 1;
}

int or_render(const or_scene *s, const or_params *p, or_result *r)
{
    if (!s || !p || !r) return -1;
    if (s->n_bins <= 0 || s->n_bins > OR_MAX_BINS) return -1;
    if (s->n_dyes < 0 || s->n_dyes > OR_MAX_DYES) return -1;
    if (s->n_emitters <= 0 || s->n_emitters > OR_MAX_EMITTERS) return -1;
    if (p->hero < 0 || p->hero > 4) return -1;
    if (p->hero > 0 && (p->macro_cell > 0 || p->paper_mode || p->frozen || p->pert_dye >= 0 ||
                        p->pert_sigma_s != 0.0)) return -1;
    if (!interfaces_supported(s, p)) return -1;
    tables *t = (tables *)malloc(sizeof(tables));
    build_tables(s, t);
    apply_params(t, p);
    apply_params_macro(s, t, p);
    int B = s->n_bins, D = s->n_dyes;
    memset(r->face, 0, sizeof(double) * 2 * 6 * B);
    memset(r->absorbed, 0, sizeof(double) * (D + 1) * B);
    if (D > 0) memset(r->emitted, 0, sizeof(double) * D * B);
    memset(r->counters, 0, sizeof(uint64_t) * OR_NCOUNTERS);
    if (r->film && s->sensor.kind)
        memset(r->film, 0, sizeof(double) * (size_t)s->sensor.width * s->sensor.height * B);
#ifdef _OPENMP
    omp_set_num_threads(p->n_threads > 0 ? p->n_threads : omp_get_num_procs());
#endif
    int64_t N = (int64_t)p->n_paths;
#pragma omp parallel
    {
        local_tally *lt = (local_tally *)calloc(1, sizeof(local_tally));
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i) {
            uint32_t ne = p->hero > 0
                ? trace_path_hero(s, t, p, p->path_offset + (uint64_t)i, lt, r->film)
                : trace_path(s, t, p, p->path_offset + (uint64_t)i, lt, r->film, NULL);
            if (r->path_events) r->path_events[i] = ne;
        }
#pragma omp critical
        {
            for (int fl = 0; fl < 2; ++fl)
                for (int f = 0; f < 6; ++f)
                    for (int b = 0; b < B; ++b) r->face[(fl * 6 + f) * B + b] += lt->face[fl][f][b];
            for (int d = 0; d <= D; ++d)
                for (int b = 0; b < B; ++b) r->absorbed[d * B + b] += lt->absorbed[d][b];
            for (int d = 0; d < D; ++d)
                for (int b = 0; b < B; ++b) r->emitted[d * B + b] += lt->emitted[d][b];
            for (int k = 0; k < OR_NCOUNTERS; ++k) r->counters[k] += lt->cnt[k];
        }
        free(lt);
    }
    /* tallies are per launched path */
    double inv = N > 0 ? 1.0 / (double)N : 0.0;
    for (int i = 0; i < 2 * 6 * B; ++i) r->face[i] *= inv;
    for (int i = 0; i < (D + 1) * B; ++i) r->absorbed[i] *= inv;
    for (int i = 0; i < D * B; ++i) r->emitted[i] *= inv;
    if (r->film && s->sensor.kind) {
        size_t n = (size_t)s->sensor.width * s->sensor.height * B;
        for (size_t i = 0; i < n; ++i) r->film[i] *= inv;
    }
    free_macro(t);
    free(t);
    return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Camera-side estimator of the paper's single-inelastic model (Sec. 4.1-4.3; Eq. 9-12).
 *
 * A path starts at the sensor: a point uniform in its pixel (pixel = path id mod W*H), a film
 * bin lambda drawn from the mixture (1/D) sum_d p_d of the dyes' emission pmfs, and the ray from
 * the sensor through that point. It walks the medium at lambda by delta tracking (scattering
 * isotropic, walls Lambertian); an absorption at lambda ends it (a dye absorption would be a
 * second inelastic event, V_f = 0; Eq. 9). At every real collision x it samples the light
 * (Eq. 12: a line in proportion to its power, p(lambda_x), and a point on it, p(x_n)) and adds
 * the emission there, the excitation-to-emission term of Eq. 10 per unit volume,
 *     J(x, lambda) = sum_d QY_d p_d(lambda) sigma_a,d(x, lambda_x) phi_x(x) / (4 pi),
 * with phi_x the uncollided excitation fluence (L_r of Eq. 5 times G of Eq. 4, transmittance
 * Eq. 6), divided by sigma_t(x, lambda) (a collision estimator: collisions occur with density
 * sigma_t T, so the sum estimates the integral of T J along the walk). The film then holds the
 * radiance of fluorescence averaged over each pixel, per unit of total source power: the same
 * quantity as the light tracer's film in paper mode. Needs sigma_t(x, lambda) > 0 wherever a
 * dye is (dyes dissolved in a scattering solvent, the paper's setting), and sources of non-zero
 * area (a pencil beam has no fluence density a camera path could find).
 * p_d(b) is the pmf realised by the fp32 CDF table (the one the light tracer samples). */
#define CAM_SPAWN 0xFFFFFFFEu

static double emission_pmf(const tables *t, int d, int b)
{
    return (double)t->cdf32[d][b] - (b > 0 ? (double)t->cdf32[d][b - 1] : 0.0);
}

/* Uncollided fluence at x at the chosen line's bin, per unit total source power (u[0] picks the
 * line, u[1], u[2] the point on a Lambertian one). */
static double excitation_fluence(const or_scene *s, const tables *t, const double x[3],
                                 const double u[3], int *bin_x)
{
    int k = sample_emitter(t, s->n_emitters, u[0]);
    const or_emitter *e = &s->emitters[k];
    *bin_x = t->em_bin[k];
    if (e->kind == 1) {
        int ax; double sg;
        normal_axis(e->dir, &ax, &sg);
        double xn[3], v[3];
        for (int i = 0; i < 3; ++i) {
            xn[i] = e->origin[i] + u[1] * e->eu[i] + u[2] * e->ev[i];
            v[i] = x[i] - xn[i];
        }
        double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (!(r2 > 0.0)) return 0.0;
        double r = sqrt(r2);
        double cn = sg * v[ax] / r;
        if (!(cn > 0.0)) return 0.0;
        double w[3] = { v[0] / r, v[1] / r, v[2] / r };
        return cn * exp(-optical_depth(s, t, xn, w, r, *bin_x)) / (OR_PI * r2);
    }
    /* collimated parallelogram: the point p of the source with x = p + l dir, l >= 0 */
    double dn = sqrt(e->dir[0] * e->dir[0] + e->dir[1] * e->dir[1] + e->dir[2] * e->dir[2]);
    double dir[3] = { e->dir[0] / dn, e->dir[1] / dn, e->dir[2] / dn };
    double n[3] = { e->eu[1] * e->ev[2] - e->eu[2] * e->ev[1], e->eu[2] * e->ev[0] - e->eu[0] * e->ev[2],
                    e->eu[0] * e->ev[1] - e->eu[1] * e->ev[0] };
    double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    double dnd = dir[0] * n[0] + dir[1] * n[1] + dir[2] * n[2];
    if (!(nn > 0.0) || dnd == 0.0) return 0.0;
    double xo[3] = { x[0] - e->origin[0], x[1] - e->origin[1], x[2] - e->origin[2] };
    double l = (xo[0] * n[0] + xo[1] * n[1] + xo[2] * n[2]) / dnd;
    if (!(l >= 0.0)) return 0.0;
    double q[3] = { xo[0] - l * dir[0], xo[1] - l * dir[1], xo[2] - l * dir[2] };
    /* q = a eu + b ev */
    double c1[3] = { q[1] * e->ev[2] - q[2] * e->ev[1], q[2] * e->ev[0] - q[0] * e->ev[2], q[0] * e->ev[1] - q[1] * e->ev[0] };
    double c2[3] = { e->eu[1] * q[2] - e->eu[2] * q[1], e->eu[2] * q[0] - e->eu[0] * q[2], e->eu[0] * q[1] - e->eu[1] * q[0] };
    double a = (c1[0] * n[0] + c1[1] * n[1] + c1[2] * n[2]) / nn;
    double b = (c2[0] * n[0] + c2[1] * n[1] + c2[2] * n[2]) / nn;
    if (!(a >= 0.0 && a < 1.0 && b >= 0.0 && b < 1.0)) return 0.0;
    double pnt[3] = { e->origin[0] + q[0], e->origin[1] + q[1], e->origin[2] + q[2] };
    double a_perp = fabs(dnd);   /* |eu x ev| |cos(normal, dir)|: the beam's cross-section */
    return exp(-optical_depth(s, t, pnt, dir, l, *bin_x)) / a_perp;
}

static void trace_camera(const or_scene *s, const tables *t, const or_params *p, uint64_t pid,
                         double *film, double film_scale, uint64_t *cnt)
{
    const or_sensor *c = &s->sensor;
    cnt[OC_PATHS]++;
    const uint64_t npix = (uint64_t)c->width * (uint64_t)c->height;
    const int pix = (int)(pid % npix);
    const int px = pix % c->width, py = pix / c->width;
    block4 S0 = rng_block(p->seed, p->medium_id, pid, CAM_SPAWN, 0);
    const double fx = (px + S0.u[0]) / c->width, fy = (py + S0.u[1]) / c->height;
    int dsel = (int)(S0.u[2] * s->n_dyes);
    if (dsel > s->n_dyes - 1) dsel = s->n_dyes - 1;
    const int bin = sample_emission_bin(t, dsel, S0.u[3]);
    double pb = 0.0;
    for (int d = 0; d < s->n_dyes; ++d) pb += emission_pmf(t, d, bin);
    pb /= s->n_dyes;
    if (!(pb > 0.0)) return;
    double o[3], w[3];
    if (c->kind == 1) {
        double vn = sqrt(c->view[0] * c->view[0] + c->view[1] * c->view[1] + c->view[2] * c->view[2]);
        for (int k = 0; k < 3; ++k) {
            o[k] = c->origin[k] + fx * c->U[k] + fy * c->V[k];
            w[k] = -c->view[k] / vn;
        }
    } else {
        double X = (2.0 * fx - 1.0) * t->tan_half * t->aspect, Y = (2.0 * fy - 1.0) * t->tan_half;
        double d[3], dl = 0.0;
        for (int k = 0; k < 3; ++k) { d[k] = c->view[k] + X * c->U[k] + Y * c->V[k]; dl += d[k] * d[k]; }
        dl = sqrt(dl);
        for (int k = 0; k < 3; ++k) { o[k] = c->origin[k]; w[k] = d[k] / dl; }
    }
    /* enter the box; the entry face must be open (walls are opaque from outside) */
    double t_in = -INFINITY, t_out = INFINITY;
    int f_in = -1;
    for (int k = 0; k < 3; ++k) {
        if (w[k] == 0.0) {
            if (o[k] < s->lo[k] || o[k] > s->hi[k]) return;
            continue;
        }
        double ta = (s->lo[k] - o[k]) / w[k], tb = (s->hi[k] - o[k]) / w[k];
        int fa = 2 * k, fb = 2 * k + 1;
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; int fi = fa; fa = fb; fb = fi; }
        if (ta > t_in) { t_in = ta; f_in = fa; }
        if (tb < t_out) t_out = tb;
    }
    if (!(t_out > t_in) || !(t_out > 0.0)) return;
    double x[3];
    if (t_in > 0.0) {
        if (s->wall_mask & (1 << f_in)) return;
        for (int k = 0; k < 3; ++k) x[k] = o[k] + t_in * w[k];
    } else {
        for (int k = 0; k < 3; ++k) x[k] = o[k];
    }
    double beta = 1.0;
    int64_t n_events = 0;
    for (int64_t step = 0;; ++step) {
        if (step >= p->max_steps) { cnt[OC_STEP_BUDGET]++; break; }
        cnt[OC_STEPS]++;
        block4 B0 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 0);
        int face;
        double te = exit_distance(s, x, w, &face);
        double sb = t->majorant[bin];
        double tf = sb > 0.0 ? -log(1.0 - B0.u[0]) / sb : INFINITY;
        if (tf >= te) {
            for (int k = 0; k < 3; ++k) x[k] += te * w[k];
            if (face >= 0 && (s->wall_mask & (1 << face))) {
                if (n_events == p->max_events) { cnt[OC_CAP_HITS]++; break; }
                n_events++;
                cnt[OC_EVENTS]++;
                cnt[OC_WALL_BOUNCES]++;
                block4 B2 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 2);
                if (p->analog) {
                    if (!(B2.u[0] < s->wall_albedo)) { cnt[OC_ABSORBED_DEAD]++; break; }
                } else {
                    beta *= s->wall_albedo;
                    if (beta == 0.0) { cnt[OC_ABSORBED_DEAD]++; break; }
                }
                int ax = face / 2;
                double sg = (face & 1) ? -1.0 : 1.0;
                x[ax] = (face & 1) ? s->hi[ax] : s->lo[ax];
                block4 B1 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 1);
                cosine_dir(B0.u[3], B1.u[0], ax, sg, w);
                if (n_events >= p->n_rr) {
                    double q = beta < 1.0 ? beta : 1.0;
                    if (!(B2.u[1] < q)) { cnt[OC_RR_KILLS]++; break; }
                    beta /= q;
                }
                continue;
            }
            cnt[OC_ESCAPES]++;
            break;
        }
        for (int k = 0; k < 3; ++k) x[k] += tf * w[k];
        coeffs cf = coeffs_at_p(s, t, x, bin, 0);
        if (cf.total > sb) cnt[OC_MAJORANT_VIOLATIONS]++;
        if (!(B0.u[1] * sb < cf.total)) { cnt[OC_NULLS]++; continue; }
        if (n_events == p->max_events) { cnt[OC_CAP_HITS]++; break; }
        n_events++;
        cnt[OC_EVENTS]++;
        block4 B1 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 1);
        /* emission at this collision, through one light sample */
        int bx;
        double phi = excitation_fluence(s, t, x, &B1.u[1], &bx);
        if (phi > 0.0) {
            coeffs cx = coeffs_at_p(s, t, x, bx, 0);
            double src = 0.0;
            for (int d = 0; d < s->n_dyes; ++d) src += t->qy[d] * emission_pmf(t, d, bin) * cx.dye[d];
            double val = beta * src * phi / (4.0 * OR_PI * cf.total * pb) * film_scale;
            if (val != 0.0) {
                size_t idx = ((size_t)py * c->width + px) * t->B + bin;
#pragma omp atomic
                film[idx] += val;
                cnt[OC_CONNECTIONS]++;
            }
        }
        /* the event at lambda: scattering continues, any absorption ends the walk */
        if (!(B0.u[2] * cf.total < cf.scat)) {
            if (B0.u[2] * cf.total < cf.total - cf.bg) cnt[OC_VF_REJECTED]++;
            else cnt[OC_ABSORBED_DEAD]++;
            break;
        }
        cnt[OC_SCATTERS]++;
        iso_dir(B0.u[3], B1.u[0], w);
        if (n_events >= p->n_rr) {
            double q = beta < 1.0 ? beta : 1.0;
            block4 B2 = rng_block(p->seed, p->medium_id, pid, (uint32_t)step, 2);
            if (!(B2.u[1] < q)) { cnt[OC_RR_KILLS]++; break; }
            beta /= q;
        }
    }
}

/* Camera-side render: film [H][W][n_bins] of fluorescence radiance per unit source power.
 * n_paths and path_offset must be multiples of W*H (each pixel gets the same number of
 * paths). Returns -2 without a sensor or dyes, -3 for a source of zero area. */
int or_render_camera(const or_scene *s, const or_params *p, double *film, uint64_t *counters)
{
    if (!s || !p || !film || !counters) return -1;
    if (s->n_bins <= 0 || s->n_bins > OR_MAX_BINS) return -1;
    if (s->n_dyes <= 0 || s->n_dyes > OR_MAX_DYES || s->sensor.kind == 0) return -2;
    if (s->n_emitters <= 0 || s->n_emitters > OR_MAX_EMITTERS) return -1;
    if (s->ior > 1.0 || s->wall_gloss > 0.0) return -1;   /* index-matched, Lambertian only */
    for (int k = 0; k < s->n_emitters; ++k) {
        const or_emitter *e = &s->emitters[k];
        double n[3] = { e->eu[1] * e->ev[2] - e->eu[2] * e->ev[1], e->eu[2] * e->ev[0] - e->eu[0] * e->ev[2],
                        e->eu[0] * e->ev[1] - e->eu[1] * e->ev[0] };
        if (!(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] > 0.0)) return -3;
    }
    const uint64_t npix = (uint64_t)s->sensor.width * (uint64_t)s->sensor.height;
    if (p->n_paths % npix != 0 || p->path_offset % npix != 0) return -1;
    tables *t = (tables *)malloc(sizeof(tables));
    build_tables(s, t);
    apply_params(t, p);
    memset(film, 0, sizeof(double) * (size_t)npix * s->n_bins);
    memset(counters, 0, sizeof(uint64_t) * OR_NCOUNTERS);
#ifdef _OPENMP
    omp_set_num_threads(p->n_threads > 0 ? p->n_threads : omp_get_num_procs());
#endif
    const int64_t N = (int64_t)p->n_paths;
    const double film_scale = N > 0 ? (double)npix / (double)N : 0.0;
#pragma omp parallel
    {
        uint64_t cnt[OR_NCOUNTERS];
        memset(cnt, 0, sizeof(cnt));
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < N; ++i)
            trace_camera(s, t, p, p->path_offset + (uint64_t)i, film, film_scale, cnt);
#pragma omp critical
        for (int k = 0; k < OR_NCOUNTERS; ++k) counters[k] += cnt[k];
    }
    free(t);
    return 0;
}

/* Raw Philox blocks, for statistical tests of the generator. */
void or_philox(uint32_t seed, uint32_t medium, const uint32_t *ctr /*[n][4]*/, int64_t n,
               uint32_t *out /*[n][4]*/)
{
    uint32_t key[2] = { seed, medium };
    for (int64_t i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Emission-bin sampling for the scene's dye d at n given uniforms (fp32-decided CDF). */
int or_sample_emission(const or_scene *s, int d, const double *u, int64_t n, int32_t *out)
{
    if (d < 0 || d >= s->n_dyes) return -1;
    tables *t = (tables *)malloc(sizeof(tables));
    build_tables(s, t);
    for (int64_t i = 0; i < n; ++i) out[i] = sample_emission_bin(t, d, u[i]);
    free(t);
    return 0;
}

void or_iso_dir(const double *u1, const double *u2, int64_t n, double *out /*[n][3]*/)
{
    for (int64_t i = 0; i < n; ++i) iso_dir(u1[i], u2[i], out + 3 * i);
}

void or_cosine_dir(const double *u1, const double *u2, int64_t n, int axis, double sign,
                   double *out)
{
    for (int64_t i = 0; i < n; ++i) cosine_dir(u1[i], u2[i], axis, sign, out + 3 * i);
}

/* Optical depth along [x0, x0 + L w] at bin (exact, Eq. 6), and the majorant table. */
double or_optical_depth(const or_scene *s, const double *x0, const double *w, double L, int bin)
{
    tables *t = (tables *)malloc(sizeof(tables));
    build_tables(s, t);
    double tau = optical_depth(s, t, x0, w, L, bin);
    free(t);
    return tau;
}

/* sigma_t(x, bin) at n points ([n][3]) by the nearest-voxel lookup the tracking uses (Sec. 4.1),
 * and the row-major index of the voxel read (-1 for a medium without grids). */
void or_sigma_t_at(const or_scene *s, const double *pts, int64_t n, int bin, double *out_sigma,
                   int64_t *out_voxel)
{
    tables *t = (tables *)malloc(sizeof(tables));
    build_tables(s, t);
    for (int64_t i = 0; i < n; ++i) {
        const double x[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
        out_sigma[i] = coeffs_at_p(s, t, x, bin, 0).total;
        out_voxel[i] = t->homogeneous ? -1 : (int64_t)voxel_index(s, x);
    }
    free(t);
}

void or_majorant(const or_scene *s, double *out)
{
    tables *t = (tables *)malloc(sizeof(tables));
    build_tables(s, t);
    for (int i = 0; i < s->n_bins; ++i) out[i] = t->majorant[i];
    free(t);
}

int or_counters_count(void) { return OR_NCOUNTERS; }

/* Reference gradient of sum_j adj[j] * I_j with respect to every dye concentration voxel and
 * sigma_s, for the frozen-sampling estimator I_j of or_render over the same paths (same seed,
 * path ids and majorant). Per path, each tracking decision contributes d log p(decision) times
 * the adjoint-weighted sensor contributions that follow it:
 *   null collision:      d log(1 - sigma_t/sigma_bar) = -d sigma_t / (sigma_bar - sigma_t)
 *   real, particle e:    d log(sigma_e / sigma_bar)   =  d sigma_e / sigma_e
 * and each sensor contribution its own transmittance derivative d log T = -d tau (Eq. 6, the
 * exact piecewise-constant optical depth). d sigma_t / d c_d[v] = eps_d a_d(lambda) inside voxel
 * v; d sigma_t / d sigma_s = s(x). grad_c [n_dyes][nz][ny][nx] (grid scenes only; may be NULL),
 * grad_sigma_s [1]. */
int or_adjoint(const or_scene *s, const or_params *p, const double *adj, double *grad_c,
               double *grad_sigma_s)
{
    if (!s || !p || !adj || !grad_sigma_s) return -1;
    if (s->sensor.kind == 0) return -1;
    if (s->n_bins <= 0 || s->n_bins > OR_MAX_BINS || s->n_dyes > OR_MAX_DYES) return -1;
    if (!interfaces_supported(s, p)) return -1;
    if (s->n_emitters <= 0 || s->n_emitters > OR_MAX_EMITTERS) return -1;
    tables *t = (tables *)malloc(sizeof(tables));
    build_tables(s, t);
    apply_params(t, p);
    apply_params_macro(s, t, p);
    t->pert_dye = -1;
    t->pert_sigma_s = 0.0;
    t->frozen = 0;
    const int D = s->n_dyes;
    const int have_grid = s->conc != NULL && grad_c != NULL;
    const size_t nv = have_grid ? (size_t)nvox(s) : 0;
    if (have_grid) memset(grad_c, 0, sizeof(double) * (size_t)D * nv);
    *grad_sigma_s = 0.0;
#ifdef _OPENMP
    omp_set_num_threads(p->n_threads > 0 ? p->n_threads : omp_get_num_procs());
#endif
    const int64_t N = (int64_t)p->n_paths;
    const double inv_n = N > 0 ? 1.0 / (double)N : 0.0;
#pragma omp parallel
    {
        local_tally *lt = (local_tally *)calloc(1, sizeof(local_tally));
        adj_path A;
        memset(&A, 0, sizeof(A));
        A.adj = adj;
        A.inv_n = inv_n;
#pragma omp for schedule(dynamic, 32)
        for (int64_t i = 0; i < N; ++i) {
            A.n_dec = 0;
            A.n_con = 0;
            trace_path(s, t, p, p->path_offset + (uint64_t)i, lt, NULL, &A);
            double total = 0.0;
            for (int64_t k = 0; k < A.n_con; ++k) total += A.con[k].a;
            if (total == 0.0 && A.n_con == 0) continue;
            double pre = 0.0;
            int64_t ci = 0;
            for (int64_t k = 0; k < A.n_dec; ++k) {
                const dec_rec *r = &A.dec[k];
                while (ci < A.n_con && A.con[ci].step < r->step) pre += A.con[ci++].a;
                const double suffix = total - pre;
                if (suffix == 0.0) continue;
                if (r->kind == 0) {
                    const double den = r->sigma_bar - r->sigma_t;
                    if (have_grid)
                        for (int d = 0; d < D; ++d) {
                            const double g = -suffix * t->sig_a[d][r->bin] / den;
                            if (g != 0.0) {
#pragma omp atomic
                                grad_c[(size_t)d * nv + r->voxel] += g;
                            }
                        }
                    if (r->solvent != 0.0) {
                        const double g = -suffix * r->solvent / den;
#pragma omp atomic
                        *grad_sigma_s += g;
                    }
                } else if (r->kind == 1) {
                    const double g = suffix / s->sigma_s;
#pragma omp atomic
                    *grad_sigma_s += g;
                } else if (r->kind == 2 && have_grid) {
                    const double g = suffix / r->conc;
#pragma omp atomic
                    grad_c[(size_t)r->dye * nv + r->voxel] += g;
                }
            }
            for (int64_t k = 0; k < A.n_con; ++k) {
                const con_rec *c = &A.con[k];
                tau_grad g = { have_grid ? grad_c : NULL, grad_sigma_s, -c->a };
                optical_depth_g(s, t, c->x, c->dir, c->L, c->bin, 0, &g);
            }
        }
        free(A.dec);
        free(A.con);
        free(lt);
    }
    free_macro(t);
    free(t);
    return 0;
}
