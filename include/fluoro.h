/*
 * fluoro.h -- C ABI of the GB300 (sm_103a) fluorescent participating-media light tracer.
 *
 * Method: Abdellah et al., "A Physically Plausible Model for Rendering Highly Scattering
 * Fluorescent Participating Media" (arXiv 1706.03024). Photons of one wavelength each are traced
 * through a scattering medium holding fluorescent dyes (Sec. 4.1); at a dye absorption the photon
 * is re-emitted with probability QY at a wavelength drawn from the dye's normalised emission
 * spectrum (Eq. 10), isotropically (Sec. 2.1); transmittance follows Beer-Lambert (Eq. 6); the
 * sensor is reached by three-point connections (Eq. 3-5); the estimator averages over paths and
 * source lines (Eq. 12).
 *
 * Conventions for every entry point:
 *   - Return value: FLR_OK (0) or a negative FLR_ERR_* code. Nothing throws across the ABI.
 *     flr_last_error(ctx) gives a one-line description of the last failure on that context.
 *   - "host" pointers are CPU memory read during the call and not retained. "device" pointers
 *     are CUDA global memory on the context's device, owned by the caller, and must stay valid
 *     until the work queued on the given stream has finished.
 *   - Streams are passed as void* holding a cudaStream_t (NULL = the legacy default stream).
 *     Render calls are asynchronous on that stream; flr_read_tallies and flr_status synchronise.
 *   - Spectra are sampled on a uniform grid of n_bins bin centres lambda_i = lambda0 + i dlambda.
 *   - Faces of the box are numbered (-x, +x, -y, +y, -z, +z) = 0..5.
 *   - Voxel grids are fp32 [nz][ny][nx] (x fastest) spanning the medium's box; lookups take the
 *     nearest voxel (piecewise-constant field).
 *   - One context is used by one host thread at a time.
 */
#ifndef FLUORO_H
#define FLUORO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLR_OK 0
#define FLR_ERR_ARG (-1)     /* invalid argument; nothing was changed or launched           */
#define FLR_ERR_CUDA (-2)    /* a CUDA call failed; see flr_last_error                       */
#define FLR_ERR_OOM (-3)     /* device allocation failed                                     */
#define FLR_ERR_BUDGET (-4)  /* a device loop budget ran out (paths were cut short)          */
#define FLR_ERR_STATE (-5)   /* call out of order (e.g. render before a medium is set)       */
#define FLR_ERR_CHECK (-6)   /* checked build: a device index was out of range (the access
                                was skipped); see flr_last_error                             */

#define FLR_MAX_BINS 128
#define FLR_MAX_DYES 1024           /* dye table size                                      */
#define FLR_MAX_DYES_PER_MEDIUM 4
#define FLR_MAX_SOURCES 65536
#define FLR_MAX_LINES 8
#define FLR_MAX_EMITTERS 32         /* spectral lines over all sources of one medium       */
#define FLR_NCOUNTERS 21

#define FLR_SOURCE_COLLIMATED 0
#define FLR_SOURCE_LAMBERTIAN 1

#define FLR_SENSOR_NONE 0
#define FLR_SENSOR_ORTHO 1
#define FLR_SENSOR_PINHOLE 2

#define FLR_FORM_PLAIN 0      /* one thread per path, nested loops                          */
#define FLR_FORM_WAVEFRONT 1  /* persistent, path regeneration, sensor connections regrouped */
#define FLR_FORM_WAVEFRONT_WARP 2  /* as WAVEFRONT, regrouping per warp instead of per block */
#define FLR_FORM_WAVEFRONT_POOL 3  /* per-warp pools of paths in shared memory, regrouped by event
                                      type every round: free flights and collision events each run
                                      on full warps (flr_render only; one majorant per bin, with or
                                      without skip_cell; blocks of 128 threads) */

/* Counter indices of flr_read_tallies' counters array. */
enum {
    FLR_C_PATHS = 0, FLR_C_EVENTS, FLR_C_NULLS, FLR_C_ESCAPES, FLR_C_ABSORBED_DEAD,
    FLR_C_RR_KILLS, FLR_C_CAP_HITS, FLR_C_STEP_BUDGET, FLR_C_CONNECTIONS, FLR_C_VF_REJECTED,
    FLR_C_WALL_BOUNCES, FLR_C_EMISSIONS, FLR_C_SCATTERS, FLR_C_DYE_ABSORPTIONS, FLR_C_STEPS,
    FLR_C_MAJORANT_VIOLATIONS, /* tracking points where sigma_t exceeded the majorant          */
    FLR_C_CONNECT_STEPS,       /* ratio-tracking steps of sensor connections                    */
    FLR_C_CONNECT_BUDGET,      /* connections cut by the ratio-tracking step budget             */
    FLR_C_NONFINITE,           /* paths ended because a weight or position became non-finite   */
    FLR_C_CELL_WALKS,          /* local-majorant cells visited by free flights and marches      */
    FLR_C_IFACE_REFLECTIONS    /* Fresnel reflections at dielectric faces (entry reflections
                                  included); those inside the medium also count as events       */
};

typedef struct flr_ctx flr_ctx;

/* A light source: a parallelogram origin + a*eu + b*ev (a, b uniform in [0,1); eu = ev = 0 gives
 * a point or pencil beam) emitting n_lines monochromatic lines (Sec. 5: each scene is lit at the
 * dyes' excitation peaks). COLLIMATED sources emit along dir; LAMBERTIAN sources emit a cosine
 * distribution about the axis-aligned normal dir. A line is chosen with probability proportional
 * to its power over all lines of the medium's sources (p(lambda_x), Eq. 12); each line snaps to
 * the nearest bin centre (ties to the lower bin). */
typedef struct flr_source {
    int kind;
    float origin[3], eu[3], ev[3], dir[3];
    int n_lines;
    float lambda_nm[FLR_MAX_LINES];
    float power[FLR_MAX_LINES];
} flr_source;

/* A participating medium in an axis-aligned box (Sec. 4.1: solvent particles plus dyes).
 *   sigma_t(x, lambda) = s(x) (sigma_s + sigma_a0) + sum_d eps_d a_d(lambda) c_d(x)
 * with s(x) the solvent mask (1 where no mask is given), eps_d a_d the dye's absorption
 * (set by flr_set_dyes) and c_d the concentration (grid or uniform). Faces whose bit is set in
 * wall_mask are walls of albedo wall_albedo; the others are open.
 * Interfaces and glossy walls (the glass vials and the glossy Cornell box of Sec. 5, which the
 * paper does not specify; these are the physically standard choices):
 *   ior > 1 makes every open face a smooth dielectric interface between the solution (index ior)
 *   and the outside (index 1): a photon reaching it from inside is reflected with the Fresnel
 *   reflectance of unpolarised light (always beyond the critical angle) and otherwise escapes; a
 *   source whose parallelogram lies in an open face's plane, pointing inward, enters through it
 *   (the reflected share is tallied as escaping through that face, the rest refracts by Snell's
 *   law). The sensor must then be orthographic with its view along a face normal (connections
 *   leave the face at normal incidence with (1 - F) / ior^2 of the radiance); pinhole sensors,
 *   hero paths, the paper's model, the camera-side estimator and the batched form are
 *   index-matched only (FLR_ERR_ARG). ior 0 or 1: index-matched.
 *   Wall BRDF: wall_albedo [(1 - g)/pi + g (e + 2)/(2 pi) cos^e alpha] with g = wall_gloss in
 *   [0, 1], e = wall_exponent >= 0 and alpha the angle between the outgoing direction and the
 *   mirror direction of the incoming one: a diffuse lobe plus a normalised Phong lobe. Sensor
 *   connections evaluate the whole BRDF; the path continues in the Phong lobe with probability g
 *   (weight (e + 2)/(e + 1) cos theta_o; a direction below the wall ends it), else in the diffuse
 *   lobe. g = 0: Lambertian. The batched form, hero paths, the paper's model and the camera-side
 *   estimator take Lambertian walls only. */
typedef struct flr_medium {
    float lo[3], hi[3];          /* box, cm                                                    */
    int dims[3];                 /* nx, ny, nz of the grids, each 1..4096, nx*ny*nz below 2^31
                                    also once each is rounded up to a multiple of 4 (the library
                                    stores the grids in 4^3-voxel bricks; FLR_ERR_ARG otherwise);
                                    ignored when no grid is given */
    int n_dyes;                  /* 0..FLR_MAX_DYES_PER_MEDIUM                                 */
    int dye_ids[FLR_MAX_DYES_PER_MEDIUM];        /* rows of the dye table                     */
    const float *conc[FLR_MAX_DYES_PER_MEDIUM];  /* device grids, or NULL => conc_uniform[d]  */
    float conc_uniform[FLR_MAX_DYES_PER_MEDIUM];
    const uint8_t *solvent;      /* device [nz][ny][nx] 0/1 mask, or NULL (solvent everywhere) */
    float sigma_s, sigma_a0;     /* solvent scattering and flat background absorption, cm^-1  */
    int wall_mask;
    float wall_albedo;
    int source_first, source_count;  /* rows of the source table; count 0 = all sources      */
    float ior;                   /* refractive index of the solution (0 or 1: index-matched)   */
    float wall_gloss, wall_exponent;  /* glossy share and Phong exponent of the walls' BRDF   */
} flr_medium;

/* The sensor. ORTHO: a film rectangle origin + s U + t V (s, t in [0,1)) recording radiance
 * that travels along +view (unit, normal to the film); pixel (px, py) = (floor(s W), floor(t H)).
 * PINHOLE: eye at origin, orthonormal right U, up V, forward view, vertical field of view
 * fov_y_deg, aspect W/H; image-plane coordinates at unit distance map to pixels with row 0 at
 * the bottom. Both films record radiance averaged over the pixel's area on the film (pinhole:
 * on the unit-distance image plane). The eye must lie outside the medium's box. */
typedef struct flr_sensor {
    int kind;
    int width, height;
    float origin[3], U[3], V[3], view[3];
    float fov_y_deg;
} flr_sensor;

/* Per-render parameters. */
typedef struct flr_params {
    uint64_t n_paths;            /* photon paths to trace                                      */
    uint64_t path_offset;        /* first path id (paths are path_offset .. +n_paths-1)         */
    uint32_t seed;               /* Philox key word 0                                          */
    uint32_t medium_id;          /* Philox key word 1                                          */
    int n_rr;                    /* Russian roulette once a path has n_rr real events           */
    int max_inelastic;           /* <0: unlimited re-emissions; k: the (k+1)-th dye absorption
                                    ends the path (k = 1 is the paper's single inelastic event,
                                    Sec. 4.1 and V_f of Eq. 9)                                 */
    int analog;                  /* 0: weight *= QY (and wall albedo); 1: survival coins        */
    int form;                    /* FLR_FORM_PLAIN, FLR_FORM_WAVEFRONT, FLR_FORM_WAVEFRONT_WARP or
                                    FLR_FORM_WAVEFRONT_POOL (flr_render; the pool form without
                                    macro_cell and hero); flr_render_camera and flr_adjoint take
                                    the first three */
    int64_t max_events;          /* a real collision once n_events == max_events ends the path */
    int64_t max_steps;           /* tracking-step budget per path                               */
    float *film;                 /* device [H][W][n_bins] fp32, or NULL                         */
    uint32_t *path_events;       /* device [n_paths] real events per path, or NULL              */
    int accumulate;              /* 0: clear tallies and film first; 1: add to them             */
    int block_size;              /* threads per block; 0 = library default (the warp-regrouped
                                    form and the adjoint's passes use at most 128)              */
    int blocks_per_sm;           /* resident blocks per SM; 0 = occupancy maximum               */
    int regroup_interval;        /* wavefront: tracking steps between connection flushes; 0 auto */
    int macro_cell;              /* > 0: free flights and transmittance marches use local
                                    majorants over cells of macro_cell^3 voxels (each the maximum
                                    of sigma_t over the cell and a one-voxel halo), walked by DDA;
                                    0: one majorant per bin. Same estimator, fewer null steps in
                                    sparse media. Single-scene renders and the adjoint only. */
    int skip_cell;               /* > 0 (with macro_cell = 0): after a null collision where
                                    sigma_t = 0, leave the largest cube of skip_cell^3-voxel cells
                                    around it that holds no matter and restart the free flight at
                                    its boundary (exact: every tentative collision inside would be
                                    a null); transmittance marches leap the same way. Gives no
                                    gradient for voxels in such cubes. 0: off. */
    float majorant_margin;       /* >= 0: every majorant (global or local) is multiplied by
                                    1 + majorant_margin. A margin keeps null-collision scores of
                                    the adjoint, -d sigma_t / (sigma_bar - sigma_t), bounded; the
                                    forward pays about that fraction of extra null steps. Replays
                                    (flr_adjoint) must use the forward's value. */
    int paper_mode;              /* 1: the paper's single-inelastic model (Sec. 4.1): excitation
                                    light reaches a dye only uncollided (a scattering event or
                                    wall bounce before the first emission ends the path), a second
                                    dye absorption ends the path (V_f of Eq. 9), and only vertices
                                    after the emission connect to the sensor, so the film holds
                                    fluorescence alone. Rejected paths count as vf_rejected.
                                    flr_render and the batch only; 0: the full RTE. */
    int hero;                    /* 1..4: hero-wavelength paths (spectral multiple importance
                                    sampling, Wilkie et al. 2014, cited in Sec. 3): a path carries
                                    up to `hero` wavelengths, the hero's source lines (the lines
                                    of one source, in blocks of `hero`) and after a re-emission
                                    the block of `hero` consecutive bins holding the drawn bin;
                                    the hero takes every decision, free flights use the largest
                                    member majorant, and every tally and film contribution is
                                    split among the members by the balance heuristic. Same
                                    expectation as one wavelength per path; with 1 the same
                                    paths and tallies. flr_render with FLR_FORM_PLAIN or
                                    FLR_FORM_WAVEFRONT_WARP (blocks of 128, regroup 1), no
                                    macro_cell, no paper_mode (else FLR_ERR_ARG). 0: one
                                    wavelength per path. */
} flr_params;

/* Create a context on CUDA device `cuda_device`. Allocates the small tally buffers. */
int flr_create(flr_ctx **out, int cuda_device);
/* Release a context and everything it allocated (not caller-owned buffers). NULL is allowed. */
void flr_destroy(flr_ctx *ctx);

/* Spectral grid (Sec. 4.2: per-wavelength transport; the paper samples every 1 nm, this library
 * takes any uniform grid of 1..FLR_MAX_BINS bins). Resets the dye table. */
int flr_set_spectrum(flr_ctx *ctx, float lambda0_nm, float dlambda_nm, int n_bins);

/* Dye table (Sec. 4.1, Eq. 10). host abs_shape [n][n_bins]: absorption (excitation) spectrum
 * a_d, peak-normalised; host emit_spec [n][n_bins]: emission spectrum f_m, any positive scale;
 * host eps [n]: napierian absorption coefficient in cm^-1 per unit concentration at the
 * absorption peak; host qy [n] in [0,1]. The emission pmf is f_m(lambda_i) / sum_j f_m(lambda_j);
 * the library builds each dye's CDF in fp64 and rounds it to fp32. FLR_ERR_ARG on negative or
 * non-finite values, an all-zero emission spectrum, QY outside [0,1] or n outside 1..FLR_MAX_DYES. */
int flr_set_dyes(flr_ctx *ctx, int n, const float *abs_shape, const float *emit_spec,
                 const float *eps, const float *qy);

/* Light sources (host array of n, copied). */
int flr_set_sources(flr_ctx *ctx, int n, const flr_source *sources);

/* The medium of single-scene renders. Copies the dye grids (device, caller-owned, read here only)
 * into a library-owned interleaved layout and reads their maxima back to build the per-bin
 * majorant, so this call synchronises the device. Grids must be finite and non-negative. */
int flr_set_medium(flr_ctx *ctx, const flr_medium *medium);
/* The same upload ordered on `stream` instead of the whole device: the grids are read on
 * `stream` (the caller orders their writes before it), packed, and their maxima read back with
 * one copy, which synchronises `stream` only; negative or non-finite values give FLR_ERR_ARG as
 * above. Renders of this context still in flight on another stream must be ordered before
 * `stream` by the caller (the upload overwrites the context's packed grid). Lets a caller
 * overlap one context's upload and render with another context's work (a stream of scenes). */
int flr_set_medium_async(flr_ctx *ctx, const flr_medium *medium, void *stream);

/* The sensor (host struct, copied). kind NONE disables the film. */
int flr_set_sensor(flr_ctx *ctx, const flr_sensor *sensor);

/* Trace p->n_paths paths of the single scene on `stream`: face, absorption and emission tallies
 * accumulate inside the context (read them with flr_read_tallies); film contributions, already
 * divided by p->n_paths, are summed exactly in 64-bit fixed point (units of 2^-32; at most 2^32
 * per film value and launch) in a film-sized context buffer (8 bytes per film value, allocated on
 * the first launch with a film), then written to p->film (accumulate = 0) or added to it when the
 * launch ends: the film does not depend on the order of the contributions. Every form traces the
 * same paths (Sec. 3, Eq. 12; fixed-point tallies identical bit for bit). For a
 * medium with grids, no solvent mask and sigma_s + sigma_a0 at least 0.9 of every bin's majorant,
 * the plain and warp forms run kernels that take a decision without reading the grid where a bound
 * settles it (sigma_t >= sigma_s + sigma_a0 everywhere: a sure scatter; a transmittance march
 * whose roulette coin fails against the bound of its estimate); the results are the same. */
int flr_render(flr_ctx *ctx, const flr_params *p, void *stream);

/* The paper's own estimator of its single-inelastic model (Sec. 4.1-4.3, Eq. 12): paths start
 * at the sensor, at an emission bin drawn from the mixture of the dyes' emission pmfs, and walk
 * the medium at that wavelength by delta tracking (isotropic scattering, Lambertian walls; an
 * absorption ends the walk, since a dye absorption would be a second inelastic event). At every
 * real collision one light sample (a line in proportion to its power, a point on it) gives the
 * uncollided excitation fluence (Eq. 4-6; transmittance by ratio tracking), and the collision adds
 * sum_d QY_d p_d(lambda) sigma_a,d(x, lambda_x) fluence / (4 pi sigma_t(x, lambda)) (Eq. 10) to
 * its pixel and bin. p->film (device [H][W][n_bins], required) receives fluorescence radiance
 * averaged over each pixel per unit total source power: the quantity flr_render writes with
 * p->paper_mode = 1. Path id i renders pixel i mod (W*H): p->n_paths and p->path_offset must be
 * multiples of W*H. Uses n_paths, path_offset, seed, medium_id, n_rr, analog, max_events,
 * max_steps, film, accumulate (0 clears the film and the counters), block_size and form
 * (FLR_FORM_PLAIN: one thread per path; the wavefront forms: warp-regrouped light samples; the
 * film summed in fixed point as flr_render sums it); the rest is ignored. Requires a sensor and dyes, and sources of non-zero area (a pencil beam has no fluence
 * density a camera path could meet: FLR_ERR_ARG). sigma_t must be positive wherever a dye is (the
 * dyes dissolved in a scattering solvent, the paper's setting): the collision estimator cannot
 * see emission where the medium never collides. Counters: paths, events (real collisions and wall
 * bounces), nulls, connections (light samples that reached the collision), vf_rejected (dye
 * absorptions at the emission wavelength), escapes and the budgets. */
int flr_render_camera(flr_ctx *ctx, const flr_params *p, void *stream);

/* Synchronise `stream` and copy out the tallies accumulated since the last clear, divided by the
 * number of paths traced since then. host face [2][6][n_bins] (escaped weight per
 * [fluoresced][face][bin]); host absorbed [n_dyes+1][n_bins] (last row: background absorption);
 * host emitted [n_dyes][n_bins]; host counters [FLR_NCOUNTERS] (raw counts). Any output may be
 * NULL. n_dyes is the current medium's. */
int flr_read_tallies(flr_ctx *ctx, double *face, double *absorbed, double *emitted,
                     uint64_t *counters, void *stream);

/* Adjoint of the single-scene render by path replay (the paper has no derivatives; the estimator
 * differentiated is the one flr_render evaluates). For the same paths as flr_render with the same
 * p (n_paths, path_offset, seed, medium_id and every mode flag), adds to device grad_conc
 * [n_dyes][nz][ny][nx] (the medium's grid layout; may be NULL, and must be NULL for a medium
 * without grids) and device grad_sigma_s [1] (may be NULL) the gradient of
 * L = sum_j adj_film[j] * film[j] with respect to every concentration voxel and sigma_s, with the
 * sampling decisions held at the current values (frozen-sampling estimator): null collisions
 * score -d sigma_t/(sigma_bar - sigma_t), real collisions with particle e score
 * d sigma_e/sigma_e (Sec. 4.1 shares), each score multiplied by the adjoint-weighted film
 * contributions that follow it; every contribution adds its ratio-tracking transmittance
 * derivative (Eq. 6). device adj_film [H][W][n_bins] (the sensor's film layout). The gradients are
 * zeroed first unless p->accumulate. Requires a sensor; asynchronous on `stream`.
 * The score estimator is unbiased only where every parameter-dependent decision has positive
 * probability: render and replay with p->majorant_margin > 0 (a null at the voxel attaining a
 * tight majorant is never sampled), keep concentrations positive (a dye collision at c = 0 is
 * never sampled), and note that local majorants (p->macro_cell > 0) give no gradient in cells that
 * hold no matter. */
int flr_adjoint(flr_ctx *ctx, const flr_params *p, const float *adj_film, float *grad_conc,
                float *grad_sigma_s, void *stream);

/* Diagnostic for derivative checks of flr_adjoint (the paper has no derivatives). For the same
 * paths as flr_adjoint with the same p, writes to device out [p->n_paths] (fp64, path i of the
 * launch at out[i]) S_i = sum_k adj_film[pixel_k][bin_k] value_k(theta) W_k(theta): the path's
 * adjoint-weighted film contributions under the frozen-sampling estimator at a perturbed medium
 * theta = (dye slot pert_dye's concentration in voxel pert_voxel plus pert_delta (pert_dye -1:
 * none), sigma_s plus pert_sigma_s). Every decision is sampled in the current medium as flr_adjoint
 * replays it; the decisions theta changes enter through their likelihood ratios W (null collision
 * (sigma_bar - sigma_t(theta)) / (sigma_bar - sigma_t), real collision with particle e
 * sigma_e(theta) / sigma_e, Sec. 4.1), and each transmittance (Eq. 6) is the ratio-tracking
 * product at theta over the same points, with flr_adjoint's roulette rule decided at the current
 * medium. The sums are deterministic per path, so central differences
 * (S_i(+h) - S_i(-h)) / 2h with common random numbers are smooth and sum to flr_adjoint's
 * gradient up to O(h^2). p->macro_cell, skip_cell, paper_mode and hero must be 0 (FLR_ERR_ARG);
 * a concentration perturbation needs a medium with grids. Asynchronous on `stream`. */
int flr_debug_frozen_sums(flr_ctx *ctx, const flr_params *p, const float *adj_film, int pert_dye,
                          int64_t pert_voxel, float pert_delta, float pert_sigma_s, double *out,
                          void *stream);

/* Batched persistent form (independent media in one launch). flr_batch_prepare validates n_media
 * media (each as flr_set_medium would; source rows via source_first/source_count, at most 8 lines
 * per medium; the sensor is not used), copies their grids into one library-owned interleaved
 * arena, builds per-medium spectral tables and majorants, splits host n_paths [n_media] into a
 * device work queue of path-id chunks ordered by expected path length, and captures the launch
 * (tally reset + one persistent kernel) in a CUDA graph. Medium m draws its random numbers under
 * the key (p->seed, p->medium_id + m), so it traces exactly the paths a single-scene render of that
 * medium with medium_id = p->medium_id + m traces. Synchronises the device. */
int flr_batch_prepare(flr_ctx *ctx, int n_media, const flr_medium *media, const uint64_t *n_paths,
                      const flr_params *p);
/* Launch the prepared batch (graph replay) on `stream`; per-medium tallies are cleared first. */
int flr_batch_launch(flr_ctx *ctx, void *stream);
/* Synchronise `stream` and copy per-medium tallies, each divided by that medium's path count:
 * host face [M][2][6][n_bins]; host absorbed [M][FLR_MAX_DYES_PER_MEDIUM+1][n_bins] (rows
 * 0..D_m-1 dyes, row D_m background); host emitted [M][FLR_MAX_DYES_PER_MEDIUM][n_bins]; host
 * counters [FLR_NCOUNTERS] summed over media. Any output may be NULL. */
int flr_batch_read(flr_ctx *ctx, double *face, double *absorbed, double *emitted,
                   uint64_t *counters, void *stream);
/* flr_batch_prepare followed by flr_batch_launch. */
int flr_render_batch(flr_ctx *ctx, int n_media, const flr_medium *media, const uint64_t *n_paths,
                     const flr_params *p, void *stream);

/* Single-scene render that allocates nothing on the device (the paper has no counterpart; it is a
 * service for callers that cannot call cudaMalloc, such as code whose device memory is owned by
 * another allocator, or hosts with a fixed memory budget that forbid allocation at run time).
 * It takes the whole scene by argument, with no context: the spectrum, the dye table (host arrays
 * as flr_set_dyes takes them; medium->dye_ids index into them), the medium (device grids, as
 * flr_set_medium takes them), the sources (medium->source_first/count index into them), the
 * sensor (may be NULL or kind NONE), the parameters (p->film and p->path_events as flr_render),
 * and host outputs laid out as flr_read_tallies writes them (any may be NULL; tallies divided by
 * p->n_paths). All scratch -- spectral tables, fixed-point tallies, counters, the work counter and
 * the interleaved copy of the grids -- lives in one static device array of 4 MiB + 64 KiB that
 * every GPU loading this library holds until the process exits; media with more than
 * FLR_NOALLOC_MAX_VOXELS voxels (counted with each dimension rounded up to a multiple of 4) are
 * rejected with FLR_ERR_ARG. It renders the full RTE with one
 * majorant per bin: p->paper_mode, p->macro_cell, p->skip_cell, p->majorant_margin and p->hero
 * must be 0 (FLR_ERR_ARG otherwise; the array has no room for cell grids). The first call on a
 * device looks up that array's device address (with that device current) and keeps it for the
 * life of the process, so make that first call before any stream capture, and do not call this
 * entry point on a device after cudaDeviceReset. Every call uses the same array and clears what
 * must start at zero, so calls that overlap on the GPU (other streams, other host threads) race
 * with each other. The call synchronises `stream` (it reads grid maxima and the tallies back).
 * It returns FLR_ERR_BUDGET (outputs written) when a path or a connection ran out of its step
 * budget, and in the checked build FLR_ERR_CHECK when a device index was out of range. With no
 * room for a fixed-point accumulator, film contributions go to p->film by fp32 atomics: the film
 * equals flr_render's up to the order (and rounding) of fp32 additions. */
#define FLR_NOALLOC_MAX_VOXELS (1 << 18)
int flr_render_noalloc(float lambda0_nm, float dlambda_nm, int n_bins, int n_dyes,
                       const float *abs_shape, const float *emit_spec, const float *eps,
                       const float *qy, const flr_medium *medium, int n_sources,
                       const flr_source *sources, const flr_sensor *sensor, const flr_params *p,
                       double *face, double *absorbed, double *emitted, uint64_t *counters,
                       void *stream);

/* Synchronise the device and report, then clear, the context's device error word: FLR_ERR_BUDGET
 * if a launch of this context since the previous flr_status cut a path or a sensor connection
 * short at its step budget (max_steps, or 65,536 ratio-tracking steps; the tallies stay valid
 * for the paths that finished, and the counters step_budget / connect_budget say how many),
 * FLR_OK if clean. In the checked build it also reports, and clears, the first device index
 * found out of range since the last call (FLR_ERR_CHECK; any context of the process sees it). */
int flr_status(flr_ctx *ctx);
const char *flr_last_error(flr_ctx *ctx);

/* 1 if this library is the checked build (libfluoro_checked.so, compiled with FLR_CHECKED): every
 * grid, table, film, tally, gradient and queue index is tested on the device before its access; a
 * failed test skips the access and is recorded for flr_status, nothing traps. 0 otherwise. */
int flr_checked_build(void);
/* Diagnostics of the checked build: tests `index` in [0, bound) on the device (on `stream`) the
 * way every checked access is tested, so a violation can be provoked without touching memory.
 * A no-op in the normal build. FLR_ERR_CUDA if the launch fails. */
int flr_debug_check(int64_t index, int64_t bound, void *stream);

/* Diagnostics. Philox4x32-10 (Salmon et al., SC'11) blocks for device counters ctr [n][4] under
 * the key (seed, medium) into device out [n][4]; both 16-byte aligned (FLR_ERR_ARG otherwise). */
int flr_debug_philox(uint32_t seed, uint32_t medium, const uint32_t *ctr, int64_t n,
                     uint32_t *out, void *stream);
/* Emission bins drawn by the current medium's dye slot `dye` for device uniforms u [n]
 * (24-bit values in [0,1)) into device out [n]: min{ i : CDF[i] > u } (Eq. 10). */
int flr_debug_sample_emission(flr_ctx *ctx, int dye, const float *u, int64_t n, int32_t *out,
                              void *stream);

/* Debug: sigma_t(x, bin) of the current medium at n points (device [n][3] fp32, box
 * coordinates) by the lookup every kernel uses (Sec. 4.1: s(x)(sigma_s + sigma_a0) +
 * sum_d sig_a[d][bin] c_d(x), nearest voxel, fp32), into sigma_t (device [n] fp32), and the
 * row-major index z*ny*nx + y*nx + x of the voxel read into voxel (device [n], may be NULL; -1
 * for a medium without grids). Points outside the box take the nearest voxel (clamped).
 * FLR_ERR_ARG for a bin outside [0, n_bins), n < 0 or host pointers; FLR_ERR_STATE without a
 * medium. */
int flr_debug_sigma_t(flr_ctx *ctx, const float *points, int64_t n, int bin, float *sigma_t,
                      int32_t *voxel, void *stream);

/* Debug (failure injection on the host): the k-th device allocation the library makes from now on
 * fails as out of memory (the calling entry point returns FLR_ERR_OOM, or FLR_ERR_CUDA where the
 * failure surfaces as another CUDA error); the counter then stays at 0, and k = 0 disables it.
 * Process-wide (all contexts, all threads). FLR_ERR_ARG for k < 0. No device fault is made. */
int flr_debug_fail_alloc(int64_t k);

#ifdef __cplusplus
}
#endif

#endif /* FLUORO_H */
