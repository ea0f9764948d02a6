// fluoro_internal.cuh -- structures shared by the C-ABI host code and the sm_103a kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fluoro.h"

namespace flr {

constexpr int MAXD = FLR_MAX_DYES_PER_MEDIUM;
constexpr uint32_t STEP_SPAWN = 0xFFFFFFFFu;
constexpr int MAX_CONNECT_STEPS = 1 << 16;   // ratio-tracking steps per sensor connection
// Roulette on a transmittance estimate T below RT_RR_THRESHOLD: it survives with probability
// T / RT_RR_THRESHOLD and continues as RT_RR_THRESHOLD (unbiased: E = T), so marches from deep
// inside a dense region end after a step or two. Measured on the Cornell box (film RMSE against a
// 16x reference, time per step): 0.05 -> 0.3 costs 0.08 % of RMSE and saves 4.3 % of the time. The
// adjoint replay keeps the gentler rule below RT_RR_ADJ_THRESHOLD (survival 1/2, T doubled): its
// derivative samples carry the contribution as a factor, and a boost of up to RT_RR_THRESHOLD / T
// would make them heavy-tailed.
constexpr float RT_RR_THRESHOLD = 0.3f;
constexpr float RT_RR_ADJ_THRESHOLD = 1e-3f;

// Layout of the per-medium spectral tables (fp32, global memory, staged into shared memory):
//   sig_a[B][MAXD]   eps_d * a_d(lambda_b), per unit concentration      (Sec. 4.1); the MAXD
//                    dyes of one bin are one 16-byte vector
//   cdf[MAXD][B]     emission CDF, fp64-built and rounded, last = 1      (Eq. 10)
//   majorant[B]      sigma_bar(lambda_b) >= sigma_t(x, lambda_b) for all x
//   inv_majorant[B]  1 / sigma_bar(lambda_b) (0 where sigma_bar = 0)
//   qy[MAXD]
// The size is padded to a multiple of 4 floats so that consecutive media's tables stay 16-byte
// aligned.
__host__ __device__ constexpr int tab_sig_a(int B) { return 0; }
__host__ __device__ constexpr int tab_sig_a_at(int B, int d, int b) { return b * MAXD + d; }
__host__ __device__ constexpr int tab_cdf(int B) { return MAXD * B; }
__host__ __device__ constexpr int tab_majorant(int B) { return 2 * MAXD * B; }
__host__ __device__ constexpr int tab_inv_majorant(int B) { return 2 * MAXD * B + B; }
__host__ __device__ constexpr int tab_qy(int B) { return 2 * MAXD * B + 2 * B; }
__host__ __device__ constexpr int tab_size(int B) { return (2 * MAXD * B + 2 * B + MAXD + 3) & ~3; }

// Fixed-point tallies (u64, 2^-24 units of photon weight): face[2][6][B], absorbed[MAXD+1][B],
// emitted[MAXD][B]. Integer sums make every launch form and thread order give identical bits.
__host__ __device__ constexpr int tal_face(int B) { return 0; }
__host__ __device__ constexpr int tal_absorbed(int B) { return 12 * B; }
__host__ __device__ constexpr int tal_emitted(int B) { return 12 * B + (MAXD + 1) * B; }
__host__ __device__ constexpr int tal_size(int B) { return 12 * B + (2 * MAXD + 1) * B; }
constexpr double TALLY_ONE = 16777216.0;  // 2^24

// The library's interleaved concentration grid (one float4 of up to four dyes per voxel) is stored
// in bricks of 4^3 voxels: x fastest inside a brick, bricks x fastest over the grid padded to
// whole bricks. A free flight or a ratio-tracking step moves a few voxels, so consecutive lookups
// of a path, and those of nearby paths, fall in the same 1 KB brick (the same cache lines and DRAM
// page) far more often than in a row-major layout, where a step in z jumps nx * ny voxels.
constexpr int GRID_BRICK = 4;
__host__ __device__ inline int grid_bricks(int n) { return (n + GRID_BRICK - 1) / GRID_BRICK; }
__host__ __device__ inline long long packed_voxels(const int dims[3])
{
    return (long long)grid_bricks(dims[0]) * grid_bricks(dims[1]) * grid_bricks(dims[2]) *
           (GRID_BRICK * GRID_BRICK * GRID_BRICK);
}
// Index in the packed grid of voxel (ix, iy, iz); bdims = bricks per axis.
__host__ __device__ inline int packed_index(int ix, int iy, int iz, const int bdims[3])
{
    const int b = ((iz >> 2) * bdims[1] + (iy >> 2)) * bdims[0] + (ix >> 2);
    return (b << 6) | ((iz & 3) << 4) | ((iy & 3) << 2) | (ix & 3);
}

struct EmitterDev {
    float origin[3], eu[3], ev[3], dir[3];
    int kind, bin, axis;
    float sign;
    int entry;                         // dielectric face the source enters through, or -1
};

// Scene description passed by value to the kernels (lives in the constant bank).
struct SceneDev {
    int B, D;
    float lo[3], hi[3], vox_scale[3];  // vox_scale = dims / (hi - lo)
    int dims[3];
    int bdims[3];                      // bricks per axis of the packed grid
    int homogeneous;                   // no grid and no solvent mask
    const float4 *grid;                // [nvox] interleaved concentrations of the medium's dyes
    const uint8_t *solvent;            // [nvox] or nullptr
    float conc_uniform[MAXD];
    float sigma_s, sigma_a0;
    int wall_mask;
    float wall_albedo;
    const float *tables;               // tab_size(B) floats
    int n_emitters;
    float em_cdf[FLR_MAX_EMITTERS];
    EmitterDev em[FLR_MAX_EMITTERS];
    // the lines of one source are consecutive emitters: emitter k's source spans emitters
    // em_group_first[k] .. em_group_first[k] + em_group_n[k] - 1 (hero-wavelength sets)
    int em_group_first[FLR_MAX_EMITTERS], em_group_n[FLR_MAX_EMITTERS];
    int sensor_kind, W, H;
    float s_origin[3], s_U[3], s_V[3], s_view[3];  // ortho: U, V pre-divided by |U|^2, |V|^2
    float tan_x, tan_y, inv_A_pix;
    float cam_U[3], cam_V[3];          // ortho: full film edges (camera rays start on the film)
    float inv_tan_x, inv_tan_y;
    // local majorants (macro cells); mc == 0: one majorant per bin. sk > 0: empty-space leaps
    // after null collisions (global majorant) over the same cell grid
    int mc, sk;
    int mc_dims[3];
    float mc_size[3], mc_inv[3];       // cell edge (cm) and its inverse
    const float4 *mc_c;                // per-cell maximum concentration of each dye
    const float *mc_s;                 // per-cell maximum of the solvent mask
    float maj_margin;                  // local majorants are multiplied by this (>= 1)
    const uint8_t *mc_dist;            // 0: cell may hold matter; k >= 1: every cell within
                                       // Chebyshev distance k - 1 is empty (leaping)
    // interfaces and glossy walls (flr_medium::ior, wall_gloss, wall_exponent): iface != 0 when
    // either is on; open faces are dielectric when ior > 1; iface_exit = (1 - F(0)) / ior^2, the
    // share of radiance a connection carries out through a dielectric face at normal incidence
    int iface, dielectric;
    float ior, inv_ior, iface_exit;
    float wall_gloss, wall_exp;
    // 1: launch the instances that settle decisions without a grid read where a bound fixes them
    // (grids, no solvent mask, and sigma_s + sigma_a0 at least 0.9 of every bin's majorant, so
    // that the bounds decide most steps)
    int lazy;
};

// Per-launch run parameters.
struct RunDev {
    uint64_t n_paths, path_offset;
    uint32_t seed, medium_id;
    int n_rr, max_inelastic, analog;
    long long max_events, max_steps;
    float film_scale;                  // 1 / n_paths
    float *film;
    unsigned long long *film_fx;       // the launch's film sums in fixed point (FILM_FX_ONE), or
                                       // NULL: contributions go to `film` by fp32 atomics
    uint32_t *path_events;
    unsigned long long *tallies;       // tal_size(B)
    unsigned long long *counters;      // FLR_NCOUNTERS
    int *error_word;
    unsigned long long *work_counter;  // dynamic path distribution (wavefront form)
    int regroup;                       // wavefront: tracking steps between connection flushes
    int paper_mode;                    // the paper's single-inelastic model (flr_params)
    int hero;                          // wavelengths per hero path (flr_params); 0 = one
    uint32_t rk[20];                   // Philox round keys of (seed, medium_id): k0[10], k1[10]
};

// Fills RunDev::rk with the Philox4x32-10 key schedule of (seed, medium_id): round r uses
// k0 = seed + r * 0x9E3779B9 and k1 = medium_id + r * 0xBB67AE85 (mod 2^32).
inline void set_round_keys(RunDev &R)
{
    uint32_t k0 = R.seed, k1 = R.medium_id;
    for (int r = 0; r < 10; ++r) {
        R.rk[r] = k0;
        R.rk[10 + r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// One medium of a batched launch (global memory; read per lane through the read-only path).
constexpr int BATCH_MAX_LINES = 8;
struct MediumDev {
    float lo[3], hi[3], vox_scale[3];
    int dims[3];
    int bdims[3];                      // bricks per axis of the packed grid
    int homogeneous, D;
    const float4 *grid;                // interleaved concentrations inside the batch arena
    const uint8_t *solvent;
    float conc_uniform[MAXD];
    float sigma_s, sigma_a0;
    int wall_mask;
    float wall_albedo;
    const float *tables;               // tab_size(B) floats
    unsigned long long *tallies;       // tal_size(B) fixed-point tallies of this medium
    uint32_t key1;                     // Philox key word 1 (the medium id)
    int n_emitters;
    float em_cdf[BATCH_MAX_LINES];
    EmitterDev em[BATCH_MAX_LINES];
};

static_assert(sizeof(MediumDev) % 8 == 0, "MediumDev array elements keep 8-byte alignment");

// A work item of the batched queue: `count` consecutive path ids of one medium.
struct ChunkDev {
    int medium;
    uint32_t count;
    unsigned long long start;
};

struct BatchDev {
    int B;
    int n_chunks;
    const MediumDev *media;
    const ChunkDev *chunks;
    unsigned long long *head;          // next chunk (device counter)
};

// Adjoint inputs and outputs (device): adj [H][W][B] = dL/dI; grad_c [D][nvox] (or nullptr);
// grad_sigma_s [1] (or nullptr).
struct AdjDev {
    const float *adj;
    float *grad_c;
    long long nvox;
    float *grad_sigma_s;
    // two-pass replay of the warp-regrouped form: a_k of the first K connections of each path of
    // the launch ([n_paths][K], zeroed before pass 1) and the sum of the later ones ([n_paths])
    float *ak;
    float *ovf;
    int K;
};

// Host-side launchers (fluoro_kernels.cu).
cudaError_t launch_adjoint(const SceneDev &S, const RunDev &R, const AdjDev &A, int block,
                           int blocks_per_sm, cudaStream_t st);
// form PLAIN: one thread per camera path; otherwise warp-regrouped (R.work_counter zeroed)
cudaError_t launch_camera(const SceneDev &S, const RunDev &R, int form, int block, cudaStream_t st);
// pass 1 (weights) or pass 2 (gradients) of the warp-regrouped adjoint; R.work_counter zeroed
cudaError_t launch_adjoint_warp(const SceneDev &S, const RunDev &R, const AdjDev &A, int pass,
                                int block, int blocks_per_sm, cudaStream_t st);
cudaError_t launch_batch(const BatchDev &Bt, const RunDev &R, int block, int blocks_per_sm,
                         cudaStream_t st);
int batch_occupancy_blocks_per_sm(int block);
// Film contributions are summed per launch as integers in units of 2^-32 of the film's unit: exact,
// so the sum does not depend on the order of the additions (up to 2^32 per film value).
constexpr float FILM_FX_ONE = 4294967296.0f;
constexpr double FILM_FX_INV = 1.0 / 4294967296.0;
// film[j] = fx[j] * 2^-32 (add = 0) or film[j] + fx[j] * 2^-32 (add = 1), j < n, through fp64.
cudaError_t launch_film_fold(float *film, const unsigned long long *fx, size_t n, int add, cudaStream_t st);
cudaError_t launch_trace(const SceneDev &S, const RunDev &R, int form, int block, int blocks_per_sm,
                         cudaStream_t st);
cudaError_t launch_build_macro(const float4 *grid, float4 uniform, const uint8_t *solvent,
                               const int dims[3], int cell, const int mdims[3], float4 *out_c,
                               float *out_s, cudaStream_t st);
cudaError_t launch_empty_distance(const float4 *mc, const float *ms, const int mdims[3],
                                  int solvent_matter, int cap, uint8_t *out, uint8_t *tmp,
                                  cudaStream_t st);
cudaError_t launch_grid_max(const float *g, long long n, unsigned int *out_bits, int *neg_flag,
                            cudaStream_t st);
// interleaves the dyes' row-major grids into the bricked layout (packed_voxels(dims) float4s)
cudaError_t launch_pack_grid(const float *const *conc, const float *uniform, int D, const int dims[3],
                             float4 *out, cudaStream_t st);
cudaError_t launch_solvent_any(const uint8_t *s, long long n, unsigned int *out, cudaStream_t st);
cudaError_t launch_philox(uint32_t seed, uint32_t medium, const uint32_t *ctr, long long n,
                          uint32_t *out, cudaStream_t st);
// frozen-sampling per-path sums of adj x film contributions at a perturbed medium (diagnostic)
cudaError_t launch_frozen_sums(const SceneDev &S, const RunDev &R, int pert_dye, long long pert_voxel,
                               float pert_delta, float pert_dsig, const float *adj, double *out,
                               cudaStream_t st);
cudaError_t launch_debug_sigma_t(const SceneDev &S, const float *pts, long long n, int bin, float *out,
                                 int32_t *vox, cudaStream_t st);
cudaError_t launch_sample_emission(const SceneDev &S, int dye, const float *u, long long n,
                                   int32_t *out, cudaStream_t st);
int trace_block_default();
// Checked build (-DFLR_CHECKED): 1 if this library tests every index before its access
int checked_build();
// Reads and clears the first recorded index violation: bit 63 set, site in bits 56..62, index in
// bits 0..55; 0 when none (always 0 in the normal build)
cudaError_t check_word_take(unsigned long long *word);
// Tests `index` in [0, bound) on the device like any checked access (debug entry)
cudaError_t launch_debug_check(long long index, long long bound, cudaStream_t st);
int device_sms();
int trace_smem_bytes(int B, int form, int block);
int occupancy_blocks_per_sm(int B, int form, int block);

}  // namespace flr
