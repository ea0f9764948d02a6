// fluoro_kernels.cu -- sm_103a kernels of the fluorescent participating-media light tracer.
//
// Light (photon) tracing of the per-wavelength fluorescent RTE (Sec. 4.2, Eq. 9 and 11) with the
// estimator structure of Eq. 12:
//   spawn      a photon of unit power at a source line chosen in proportion to power
//   free flight  delta tracking against the per-wavelength majorant (Eq. 6 sampled exactly)
//   collision  particle type in proportion to its coefficient: solvent scatterer, dye d
//              (eps_d a_d(lambda) c_d), or background absorber (Sec. 4.1)
//   scatter    isotropic (Sec. 2.1)
//   dye        weight *= QY (or a QY coin), new wavelength from the emission CDF (Eq. 10),
//              isotropic direction (Sec. 2.1)
//   walls      Lambertian reflection
//   roulette   once n_events >= n_rr, survive with q = min(1, w), w /= q
//   sensor     every scatter, emission, wall and Lambertian-light vertex connects to the film:
//              intensity x transmittance (ratio tracking, Eq. 6) x importance (Eq. 3-5)
//   tallies    escaped weight per [fluoresced][face][bin]; absorbed / emitted per dye and bin
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by (seed, medium), counter
// (path_lo, step, slot, path_hi). Slot 0 of a tracking step gives (u_dist, u_real, u_event,
// u_dir1), slot 1 (u_dir2, u_emit, u_rr, u_coin); slot 2 seeds the xoshiro128** stream of the
// step's sensor connection (its ratio-tracking march). Spawn uses step 0xFFFFFFFF. Uniforms are
// 24-bit: u = (x >> 8) 2^-24.
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "fluoro_internal.cuh"

namespace flr {

namespace {

constexpr float INV_4PI = 0.0795774715459476679f;
constexpr float INV_PI = 0.318309886183790672f;
constexpr float TWO_PI = 6.28318530717958648f;

// ---------------------------------------------------------------------------------------------
// Philox4x32-10: ten rounds, each two 32x32->64 products of the even words with the round
// multipliers, mixed with the odd words and the key; the key advances by the Weyl constants.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

struct U4 { float a, b, c, d; };


__device__ __forceinline__ U4 draw(uint32_t seed, uint32_t medium, uint64_t pid, uint32_t step,
                                   uint32_t slot)
{
    const uint4 o = philox(make_uint4((uint32_t)pid, step, slot, (uint32_t)(pid >> 32)), seed, medium);
    return U4{u24(o.x), u24(o.y), u24(o.z), u24(o.w)};
}

// The same Philox4x32-10 block with the launch's key schedule read from the kernel parameters
// (RunDev::rk, filled by set_round_keys): the round keys of a single-scene launch are constants, so
// the rounds take them as operands instead of recomputing them for every block.
__device__ __forceinline__ U4 draw_rk(const RunDev &R, uint64_t pid, uint32_t step, uint32_t slot)
{
    uint4 c = make_uint4((uint32_t)pid, step, slot, (uint32_t)(pid >> 32));
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ R.rk[r], lo1, hi0 ^ c.w ^ R.rk[10 + r], lo0);
    }
    return U4{u24(c.x), u24(c.y), u24(c.z), u24(c.w)};
}

// The raw words of that block.
__device__ __forceinline__ uint4 draw_raw_rk(const RunDev &R, uint64_t pid, uint32_t step, uint32_t slot)
{
    uint4 c = make_uint4((uint32_t)pid, step, slot, (uint32_t)(pid >> 32));
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ R.rk[r], lo1, hi0 ^ c.w ^ R.rk[10 + r], lo0);
    }
    return c;
}

// Uniforms of one sensor connection's ratio-tracking march: the xoshiro128** generator (Blackman and
// Vigna, "Scrambled linear pseudorandom number generators", ACM TOMS 2021) seeded with the Philox
// block of the connection's counter (path, step, slot 2). A march draws one uniform per step (and
// one more for a roulette), always the next of its stream, so every lane of a warp pays the same
// dozen integer operations per step instead of a whole Philox block whenever its own four-uniform
// block runs out (which, with the lanes' marches at different points, is nearly every step for
// some lane). Every form and replay of a connection draws the same stream. The oracle evaluates
// transmittances exactly (reading 17), so nothing on its side depends on these numbers.
struct MarchRng {
    uint32_t s0, s1, s2, s3;
};

__device__ __forceinline__ MarchRng march_rng(const RunDev &R, uint64_t pid, uint32_t step, uint32_t slot = 2u)
{
    const uint4 b = draw_raw_rk(R, pid, step, slot);
    MarchRng g{b.x, b.y, b.z, b.w};
    if ((b.x | b.y | b.z | b.w) == 0u) g.s0 = 1u;   // the all-zero state would stay zero
    return g;
}

__device__ __forceinline__ float march_next(MarchRng &g)
{
    const uint32_t r = __funnelshift_l(g.s1 * 5u, g.s1 * 5u, 7) * 9u;
    const uint32_t t = g.s1 << 9;
    g.s2 ^= g.s0;
    g.s3 ^= g.s1;
    g.s1 ^= g.s2;
    g.s0 ^= g.s3;
    g.s2 ^= t;
    g.s3 = __funnelshift_l(g.s3, g.s3, 11);
    return u24(r);
}

// ---------------------------------------------------------------------------------------------
// Checked build (-DFLR_CHECKED, libfluoro_checked.so): every grid, table, film, tally, gradient
// and queue index is tested before its access. A failed test skips the access and records the
// first (site, index) in g_check_word, which flr_status reports as FLR_ERR_CHECK; nothing traps.
// In the normal build FLR_CHK is the constant true: the tests are not compiled.
enum CheckSite { CK_DEBUG = 1, CK_GRID = 2, CK_FILM = 3, CK_TALLY = 4, CK_GRAD = 5, CK_ADJ_STORE = 6,
                 CK_QUEUE = 7, CK_CELL = 8 };
#ifdef FLR_CHECKED
__device__ unsigned long long g_check_word;
__device__ __forceinline__ bool check_index(bool ok, int site, long long idx)
{
    if (!ok)
        atomicCAS(&g_check_word, 0ull,
                  (1ull << 63) | ((unsigned long long)(site & 0x7F) << 56) |
                      ((unsigned long long)idx & 0x00FFFFFFFFFFFFFFull));
    return ok;
}
#define FLR_CHK(ok, site, idx) check_index((ok), (site), (long long)(idx))
#else
#define FLR_CHK(ok, site, idx) true
#endif

// Film accumulation at index idx of the [H][W][B] film. With an accumulator (R.film_fx) a
// contribution adds round(val * 2^32) to a 64-bit integer, so the launch's sum is exact: a bin that
// millions of paths reach keeps every contribution (an fp32 sum stops growing once the bin exceeds
// 2^24 times a contribution), the result does not depend on the order of the additions, and the
// L2 serialises integer additions to one address faster than fp32 ones. Without an accumulator
// (the no-allocation entry point) the contribution goes to the fp32 film directly.
__device__ __forceinline__ void film_add(const SceneDev &S, const RunDev &R, size_t idx, float val)
{
    if (!FLR_CHK(idx < (size_t)S.W * S.H * S.B, CK_FILM, (long long)idx)) return;
    if (R.film_fx == nullptr) {
        atomicAdd(&R.film[idx], val);
        return;
    }
    const unsigned long long fx = __float2ull_rn(val * FILM_FX_ONE);
    if (fx) atomicAdd(&R.film_fx[idx], fx);
}

// ---------------------------------------------------------------------------------------------
// Shared-memory view: spectral tables, block tallies, block counters.
struct Smem {
    const float *sig_a, *cdf, *maj, *inv_maj, *qy;
    unsigned long long *tal;   // shared memory, or the launch's global tallies (tal_global)
    unsigned long long *cnt;
    bool tal_global;
};

// Frequent counters live in registers; the rest go straight to shared memory.
struct RegCnt {
    uint32_t steps, nulls, events, scatters, connections, connect_steps, cell_walks;
};

// Adds one per calling lane. The lanes that arrive together add once, through their lowest lane,
// instead of queueing on one shared-memory word.
__device__ __forceinline__ void cnt_add(const Smem &sm, int k)
{
    const unsigned mask = __activemask();
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(&sm.cnt[k], (unsigned long long)__popc(mask));
}

__device__ __forceinline__ void tally_add(const Smem &sm, int idx, float w)
{
    const unsigned long long fx = __float2ull_rn(w * 16777216.0f);
    if (fx) atomicAdd(&sm.tal[idx], fx);
}

// ---------------------------------------------------------------------------------------------
// Medium accessors. The tracking code is written once against this interface:
//   MedS  single scene: geometry from the kernel parameters (constant bank), spectral tables and
//         tallies in shared memory.
//   MedB  one medium of a batched launch, per lane: fields read from global memory through the
//         read-only path, tables in global memory (L1-resident), tallies in global memory.
// OPT = false compiles the local-majorant and empty-space paths out (the plain baseline kernel);
// MC = false compiles the local-majorant path alone out (launched whenever the scene has none:
// the smaller code keeps the warp-regrouped kernel's loops in the instruction cache); IF = false
// compiles dielectric faces and glossy walls out (scenes with index-matched faces and Lambertian
// walls). LZ = true compiles in the decisions taken without a grid read (minorant_known; launched
// for media with grids and no solvent mask).
template <bool OPT, bool MC = OPT, bool IF = true, bool LZ = false>
struct MedS_ {
    static constexpr bool kLazy = LZ;
    const SceneDev &S;
    const Smem &sm;
    __device__ __forceinline__ int B() const { return S.B; }
    __device__ __forceinline__ int D() const { return S.D; }
    __device__ __forceinline__ float lo(int k) const { return S.lo[k]; }
    __device__ __forceinline__ float hi(int k) const { return S.hi[k]; }
    __device__ __forceinline__ float vox_scale(int k) const { return S.vox_scale[k]; }
    __device__ __forceinline__ int dims(int k) const { return S.dims[k]; }
    __device__ __forceinline__ const int *bdims() const { return S.bdims; }
    __device__ __forceinline__ bool homogeneous() const { return S.homogeneous != 0; }
    __device__ __forceinline__ const float4 *grid() const { return S.grid; }
    __device__ __forceinline__ const uint8_t *solvent() const { return S.solvent; }
    __device__ __forceinline__ float4 conc_uniform() const
    {
        return make_float4(S.conc_uniform[0], S.conc_uniform[1], S.conc_uniform[2], S.conc_uniform[3]);
    }
    __device__ __forceinline__ float sigma_s() const { return S.sigma_s; }
    __device__ __forceinline__ float sigma_a0() const { return S.sigma_a0; }
    __device__ __forceinline__ int wall_mask() const { return S.wall_mask; }
    __device__ __forceinline__ float wall_albedo() const { return S.wall_albedo; }
    __device__ __forceinline__ float sig_a(int d, int b) const { return sm.sig_a[tab_sig_a_at(S.B, d, b)]; }
    __device__ __forceinline__ float4 sig_a4(int b) const { return reinterpret_cast<const float4 *>(sm.sig_a)[b]; }
    __device__ __forceinline__ float maj(int b) const { return sm.maj[b]; }
    __device__ __forceinline__ float inv_maj(int b) const { return sm.inv_maj[b]; }
    __device__ __forceinline__ float qy(int d) const { return sm.qy[d]; }
    __device__ __forceinline__ const float *cdf(int d) const { return sm.cdf + d * S.B; }
    __device__ __forceinline__ void tally(int idx, float w) const
    {
        if (FLR_CHK(idx >= 0 && idx < tal_size(S.B), CK_TALLY, idx)) tally_add(sm, idx, w);
    }
    __device__ __forceinline__ bool sensor() const { return S.sensor_kind != FLR_SENSOR_NONE; }
    __device__ __forceinline__ int n_emitters() const { return S.n_emitters; }
    __device__ __forceinline__ float em_cdf(int k) const { return S.em_cdf[k]; }
    __device__ __forceinline__ const EmitterDev &em(int k) const { return S.em[k]; }
    __device__ __forceinline__ uint32_t key1(const RunDev &R) const { return R.medium_id; }
    __device__ __forceinline__ U4 rng(const RunDev &R, uint64_t pid, uint32_t step, uint32_t slot) const
    {
        return draw_rk(R, pid, step, slot);
    }
    __device__ __forceinline__ bool macro() const { return OPT && MC && S.mc > 0; }
    __device__ __forceinline__ float margin() const { return S.maj_margin; }
    __device__ __forceinline__ int mc_dims(int k) const { return S.mc_dims[k]; }
    __device__ __forceinline__ float mc_size(int k) const { return S.mc_size[k]; }
    __device__ __forceinline__ float mc_inv(int k) const { return S.mc_inv[k]; }
    __device__ __forceinline__ bool cell_ok(int c) const
    {
        return FLR_CHK(c >= 0 && c < S.mc_dims[0] * S.mc_dims[1] * S.mc_dims[2], CK_CELL, c);
    }
    __device__ __forceinline__ float4 mc_conc(int c) const
    {
        return cell_ok(c) ? __ldg(&S.mc_c[c]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __device__ __forceinline__ float mc_solvent(int c) const { return cell_ok(c) ? __ldg(&S.mc_s[c]) : 0.0f; }
    __device__ __forceinline__ int mc_empty_radius(int c) const { return cell_ok(c) ? (int)__ldg(&S.mc_dist[c]) : 0; }
    __device__ __forceinline__ bool skip() const { return OPT && S.sk > 0; }
    __device__ __forceinline__ bool iface() const { return IF && S.iface != 0; }
    __device__ __forceinline__ bool dielectric() const { return S.dielectric != 0; }
    __device__ __forceinline__ float ior() const { return S.ior; }
    __device__ __forceinline__ float inv_ior() const { return S.inv_ior; }
    __device__ __forceinline__ float wall_gloss() const { return S.wall_gloss; }
    __device__ __forceinline__ float wall_exp() const { return S.wall_exp; }
    // unit direction from x toward the sensor (orthographic: the view direction)
    __device__ __forceinline__ float3 sensor_dir(float3 x) const
    {
        if (S.sensor_kind == FLR_SENSOR_ORTHO) return make_float3(S.s_view[0], S.s_view[1], S.s_view[2]);
        const float vx = S.s_origin[0] - x.x, vy = S.s_origin[1] - x.y, vz = S.s_origin[2] - x.z;
        const float ir = rsqrtf(vx * vx + vy * vy + vz * vz);
        return make_float3(vx * ir, vy * ir, vz * ir);
    }
};
using MedS = MedS_<true>;

__device__ __forceinline__ void tally_add_global(unsigned long long *t, int idx, float w)
{
    const unsigned long long fx = __float2ull_rn(w * 16777216.0f);
    if (fx) atomicAdd(&t[idx], fx);
}

struct MedB {
    static constexpr bool kLazy = false;
    const MediumDev *__restrict__ md;
    int B_;
    __device__ __forceinline__ int B() const { return B_; }
    __device__ __forceinline__ int D() const { return __ldg(&md->D); }
    __device__ __forceinline__ float lo(int k) const { return __ldg(&md->lo[k]); }
    __device__ __forceinline__ float hi(int k) const { return __ldg(&md->hi[k]); }
    __device__ __forceinline__ float vox_scale(int k) const { return __ldg(&md->vox_scale[k]); }
    __device__ __forceinline__ int dims(int k) const { return __ldg(&md->dims[k]); }
    __device__ __forceinline__ const int *bdims() const { return md->bdims; }
    __device__ __forceinline__ bool homogeneous() const { return __ldg(&md->homogeneous) != 0; }
    __device__ __forceinline__ const float4 *grid() const
    {
        return reinterpret_cast<const float4 *>(__ldg(reinterpret_cast<const unsigned long long *>(&md->grid)));
    }
    __device__ __forceinline__ const uint8_t *solvent() const
    {
        return reinterpret_cast<const uint8_t *>(__ldg(reinterpret_cast<const unsigned long long *>(&md->solvent)));
    }
    __device__ __forceinline__ float4 conc_uniform() const
    {
        // scalar loads: the field is only 8-byte aligned inside MediumDev
        return make_float4(__ldg(&md->conc_uniform[0]), __ldg(&md->conc_uniform[1]),
                           __ldg(&md->conc_uniform[2]), __ldg(&md->conc_uniform[3]));
    }
    __device__ __forceinline__ float sigma_s() const { return __ldg(&md->sigma_s); }
    __device__ __forceinline__ float sigma_a0() const { return __ldg(&md->sigma_a0); }
    __device__ __forceinline__ int wall_mask() const { return __ldg(&md->wall_mask); }
    __device__ __forceinline__ float wall_albedo() const { return __ldg(&md->wall_albedo); }
    __device__ __forceinline__ const float *tables() const
    {
        return reinterpret_cast<const float *>(__ldg(reinterpret_cast<const unsigned long long *>(&md->tables)));
    }
    __device__ __forceinline__ float sig_a(int d, int b) const { return __ldg(tables() + tab_sig_a(B_) + tab_sig_a_at(B_, d, b)); }
    __device__ __forceinline__ float4 sig_a4(int b) const
    {
        return __ldg(reinterpret_cast<const float4 *>(tables() + tab_sig_a(B_)) + b);
    }
    __device__ __forceinline__ float maj(int b) const { return __ldg(tables() + tab_majorant(B_) + b); }
    __device__ __forceinline__ float inv_maj(int b) const { return __ldg(tables() + tab_inv_majorant(B_) + b); }
    __device__ __forceinline__ float qy(int d) const { return __ldg(tables() + tab_qy(B_) + d); }
    __device__ __forceinline__ const float *cdf(int d) const { return tables() + tab_cdf(B_) + d * B_; }
    __device__ __forceinline__ void tally(int idx, float w) const
    {
        if (!FLR_CHK(idx >= 0 && idx < tal_size(B_), CK_TALLY, idx)) return;
        tally_add_global(reinterpret_cast<unsigned long long *>(
                             __ldg(reinterpret_cast<const unsigned long long *>(&md->tallies))),
                         idx, w);
    }
    __device__ __forceinline__ bool sensor() const { return false; }
    __device__ __forceinline__ int n_emitters() const { return __ldg(&md->n_emitters); }
    __device__ __forceinline__ float em_cdf(int k) const { return __ldg(&md->em_cdf[k]); }
    __device__ __forceinline__ const EmitterDev &em(int k) const { return md->em[k]; }
    __device__ __forceinline__ uint32_t key1(const RunDev &) const { return __ldg(&md->key1); }
    __device__ __forceinline__ U4 rng(const RunDev &R, uint64_t pid, uint32_t step, uint32_t slot) const
    {
        return draw(R.seed, key1(R), pid, step, slot);
    }
    __device__ __forceinline__ bool macro() const { return false; }
    __device__ __forceinline__ float margin() const { return 1.0f; }
    __device__ __forceinline__ int mc_dims(int) const { return 1; }
    __device__ __forceinline__ float mc_size(int) const { return 1.0f; }
    __device__ __forceinline__ float mc_inv(int) const { return 1.0f; }
    __device__ __forceinline__ float4 mc_conc(int) const { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ float mc_solvent(int) const { return 0.0f; }
    __device__ __forceinline__ int mc_empty_radius(int) const { return 0; }
    __device__ __forceinline__ bool skip() const { return false; }
    __device__ __forceinline__ bool iface() const { return false; }
    __device__ __forceinline__ bool dielectric() const { return false; }
    __device__ __forceinline__ float ior() const { return 1.0f; }
    __device__ __forceinline__ float inv_ior() const { return 1.0f; }
    __device__ __forceinline__ float wall_gloss() const { return 0.0f; }
    __device__ __forceinline__ float wall_exp() const { return 0.0f; }
    __device__ __forceinline__ float3 sensor_dir(float3) const { return make_float3(0.f, 0.f, 1.f); }
};

// ---------------------------------------------------------------------------------------------
// Medium (Sec. 4.1): sigma_t = s(x)(sigma_s + sigma_a0) + sum_d sig_a[d][b] c_d(x), nearest voxel.
struct Coeffs {
    float scat, bg, total;
    float dye[MAXD];
};

// Nearest voxel of x (clamped to the grid): its (ix, iy, iz).
template <class M>
__device__ __forceinline__ int3 voxel_ijk(const M &m, float3 x)
{
    int ix = __float2int_rd((x.x - m.lo(0)) * m.vox_scale(0));
    int iy = __float2int_rd((x.y - m.lo(1)) * m.vox_scale(1));
    int iz = __float2int_rd((x.z - m.lo(2)) * m.vox_scale(2));
    ix = min(max(ix, 0), m.dims(0) - 1);
    iy = min(max(iy, 0), m.dims(1) - 1);
    iz = min(max(iz, 0), m.dims(2) - 1);
    return make_int3(ix, iy, iz);
}

// Row-major [nz][ny][nx] index of the nearest voxel: the caller's layout (solvent mask, gradients).
template <class M>
__device__ __forceinline__ int voxel_of(const M &m, float3 x)
{
    const int3 c = voxel_ijk(m, x);
    return (c.z * m.dims(1) + c.y) * m.dims(0) + c.x;
}

template <class M>
__device__ __forceinline__ Coeffs coeffs_at(const M &m, float3 x, int b)
{
    float s = 1.0f;
    float4 c = m.conc_uniform();
    if (!m.homogeneous()) {
        const int3 q = voxel_ijk(m, x);
        const int v = (q.z * m.dims(1) + q.y) * m.dims(0) + q.x;
        const float4 *g = m.grid();
        const uint8_t *sv = m.solvent();
        if (FLR_CHK(v >= 0 && v < m.dims(0) * m.dims(1) * m.dims(2), CK_GRID, v)) {
            if (g) c = __ldg(&g[packed_index(q.x, q.y, q.z, m.bdims())]);
            if (sv) s = __ldg(&sv[v]) ? 1.0f : 0.0f;
        }
    }
    Coeffs k;
    k.scat = s * m.sigma_s();
    k.bg = s * m.sigma_a0();
    k.total = k.scat + k.bg;
    const float cc[4] = {c.x, c.y, c.z, c.w};
    const float4 sa = m.sig_a4(b);
    const float ss[4] = {sa.x, sa.y, sa.z, sa.w};
    const int D = m.D();
#pragma unroll
    for (int d = 0; d < MAXD; ++d) {
        k.dye[d] = (d < D) ? ss[d] * cc[d] : 0.0f;
        k.total += k.dye[d];
    }
    return k;
}

template <class M>
__device__ __forceinline__ float sigma_t_at(const M &m, float3 x, int b)
{
    return coeffs_at(m, x, b).total;
}

// Distance to leave the box along w (inverse direction given), face index 0..5 or -1; ties to
// the lowest face index.
template <class M>
__device__ __forceinline__ float exit_distance(const M &m, float3 x, float3 w, float3 iw, int &face)
{
    float best = FLT_MAX;
    face = -1;
    const float xs[3] = {x.x, x.y, x.z}, ws[3] = {w.x, w.y, w.z}, is[3] = {iw.x, iw.y, iw.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (ws[k] == 0.0f) continue;
        const bool pos = ws[k] > 0.0f;
        float t = ((pos ? m.hi(k) : m.lo(k)) - xs[k]) * is[k];
        t = fmaxf(t, 0.0f);
        if (t < best) { best = t; face = 2 * k + (pos ? 1 : 0); }
    }
    return best;
}

// The hardware's approximate square root (PTX sqrt.approx.f32, relative error about 2^-23):
// enough for sampled directions, cheaper than the correctly rounded sqrtf.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Componentwise inverse of a direction (0 for a zero component). The approximate reciprocal
// (2 ulp) is plenty for distances to planes and cost 7 % less time per Cornell-box step than the
// correctly rounded one.
__device__ __forceinline__ float3 inv_dir(float3 w)
{
    return make_float3(w.x != 0.0f ? __fdividef(1.0f, w.x) : 0.0f, w.y != 0.0f ? __fdividef(1.0f, w.y) : 0.0f,
                       w.z != 0.0f ? __fdividef(1.0f, w.z) : 0.0f);
}

// ---------------------------------------------------------------------------------------------
// Local majorants. Cell c covers macro_cell^3 voxels; its majorant is evaluated with exactly the
// operation order of coeffs_at (solvent scattering, solvent absorption, then each dye), so with
// cell maxima of every input the fp32 result bounds sigma_t anywhere in the cell (IEEE rounding is
// monotone). A DDA walks the cells along a ray spending an optical budget tau = -ln(1 - u).
template <class M>
__device__ __forceinline__ float cell_majorant(const M &m, int cell, int b)
{
    const float sv = m.mc_solvent(cell);
    const float4 c = m.mc_conc(cell);
    float total = sv * m.sigma_s() + sv * m.sigma_a0();
    const float cc[4] = {c.x, c.y, c.z, c.w};
    const int D = m.D();
#pragma unroll
    for (int d = 0; d < MAXD; ++d) total += (d < D) ? m.sig_a(d, b) * cc[d] : 0.0f;
    return total;
}

struct Dda {
    int cx, cy, cz, sx, sy, sz;
    float tmx, tmy, tmz, tdx, tdy, tdz;
    float t;
};

template <class M>
__device__ __forceinline__ void dda_axis(const M &m, int k, float x, float w, float iw, int &c, int &st,
                                         float &tm, float &td)
{
    const float cs = m.mc_size(k);
    c = min(max(__float2int_rd((x - m.lo(k)) * m.mc_inv(k)), 0), m.mc_dims(k) - 1);
    if (w > 0.0f) {
        st = 1;
        tm = (m.lo(k) + (float)(c + 1) * cs - x) * iw;
        td = cs * iw;
    } else if (w < 0.0f) {
        st = -1;
        tm = (m.lo(k) + (float)c * cs - x) * iw;
        td = -cs * iw;
    } else {
        st = 0;
        tm = FLT_MAX;
        td = FLT_MAX;
    }
}

template <class M>
__device__ __forceinline__ void dda_init(const M &m, Dda &d, float3 x, float3 w, float3 iw)
{
    dda_axis(m, 0, x.x, w.x, iw.x, d.cx, d.sx, d.tmx, d.tdx);
    dda_axis(m, 1, x.y, w.y, iw.y, d.cy, d.sy, d.tmy, d.tdy);
    dda_axis(m, 2, x.z, w.z, iw.z, d.cz, d.sz, d.tmz, d.tdz);
    d.t = 0.0f;
}

// Spends tau from d.t on; returns the tentative distance (and its cell's majorant times the
// margin factor in sb), or FLT_MAX once t_end is reached first. Ties between axes go to the lowest
// axis.
template <class M>
__device__ __forceinline__ float dda_advance(const M &m, Dda &d, int b, float tau, float t_end, float &sb,
                                             uint32_t &walks)
{
    const int mx = m.mc_dims(0), my = m.mc_dims(1), mz = m.mc_dims(2);
    for (int guard = 0; guard < (1 << 16); ++guard) {
        ++walks;
        const int cell = (d.cz * my + d.cy) * mx + d.cx;
        const int k = m.mc_empty_radius(cell);
        if (k > 0) {
            // the cube of cells within Chebyshev distance k - 1 holds no matter (majorant 0): leave
            // it in one move, spending no optical budget
            const float kx = d.tmx + (float)(k - 1) * d.tdx;
            const float ky = d.tmy + (float)(k - 1) * d.tdy;
            const float kz = d.tmz + (float)(k - 1) * d.tdz;
            int ax = 0;
            float tn = kx;
            if (ky < tn) { ax = 1; tn = ky; }
            if (kz < tn) { ax = 2; tn = kz; }
            if (tn >= t_end) { d.t = t_end; sb = 0.0f; return FLT_MAX; }
            d.t = fmaxf(tn, d.t);
            // cross k boundaries on the exit axis, and those the ray passes on the other two
            const int nx = ax == 0 ? k : (d.tmx <= tn ? min(k - 1, (int)((tn - d.tmx) / d.tdx) + 1) : 0);
            const int ny = ax == 1 ? k : (d.tmy <= tn ? min(k - 1, (int)((tn - d.tmy) / d.tdy) + 1) : 0);
            const int nz = ax == 2 ? k : (d.tmz <= tn ? min(k - 1, (int)((tn - d.tmz) / d.tdz) + 1) : 0);
            d.cx += d.sx * nx;
            d.cy += d.sy * ny;
            d.cz += d.sz * nz;
            d.tmx += (float)nx * d.tdx;
            d.tmy += (float)ny * d.tdy;
            d.tmz += (float)nz * d.tdz;
            if (d.cx < 0 || d.cx >= mx || d.cy < 0 || d.cy >= my || d.cz < 0 || d.cz >= mz) {
                sb = 0.0f;
                return FLT_MAX;
            }
            continue;
        }
        const float sbc = cell_majorant(m, cell, b) * m.margin();
        int ax = 0;
        float tn = d.tmx;
        if (d.tmy < tn) { ax = 1; tn = d.tmy; }
        if (d.tmz < tn) { ax = 2; tn = d.tmz; }
        const float t1 = fmaxf(fminf(tn, t_end), d.t);
        const float opt = sbc * (t1 - d.t);
        if (sbc > 0.0f && tau < opt) {
            d.t += tau / sbc;
            sb = sbc;
            return d.t;
        }
        tau -= opt;
        d.t = t1;
        if (t1 >= t_end) { sb = sbc; return FLT_MAX; }
        bool out;
        if (ax == 0) {
            d.cx += d.sx;
            d.tmx += d.tdx;
            out = d.cx < 0 || d.cx >= mx;
        } else if (ax == 1) {
            d.cy += d.sy;
            d.tmy += d.tdy;
            out = d.cy < 0 || d.cy >= my;
        } else {
            d.cz += d.sz;
            d.tmz += d.tdz;
            out = d.cz < 0 || d.cz >= mz;
        }
        if (out) { sb = sbc; return FLT_MAX; }
    }
    sb = 0.0f;
    return FLT_MAX;
}

// The cell of x and its stored distance to matter (.w), read on its own so that a caller can issue
// this load beside the medium lookup at the same point instead of after it (6 % on the Cornell
// box); empty_cube_exit_at then finishes the exit distance.
template <class M>
__device__ __forceinline__ int4 empty_cell(const M &m, float3 x)
{
    const int cx = min(max(__float2int_rd((x.x - m.lo(0)) * m.mc_inv(0)), 0), m.mc_dims(0) - 1);
    const int cy = min(max(__float2int_rd((x.y - m.lo(1)) * m.mc_inv(1)), 0), m.mc_dims(1) - 1);
    const int cz = min(max(__float2int_rd((x.z - m.lo(2)) * m.mc_inv(2)), 0), m.mc_dims(2) - 1);
    return make_int4(cx, cy, cz, m.mc_empty_radius((cz * m.mc_dims(1) + cy) * m.mc_dims(0) + cx));
}

// Distance along (x, w) to leave the empty cube of cells around x (0 when x's cell may hold
// matter): the cube of cells within Chebyshev distance k - 1 of x's cell c, k = c.w its stored
// distance.
template <class M>
__device__ __forceinline__ float empty_cube_exit_at(const M &m, int4 c, float3 x, float3 w, float3 iw)
{
    const int k = c.w;
    if (k == 0) return 0.0f;
    float best = FLT_MAX;
    const float xs[3] = {x.x, x.y, x.z}, ws[3] = {w.x, w.y, w.z}, is[3] = {iw.x, iw.y, iw.z};
    const int cs_[3] = {c.x, c.y, c.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ws[a] == 0.0f) continue;
        const float edge = ws[a] > 0.0f ? (float)(cs_[a] + k) : (float)(cs_[a] - k + 1);
        const float t = (m.lo(a) + edge * m.mc_size(a) - xs[a]) * is[a];
        best = fminf(best, t);
    }
    return fmaxf(best, 0.0f);
}

// The same in one call.
template <class M>
__device__ __forceinline__ float empty_cube_exit(const M &m, float3 x, float3 w, float3 iw)
{
    const int cx = min(max(__float2int_rd((x.x - m.lo(0)) * m.mc_inv(0)), 0), m.mc_dims(0) - 1);
    const int cy = min(max(__float2int_rd((x.y - m.lo(1)) * m.mc_inv(1)), 0), m.mc_dims(1) - 1);
    const int cz = min(max(__float2int_rd((x.z - m.lo(2)) * m.mc_inv(2)), 0), m.mc_dims(2) - 1);
    const int k = m.mc_empty_radius((cz * m.mc_dims(1) + cy) * m.mc_dims(0) + cx);
    if (k == 0) return 0.0f;
    float best = FLT_MAX;
    const float xs[3] = {x.x, x.y, x.z}, ws[3] = {w.x, w.y, w.z}, is[3] = {iw.x, iw.y, iw.z};
    const int cs_[3] = {cx, cy, cz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ws[a] == 0.0f) continue;
        const float edge = ws[a] > 0.0f ? (float)(cs_[a] + k) : (float)(cs_[a] - k + 1);
        const float t = (m.lo(a) + edge * m.mc_size(a) - xs[a]) * is[a];
        best = fminf(best, t);
    }
    return fmaxf(best, 0.0f);
}

// ---------------------------------------------------------------------------------------------
// Directions (Sec. 2.1: isotropic scattering and emission; Lambertian walls and lights).
// Cosine-weighted about sign * e_axis, tangents e_{axis+1}, e_{axis+2}.
__device__ __forceinline__ float3 cosine_dir(float u1, float u2, int axis, float sign)
{
    const float r = sqrt_approx(u1);
    float s, c;
    __sincosf(TWO_PI * u2, &s, &c);
    const float zl = sqrt_approx(fmaxf(0.0f, 1.0f - u1));
    const float a = sign * zl, bx = r * c, by = r * s;
    // component axis = a, (axis+1)%3 = bx, (axis+2)%3 = by
    if (axis == 0) return make_float3(a, bx, by);
    if (axis == 1) return make_float3(by, a, bx);
    return make_float3(bx, by, a);
}

__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ void set_comp(float3 &v, int k, float a)
{
    if (k == 0) v.x = a; else if (k == 1) v.y = a; else v.z = a;
}

// ---------------------------------------------------------------------------------------------
// Dielectric faces and glossy walls (Sec. 5's glass vials and glossy Cornell box; the paper does not
// specify them, these are the standard choices). Reflectance of unpolarised light at a smooth
// interface from index n1 into n2 for a ray meeting it at cos_i, eta = n1 / n2 (Fresnel's
// equations divided through by n2); beyond the critical angle everything is reflected. cos_t: the
// refracted ray's cosine (Snell: sin_t = eta sin_i).
__device__ __forceinline__ float fresnel_refl(float cos_i, float eta, float &cos_t)
{
    const float sin_t2 = eta * eta * fmaxf(0.0f, 1.0f - cos_i * cos_i);
    if (sin_t2 >= 1.0f) {
        cos_t = 0.0f;
        return 1.0f;
    }
    const float ct = sqrtf(1.0f - sin_t2);
    cos_t = ct;
    const float rs = (eta * cos_i - ct) / (eta * cos_i + ct);
    const float rp = (cos_i - eta * ct) / (cos_i + eta * ct);
    return 0.5f * (rs * rs + rp * rp);
}

// Normalised Phong lobe about the unit vector r: cos alpha = u1^(1/(e+1)), azimuth 2 pi u2 in r's
// tangent frame (Duff et al., "Building an orthonormal basis, revisited", JCGT 2017).
__device__ __forceinline__ float3 phong_dir(float u1, float u2, float3 r, float e)
{
    const float ca = __powf(u1, 1.0f / (e + 1.0f));
    const float sa = sqrtf(fmaxf(0.0f, 1.0f - ca * ca));
    float sn, cs;
    __sincosf(TWO_PI * u2, &sn, &cs);
    const float sg = copysignf(1.0f, r.z);
    const float a = -1.0f / (sg + r.z);
    const float b = r.x * r.y * a;
    const float3 t1 = make_float3(1.0f + sg * r.x * r.x * a, sg * b, -sg * r.x);
    const float3 t2 = make_float3(b, sg + r.y * r.y * a, -r.y);
    const float p = sa * cs, q = sa * sn;
    return make_float3(p * t1.x + q * t2.x + ca * r.x, p * t1.y + q * t2.y + ca * r.y,
                       p * t1.z + q * t2.z + ca * r.z);
}

// The wall BRDF without its albedo, times cos_o, toward o for a photon with mirror direction r:
// (1 - g) cos_o / pi + g (e + 2)/(2 pi) cos^e alpha cos_o.
__device__ __forceinline__ float wall_lobe_cos(float g, float e, float3 r, float3 o, float cos_o)
{
    const float ca = r.x * o.x + r.y * o.y + r.z * o.z;
    const float lobe = ca > 0.0f ? (e + 2.0f) * (0.5f * INV_PI) * __powf(ca, e) : 0.0f;
    return ((1.0f - g) * INV_PI + g * lobe) * cos_o;
}

// Vertex kind of a connection whose weight already holds the vertex's intensity toward the sensor
// (glossy wall vertices): the connection multiplies by importance and transmittance only.
constexpr int LAMB_WEIGHTED = 6;

// ---------------------------------------------------------------------------------------------
// Sensor connection (Eq. 3-6). `lamb` < 0: isotropic vertex, intensity w/(4 pi); otherwise a
// Lambertian vertex with normal sign*e_axis (lamb = 2*axis + (sign > 0)), intensity w cos/pi.
// Transmittance: analytic in homogeneous media, else ratio tracking
//   T = prod_k (1 - sigma_t(x_k)/sigma_bar) over majorant-distributed points x_k,
// with roulette once the estimate falls below RT_RR_THRESHOLD (survival T / RT_RR_THRESHOLD; in the
// adjoint replay survival 1/2 below RT_RR_ADJ_THRESHOLD).
// Geometry of a connection: direction to the sensor, distance to leave the box, intensity x
// importance (f * geom) and the film pixel; ok = false when the vertex does not see the sensor.
struct ConnGeom {
    float3 dir, idr;   // direction to the sensor and its componentwise inverse
    float tl, gf;
    int pix;
    bool ok;
};

__device__ __forceinline__ ConnGeom connect_geom(const SceneDev &S, const Smem &sm, float3 x, int lamb)
{
    ConnGeom g;
    g.ok = false;
    float geom, r2 = 0.0f;
    int px, py;
    float3 dir;
    if (S.sensor_kind == FLR_SENSOR_ORTHO) {
        dir = make_float3(S.s_view[0], S.s_view[1], S.s_view[2]);
        const float dx = x.x - S.s_origin[0], dy = x.y - S.s_origin[1], dz = x.z - S.s_origin[2];
        const float su = dx * S.s_U[0] + dy * S.s_U[1] + dz * S.s_U[2];
        const float sv = dx * S.s_V[0] + dy * S.s_V[1] + dz * S.s_V[2];
        if (!(su >= 0.0f && su < 1.0f && sv >= 0.0f && sv < 1.0f)) return g;
        px = min(__float2int_rd(su * (float)S.W), S.W - 1);
        py = min(__float2int_rd(sv * (float)S.H), S.H - 1);
        geom = S.inv_A_pix;
    } else {
        const float vx = x.x - S.s_origin[0], vy = x.y - S.s_origin[1], vz = x.z - S.s_origin[2];
        r2 = vx * vx + vy * vy + vz * vz;
        const float zf = vx * S.s_view[0] + vy * S.s_view[1] + vz * S.s_view[2];
        if (!(zf > 0.0f)) return g;
        const float izf = __fdividef(1.0f, zf);
        const float X = (vx * S.s_U[0] + vy * S.s_U[1] + vz * S.s_U[2]) * izf;
        const float Y = (vx * S.s_V[0] + vy * S.s_V[1] + vz * S.s_V[2]) * izf;
        const float sx = 0.5f * (X * S.inv_tan_x + 1.0f);
        const float sy = 0.5f * (Y * S.inv_tan_y + 1.0f);
        if (!(sx >= 0.0f && sx < 1.0f && sy >= 0.0f && sy < 1.0f)) return g;
        px = min(__float2int_rd(sx * (float)S.W), S.W - 1);
        py = min(__float2int_rd(sy * (float)S.H), S.H - 1);
        const float ir = rsqrtf(r2);
        dir = make_float3(-vx * ir, -vy * ir, -vz * ir);
        const float ct = zf * ir;
        geom = __fdividef(S.inv_A_pix, r2 * ct * ct * ct);
    }
    float f;
    if (lamb == LAMB_WEIGHTED) {
        f = 1.0f;
    } else if (lamb >= 0) {
        const int axis = lamb >> 1;
        const float co = (lamb & 1) ? comp(dir, axis) : -comp(dir, axis);
        if (!(co > 0.0f)) return g;
        f = co * INV_PI;
    } else {
        f = INV_4PI;
    }
    const MedS m{S, sm};
    int face;
    const float3 idr = inv_dir(dir);
    const float tl = exit_distance(m, x, dir, idr, face);
    if (face < 0) return g;
    if (S.wall_mask & (1 << face)) return g;
    // out through a dielectric face at normal incidence: (1 - F(0)) / ior^2 of the radiance
    if (S.dielectric) f *= S.iface_exit;
    if (S.sensor_kind == FLR_SENSOR_PINHOLE && tl * tl > r2) return g;
    g.dir = dir;
    g.idr = idr;
    g.tl = tl;
    g.gf = f * geom;
    g.pix = py * S.W + px;
    g.ok = true;
    return g;
}

// Transmittance estimate along the connection (Eq. 6): analytic in homogeneous media, else ratio
// tracking T = prod_k (1 - sigma_t(x_k)/sigma_bar) over majorant-distributed points with roulette
// below RT_RR_THRESHOLD (ADJ: the adjoint's rule). The sink G sees every ratio-tracking point (the adjoint
// accumulates d log T there); NoSink is the forward's.
struct NoSink {
    __device__ __forceinline__ void point(float3, int, float, float) const {}
    __device__ __forceinline__ void homogeneous(float) const {}
};

template <class G, bool OPT = true, bool MC = OPT, bool ADJ = false, uint32_t SLOT0 = 2u, bool LZ = false>
__device__ __forceinline__ float transmittance(const SceneDev &S, const RunDev &R, const Smem &sm,
                                               float3 x, float3 dir, float tl, int b, uint64_t pid,
                                               uint32_t step, RegCnt &rc, const G &sink)
{
    const MedS_<OPT, MC> m{S, sm};
    const float sb = sm.maj[b];
    float T = 1.0f;
    if (!(sb > 0.0f)) return T;
    if (S.homogeneous) {
        sink.homogeneous(tl);
        return __expf(-sigma_t_at(m, x, b) * tl);
    }
    if (OPT && MC && S.mc > 0) {
        // ratio tracking against the local majorants: one uniform per tentative point
        Dda dd;
        dda_init(m, dd, x, dir, inv_dir(dir));
        MarchRng rg = march_rng(R, pid, step, SLOT0);
        int it = 0;
        for (; it < MAX_CONNECT_STEPS; ++it) {
            const float u = march_next(rg);
            float sbc;
            const float t = dda_advance(m, dd, b, -__logf(1.0f - u), tl, sbc, rc.cell_walks);
            if (t >= tl) break;
            rc.connect_steps++;
            const float3 p = make_float3(x.x + t * dir.x, x.y + t * dir.y, x.z + t * dir.z);
            const float st = sigma_t_at(m, p, b);
            sink.point(p, b, st, sbc);
            T *= fmaxf(0.0f, 1.0f - st / sbc);
            if (T < (ADJ ? RT_RR_ADJ_THRESHOLD : RT_RR_THRESHOLD)) {
                const float u2 = march_next(rg);
                if (ADJ ? u2 < 0.5f : u2 * RT_RR_THRESHOLD < T) {
                    T = ADJ ? 2.0f * T : RT_RR_THRESHOLD;
                } else {
                    T = 0.0f;
                    break;
                }
            }
        }
        if (it == MAX_CONNECT_STEPS) {
            T = 0.0f;
            cnt_add(sm, FLR_C_CONNECT_BUDGET);
        }
        return T;
    }
    const float isb = sm.inv_maj[b];
    float t = 0.0f;
    MarchRng rg = march_rng(R, pid, step, SLOT0);
    int it = 0;
    constexpr bool LAZY = LZ && !ADJ && std::is_same<G, NoSink>::value;
    for (; it < MAX_CONNECT_STEPS; ++it) {
        const float u = march_next(rg);
        t -= __logf(1.0f - u) * isb;
        if (t >= tl) break;
        rc.connect_steps++;
        float u2 = -1.0f;   // the roulette coin, when the bound below draws it first
        if (LAZY && !S.homogeneous && S.solvent == nullptr) {
            // a coin that fails against the bound of the updated estimate ends the march
            // whatever sigma_t is here (minorant_known)
            const float tu = T * fmaxf(0.0f, 1.0f - (S.sigma_s + S.sigma_a0) * isb);
            if (tu < RT_RR_THRESHOLD) {
                u2 = march_next(rg);
                if (!(u2 * RT_RR_THRESHOLD < tu)) {
                    T = 0.0f;
                    break;
                }
            }
        }
        const float3 p = make_float3(x.x + t * dir.x, x.y + t * dir.y, x.z + t * dir.z);
        const float st = sigma_t_at(m, p, b);
        sink.point(p, b, st, sb);
        T *= fmaxf(0.0f, 1.0f - st * isb);
        if (OPT && S.sk > 0 && st == 0.0f) {
            // no matter in the cube around this point: continue sampling from its far side
            const float tl2 = empty_cube_exit(m, p, dir, inv_dir(dir));
            if (tl2 > 0.0f) {
                t += tl2;
                rc.cell_walks++;
            }
        }
        if (T < (ADJ ? RT_RR_ADJ_THRESHOLD : RT_RR_THRESHOLD)) {
            if (u2 < 0.0f) u2 = march_next(rg);
            if (ADJ ? u2 < 0.5f : u2 * RT_RR_THRESHOLD < T) {
                T = ADJ ? 2.0f * T : RT_RR_THRESHOLD;
            } else {
                T = 0.0f;
                break;
            }
        }
    }
    if (it == MAX_CONNECT_STEPS) {
        T = 0.0f;
        cnt_add(sm, FLR_C_CONNECT_BUDGET);
    }
    return T;
}

// Sensor connection (Eq. 3-6). `lamb` < 0: isotropic vertex, intensity w/(4 pi); otherwise a
// Lambertian vertex with normal sign*e_axis (lamb = 2*axis + (sign > 0)), intensity w cos/pi.
template <bool OPT = true, bool LZ = false>
__device__ __forceinline__ void connect(const SceneDev &S, const RunDev &R, const Smem &sm,
                                        float3 x, int b, float w, int lamb, uint64_t pid,
                                        uint32_t step, RegCnt &rc)
{
    const ConnGeom g = connect_geom(S, sm, x, lamb);
    if (!g.ok) return;
    rc.connections++;
    const float T = transmittance<NoSink, OPT, OPT, false, 2u, LZ>(S, R, sm, x, g.dir, g.tl, b, pid, step, rc,
                                                                 NoSink{});
    const float val = w * g.gf * T * R.film_scale;
    if (val > 0.0f) film_add(S, R, (size_t)g.pix * S.B + b, val);
}

// ---------------------------------------------------------------------------------------------
// Path state and one tracking step.
struct Path {
    float3 x, w, iw;
    float wt;
    int bin;
    uint32_t step;
    int n_events, n_inel, fl;
    uint64_t pid;
    bool alive;
};

// A connection requested by a step: position, bin, weight, vertex kind, and the RNG coordinates.
struct Conn {
    float3 x;
    float w;
    int bin, lamb;
    uint64_t pid;
    uint32_t step;
    bool valid;
};

__device__ __forceinline__ int sample_cdf(const float *cdf, int B, float u)
{
    // min{ i : cdf[i] > u }; cdf is non-decreasing with cdf[B-1] = 1 > u.
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ void finish(const RunDev &R, Path &p)
{
    p.alive = false;
    if (R.path_events) R.path_events[p.pid - R.path_offset] = (uint32_t)p.n_events;
}

template <class M>
__device__ __forceinline__ Conn spawn(const M &m, const RunDev &R, const Smem &sm, uint64_t pid,
                                      Path &p, int *emitter = nullptr)
{
    cnt_add(sm, FLR_C_PATHS);
    const U4 s0 = m.rng(R, pid, STEP_SPAWN, 0u);
    int k = 0;
    const int ne = m.n_emitters();
    while (k < ne - 1 && !(m.em_cdf(k) > s0.a)) ++k;
    if (emitter) *emitter = k;
    const EmitterDev &e = m.em(k);
    p.x = make_float3(e.origin[0] + s0.b * e.eu[0] + s0.c * e.ev[0],
                      e.origin[1] + s0.b * e.eu[1] + s0.c * e.ev[1],
                      e.origin[2] + s0.b * e.eu[2] + s0.c * e.ev[2]);
    p.bin = e.bin;
    p.wt = 1.0f;
    p.step = 0;
    p.n_events = 0;
    p.n_inel = 0;
    p.fl = 0;
    p.pid = pid;
    p.alive = true;
    Conn c;
    c.valid = false;
    if (e.kind == FLR_SOURCE_LAMBERTIAN) {
        const U4 s1 = m.rng(R, pid, STEP_SPAWN, 1u);
        p.w = cosine_dir(s0.d, s1.a, e.axis, e.sign);
        if (m.sensor() && !R.paper_mode) {   // the paper's film holds fluorescence only
            c = Conn{p.x, p.wt, p.bin, 2 * e.axis + (e.sign > 0.0f ? 1 : 0), pid, STEP_SPAWN, true};
        }
    } else {
        p.w = make_float3(e.dir[0], e.dir[1], e.dir[2]);
    }
    if (m.iface() && e.entry >= 0) {
        // entering the solution through a dielectric face (coin: spawn slot 1, word 1): the
        // Fresnel-reflected share leaves through that face, the rest refracts inward by Snell
        const U4 s1 = m.rng(R, pid, STEP_SPAWN, 1u);
        const int f = e.entry, k = f >> 1;
        const float wk = comp(p.w, k);
        float ct;
        const float F = fresnel_refl(fabsf(wk), m.inv_ior(), ct);
        if (s1.b < F) {
            cnt_add(sm, FLR_C_IFACE_REFLECTIONS);
            m.tally(tal_face(m.B()) + f * m.B() + p.bin, p.wt);
            cnt_add(sm, FLR_C_ESCAPES);
            finish(R, p);
            return c;
        }
        const float eta = m.inv_ior();
        p.w = make_float3(p.w.x * eta, p.w.y * eta, p.w.z * eta);
        set_comp(p.w, k, wk > 0.0f ? ct : -ct);
    }
    p.iw = inv_dir(p.w);
    return c;
}

// Decisions that need no grid read. Where a medium has grids but no solvent mask (s(x) = 1), every
// point has sigma_t >= sigma_s + sigma_a0 (the dye terms are >= 0) and sigma_t <= sigma_bar. So a
// tentative collision with u_real sigma_bar < sigma_s + sigma_a0 is real, and then a scatter if
// u_event sigma_bar < sigma_s, whatever the concentrations there; and a ratio-tracking step whose
// roulette coin fails against T (1 - (sigma_s + sigma_a0) / sigma_bar), an upper bound of the
// updated estimate, ends its march whatever they are. The bounds are formed with the operations
// coeffs_at and the march use (fp32 rounding is monotone), so a decision taken from them is the
// one the grid read would give: the same paths, tallies and film, fewer reads. In the dense
// scattering media of high albedo most decisions are of this kind. Forward passes only: the
// adjoint's observers need the coefficients at every point.
template <class M>
__device__ __forceinline__ bool minorant_known(const M &m)
{
    return M::kLazy && !m.homogeneous() && m.solvent() == nullptr;
}

// Observer of the tracking decisions (the adjoint replay scores them); NoObs is the forward's.
struct NoObs {
    __device__ __forceinline__ void null_event(float3, int, const Coeffs &, float) const {}
    __device__ __forceinline__ void real_event(float3, int, const Coeffs &, int) const {}
};

// One tracking step (null or real collision, wall bounce or escape). Returns the connection the
// step asks for, if any.
template <class M, class Obs = NoObs>
__device__ __forceinline__ Conn track_step(const M &m, const RunDev &R, const Smem &sm, Path &p,
                                           RegCnt &rc, const Obs &obs = Obs())
{
    Conn c;
    c.valid = false;
    if ((long long)p.step >= R.max_steps) {
        cnt_add(sm, FLR_C_STEP_BUDGET);
        finish(R, p);
        return c;
    }
    rc.steps++;
    const U4 b0 = m.rng(R, p.pid, p.step, 0u);
    // The second block serves real events and wall bounces only, but some lane of a warp nearly
    // always needs it: drawing it here, beside the first, overlaps the two Philox chains.
    const U4 b1 = m.rng(R, p.pid, p.step, 1u);
    int face;
    const float te = exit_distance(m, p.x, p.w, p.iw, face);
    float sb, tf;
    if (m.macro()) {
        Dda dd;
        dda_init(m, dd, p.x, p.w, p.iw);
        tf = dda_advance(m, dd, p.bin, -__logf(1.0f - b0.a), te, sb, rc.cell_walks);
    } else {
        sb = m.maj(p.bin);
        tf = sb > 0.0f ? -__logf(1.0f - b0.a) * m.inv_maj(p.bin) : FLT_MAX;
    }
    const uint32_t step = p.step;
    p.step++;
    // the new direction: isotropic (dax < 0) or cosine about dsg * e_dax, from (du1, du2)
    int dax = -1;
    float dsg = 1.0f, du1 = b0.d, du2 = b1.a;
    int gw = 0;   // glossy wall bounce: 1 diffuse lobe, 2 Phong lobe (direction already drawn)
    if (tf >= te) {
        p.x = make_float3(p.x.x + te * p.w.x, p.x.y + te * p.w.y, p.x.z + te * p.w.z);
        if (face < 0) {  // no direction component: cannot happen for unit directions
            cnt_add(sm, FLR_C_NONFINITE);
            finish(R, p);
            return c;
        }
        if (!(m.wall_mask() & (1 << face))) {
            if (m.iface() && m.dielectric()) {
                // a dielectric face from inside: Fresnel reflection (an event; the coin is the
                // step's unused u_real), else refraction out of the solution (an escape)
                const int k = face >> 1;
                float ct;
                const float F = fresnel_refl(fabsf(comp(p.w, k)), m.ior(), ct);
                if (b0.b < F) {
                    if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
                    p.n_events++;
                    rc.events++;
                    cnt_add(sm, FLR_C_IFACE_REFLECTIONS);
                    set_comp(p.w, k, -comp(p.w, k));
                    set_comp(p.x, k, (face & 1) ? m.hi(k) : m.lo(k));
                    p.iw = inv_dir(p.w);
                    if (p.n_events >= R.n_rr) {
                        const float q = fminf(p.wt, 1.0f);
                        if (!(b1.c < q)) { cnt_add(sm, FLR_C_RR_KILLS); finish(R, p); return c; }
                        p.wt = p.wt < 1.0f ? 1.0f : p.wt;
                    }
                    return c;
                }
            }
            m.tally(tal_face(m.B()) + (p.fl * 6 + face) * m.B() + p.bin, p.wt);
            cnt_add(sm, FLR_C_ESCAPES);
            finish(R, p);
            return c;
        }
        // the paper's model drops excitation light reflected by a wall before any emission
        if (R.paper_mode && !p.fl) { cnt_add(sm, FLR_C_VF_REJECTED); finish(R, p); return c; }
        if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
        p.n_events++;
        rc.events++;
        cnt_add(sm, FLR_C_WALL_BOUNCES);
        if (R.analog) {
            if (!(b1.d < m.wall_albedo())) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
        } else {
            p.wt *= m.wall_albedo();
            if (p.wt == 0.0f) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
        }
        dax = face >> 1;
        dsg = (face & 1) ? -1.0f : 1.0f;
        if (dax == 0) p.x.x = (face & 1) ? m.hi(0) : m.lo(0);
        else if (dax == 1) p.x.y = (face & 1) ? m.hi(1) : m.lo(1);
        else p.x.z = (face & 1) ? m.hi(2) : m.lo(2);
        du1 = b0.c;
        du2 = b0.d;
        if (m.iface() && m.wall_gloss() > 0.0f) {
            // glossy wall: the sensor sees the whole BRDF (evaluated here, so the connection carries
            // it in its weight); the path continues in the Phong lobe about the mirror direction
            // with probability g (lobe choice: u_dir2; weight (e + 2)/(e + 1) cos_o, ended below
            // the wall), else in the diffuse lobe
            float3 r = p.w;
            set_comp(r, dax, -comp(r, dax));
            const float g = m.wall_gloss(), e = m.wall_exp();
            gw = 1;
            if (m.sensor()) {
                const float3 od = m.sensor_dir(p.x);
                const float co = dsg * comp(od, dax);
                if (co > 0.0f) c = Conn{p.x, p.wt * wall_lobe_cos(g, e, r, od, co), p.bin, LAMB_WEIGHTED, p.pid, step, true};
            }
            if (b1.a < g) {
                p.w = phong_dir(du1, du2, r, e);
                const float co = dsg * comp(p.w, dax);
                if (!(co > 0.0f)) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
                p.wt *= (e + 2.0f) / (e + 1.0f) * co;
                gw = 2;
            }
        }
    } else {
        p.x = make_float3(p.x.x + tf * p.w.x, p.x.y + tf * p.w.y, p.x.z + tf * p.w.z);
        // a real scatter whatever the concentrations (minorant_known): no grid read
        const bool sure = std::is_same<Obs, NoObs>::value && minorant_known(m) &&
                          b0.b * sb < m.sigma_s() + m.sigma_a0() && b0.c * sb < m.sigma_s();
        Coeffs k;
        if (!sure) {
            // the empty-space distance is read beside the coefficients, not after them
            const int4 ec = m.skip() ? empty_cell(m, p.x) : make_int4(0, 0, 0, 0);
            k = coeffs_at(m, p.x, p.bin);
            if (k.total > sb) cnt_add(sm, FLR_C_MAJORANT_VIOLATIONS);
            if (!(b0.b * sb < k.total)) {
                rc.nulls++;
                obs.null_event(p.x, p.bin, k, sb);
                if (m.skip() && k.total == 0.0f) {
                    // every tentative collision in the empty cube around here would be a null: leave it
                    float tl = empty_cube_exit_at(m, ec, p.x, p.w, p.iw);
                    if (tl > 0.0f) {
                        tl = fminf(tl, te - tf);
                        p.x = make_float3(p.x.x + tl * p.w.x, p.x.y + tl * p.w.y, p.x.z + tl * p.w.z);
                        rc.cell_walks++;
                    }
                }
                return c;
            }
        }
        if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
        p.n_events++;
        rc.events++;
        // particle type in proportion to its coefficient (Sec. 4.1)
        int ev = -1;
        const int D = m.D();
        if (!sure) {
            const float ue = b0.c * k.total;
            float acc = k.scat;
            if (!(ue < acc)) {
                ev = D;
#pragma unroll
                for (int d = 0; d < MAXD; ++d) {
                    if (d < D && ev == D) {
                        acc += k.dye[d];
                        if (ue < acc) ev = d;
                    }
                }
            }
            obs.real_event(p.x, p.bin, k, ev);
        }
        if (ev < 0) {
            rc.scatters++;
            // the paper's model drops scattered excitation light (Sec. 4.1)
            if (R.paper_mode && !p.fl) { cnt_add(sm, FLR_C_VF_REJECTED); finish(R, p); return c; }
        } else if (ev < D) {
            cnt_add(sm, FLR_C_DYE_ABSORPTIONS);
            m.tally(tal_absorbed(m.B()) + ev * m.B() + p.bin, p.wt);
            if ((R.max_inelastic >= 0 && p.n_inel >= R.max_inelastic) || (R.paper_mode && p.n_inel >= 1)) {
                cnt_add(sm, FLR_C_VF_REJECTED);
                finish(R, p);
                return c;
            }
            if (R.analog) {
                if (!(b1.d < m.qy(ev))) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
            } else {
                p.wt *= m.qy(ev);
                if (p.wt == 0.0f) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
            }
            p.bin = sample_cdf(m.cdf(ev), m.B(), b1.b);
            m.tally(tal_emitted(m.B()) + ev * m.B() + p.bin, p.wt);
            cnt_add(sm, FLR_C_EMISSIONS);
            p.n_inel++;
            p.fl = 1;
        } else {
            m.tally(tal_absorbed(m.B()) + D * m.B() + p.bin, p.wt);
            cnt_add(sm, FLR_C_ABSORBED_DEAD);
            finish(R, p);
            return c;
        }
    }
    // One direction sampler for scattering and emission (isotropic: z = 1 - 2 u1, phi = 2 pi u2)
    // and wall bounces (cosine-weighted, the operations of cosine_dir): a warp whose lanes scatter
    // and bounce runs it once instead of both (measured 3 % on the Cornell box).
    if (gw != 2) {
        const float u1 = du1;
        float sn, cs;
        __sincosf(TWO_PI * du2, &sn, &cs);
        float a, r;
        if (dax < 0) {
            a = 1.0f - 2.0f * u1;
            r = sqrt_approx(fmaxf(0.0f, 1.0f - a * a));
        } else {
            r = sqrt_approx(u1);
            a = dsg * sqrt_approx(fmaxf(0.0f, 1.0f - u1));
        }
        const float bx = r * cs, by = r * sn;
        p.w = dax == 0 ? make_float3(a, bx, by) : (dax == 1 ? make_float3(by, a, bx) : make_float3(bx, by, a));
    }
    p.iw = inv_dir(p.w);
    if (m.sensor() && gw == 0) c = Conn{p.x, p.wt, p.bin, dax < 0 ? -1 : 2 * dax + (dsg > 0.0f ? 1 : 0), p.pid, step, true};
    if (p.n_events >= R.n_rr) {
        const float q = fminf(p.wt, 1.0f);
        if (!(b1.c < q)) { cnt_add(sm, FLR_C_RR_KILLS); finish(R, p); return c; }
        p.wt = p.wt < 1.0f ? 1.0f : p.wt;   // w / min(w, 1), exactly
    }
    if (!(isfinite(p.wt) && isfinite(p.x.x) && isfinite(p.x.y) && isfinite(p.x.z))) {
        cnt_add(sm, FLR_C_NONFINITE);
        finish(R, p);
        c.valid = false;
    }
    return c;
}

// ---------------------------------------------------------------------------------------------
// Block prologue / epilogue: stage tables, zero and flush block tallies and counters.
struct SmemLayout {
    int tab_floats, tal_off_bytes, cnt_off_bytes, queue_off_bytes, total_bytes;
    bool tal_global;   // tallies go straight to global memory (their shared space holds queues)
};

// Per-warp connection queue of the warp-regrouped form: capacity and drain threshold. A drain starts
// once WQ_DRAIN records wait; one tracking round adds at most 32, so the queue never wraps. Longer
// queues drain less often and amortise each drain's tail (measured on the Cornell box: 128 -> 256 ->
// 320 records gave 26.0 -> 24.0 -> 23.6 ms per step, with the drains of that time); five blocks of
// 128 threads (WARP_BLOCK, at most 102 registers) per SM measured 3 % faster than two blocks of 256
// with 416-record queues. With drains that claim every iteration the optimum moved down: 256
// records (drained at 224) gave 12.93 ms, against 13.14 (320 / 288), 12.97 (224 / 192), 13.2
// (192 / 160) and 13.45 ms (160 / 128); the block count stays five (registers), and the shared
// memory no longer held by queues is left to the L1. The adjoint's and the local-majorant
// instances keep four blocks (128 registers): with five they spill.
constexpr int WARP_BLOCK = 128;   // threads per block of the warp-regrouped form
constexpr int WQ_CAP = 256;
constexpr int WQ_DRAIN = 224;
constexpr int SPAWN_MIN = 8;   // lanes that start new paths together
static_assert(WQ_DRAIN + 31 < WQ_CAP, "warp queue overflow");

// Path-pool form (k_trace_pool): slots per warp, connection queue, per-warp shared memory.
constexpr int POOL_SLOTS = 64;   // lane l keeps the states of slots l and l + 32
static_assert(POOL_SLOTS == 64, "k_trace_pool's slot bookkeeping assumes two slots per lane");
// Queues of 160 records (drained at 128) let five blocks of 128 threads share an SM: measured on
// the Cornell box 14.46 ms per step against 15.45 ms with 224 records and four blocks, 14.97 ms
// with 128 records and 15.46 ms with 192.
constexpr int PQ_CAP = 160;    // connection records per warp
constexpr int PQ_DRAIN = 128;  // a round adds at most 32 records, so the queue never wraps
static_assert(PQ_DRAIN + 31 < PQ_CAP, "pool queue overflow");
constexpr int POOL_WORDS = 19; // 4-byte fields per slot
enum { PS_FREE = 0, PS_TRACK = 1, PS_EVENT = 2 };
constexpr int POOL_WARP_BYTES = PQ_CAP * 32 + POOL_WORDS * POOL_SLOTS * 4 + POOL_SLOTS + 32 * 4 + 16;
static_assert(POOL_WARP_BYTES % 16 == 0, "per-warp pool keeps 16-byte alignment");

__host__ __device__ inline SmemLayout smem_layout(int B, int form, int block)
{
    SmemLayout L;
    L.tab_floats = tab_size(B);
    int off = ((L.tab_floats * 4 + 15) / 16) * 16;
    L.tal_off_bytes = off;
    L.tal_global = form == FLR_FORM_WAVEFRONT_WARP || form == FLR_FORM_WAVEFRONT_POOL;
    if (!L.tal_global) off += tal_size(B) * 8;
    L.cnt_off_bytes = off;
    off += FLR_NCOUNTERS * 8;
    off = ((off + 15) / 16) * 16;
    L.queue_off_bytes = off;
    if (form == FLR_FORM_WAVEFRONT) off += 2 * block * 32 + 16;
    if (form == FLR_FORM_WAVEFRONT_WARP) off += (block / 32) * (WQ_CAP * 32 + 8);
    if (form == FLR_FORM_WAVEFRONT_POOL) off += (block / 32) * POOL_WARP_BYTES;
    L.total_bytes = off;
    return L;
}

__device__ __forceinline__ Smem block_prologue(const SceneDev &S, unsigned char *raw, const SmemLayout &L,
                                               unsigned long long *global_tal)
{
    float *tab = reinterpret_cast<float *>(raw);
    for (int i = threadIdx.x; i < L.tab_floats; i += blockDim.x) tab[i] = S.tables[i];
    unsigned long long *tal = L.tal_global ? global_tal
                                           : reinterpret_cast<unsigned long long *>(raw + L.tal_off_bytes);
    if (!L.tal_global)
        for (int i = threadIdx.x; i < tal_size(S.B); i += blockDim.x) tal[i] = 0ull;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(raw + L.cnt_off_bytes);
    for (int i = threadIdx.x; i < FLR_NCOUNTERS; i += blockDim.x) cnt[i] = 0ull;
    __syncthreads();
    Smem sm;
    sm.sig_a = tab + tab_sig_a(S.B);
    sm.cdf = tab + tab_cdf(S.B);
    sm.maj = tab + tab_majorant(S.B);
    sm.inv_maj = tab + tab_inv_majorant(S.B);
    sm.qy = tab + tab_qy(S.B);
    sm.tal = tal;
    sm.cnt = cnt;
    sm.tal_global = L.tal_global;
    return sm;
}

// Sets the launch's error word when a path or a connection of this block ran out of its step
// budget (flr_status then reports FLR_ERR_BUDGET). Called by every thread after a block barrier.
__device__ __forceinline__ void budget_flag(const RunDev &R, const Smem &sm)
{
    if (threadIdx.x == 0 && R.error_word && (sm.cnt[FLR_C_STEP_BUDGET] | sm.cnt[FLR_C_CONNECT_BUDGET]))
        atomicOr(R.error_word, 1);
}

__device__ __forceinline__ void block_epilogue(const SceneDev &S, const RunDev &R, const Smem &sm,
                                               const RegCnt &rc)
{
    const unsigned vals[7] = {rc.steps, rc.nulls, rc.events, rc.scatters, rc.connections,
                              rc.connect_steps, rc.cell_walks};
    const int idx[7] = {FLR_C_STEPS, FLR_C_NULLS, FLR_C_EVENTS, FLR_C_SCATTERS, FLR_C_CONNECTIONS,
                        FLR_C_CONNECT_STEPS, FLR_C_CELL_WALKS};
    // 32-bit per-thread counters; warp sums are widened before they can overflow
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        unsigned long long v = vals[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sm.cnt[idx[i]], v);
    }
    __syncthreads();
    budget_flag(R, sm);
    if (!sm.tal_global)
        for (int i = threadIdx.x; i < tal_size(S.B); i += blockDim.x)
            if (sm.tal[i]) atomicAdd(&R.tallies[i], sm.tal[i]);
    for (int i = threadIdx.x; i < FLR_NCOUNTERS; i += blockDim.x)
        if (sm.cnt[i]) atomicAdd(&R.counters[i], sm.cnt[i]);
}

// ---------------------------------------------------------------------------------------------
// Plain form: one thread per path, grid-stride over path ids, connections made inline.
template <bool OPT, bool IF, bool LZ = false>
__global__ void __launch_bounds__(256) k_trace_plain(SceneDev S, RunDev R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_PLAIN, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS_<OPT, OPT, IF, LZ> m{S, sm};
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R.n_paths; i += stride) {
        Path p;
        Conn c = spawn(m, R, sm, R.path_offset + i, p);
        if (c.valid) connect<OPT, LZ>(S, R, sm, c.x, c.bin, c.w, c.lamb, c.pid, c.step, rc);
        while (p.alive) {
            c = track_step(m, R, sm, p, rc);
            if (c.valid) connect<OPT, LZ>(S, R, sm, c.x, c.bin, c.w, c.lamb, c.pid, c.step, rc);
        }
    }
    block_epilogue(S, R, sm, rc);
}


// ---------------------------------------------------------------------------------------------
// Hero-wavelength paths (spectral MIS; Wilkie et al., "Hero wavelength spectral sampling", EGSR
// 2014, which the paper's Sec. 3 cites against the cost of per-wavelength transport). A path carries
// a set of up to HERO_MAX wavelengths: the hero drives every decision exactly as a single-wavelength
// path would, and every tally is split among the members by the balance heuristic,
//     q_j = P(j) p(path | j) / sum_k P(k) p(path | k),
// P(k) the probability of drawing member k as the hero, p(path | k) the density of the decisions
// since the set was drawn at member k's wavelength. The set is the block of a fixed partition that
// holds the hero: the hero's source lines (consecutive emitters of one source) in blocks of C, and
// after a re-emission the emission bins [C floor(b/C), C floor(b/C) + C). Free flights use the set's
// majorant max_k sigma_bar(lambda_k), so only null collisions (and, for the absorbed tally, the dye
// absorption itself) change q; scattering, walls and background absorption are grey. A re-emission
// does not depend on which member was absorbed, so the path goes on with weight w QY and a fresh
// set. With C = 1 every decision and tally is the single-wavelength path's.
constexpr int HERO_MAX = 4;

struct HeroSet {
    int n, hero;
    int bin[HERO_MAX];
    float q[HERO_MAX];   // balance-heuristic weights, sum 1
    float sb, isb;       // the set's majorant and its tabulated inverse
};

// The matter at a point, read once for all members: solvent indicator and the dyes' concentrations.
struct MatterPt {
    float s;
    float4 c;
};

template <class M>
__device__ __forceinline__ MatterPt matter_at(const M &m, float3 x)
{
    MatterPt r{1.0f, m.conc_uniform()};
    if (!m.homogeneous()) {
        const int3 q = voxel_ijk(m, x);
        const int v = (q.z * m.dims(1) + q.y) * m.dims(0) + q.x;
        const float4 *g = m.grid();
        const uint8_t *sv = m.solvent();
        if (FLR_CHK(v >= 0 && v < m.dims(0) * m.dims(1) * m.dims(2), CK_GRID, v)) {
            if (g) r.c = __ldg(&g[packed_index(q.x, q.y, q.z, m.bdims())]);
            if (sv) r.s = __ldg(&sv[v]) ? 1.0f : 0.0f;
        }
    }
    return r;
}

// The coefficients of coeffs_at, in its operation order, from a point already read.
template <class M>
__device__ __forceinline__ Coeffs coeffs_of(const M &m, const MatterPt &pt, int b)
{
    Coeffs k;
    k.scat = pt.s * m.sigma_s();
    k.bg = pt.s * m.sigma_a0();
    k.total = k.scat + k.bg;
    const float cc[4] = {pt.c.x, pt.c.y, pt.c.z, pt.c.w};
    const float4 sa = m.sig_a4(b);
    const float ss[4] = {sa.x, sa.y, sa.z, sa.w};
    const int D = m.D();
#pragma unroll
    for (int d = 0; d < MAXD; ++d) {
        k.dye[d] = (d < D) ? ss[d] * cc[d] : 0.0f;
        k.total += k.dye[d];
    }
    return k;
}

// k.dye[d] for a run-time d, by selects (an indexed read would put the array in local memory).
__device__ __forceinline__ float dye_of(const Coeffs &k, int d)
{
    return d == 0 ? k.dye[0] : (d == 1 ? k.dye[1] : (d == 2 ? k.dye[2] : k.dye[3]));
}

// Normalises the weights and takes the set's majorant (the member bin with the largest).
template <class M>
__device__ __forceinline__ void hero_close(const M &m, HeroSet &h)
{
    if (h.n == 1) {
        h.q[0] = 1.0f;
    } else {
        float z = 0.0f;
#pragma unroll
        for (int j = 0; j < HERO_MAX; ++j) z += j < h.n ? h.q[j] : 0.0f;
        const float iz = 1.0f / z;
#pragma unroll
        for (int j = 0; j < HERO_MAX; ++j) h.q[j] = j < h.n ? h.q[j] * iz : 0.0f;
    }
    int bm = h.bin[0];
#pragma unroll
    for (int j = 1; j < HERO_MAX; ++j)
        if (j < h.n && m.maj(h.bin[j]) > m.maj(bm)) bm = h.bin[j];
    h.sb = m.maj(bm);
    h.isb = m.inv_maj(bm);
}

// The hero's source lines: emitters first .. first + n - 1 of its source, in blocks of C.
template <class M>
__device__ __forceinline__ void hero_lines(const M &m, const SceneDev &S, int k, int C, HeroSet &h)
{
    const int g0 = S.em_group_first[k], gn = S.em_group_n[k];
    const int first = g0 + ((k - g0) / C) * C;
    h.n = min(C, g0 + gn - first);
    h.hero = k - first;
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j) {
        const int e = min(first + j, m.n_emitters() - 1);
        h.bin[j] = S.em[e].bin;
        h.q[j] = m.em_cdf(e) - (e > 0 ? m.em_cdf(e - 1) : 0.0f);
    }
    hero_close(m, h);
}

// The emission block of bin b of dye d: bins [C floor(b/C), ...), weights the realised pmf.
template <class M>
__device__ __forceinline__ void hero_emission(const M &m, int d, int b, int C, HeroSet &h)
{
    const int first = (b / C) * C;
    h.n = min(C, m.B() - first);
    h.hero = b - first;
    const float *cdf = m.cdf(d);
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j) {
        const int bj = min(first + j, m.B() - 1);
        h.bin[j] = bj;
        h.q[j] = cdf[bj] - (bj > 0 ? cdf[bj - 1] : 0.0f);
    }
    hero_close(m, h);
}

// Sensor connection of a vertex for every member: shared geometry, one ratio-tracking march against
// the set's majorant estimating every member's transmittance; the roulette acts on the weighted sum
// sum_k q_k T_k (with one member: the single-wavelength rule exactly).
template <class M>
__device__ __forceinline__ void connect_hero(const M &m, const SceneDev &S, const RunDev &R,
                                             const Smem &sm, float3 x, const HeroSet &h, float w,
                                             int lamb, uint64_t pid, uint32_t step, RegCnt &rc)
{
    const ConnGeom g = connect_geom(S, sm, x, lamb);
    if (!g.ok) return;
    rc.connections++;
    float T[HERO_MAX];
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j) T[j] = 1.0f;
    if (S.homogeneous) {
        const MatterPt pt = matter_at(m, x);
#pragma unroll
        for (int j = 0; j < HERO_MAX; ++j)
            if (j < h.n) T[j] = __expf(-coeffs_of(m, pt, h.bin[j]).total * g.tl);
    } else if (h.sb > 0.0f) {
        float t = 0.0f;
        MarchRng rg = march_rng(R, pid, step);
        int it = 0;
        for (; it < MAX_CONNECT_STEPS; ++it) {
            const float u = march_next(rg);
            t -= __logf(1.0f - u) * h.isb;
            if (t >= g.tl) break;
            rc.connect_steps++;
            const float3 p = make_float3(x.x + t * g.dir.x, x.y + t * g.dir.y, x.z + t * g.dir.z);
            const MatterPt pt = matter_at(m, p);
            float Tq = 0.0f, st_h = 0.0f;
#pragma unroll
            for (int j = 0; j < HERO_MAX; ++j) {
                if (j < h.n) {
                    const float st = coeffs_of(m, pt, h.bin[j]).total;
                    if (j == h.hero) st_h = st;
                    T[j] *= fmaxf(0.0f, 1.0f - st * h.isb);
                    Tq += h.q[j] * T[j];
                }
            }
            if (h.n == 1) Tq = T[0];
            if (S.sk > 0 && st_h == 0.0f) {
                // the cube around this point holds no matter at any wavelength
                const float tl2 = empty_cube_exit(m, p, g.dir, inv_dir(g.dir));
                if (tl2 > 0.0f) {
                    t += tl2;
                    rc.cell_walks++;
                }
            }
            if (Tq < RT_RR_THRESHOLD) {
                const float u2 = march_next(rg);
                if (u2 * RT_RR_THRESHOLD < Tq) {
                    if (h.n == 1) {
                        T[0] = RT_RR_THRESHOLD;
                    } else {
                        const float sc = RT_RR_THRESHOLD / Tq;
#pragma unroll
                        for (int j = 0; j < HERO_MAX; ++j) T[j] *= sc;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < HERO_MAX; ++j) T[j] = 0.0f;
                    break;
                }
            }
        }
        if (it == MAX_CONNECT_STEPS) {
#pragma unroll
            for (int j = 0; j < HERO_MAX; ++j) T[j] = 0.0f;
            cnt_add(sm, FLR_C_CONNECT_BUDGET);
        }
    }
    const float base = w * g.gf;
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j) {
        if (j < h.n) {
            const float val = (h.n == 1 ? base * T[j] : base * h.q[j] * T[j]) * R.film_scale;
            if (val > 0.0f) film_add(S, R, (size_t)g.pix * S.B + h.bin[j], val);
        }
    }
}

// Tally w split among the members: row + bin_j gets w q_j.
template <class M>
__device__ __forceinline__ void hero_tally(const M &m, int row, const HeroSet &h, float w)
{
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j)
        if (j < h.n) m.tally(row + h.bin[j], h.n == 1 ? w : w * h.q[j]);
}

// One tracking step of a hero path: the single-wavelength step (track_step) with the set's
// majorant, the weights re-balanced at null collisions and the tallies split among the members.
template <class M>
__device__ __forceinline__ Conn track_step_hero(const M &m, const RunDev &R, const Smem &sm, Path &p,
                                                HeroSet &h, RegCnt &rc)
{
    Conn c;
    c.valid = false;
    if ((long long)p.step >= R.max_steps) {
        cnt_add(sm, FLR_C_STEP_BUDGET);
        finish(R, p);
        return c;
    }
    rc.steps++;
    const U4 b0 = m.rng(R, p.pid, p.step, 0u);
    const U4 b1 = m.rng(R, p.pid, p.step, 1u);
    int face;
    const float te = exit_distance(m, p.x, p.w, p.iw, face);
    const float sb = h.sb;
    const float tf = sb > 0.0f ? -__logf(1.0f - b0.a) * h.isb : FLT_MAX;
    const uint32_t step = p.step;
    p.step++;
    int dax = -1;
    float dsg = 1.0f, du1 = b0.d, du2 = b1.a;
    if (tf >= te) {
        p.x = make_float3(p.x.x + te * p.w.x, p.x.y + te * p.w.y, p.x.z + te * p.w.z);
        if (face < 0) {
            cnt_add(sm, FLR_C_NONFINITE);
            finish(R, p);
            return c;
        }
        if (!(m.wall_mask() & (1 << face))) {
            hero_tally(m, tal_face(m.B()) + (p.fl * 6 + face) * m.B(), h, p.wt);
            cnt_add(sm, FLR_C_ESCAPES);
            finish(R, p);
            return c;
        }
        if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
        p.n_events++;
        rc.events++;
        cnt_add(sm, FLR_C_WALL_BOUNCES);
        if (R.analog) {
            if (!(b1.d < m.wall_albedo())) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
        } else {
            p.wt *= m.wall_albedo();
            if (p.wt == 0.0f) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
        }
        dax = face >> 1;
        dsg = (face & 1) ? -1.0f : 1.0f;
        if (dax == 0) p.x.x = (face & 1) ? m.hi(0) : m.lo(0);
        else if (dax == 1) p.x.y = (face & 1) ? m.hi(1) : m.lo(1);
        else p.x.z = (face & 1) ? m.hi(2) : m.lo(2);
        du1 = b0.c;
        du2 = b0.d;
    } else {
        p.x = make_float3(p.x.x + tf * p.w.x, p.x.y + tf * p.w.y, p.x.z + tf * p.w.z);
        const int4 ec = m.skip() ? empty_cell(m, p.x) : make_int4(0, 0, 0, 0);
        const MatterPt pt = matter_at(m, p.x);
        const Coeffs k = coeffs_of(m, pt, p.bin);
        if (k.total > sb) cnt_add(sm, FLR_C_MAJORANT_VIOLATIONS);
        if (!(b0.b * sb < k.total)) {
            rc.nulls++;
            if (h.n > 1) {
                // member j's null probability over the hero's
                const float inull = 1.0f / (sb - k.total);
                float z = 0.0f;
#pragma unroll
                for (int j = 0; j < HERO_MAX; ++j) {
                    if (j < h.n && j != h.hero) {
                        const float st = coeffs_of(m, pt, h.bin[j]).total;
                        if (st > sb) cnt_add(sm, FLR_C_MAJORANT_VIOLATIONS);
                        h.q[j] *= fmaxf(0.0f, sb - st) * inull;
                    }
                    z += j < h.n ? h.q[j] : 0.0f;
                }
                const float iz = 1.0f / z;
#pragma unroll
                for (int j = 0; j < HERO_MAX; ++j) h.q[j] *= iz;
            }
            if (m.skip() && k.total == 0.0f) {
                float tl = empty_cube_exit_at(m, ec, p.x, p.w, p.iw);
                if (tl > 0.0f) {
                    tl = fminf(tl, te - tf);
                    p.x = make_float3(p.x.x + tl * p.w.x, p.x.y + tl * p.w.y, p.x.z + tl * p.w.z);
                    rc.cell_walks++;
                }
            }
            return c;
        }
        if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
        p.n_events++;
        rc.events++;
        const float ue = b0.c * k.total;
        float acc = k.scat;
        int ev = -1;
        const int D = m.D();
        if (!(ue < acc)) {
            ev = D;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d < D && ev == D) {
                    acc += k.dye[d];
                    if (ue < acc) ev = d;
                }
            }
        }
        if (ev < 0) {
            rc.scatters++;
        } else if (ev < D) {
            cnt_add(sm, FLR_C_DYE_ABSORPTIONS);
            {
                // the absorbed tally: member j's probability of this dye absorption over the hero's
                HeroSet ha = h;
                if (h.n > 1) {
                    const float dh = dye_of(k, ev);   // > 0: the dye was chosen
                    float z = 0.0f;
#pragma unroll
                    for (int j = 0; j < HERO_MAX; ++j) {
                        if (j < h.n && j != h.hero) ha.q[j] *= dye_of(coeffs_of(m, pt, h.bin[j]), ev) / dh;
                        z += j < h.n ? ha.q[j] : 0.0f;
                    }
                    if (z > 0.0f && z < FLT_MAX) {
                        const float iz = 1.0f / z;
#pragma unroll
                        for (int j = 0; j < HERO_MAX; ++j) ha.q[j] *= iz;
                    } else {
                        cnt_add(sm, FLR_C_NONFINITE);
                    }
                }
                hero_tally(m, tal_absorbed(m.B()) + ev * m.B(), ha, p.wt);
            }
            if (R.max_inelastic >= 0 && p.n_inel >= R.max_inelastic) {
                cnt_add(sm, FLR_C_VF_REJECTED);
                finish(R, p);
                return c;
            }
            if (R.analog) {
                if (!(b1.d < m.qy(ev))) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
            } else {
                p.wt *= m.qy(ev);
                if (p.wt == 0.0f) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
            }
            p.bin = sample_cdf(m.cdf(ev), m.B(), b1.b);
            hero_emission(m, ev, p.bin, R.hero, h);
            hero_tally(m, tal_emitted(m.B()) + ev * m.B(), h, p.wt);
            cnt_add(sm, FLR_C_EMISSIONS);
            p.n_inel++;
            p.fl = 1;
        } else {
            hero_tally(m, tal_absorbed(m.B()) + D * m.B(), h, p.wt);
            cnt_add(sm, FLR_C_ABSORBED_DEAD);
            finish(R, p);
            return c;
        }
    }
    {
        const float u1 = du1;
        float sn, cs;
        __sincosf(TWO_PI * du2, &sn, &cs);
        float a, r;
        if (dax < 0) {
            a = 1.0f - 2.0f * u1;
            r = sqrt_approx(fmaxf(0.0f, 1.0f - a * a));
        } else {
            r = sqrt_approx(u1);
            a = dsg * sqrt_approx(fmaxf(0.0f, 1.0f - u1));
        }
        const float bx = r * cs, by = r * sn;
        p.w = dax == 0 ? make_float3(a, bx, by) : (dax == 1 ? make_float3(by, a, bx) : make_float3(bx, by, a));
    }
    p.iw = inv_dir(p.w);
    if (m.sensor()) c = Conn{p.x, p.wt, p.bin, dax < 0 ? -1 : 2 * dax + (dsg > 0.0f ? 1 : 0), p.pid, step, true};
    if (p.n_events >= R.n_rr) {
        const float q = fminf(p.wt, 1.0f);
        if (!(b1.c < q)) { cnt_add(sm, FLR_C_RR_KILLS); finish(R, p); return c; }
        p.wt = p.wt < 1.0f ? 1.0f : p.wt;
    }
    if (!(isfinite(p.wt) && isfinite(p.x.x) && isfinite(p.x.y) && isfinite(p.x.z))) {
        cnt_add(sm, FLR_C_NONFINITE);
        finish(R, p);
        c.valid = false;
    }
    return c;
}

// Plain form of the hero-wavelength tracer: one thread per path, connections inline. The
// connection of a step is made after the step, with the set as it stands then (an emission's
// connection carries the new set; the roulette that follows does not touch the set).
__global__ void __launch_bounds__(256) k_trace_hero(SceneDev S, RunDev R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_PLAIN, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS_<true, false> m{S, sm};
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R.n_paths; i += stride) {
        Path p;
        HeroSet h;
        int k = 0;
        Conn c = spawn(m, R, sm, R.path_offset + i, p, &k);
        hero_lines(m, S, k, R.hero, h);
        if (c.valid) connect_hero(m, S, R, sm, c.x, h, c.w, c.lamb, c.pid, c.step, rc);
        while (p.alive) {
            c = track_step_hero(m, R, sm, p, h, rc);
            if (c.valid) connect_hero(m, S, R, sm, c.x, h, c.w, c.lamb, c.pid, c.step, rc);
        }
    }
    block_epilogue(S, R, sm, rc);
}

// ---------------------------------------------------------------------------------------------
// Wavefront form: persistent blocks; each thread regenerates a new path (dynamic queue) as soon
// as its path ends; sensor connections are pushed to a block queue and made in batches of
// blockDim, so the ratio-tracking marches run with full warps instead of a few lanes of a
// tracking warp. Each thread steps until it has queued one connection or made `regroup` steps.
struct Queue {
    float *x, *y, *z, *w;
    int *bin_lamb;
    uint32_t *pid_lo, *pid_hi, *step;
    int *head_tail;  // [0] head, [1] tail (monotone; capacity 2 * blockDim)
};

__device__ __forceinline__ void queue_push(const Queue &q, int cap, const Conn &c)
{
    const int slot = atomicAdd(&q.head_tail[1], 1) % cap;
    q.x[slot] = c.x.x;
    q.y[slot] = c.x.y;
    q.z[slot] = c.x.z;
    q.w[slot] = c.w;
    q.bin_lamb[slot] = (c.bin & 0xFFFF) | ((c.lamb + 1) << 16);
    q.pid_lo[slot] = (uint32_t)c.pid;
    q.pid_hi[slot] = (uint32_t)(c.pid >> 32);
    q.step[slot] = c.step;
}

__device__ __forceinline__ void queue_drain(const SceneDev &S, const RunDev &R, const Smem &sm,
                                            const Queue &q, int cap, int min_batch, RegCnt &rc)
{
    // called by the whole block after a __syncthreads(); drains batches of >= min_batch entries
    while (true) {
        const int head = q.head_tail[0], tail = q.head_tail[1];
        const int n = tail - head;
        if (n <= 0 || n < min_batch) break;
        const int take = min(n, (int)blockDim.x);
        if ((int)threadIdx.x < take) {
            const int slot = (head + (int)threadIdx.x) % cap;
            const int bl = q.bin_lamb[slot];
            const uint64_t pid = ((uint64_t)q.pid_hi[slot] << 32) | q.pid_lo[slot];
            connect(S, R, sm, make_float3(q.x[slot], q.y[slot], q.z[slot]), bl & 0xFFFF, q.w[slot],
                    (bl >> 16) - 1, pid, q.step[slot], rc);
        }
        __syncthreads();
        if (threadIdx.x == 0) q.head_tail[0] = head + take;
        __syncthreads();
    }
    // rebase the ring counters (by a multiple of the capacity) so they never overflow
    if (threadIdx.x == 0) {
        const int base = q.head_tail[0] - q.head_tail[0] % cap;
        q.head_tail[0] -= base;
        q.head_tail[1] -= base;
    }
    // every thread has read head/tail before anyone pushes again
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_trace_wavefront(SceneDev S, RunDev R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_WAVEFRONT, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const int cap = 2 * blockDim.x;
    Queue q;
    {
        unsigned char *base = smem_raw + L.queue_off_bytes;
        q.x = reinterpret_cast<float *>(base);
        q.y = q.x + cap;
        q.z = q.y + cap;
        q.w = q.z + cap;
        q.bin_lamb = reinterpret_cast<int *>(q.w + cap);
        q.pid_lo = reinterpret_cast<uint32_t *>(q.bin_lamb + cap);
        q.pid_hi = q.pid_lo + cap;
        q.step = q.pid_hi + cap;
        q.head_tail = reinterpret_cast<int *>(q.step + cap);
        if (threadIdx.x == 0) { q.head_tail[0] = 0; q.head_tail[1] = 0; }
    }
    __shared__ int s_active;
    __syncthreads();
    const MedS m{S, sm};
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    Path p;
    p.alive = false;
    bool exhausted = false;
    const int regroup = R.regroup > 0 ? R.regroup : 8;
    for (long long round = 0;; ++round) {
        // stepping phase: at most `regroup` steps or one queued connection per thread
        for (int s = 0; s < regroup; ++s) {
            if (!p.alive) {
                if (exhausted) break;
                const unsigned long long i = atomicAdd(R.work_counter, 1ull);
                if (i >= R.n_paths) { exhausted = true; break; }
                const Conn c = spawn(m, R, sm, R.path_offset + i, p);
                if (c.valid) { queue_push(q, cap, c); break; }
                continue;
            }
            const Conn c = track_step(m, R, sm, p, rc);
            if (c.valid) { queue_push(q, cap, c); break; }
        }
        if (threadIdx.x == 0) s_active = 0;
        __syncthreads();
        if (p.alive || !exhausted) atomicOr(&s_active, 1);
        __syncthreads();
        const bool any = s_active != 0;
        // regrouped connection phase: full batches while work remains, everything at the end
        queue_drain(S, R, sm, q, cap, any ? (int)blockDim.x : 1, rc);
        if (!any) break;
    }
    block_epilogue(S, R, sm, rc);
}

// ---------------------------------------------------------------------------------------------
// Adjoint (path replay). For L = sum_j adj_j I_j of the film estimator over the same paths, with
// decisions frozen at the current parameters, dL/dtheta per path is
//   sum_i d log p(decision_i) * (adjoint-weighted contributions after decision i)
//   + sum_k a_k d log T_k,
// where null collisions score -d sigma_t / (sigma_bar - sigma_t), a real collision with particle e
// scores d sigma_e / sigma_e, and T_k is the ratio-tracking transmittance of contribution k
// (d log T = sum over its points of -d sigma_t / (sigma_bar - sigma_t)). d sigma_t / d c_d[v] is
// eps_d a_d(lambda) inside voxel v, d sigma_t / d sigma_s is s(x). Each path is replayed twice from
// its Philox key: pass 1 sums its contributions a_k = adj[pixel][bin] * value_k; pass 2 walks the
// decisions again with the suffix sum and re-marches each contribution with a gradient sink.
struct AdjSink {
    const SceneDev &S;
    const Smem &sm;
    const AdjDev &A;
    float scale;
    float *gsig;
    __device__ __forceinline__ void point(float3 p, int b, float st, float sb) const
    {
        const float den = sb - st;
        if (!(den > 0.0f)) return;
        const float q = -scale / den;
        const MedS m{S, sm};
        const int v = voxel_of(m, p);
        if (A.grad_c && S.grid)
            for (int d = 0; d < S.D; ++d) {
                const float g = q * sm.sig_a[tab_sig_a_at(S.B, d, b)];
                if (g != 0.0f && FLR_CHK(v >= 0 && v < A.nvox, CK_GRAD, v)) atomicAdd(&A.grad_c[(size_t)d * A.nvox + v], g);
            }
        const float sv = S.solvent ? (__ldg(&S.solvent[v]) ? 1.0f : 0.0f) : 1.0f;
        *gsig += q * sv;
    }
    __device__ __forceinline__ void homogeneous(float tl) const { *gsig += -scale * tl; }
};

struct AdjObs {
    const SceneDev &S;
    const Smem &sm;
    const AdjDev &A;
    float suffix;
    float *gsig;
    __device__ __forceinline__ void null_event(float3 x, int b, const Coeffs &k, float sb) const
    {
        if (suffix == 0.0f) return;
        const float den = sb - k.total;
        if (!(den > 0.0f)) return;
        const float q = -suffix / den;
        const MedS m{S, sm};
        int v = 0;
        if (!S.homogeneous) v = voxel_of(m, x);
        if (A.grad_c && S.grid)
            for (int d = 0; d < S.D; ++d) {
                const float g = q * sm.sig_a[tab_sig_a_at(S.B, d, b)];
                if (g != 0.0f && FLR_CHK(v >= 0 && v < A.nvox, CK_GRAD, v)) atomicAdd(&A.grad_c[(size_t)d * A.nvox + v], g);
            }
        const float sv = S.solvent ? (__ldg(&S.solvent[v]) ? 1.0f : 0.0f) : 1.0f;
        *gsig += q * sv;
    }
    __device__ __forceinline__ void real_event(float3 x, int b, const Coeffs &k, int ev) const
    {
        if (suffix == 0.0f) return;
        if (ev < 0) {
            *gsig += suffix / S.sigma_s;
        } else if (ev < S.D && A.grad_c && S.grid && k.dye[ev] > 0.0f) {
            const MedS m{S, sm};
            const int v = voxel_of(m, x);
            if (FLR_CHK(v >= 0 && v < A.nvox, CK_GRAD, v))
                atomicAdd(&A.grad_c[(size_t)ev * A.nvox + v], suffix * sm.sig_a[tab_sig_a_at(S.B, ev, b)] / k.dye[ev]);
        }
    }
};

template <bool MC = true>
__device__ __forceinline__ float adjoint_weight(const SceneDev &S, const RunDev &R, const Smem &sm,
                                                const AdjDev &A, const Conn &c, RegCnt &rc)
{
    const ConnGeom g = connect_geom(S, sm, c.x, c.lamb);
    if (!g.ok) return 0.0f;
    const float T = transmittance<NoSink, true, MC, true>(S, R, sm, c.x, g.dir, g.tl, c.bin, c.pid,
                                                          c.step, rc, NoSink{});
    const float val = c.w * g.gf * T * R.film_scale;
    if (!(val > 0.0f)) return 0.0f;
    return __ldg(&A.adj[(size_t)g.pix * S.B + c.bin]) * val;
}

__device__ __forceinline__ void adjoint_march(const SceneDev &S, const RunDev &R, const Smem &sm,
                                              const AdjDev &A, const Conn &c, float a, float *gsig,
                                              RegCnt &rc)
{
    const ConnGeom g = connect_geom(S, sm, c.x, c.lamb);
    if (!g.ok) return;
    transmittance<AdjSink, true, true, true>(S, R, sm, c.x, g.dir, g.tl, c.bin, c.pid, c.step, rc,
                                             AdjSink{S, sm, A, a, gsig});
}

__global__ void __launch_bounds__(256, 1) k_adjoint(SceneDev S, RunDev R, AdjDev A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_PLAIN, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS m{S, sm};
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    float gsig = 0.0f;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R.n_paths; i += stride) {
        const uint64_t pid = R.path_offset + i;
        // pass 1: total adjoint-weighted contribution of the path
        Path p;
        Conn c = spawn(m, R, sm, pid, p);
        float total = 0.0f;
        bool any = false;
        if (c.valid) { const float a = adjoint_weight(S, R, sm, A, c, rc); total += a; any |= a != 0.0f; }
        while (p.alive) {
            c = track_step(m, R, sm, p, rc);
            if (c.valid) { const float a = adjoint_weight(S, R, sm, A, c, rc); total += a; any |= a != 0.0f; }
        }
        if (!any) continue;
        // pass 2: scores times suffix sums, and transmittance derivatives
        float pre = 0.0f;
        c = spawn(m, R, sm, pid, p);
        if (c.valid) {
            const float a = adjoint_weight(S, R, sm, A, c, rc);
            if (a != 0.0f) adjoint_march(S, R, sm, A, c, a, &gsig, rc);
            pre += a;
        }
        AdjObs obs{S, sm, A, total - pre, &gsig};
        while (p.alive) {
            c = track_step(m, R, sm, p, rc, obs);
            if (c.valid) {
                const float a = adjoint_weight(S, R, sm, A, c, rc);
                if (a != 0.0f) adjoint_march(S, R, sm, A, c, a, &gsig, rc);
                pre += a;
                obs.suffix = total - pre;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gsig += __shfl_xor_sync(0xffffffffu, gsig, o);
    if ((threadIdx.x & 31) == 0 && gsig != 0.0f && A.grad_sigma_s) atomicAdd(A.grad_sigma_s, gsig);
    __syncthreads();
    budget_flag(R, sm);
}

// ---------------------------------------------------------------------------------------------
// Frozen-sampling evaluation (a diagnostic for derivative checks; the paper has no derivatives).
// Every path is replayed with its decisions sampled in the current medium theta_0, as flr_adjoint
// replays it, while its film contributions are those of a perturbed medium theta: dye P.dye's
// concentration in voxel P.voxel plus P.delta, and sigma_s plus P.dsig. Each decision d that
// theta changes enters through its likelihood ratio p_theta(d) / p_theta0(d):
//   null collision at x    (sigma_bar - sigma_t(theta, x)) / (sigma_bar - sigma_t(theta_0, x))
//   real collision with e  sigma_e(theta, x) / sigma_e(theta_0, x)   (Sec. 4.1 shares)
// and each transmittance is the ratio-tracking product at theta over the same points (Eq. 6); the
// roulette of a transmittance estimate takes its decision on the theta_0 estimate, as sampling
// does. Per path the result is S_p(theta) = sum_k adj[pixel_k][bin_k] value_k(theta) W_k(theta)
// (W_k the product of the ratios before contribution k), accumulated in fp64 in path order: the
// same path gives the same bits, so central differences (S_p(theta+h) - S_p(theta-h)) / 2h with
// common random numbers are smooth per path and vanish exactly for paths the perturbation does
// not touch. Their sum over paths is the derivative flr_adjoint estimates, up to O(h^2).
struct PertDev {
    int dye;          // < 0: no concentration perturbation
    long long voxel;
    float delta, dsig;
    const float *adj; // [H][W][B]
    double *out;      // [n_paths]
};

// Change of each coefficient at x (voxel v, solvent indicator sv) under the perturbation.
__device__ __forceinline__ float pert_dye_at(const SceneDev &S, const Smem &sm, const PertDev &P, int v, int b)
{
    return (P.dye >= 0 && (long long)v == P.voxel) ? sm.sig_a[tab_sig_a_at(S.B, P.dye, b)] * P.delta : 0.0f;
}

struct FrozenObs {
    const SceneDev &S;
    const Smem &sm;
    const PertDev &P;
    float *W;
    __device__ __forceinline__ void null_event(float3 x, int b, const Coeffs &k, float sb) const
    {
        const MedS_<false> m{S, sm};
        const int v = S.homogeneous ? -1 : voxel_of(m, x);
        const float sv = (S.solvent && v >= 0) ? (__ldg(&S.solvent[v]) ? 1.0f : 0.0f) : 1.0f;
        const float d = sv * P.dsig + (v >= 0 ? pert_dye_at(S, sm, P, v, b) : 0.0f);
        const float den = sb - k.total;
        if (d != 0.0f && den > 0.0f) *W *= 1.0f - d / den;
    }
    __device__ __forceinline__ void real_event(float3 x, int b, const Coeffs &k, int ev) const
    {
        if (ev < 0) {
            if (P.dsig != 0.0f && S.sigma_s > 0.0f) *W *= 1.0f + P.dsig / S.sigma_s;
        } else if (ev < S.D && ev == P.dye && !S.homogeneous && k.dye[ev] > 0.0f) {
            const MedS_<false> m{S, sm};
            const int v = voxel_of(m, x);
            const float d = pert_dye_at(S, sm, P, v, b);
            if (d != 0.0f) *W *= 1.0f + d / k.dye[ev];
        }
    }
};

// adj x value_k(theta) of one connection (0 if it does not reach the film); value_k as
// adjoint_weight computes it, the transmittance at theta with the adjoint's roulette rule.
__device__ __forceinline__ float frozen_contribution(const SceneDev &S, const RunDev &R, const Smem &sm,
                                                     const PertDev &P, const Conn &c, RegCnt &rc)
{
    const ConnGeom g = connect_geom(S, sm, c.x, c.lamb);
    if (!g.ok) return 0.0f;
    const MedS_<false> m{S, sm};
    const float sb = sm.maj[c.bin];
    float T = 1.0f;
    if (sb > 0.0f) {
        if (S.homogeneous) {
            T = __expf(-(sigma_t_at(m, c.x, c.bin) + P.dsig) * g.tl);
        } else {
            const float isb = sm.inv_maj[c.bin];
            float T0 = 1.0f, t = 0.0f;
            MarchRng rg = march_rng(R, c.pid, c.step);
            int it = 0;
            for (; it < MAX_CONNECT_STEPS; ++it) {
                const float u = march_next(rg);
                t -= __logf(1.0f - u) * isb;
                if (t >= g.tl) break;
                rc.connect_steps++;
                const float3 p = make_float3(c.x.x + t * g.dir.x, c.x.y + t * g.dir.y, c.x.z + t * g.dir.z);
                const float st = sigma_t_at(m, p, c.bin);
                const int v = voxel_of(m, p);
                const float sv = S.solvent ? (__ldg(&S.solvent[v]) ? 1.0f : 0.0f) : 1.0f;
                const float d = sv * P.dsig + pert_dye_at(S, sm, P, v, c.bin);
                const float f0 = 1.0f - st * isb;
                T0 *= fmaxf(0.0f, f0);
                T *= fmaxf(0.0f, f0 - d * isb);
                if (T0 < RT_RR_ADJ_THRESHOLD) {
                    const float u2 = march_next(rg);
                    if (u2 < 0.5f) {
                        T0 *= 2.0f;
                        T *= 2.0f;
                    } else {
                        T = 0.0f;
                        break;
                    }
                }
            }
            if (it == MAX_CONNECT_STEPS) {
                T = 0.0f;
                cnt_add(sm, FLR_C_CONNECT_BUDGET);
            }
        }
    }
    const float val = c.w * g.gf * T * R.film_scale;
    if (!(val > 0.0f)) return 0.0f;
    return __ldg(&P.adj[(size_t)g.pix * S.B + c.bin]) * val;
}

__global__ void __launch_bounds__(256) k_frozen_sums(SceneDev S, RunDev R, PertDev P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_PLAIN, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS_<false> m{S, sm};
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R.n_paths; i += stride) {
        float W = 1.0f;
        double sum = 0.0;
        const FrozenObs obs{S, sm, P, &W};
        Path p;
        Conn c = spawn(m, R, sm, R.path_offset + i, p);
        if (c.valid) sum += (double)frozen_contribution(S, R, sm, P, c, rc) * (double)W;
        while (p.alive) {
            c = track_step(m, R, sm, p, rc, obs);
            if (c.valid) sum += (double)frozen_contribution(S, R, sm, P, c, rc) * (double)W;
        }
        P.out[i] = sum;
    }
    __syncthreads();
    budget_flag(R, sm);
}

// ---------------------------------------------------------------------------------------------
// Wavefront form with per-warp regrouping and pull-based connection drains. Each warp queues its
// lanes' sensor connections in shared memory (up to WQ_CAP records). Once WQ_DRAIN records are
// waiting (or the work is done) the warp drains the queue: every lane advances its own
// ratio-tracking march by one step per iteration and claims the next record as soon as its march
// ends, so the lanes stay busy until the queue runs dry instead of waiting for the longest march
// of a fixed batch. The marches consume their random numbers exactly as transmittance() does, so
// every launch form gives the same film up to the order of the fp32 film atomics.
//
// The same kernel runs the two passes of the adjoint replay (MODE):
//   WM_RENDER       film contributions (the forward);
//   WM_ADJ_WEIGHTS  pass 1: the adjoint-weighted contribution a_k = adj[pixel][bin] * value_k of
//                   the k-th connection of each path, stored per path (the first ADJ_K of them;
//                   the rest summed per path);
//   WM_ADJ_GRAD     pass 2: replays each path with the decision scores times the suffix sums of
//                   its a_k (read back in path order) and queues the transmittance-derivative
//                   march of every contribution with a_k != 0 (scaled by a_k).
constexpr int WM_RENDER = 0;
constexpr int WM_ADJ_WEIGHTS = 1;
constexpr int WM_ADJ_GRAD = 2;
constexpr int WQ_ORD_MAX = (1 << 21) - 1;   // connection ordinals carried by a queue record

struct March {
    float3 x, dir, idir;
    float tl, t, T, isb, wg;   // wg: intensity x importance (render, pass 1) or a_k (pass 2)
    int b, pix, it, ord;
    uint64_t pid;
    MarchRng g;                // the connection's uniform stream
};

// A queued connection record: position, weight (pass 2: a_k), bin, vertex kind, ordinal along
// its path, RNG coordinates. bin < 256 (FLR_MAX_BINS), vertex kind + 1 in 0..6.
__device__ __forceinline__ void wq_push(const Queue &q, const Conn &c, float w, int ord)
{
    const int slot = atomicAdd(&q.head_tail[1], 1) % WQ_CAP;
    (void)FLR_CHK(q.head_tail[1] <= WQ_CAP, CK_QUEUE, slot);   // a wrap would overwrite a waiting record
    q.x[slot] = c.x.x;
    q.y[slot] = c.x.y;
    q.z[slot] = c.x.z;
    q.w[slot] = w;
    q.bin_lamb[slot] = (c.bin & 0xFF) | ((c.lamb + 1) << 8) | (min(ord, WQ_ORD_MAX) << 11);
    q.pid_lo[slot] = (uint32_t)c.pid;
    q.pid_hi[slot] = (uint32_t)(c.pid >> 32);
    q.step[slot] = c.step;
}

// The end of a march that reached the sensor side of the box.
template <int MODE>
__device__ __forceinline__ void march_deposit(const SceneDev &S, const RunDev &R, const AdjDev &A,
                                              const March &mc)
{
    if (MODE == WM_ADJ_GRAD) return;
    const float val = mc.wg * mc.T * R.film_scale;
    if (!(val > 0.0f)) return;
    if (MODE == WM_RENDER) {
        film_add(S, R, (size_t)mc.pix * S.B + mc.b, val);
    } else {
        const float a = __ldg(&A.adj[(size_t)mc.pix * S.B + mc.b]) * val;
        if (a == 0.0f) return;
        const uint64_t i = mc.pid - R.path_offset;
        if (!FLR_CHK(i < R.n_paths, CK_ADJ_STORE, (long long)i)) return;
        if (mc.ord < A.K) A.ak[i * A.K + mc.ord] = a;
        else atomicAdd(&A.ovf[i], a);
    }
}

// Transmittance of a connection that needs no march: the bin has no extinction anywhere, or the
// medium is homogeneous (Eq. 6 in closed form); the same cases, in the same way, as transmittance().
template <class G>
__device__ __forceinline__ float transmittance_closed(const SceneDev &S, const Smem &sm, float3 x,
                                                      float tl, int b, const G &sink)
{
    if (!(sm.maj[b] > 0.0f)) return 1.0f;
    sink.homogeneous(tl);
    return __expf(-sigma_t_at(MedS_<false>{S, sm}, x, b) * tl);
}

// Starts the connection of one queued vertex; returns true if a ratio-tracking march remains (the
// connections that need no march are finished here).
template <int MODE, bool MC>
__device__ __forceinline__ bool march_begin(const SceneDev &S, const RunDev &R, const Smem &sm,
                                            const AdjDev &A, float3 x, int b, float w, int lamb,
                                            int ord, uint64_t pid, uint32_t step, March &mc,
                                            RegCnt &rc, float &gsig)
{
    const ConnGeom g = connect_geom(S, sm, x, lamb);
    if (!g.ok) return false;
    if (MODE != WM_ADJ_GRAD) rc.connections++;
    mc.wg = MODE == WM_ADJ_GRAD ? w : w * g.gf;
    mc.pix = g.pix;
    mc.b = b;
    if (MODE == WM_ADJ_WEIGHTS) mc.ord = ord;
    mc.pid = pid;
    const float sb = sm.maj[b];
    if (!(sb > 0.0f) || S.homogeneous || (MC && S.mc > 0)) {
        const bool closed = !(sb > 0.0f) || S.homogeneous;
        if (MODE == WM_ADJ_GRAD) {
            const AdjSink sink{S, sm, A, w, &gsig};
            if (closed) transmittance_closed(S, sm, x, g.tl, b, sink);
            else transmittance<AdjSink, true, MC, true>(S, R, sm, x, g.dir, g.tl, b, pid, step, rc, sink);
        } else {
            mc.T = closed ? transmittance_closed(S, sm, x, g.tl, b, NoSink{})
                          : transmittance<NoSink, true, MC, MODE != WM_RENDER>(
                                S, R, sm, x, g.dir, g.tl, b, pid, step, rc, NoSink{});
            march_deposit<MODE>(S, R, A, mc);
        }
        return false;
    }
    mc.x = x;
    mc.dir = g.dir;
    mc.tl = g.tl;
    mc.t = 0.0f;
    mc.T = 1.0f;
    mc.isb = sm.inv_maj[b];
    mc.idir = g.idr;
    mc.it = 0;
    mc.g = march_rng(R, pid, step);
    return true;
}

__device__ __forceinline__ float march_uniform(const RunDev &, March &mc) { return march_next(mc.g); }

// One ratio-tracking step (the body of transmittance()'s loop); returns false when the march ends.
template <int MODE, bool LZ = false>
__device__ __forceinline__ bool march_step(const SceneDev &S, const RunDev &R, const Smem &sm,
                                           const AdjDev &A, March &mc, RegCnt &rc, float &gsig)
{
    if (mc.it >= MAX_CONNECT_STEPS) {
        cnt_add(sm, FLR_C_CONNECT_BUDGET);
        return false;
    }
    ++mc.it;
    const float u = march_uniform(R, mc);
    mc.t -= __logf(1.0f - u) * mc.isb;
    if (mc.t >= mc.tl) {
        march_deposit<MODE>(S, R, A, mc);
        return false;
    }
    rc.connect_steps++;
    const MedS m{S, sm};
    float u2 = -1.0f;   // the roulette coin, when the bound below draws it first
    if (MODE == WM_RENDER && LZ && !S.homogeneous && S.solvent == nullptr) {
        // upper bound of the updated estimate (minorant_known): a coin that fails against it ends
        // the march whatever sigma_t is here
        const float tu = mc.T * fmaxf(0.0f, 1.0f - (S.sigma_s + S.sigma_a0) * mc.isb);
        if (tu < RT_RR_THRESHOLD) {
            u2 = march_uniform(R, mc);
            if (!(u2 * RT_RR_THRESHOLD < tu)) return false;
        }
    }
    const float3 p = make_float3(mc.x.x + mc.t * mc.dir.x, mc.x.y + mc.t * mc.dir.y,
                                 mc.x.z + mc.t * mc.dir.z);
    const int4 ec = S.sk > 0 ? empty_cell(m, p) : make_int4(0, 0, 0, 0);
    const float st = sigma_t_at(m, p, mc.b);
    if (MODE == WM_ADJ_GRAD) AdjSink{S, sm, A, mc.wg, &gsig}.point(p, mc.b, st, sm.maj[mc.b]);
    mc.T *= fmaxf(0.0f, 1.0f - st * mc.isb);
    if (S.sk > 0 && st == 0.0f) {
        const float tl2 = empty_cube_exit_at(m, ec, p, mc.dir, mc.idir);
        if (tl2 > 0.0f) {
            mc.t += tl2;
            rc.cell_walks++;
        }
    }
    constexpr bool ADJ = MODE != WM_RENDER;
    if (mc.T < (ADJ ? RT_RR_ADJ_THRESHOLD : RT_RR_THRESHOLD)) {
        if (u2 < 0.0f) u2 = march_uniform(R, mc);
        if (ADJ ? u2 < 0.5f : u2 * RT_RR_THRESHOLD < mc.T) {
            mc.T = ADJ ? 2.0f * mc.T : RT_RR_THRESHOLD;
        } else {
            return false;
        }
    }
    return true;
}

template <int MODE, bool MC, bool IF = true, bool LZ = false>
__global__ void __launch_bounds__(WARP_BLOCK, (MODE == WM_RENDER && !MC) ? 5 : 4) k_trace_wavefront_warp(SceneDev S, RunDev R, AdjDev A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_WAVEFRONT_WARP, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS_<true, MC, IF, LZ> m{S, sm};
    constexpr unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const unsigned lower = (1u << lane) - 1u;
    Queue q;
    {
        unsigned char *base = smem_raw + L.queue_off_bytes;
        float *f = reinterpret_cast<float *>(base) + warp * WQ_CAP * 8;
        q.x = f;
        q.y = q.x + WQ_CAP;
        q.z = q.y + WQ_CAP;
        q.w = q.z + WQ_CAP;
        q.bin_lamb = reinterpret_cast<int *>(q.w + WQ_CAP);
        q.pid_lo = reinterpret_cast<uint32_t *>(q.bin_lamb + WQ_CAP);
        q.pid_hi = q.pid_lo + WQ_CAP;
        q.step = q.pid_hi + WQ_CAP;
        q.head_tail = reinterpret_cast<int *>(base + (size_t)nwarps * WQ_CAP * 32) + 2 * warp;
        if (lane == 0) { q.head_tail[0] = 0; q.head_tail[1] = 0; }
    }
    __syncwarp();
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    Path p;
    p.alive = false;
    bool exhausted = false;
    int ord = 0;                       // connections of the lane's path so far (adjoint passes)
    float tot = 0.0f, pre = 0.0f;      // pass 2: sum of the path's a_k, and of those seen so far
    float gsig = 0.0f;                 // pass 2: this lane's share of dL/dsigma_s
    const int regroup = R.regroup > 0 ? R.regroup : 1;
    while (true) {
        // Tracking: at most `regroup` steps or one queued connection per lane. Lanes whose path
        // ended wait until SPAWN_MIN of them (or all) can start new paths together: the source
        // sampling then runs for several lanes at once instead of in most rounds for one or two
        // (measured: 21.5 -> 19.5 ms per Cornell-box step with 8).
        const bool spawn_now = __popc(__ballot_sync(FULL, !p.alive && !exhausted)) >= SPAWN_MIN ||
                               __ballot_sync(FULL, p.alive) == 0u;
        for (int s = 0; s < regroup; ++s) {
            if (MODE != WM_ADJ_GRAD) {
                if (!p.alive) {
                    if (exhausted || !spawn_now) break;
                    const unsigned long long i = atomicAdd(R.work_counter, 1ull);
                    if (i >= R.n_paths) { exhausted = true; break; }
                    const Conn c = spawn(m, R, sm, R.path_offset + i, p);
                    ord = 0;
                    if (c.valid) {
                        wq_push(q, c, c.w, ord);
                        if (MODE == WM_ADJ_WEIGHTS) ++ord;
                        break;
                    }
                    continue;
                }
                const Conn c = track_step(m, R, sm, p, rc);
                if (c.valid) {
                    wq_push(q, c, c.w, MODE == WM_ADJ_WEIGHTS ? ord : 0);
                    if (MODE == WM_ADJ_WEIGHTS) ++ord;
                    break;
                }
                continue;
            }
            // pass 2 of the adjoint
            Conn c;
            if (!p.alive) {
                if (exhausted || !spawn_now) break;
                const unsigned long long i = atomicAdd(R.work_counter, 1ull);
                if (i >= R.n_paths) { exhausted = true; break; }
                c = spawn(m, R, sm, R.path_offset + i, p);
                ord = 0;
                // the path's contributions from pass 1, summed in path order
                const float *ak = A.ak + i * A.K;
                const float ov = A.ovf[i];
                bool nz = ov != 0.0f;
                tot = 0.0f;
                for (int k = 0; k < A.K; ++k) {
                    const float a = ak[k];
                    tot += a;
                    nz |= a != 0.0f;
                }
                tot += ov;
                pre = 0.0f;
                if (!nz) { p.alive = false; continue; }   // nothing to differentiate
            } else {
                c = track_step(m, R, sm, p, rc, AdjObs{S, sm, A, tot - pre, &gsig});
            }
            if (!c.valid) continue;
            const float a = ord < A.K ? __ldg(&A.ak[(p.pid - R.path_offset) * A.K + ord])
                                      : adjoint_weight<MC>(S, R, sm, A, c, rc);
            ++ord;
            pre += a;
            if (a != 0.0f) { wq_push(q, c, a, 0); break; }
        }
        __syncwarp();
        const bool any = __any_sync(FULL, p.alive || !exhausted);
        const int avail = q.head_tail[1];
        if (avail >= WQ_DRAIN || (!any && avail > 0)) {
            // pull-based drain of all `avail` records; a lane whose march ended claims the next
            // record in the next iteration (measured with the march streams: 13.14 ms per
            // Cornell-box step and 33.3 ms per 8.4M light-sheet paths, against 13.28 / 35.5 ms
            // claiming every second iteration, 13.70 / 36.3 every third and 14.20 / 37.1 every
            // fourth; every second had been fastest while marches drew Philox blocks by phase)
            March mc;
            bool active = false;
            int claimed = 0;
            for (;;) {
                const unsigned need = __ballot_sync(FULL, !active);
                if (need != 0u && !active) {
                    const int k = claimed + __popc(need & lower);
                    if (k < avail) {
                        const int bl = q.bin_lamb[k];
                        const uint64_t pid = ((uint64_t)q.pid_hi[k] << 32) | q.pid_lo[k];
                        active = march_begin<MODE, MC>(S, R, sm, A, make_float3(q.x[k], q.y[k], q.z[k]),
                                                   bl & 0xFF, q.w[k], ((bl >> 8) & 7) - 1,
                                                   MODE == WM_ADJ_WEIGHTS ? (int)((unsigned)bl >> 11) : 0,
                                                   pid, q.step[k], mc, rc,
                                                   gsig);
                    }
                }
                claimed += __popc(need);
                if (active) active = march_step<MODE, LZ>(S, R, sm, A, mc, rc, gsig);
                if (!__any_sync(FULL, active) && claimed >= avail) break;
            }
            __syncwarp();
            if (lane == 0) q.head_tail[1] = 0;
            __syncwarp();
        }
        if (!any) break;
    }
    if (MODE == WM_RENDER) {
        block_epilogue(S, R, sm, rc);
    } else {
        if (MODE == WM_ADJ_GRAD) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) gsig += __shfl_xor_sync(FULL, gsig, o);
            if (lane == 0 && gsig != 0.0f && A.grad_sigma_s) atomicAdd(A.grad_sigma_s, gsig);
        }
        __syncthreads();
        budget_flag(R, sm);
    }
}


// ---------------------------------------------------------------------------------------------
// The two halves of track_step, for the path-pool form: the free flight (block 0 of the step:
// tentative distance, null or real collision, empty-space leap, escape) and the event it leads to
// (block 1: collision type, re-emission, wall bounce or interface reflection, new direction, sensor
// connection, roulette). Together they take the decisions of track_step on the same random numbers
// in the same order, so the pool form traces exactly the paths every other form traces (tested bit
// for bit on the fixed-point tallies). Local majorants are not supported here (the pool form runs
// with one majorant per bin, with or without empty-space leaps).
enum { FL_NONE = 0, FL_MEDIUM = 1, FL_WALL = 2, FL_IFACE = 3 };

struct Flight {
    int kind, face;
    MatterPt pt;            // FL_MEDIUM: the matter at the collision point
    float u_event, u_dir1;  // block 0, words 2 and 3
};

template <class M>
__device__ __forceinline__ Flight flight_step(const M &m, const RunDev &R, const Smem &sm, Path &p, RegCnt &rc)
{
    Flight fl;
    fl.kind = FL_NONE;
    fl.face = -1;
    if ((long long)p.step >= R.max_steps) {
        cnt_add(sm, FLR_C_STEP_BUDGET);
        finish(R, p);
        return fl;
    }
    rc.steps++;
    const U4 b0 = m.rng(R, p.pid, p.step, 0u);
    fl.u_event = b0.c;
    fl.u_dir1 = b0.d;
    int face;
    const float te = exit_distance(m, p.x, p.w, p.iw, face);
    const float sb = m.maj(p.bin);
    const float tf = sb > 0.0f ? -__logf(1.0f - b0.a) * m.inv_maj(p.bin) : FLT_MAX;
    p.step++;
    if (tf >= te) {
        p.x = make_float3(p.x.x + te * p.w.x, p.x.y + te * p.w.y, p.x.z + te * p.w.z);
        if (face < 0) {
            cnt_add(sm, FLR_C_NONFINITE);
            finish(R, p);
            return fl;
        }
        fl.face = face;
        if (!(m.wall_mask() & (1 << face))) {
            if (m.iface() && m.dielectric()) {
                float ct;
                const float F = fresnel_refl(fabsf(comp(p.w, face >> 1)), m.ior(), ct);
                if (b0.b < F) {
                    fl.kind = FL_IFACE;
                    return fl;
                }
            }
            m.tally(tal_face(m.B()) + (p.fl * 6 + face) * m.B() + p.bin, p.wt);
            cnt_add(sm, FLR_C_ESCAPES);
            finish(R, p);
            return fl;
        }
        fl.kind = FL_WALL;
        return fl;
    }
    p.x = make_float3(p.x.x + tf * p.w.x, p.x.y + tf * p.w.y, p.x.z + tf * p.w.z);
    const int4 ec = m.skip() ? empty_cell(m, p.x) : make_int4(0, 0, 0, 0);
    const MatterPt pt = matter_at(m, p.x);
    const Coeffs k = coeffs_of(m, pt, p.bin);
    if (k.total > sb) cnt_add(sm, FLR_C_MAJORANT_VIOLATIONS);
    if (!(b0.b * sb < k.total)) {
        rc.nulls++;
        if (m.skip() && k.total == 0.0f) {
            float tl = empty_cube_exit_at(m, ec, p.x, p.w, p.iw);
            if (tl > 0.0f) {
                tl = fminf(tl, te - tf);
                p.x = make_float3(p.x.x + tl * p.w.x, p.x.y + tl * p.w.y, p.x.z + tl * p.w.z);
                rc.cell_walks++;
            }
        }
        return fl;
    }
    fl.kind = FL_MEDIUM;
    fl.pt = pt;
    return fl;
}

template <class M>
__device__ __forceinline__ Conn event_step(const M &m, const RunDev &R, const Smem &sm, Path &p,
                                           const Flight &fl, RegCnt &rc)
{
    Conn c;
    c.valid = false;
    const uint32_t step = p.step - 1u;
    const U4 b1 = m.rng(R, p.pid, step, 1u);
    int dax = -1;
    float dsg = 1.0f, du1 = fl.u_dir1, du2 = b1.a;
    int gw = 0;
    if (fl.kind == FL_IFACE) {
        const int face = fl.face, k = face >> 1;
        if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
        p.n_events++;
        rc.events++;
        cnt_add(sm, FLR_C_IFACE_REFLECTIONS);
        set_comp(p.w, k, -comp(p.w, k));
        set_comp(p.x, k, (face & 1) ? m.hi(k) : m.lo(k));
        p.iw = inv_dir(p.w);
        if (p.n_events >= R.n_rr) {
            const float q = fminf(p.wt, 1.0f);
            if (!(b1.c < q)) { cnt_add(sm, FLR_C_RR_KILLS); finish(R, p); return c; }
            p.wt = p.wt < 1.0f ? 1.0f : p.wt;
        }
        return c;
    }
    if (fl.kind == FL_WALL) {
        const int face = fl.face;
        if (R.paper_mode && !p.fl) { cnt_add(sm, FLR_C_VF_REJECTED); finish(R, p); return c; }
        if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
        p.n_events++;
        rc.events++;
        cnt_add(sm, FLR_C_WALL_BOUNCES);
        if (R.analog) {
            if (!(b1.d < m.wall_albedo())) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
        } else {
            p.wt *= m.wall_albedo();
            if (p.wt == 0.0f) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
        }
        dax = face >> 1;
        dsg = (face & 1) ? -1.0f : 1.0f;
        if (dax == 0) p.x.x = (face & 1) ? m.hi(0) : m.lo(0);
        else if (dax == 1) p.x.y = (face & 1) ? m.hi(1) : m.lo(1);
        else p.x.z = (face & 1) ? m.hi(2) : m.lo(2);
        du1 = fl.u_event;
        du2 = fl.u_dir1;
        if (m.iface() && m.wall_gloss() > 0.0f) {
            float3 r = p.w;
            set_comp(r, dax, -comp(r, dax));
            const float g = m.wall_gloss(), e = m.wall_exp();
            gw = 1;
            if (m.sensor()) {
                const float3 od = m.sensor_dir(p.x);
                const float co = dsg * comp(od, dax);
                if (co > 0.0f) c = Conn{p.x, p.wt * wall_lobe_cos(g, e, r, od, co), p.bin, LAMB_WEIGHTED, p.pid, step, true};
            }
            if (b1.a < g) {
                p.w = phong_dir(du1, du2, r, e);
                const float co = dsg * comp(p.w, dax);
                if (!(co > 0.0f)) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
                p.wt *= (e + 2.0f) / (e + 1.0f) * co;
                gw = 2;
            }
        }
    } else {
        const Coeffs k = coeffs_of(m, fl.pt, p.bin);
        if (p.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); finish(R, p); return c; }
        p.n_events++;
        rc.events++;
        const float ue = fl.u_event * k.total;
        float acc = k.scat;
        int ev = -1;
        const int D = m.D();
        if (!(ue < acc)) {
            ev = D;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d < D && ev == D) {
                    acc += k.dye[d];
                    if (ue < acc) ev = d;
                }
            }
        }
        if (ev < 0) {
            rc.scatters++;
            if (R.paper_mode && !p.fl) { cnt_add(sm, FLR_C_VF_REJECTED); finish(R, p); return c; }
        } else if (ev < D) {
            cnt_add(sm, FLR_C_DYE_ABSORPTIONS);
            m.tally(tal_absorbed(m.B()) + ev * m.B() + p.bin, p.wt);
            if ((R.max_inelastic >= 0 && p.n_inel >= R.max_inelastic) || (R.paper_mode && p.n_inel >= 1)) {
                cnt_add(sm, FLR_C_VF_REJECTED);
                finish(R, p);
                return c;
            }
            if (R.analog) {
                if (!(b1.d < m.qy(ev))) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
            } else {
                p.wt *= m.qy(ev);
                if (p.wt == 0.0f) { cnt_add(sm, FLR_C_ABSORBED_DEAD); finish(R, p); return c; }
            }
            p.bin = sample_cdf(m.cdf(ev), m.B(), b1.b);
            m.tally(tal_emitted(m.B()) + ev * m.B() + p.bin, p.wt);
            cnt_add(sm, FLR_C_EMISSIONS);
            p.n_inel++;
            p.fl = 1;
        } else {
            m.tally(tal_absorbed(m.B()) + D * m.B() + p.bin, p.wt);
            cnt_add(sm, FLR_C_ABSORBED_DEAD);
            finish(R, p);
            return c;
        }
    }
    if (gw != 2) {
        const float u1 = du1;
        float sn, cs;
        __sincosf(TWO_PI * du2, &sn, &cs);
        float a, r;
        if (dax < 0) {
            a = 1.0f - 2.0f * u1;
            r = sqrt_approx(fmaxf(0.0f, 1.0f - a * a));
        } else {
            r = sqrt_approx(u1);
            a = dsg * sqrt_approx(fmaxf(0.0f, 1.0f - u1));
        }
        const float bx = r * cs, by = r * sn;
        p.w = dax == 0 ? make_float3(a, bx, by) : (dax == 1 ? make_float3(by, a, bx) : make_float3(bx, by, a));
    }
    p.iw = inv_dir(p.w);
    if (m.sensor() && gw == 0) c = Conn{p.x, p.wt, p.bin, dax < 0 ? -1 : 2 * dax + (dsg > 0.0f ? 1 : 0), p.pid, step, true};
    if (p.n_events >= R.n_rr) {
        const float q = fminf(p.wt, 1.0f);
        if (!(b1.c < q)) { cnt_add(sm, FLR_C_RR_KILLS); finish(R, p); return c; }
        p.wt = p.wt < 1.0f ? 1.0f : p.wt;
    }
    if (!(isfinite(p.wt) && isfinite(p.x.x) && isfinite(p.x.y) && isfinite(p.x.z))) {
        cnt_add(sm, FLR_C_NONFINITE);
        finish(R, p);
        c.valid = false;
    }
    return c;
}

// ---------------------------------------------------------------------------------------------
// Path-pool form: regrouping by event type. Each warp keeps POOL_SLOTS paths in a shared-memory
// SoA (position, direction, weight, bin, counters, RNG coordinates, and the outcome of the last
// free flight). Every round the warp ballots the slots' states and runs one kind of work on up to
// 32 of them at once, each lane taking the k-th slot of that kind (ballot + prefix compaction):
//   track  one free flight (null collisions, leaps and escapes end here);
//   event  the collision, wall bounce or interface reflection a free flight reached;
//   spawn  new paths into free slots, claimed from the launch's work counter in one atomic.
// Event rounds run once 32 events wait (or no full tracking round is left), so both kinds of
// work run on full warps instead of splitting every step's warp between the lanes that collide
// and those that fly on. Sensor connections go to the per-warp queue and pull-based drains of the
// warp-regrouped form.

struct Pool {
    float *px, *py, *pz, *wx, *wy, *wz, *wt, *c0, *c1, *c2, *c3, *ue, *ud;
    uint32_t *step, *nev, *nin, *misc, *plo, *phi;   // misc: bin | fl << 8 | s << 9 | kind << 10 | face << 12
    uint8_t *status;
    int *scratch;
};

__device__ __forceinline__ void pool_load(const Pool &P, int s, Path &p)
{
    p.x = make_float3(P.px[s], P.py[s], P.pz[s]);
    p.w = make_float3(P.wx[s], P.wy[s], P.wz[s]);
    p.iw = inv_dir(p.w);
    p.wt = P.wt[s];
    const uint32_t mi = P.misc[s];
    p.bin = (int)(mi & 0xFFu);
    p.fl = (int)((mi >> 8) & 1u);
    p.step = P.step[s];
    p.n_events = (int)P.nev[s];
    p.n_inel = (int)P.nin[s];
    p.pid = ((uint64_t)P.phi[s] << 32) | P.plo[s];
    p.alive = true;
}

__device__ __forceinline__ void pool_store(const Pool &P, int s, const Path &p)
{
    P.px[s] = p.x.x;
    P.py[s] = p.x.y;
    P.pz[s] = p.x.z;
    P.wx[s] = p.w.x;
    P.wy[s] = p.w.y;
    P.wz[s] = p.w.z;
    P.wt[s] = p.wt;
    P.misc[s] = (uint32_t)p.bin | ((uint32_t)p.fl << 8);
    P.step[s] = p.step;
    P.nev[s] = (uint32_t)p.n_events;
    P.nin[s] = (uint32_t)p.n_inel;
    P.plo[s] = (uint32_t)p.pid;
    P.phi[s] = (uint32_t)(p.pid >> 32);
}

template <int CAP>
__device__ __forceinline__ void queue_push_cap(const Queue &q, const Conn &c)
{
    const int slot = atomicAdd(&q.head_tail[1], 1) % CAP;
    (void)FLR_CHK(q.head_tail[1] <= CAP, CK_QUEUE, slot);
    q.x[slot] = c.x.x;
    q.y[slot] = c.x.y;
    q.z[slot] = c.x.z;
    q.w[slot] = c.w;
    q.bin_lamb[slot] = (c.bin & 0xFF) | ((c.lamb + 1) << 8);
    q.pid_lo[slot] = (uint32_t)c.pid;
    q.pid_hi[slot] = (uint32_t)(c.pid >> 32);
    q.step[slot] = c.step;
}

template <bool IF>
__global__ void __launch_bounds__(WARP_BLOCK, 5) k_trace_pool(SceneDev S, RunDev R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_WAVEFRONT_POOL, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS_<true, false, IF> m{S, sm};
    constexpr unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    unsigned char *wb = smem_raw + L.queue_off_bytes + (size_t)warp * POOL_WARP_BYTES;
    Queue q;
    {
        float *f = reinterpret_cast<float *>(wb);
        q.x = f;
        q.y = q.x + PQ_CAP;
        q.z = q.y + PQ_CAP;
        q.w = q.z + PQ_CAP;
        q.bin_lamb = reinterpret_cast<int *>(q.w + PQ_CAP);
        q.pid_lo = reinterpret_cast<uint32_t *>(q.bin_lamb + PQ_CAP);
        q.pid_hi = q.pid_lo + PQ_CAP;
        q.step = q.pid_hi + PQ_CAP;
    }
    Pool P;
    {
        float *f = reinterpret_cast<float *>(wb + PQ_CAP * 32);
        float **fs[13] = {&P.px, &P.py, &P.pz, &P.wx, &P.wy, &P.wz, &P.wt, &P.c0, &P.c1, &P.c2, &P.c3, &P.ue, &P.ud};
#pragma unroll
        for (int i = 0; i < 13; ++i) *fs[i] = f + i * POOL_SLOTS;
        uint32_t *u = reinterpret_cast<uint32_t *>(f + 13 * POOL_SLOTS);
        uint32_t **us[6] = {&P.step, &P.nev, &P.nin, &P.misc, &P.plo, &P.phi};
#pragma unroll
        for (int i = 0; i < 6; ++i) *us[i] = u + i * POOL_SLOTS;
        P.status = reinterpret_cast<uint8_t *>(u + 6 * POOL_SLOTS);
        P.scratch = reinterpret_cast<int *>(P.status + POOL_SLOTS);
        q.head_tail = P.scratch + 32;
    }
    P.status[lane] = PS_FREE;
    P.status[lane + 32] = PS_FREE;
    if (lane == 0) { q.head_tail[0] = 0; q.head_tail[1] = 0; }
    __syncwarp();
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    float gsig = 0.0f;
    const AdjDev A{};
    bool exhausted = false;
    while (true) {
        const int s0 = P.status[lane], s1 = P.status[lane + 32];
        const unsigned tlo = __ballot_sync(FULL, s0 == PS_TRACK), thi = __ballot_sync(FULL, s1 == PS_TRACK);
        const unsigned elo = __ballot_sync(FULL, s0 == PS_EVENT), ehi = __ballot_sync(FULL, s1 == PS_EVENT);
        const int nT = __popc(tlo) + __popc(thi), nE = __popc(elo) + __popc(ehi);
        const int nF = POOL_SLOTS - nT - nE;
        int kind;   // 0 spawn, 1 event, 2 track, 3 done
        if (!exhausted && (nF >= 32 || (nF >= SPAWN_MIN && nT < 32 && nE < 32))) kind = 0;
        else if (nE >= 32 || (nE > 0 && nT < 32)) kind = 1;
        else if (nT > 0) kind = 2;
        else kind = exhausted ? 3 : 0;
        if (kind != 3) {
            unsigned lo, hi;
            if (kind == 0) { lo = ~(tlo | elo); hi = ~(thi | ehi); }
            else if (kind == 1) { lo = elo; hi = ehi; }
            else { lo = tlo; hi = thi; }
            const int n = min(32, __popc(lo) + __popc(hi));
            // ballot + prefix: the k-th slot of this kind goes to lane k
            if ((lo >> lane) & 1u) {
                const int r = __popc(lo & lower);
                if (r < 32) P.scratch[r] = lane;
            }
            if ((hi >> lane) & 1u) {
                const int r = __popc(lo) + __popc(hi & lower);
                if (r < 32) P.scratch[r] = lane + 32;
            }
            __syncwarp();
            const int slot = lane < n ? P.scratch[lane] : -1;
            __syncwarp();
            if (kind == 0) {
                unsigned long long base = 0ull;
                if (lane == 0) base = atomicAdd(R.work_counter, (unsigned long long)n);
                base = __shfl_sync(FULL, base, 0);
                if (base + (unsigned long long)n >= R.n_paths) exhausted = true;
                if (slot >= 0 && base + (unsigned long long)lane < R.n_paths) {
                    Path p;
                    const Conn c = spawn(m, R, sm, R.path_offset + base + (unsigned long long)lane, p);
                    if (c.valid) queue_push_cap<PQ_CAP>(q, c);
                    if (p.alive) {
                        pool_store(P, slot, p);
                        P.status[slot] = PS_TRACK;
                    }
                }
            } else if (kind == 2) {
                if (slot >= 0) {
                    Path p;
                    pool_load(P, slot, p);
                    const Flight fl = flight_step(m, R, sm, p, rc);
                    if (!p.alive) {
                        P.status[slot] = PS_FREE;
                    } else {
                        P.px[slot] = p.x.x;
                        P.py[slot] = p.x.y;
                        P.pz[slot] = p.x.z;
                        P.step[slot] = p.step;
                        if (fl.kind != FL_NONE) {
                            P.c0[slot] = fl.pt.c.x;
                            P.c1[slot] = fl.pt.c.y;
                            P.c2[slot] = fl.pt.c.z;
                            P.c3[slot] = fl.pt.c.w;
                            P.ue[slot] = fl.u_event;
                            P.ud[slot] = fl.u_dir1;
                            P.misc[slot] = (uint32_t)p.bin | ((uint32_t)p.fl << 8) |
                                           ((fl.kind == FL_MEDIUM && fl.pt.s != 0.0f) ? (1u << 9) : 0u) |
                                           ((uint32_t)fl.kind << 10) | ((uint32_t)max(fl.face, 0) << 12);
                            P.status[slot] = PS_EVENT;
                        }
                    }
                }
            } else {
                if (slot >= 0) {
                    Path p;
                    pool_load(P, slot, p);
                    const uint32_t mi = P.misc[slot];
                    Flight fl;
                    fl.kind = (int)((mi >> 10) & 3u);
                    fl.face = (int)((mi >> 12) & 7u);
                    fl.pt.s = (mi >> 9) & 1u ? 1.0f : 0.0f;
                    fl.pt.c = make_float4(P.c0[slot], P.c1[slot], P.c2[slot], P.c3[slot]);
                    fl.u_event = P.ue[slot];
                    fl.u_dir1 = P.ud[slot];
                    const Conn c = event_step(m, R, sm, p, fl, rc);
                    if (c.valid) queue_push_cap<PQ_CAP>(q, c);
                    if (!p.alive) {
                        P.status[slot] = PS_FREE;
                    } else {
                        pool_store(P, slot, p);
                        P.status[slot] = PS_TRACK;
                    }
                }
            }
            __syncwarp();
        }
        const int avail = q.head_tail[1];
        if (avail >= PQ_DRAIN || (kind == 3 && avail > 0)) {
            // pull-based drain of all `avail` records (as in k_trace_wavefront_warp)
            March mc;
            bool active = false;
            int claimed = 0;
            for (;;) {
                const unsigned need = __ballot_sync(FULL, !active);
                if (need != 0u && !active) {
                    const int k = claimed + __popc(need & lower);
                    if (k < avail) {
                        const int bl = q.bin_lamb[k];
                        const uint64_t pid = ((uint64_t)q.pid_hi[k] << 32) | q.pid_lo[k];
                        active = march_begin<WM_RENDER, false>(S, R, sm, A, make_float3(q.x[k], q.y[k], q.z[k]),
                                                               bl & 0xFF, q.w[k], ((bl >> 8) & 7) - 1, 0, pid,
                                                               q.step[k], mc, rc, gsig);
                    }
                }
                claimed += __popc(need);
                if (active) active = march_step<WM_RENDER>(S, R, sm, A, mc, rc, gsig);
                if (!__any_sync(FULL, active) && claimed >= avail) break;
            }
            __syncwarp();
            if (lane == 0) q.head_tail[1] = 0;
            __syncwarp();
        }
        if (kind == 3) break;
    }
    block_epilogue(S, R, sm, rc);
}

// ---------------------------------------------------------------------------------------------
// Warp-regrouped form of the hero-wavelength tracer: the tracking round and the pull-based drains
// of k_trace_wavefront_warp, with records that carry the member set. A record holds the vertex, the
// path weight, the members' weights q_j and packed bins, the member count, the hero's index and the
// vertex kind, and the RNG coordinates (13 words). A drain's march estimates every member's
// transmittance at once (connect_hero's march, step by step), so the film matches the plain hero
// form's up to the order of the fp32 atomics.
constexpr int HQ_CAP = 224;
constexpr int HQ_DRAIN = 192;
constexpr int HQ_WORDS = 13;
static_assert(HQ_DRAIN + 31 < HQ_CAP, "hero queue overflow");

struct HQueue {
    float *x, *y, *z, *w, *q0, *q1, *q2, *q3;
    uint32_t *bins, *nhl, *pid_lo, *pid_hi, *step;
    int *head_tail;
};

__host__ __device__ inline SmemLayout hero_warp_layout(int B, int block)
{
    SmemLayout L;
    L.tab_floats = tab_size(B);
    int off = ((L.tab_floats * 4 + 15) / 16) * 16;
    L.tal_off_bytes = off;
    L.tal_global = true;
    L.cnt_off_bytes = off;
    off += FLR_NCOUNTERS * 8;
    off = ((off + 15) / 16) * 16;
    L.queue_off_bytes = off;
    off += (block / 32) * (HQ_CAP * HQ_WORDS * 4 + 8);
    L.total_bytes = off;
    return L;
}

__device__ __forceinline__ void hq_push(const HQueue &q, const Conn &c, const HeroSet &h)
{
    const int slot = atomicAdd(&q.head_tail[1], 1);
    if (!FLR_CHK(slot < HQ_CAP, CK_QUEUE, slot)) return;
    q.x[slot] = c.x.x;
    q.y[slot] = c.x.y;
    q.z[slot] = c.x.z;
    q.w[slot] = c.w;
    q.q0[slot] = h.q[0];
    q.q1[slot] = h.n > 1 ? h.q[1] : 0.0f;
    q.q2[slot] = h.n > 2 ? h.q[2] : 0.0f;
    q.q3[slot] = h.n > 3 ? h.q[3] : 0.0f;
    q.bins[slot] = (uint32_t)(h.bin[0] & 0xFF) | ((uint32_t)(h.bin[1] & 0xFF) << 8) |
                   ((uint32_t)(h.bin[2] & 0xFF) << 16) | ((uint32_t)(h.bin[3] & 0xFF) << 24);
    q.nhl[slot] = (uint32_t)h.n | ((uint32_t)h.hero << 3) | ((uint32_t)(c.lamb + 1) << 5);
    q.pid_lo[slot] = (uint32_t)c.pid;
    q.pid_hi[slot] = (uint32_t)(c.pid >> 32);
    q.step[slot] = c.step;
}

struct HMarch {
    March mc;             // geometry, march state and RNG coordinates (wg: weight x importance)
    float T[HERO_MAX], q[HERO_MAX];
    uint32_t bins;
    int n, hero;
};

__device__ __forceinline__ int hm_bin(const HMarch &hm, int j) { return (int)((hm.bins >> (8 * j)) & 0xFFu); }

__device__ __forceinline__ void hero_deposit(const SceneDev &S, const RunDev &R, const HMarch &hm)
{
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j) {
        if (j < hm.n) {
            const float val = (hm.n == 1 ? hm.mc.wg * hm.T[j] : hm.mc.wg * hm.q[j] * hm.T[j]) * R.film_scale;
            if (val > 0.0f) film_add(S, R, (size_t)hm.mc.pix * S.B + hm_bin(hm, j), val);
        }
    }
}

// Starts the connection of one queued hero vertex; returns true if a march remains.
__device__ __forceinline__ bool hero_march_begin(const SceneDev &S, const RunDev &R, const Smem &sm,
                                                 const HQueue &q, int k, HMarch &hm, RegCnt &rc)
{
    const uint32_t nhl = q.nhl[k];
    const float3 x = make_float3(q.x[k], q.y[k], q.z[k]);
    const ConnGeom g = connect_geom(S, sm, x, (int)((nhl >> 5) & 7u) - 1);
    if (!g.ok) return false;
    rc.connections++;
    const MedS_<true, false> m{S, sm};
    hm.n = (int)(nhl & 7u);
    hm.hero = (int)((nhl >> 3) & 3u);
    hm.bins = q.bins[k];
    hm.q[0] = q.q0[k];
    hm.q[1] = q.q1[k];
    hm.q[2] = q.q2[k];
    hm.q[3] = q.q3[k];
    hm.mc.wg = q.w[k] * g.gf;
    hm.mc.pix = g.pix;
    int bm = hm_bin(hm, 0);
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j) {
        hm.T[j] = 1.0f;
        if (j > 0 && j < hm.n && m.maj(hm_bin(hm, j)) > m.maj(bm)) bm = hm_bin(hm, j);
    }
    const float sb = m.maj(bm);
    if (S.homogeneous) {
        const MatterPt pt = matter_at(m, x);
#pragma unroll
        for (int j = 0; j < HERO_MAX; ++j)
            if (j < hm.n) hm.T[j] = __expf(-coeffs_of(m, pt, hm_bin(hm, j)).total * g.tl);
        hero_deposit(S, R, hm);
        return false;
    }
    if (!(sb > 0.0f)) {
        hero_deposit(S, R, hm);
        return false;
    }
    hm.mc.x = x;
    hm.mc.dir = g.dir;
    hm.mc.idir = g.idr;
    hm.mc.tl = g.tl;
    hm.mc.t = 0.0f;
    hm.mc.isb = m.inv_maj(bm);
    hm.mc.it = 0;
    hm.mc.pid = ((uint64_t)q.pid_hi[k] << 32) | q.pid_lo[k];
    hm.mc.g = march_rng(R, hm.mc.pid, q.step[k]);
    return true;
}

// One step of a hero march (the loop body of connect_hero's march); false when the march ends.
__device__ __forceinline__ bool hero_march_step(const SceneDev &S, const RunDev &R, const Smem &sm,
                                                HMarch &hm, RegCnt &rc)
{
    March &mc = hm.mc;
    if (mc.it >= MAX_CONNECT_STEPS) {
        cnt_add(sm, FLR_C_CONNECT_BUDGET);
        return false;
    }
    ++mc.it;
    const float u = march_uniform(R, mc);
    mc.t -= __logf(1.0f - u) * mc.isb;
    if (mc.t >= mc.tl) {
        hero_deposit(S, R, hm);
        return false;
    }
    rc.connect_steps++;
    const MedS_<true, false> m{S, sm};
    const float3 p = make_float3(mc.x.x + mc.t * mc.dir.x, mc.x.y + mc.t * mc.dir.y,
                                 mc.x.z + mc.t * mc.dir.z);
    const int4 ec = S.sk > 0 ? empty_cell(m, p) : make_int4(0, 0, 0, 0);
    const MatterPt pt = matter_at(m, p);
    float Tq = 0.0f, st_h = 0.0f;
#pragma unroll
    for (int j = 0; j < HERO_MAX; ++j) {
        if (j < hm.n) {
            const float st = coeffs_of(m, pt, hm_bin(hm, j)).total;
            if (j == hm.hero) st_h = st;
            hm.T[j] *= fmaxf(0.0f, 1.0f - st * mc.isb);
            Tq += hm.q[j] * hm.T[j];
        }
    }
    if (hm.n == 1) Tq = hm.T[0];
    if (S.sk > 0 && st_h == 0.0f) {
        const float tl2 = empty_cube_exit_at(m, ec, p, mc.dir, mc.idir);
        if (tl2 > 0.0f) {
            mc.t += tl2;
            rc.cell_walks++;
        }
    }
    if (Tq < RT_RR_THRESHOLD) {
        const float u2 = march_uniform(R, mc);
        if (u2 * RT_RR_THRESHOLD < Tq) {
            if (hm.n == 1) {
                hm.T[0] = RT_RR_THRESHOLD;
            } else {
                const float sc = RT_RR_THRESHOLD / Tq;
#pragma unroll
                for (int j = 0; j < HERO_MAX; ++j) hm.T[j] *= sc;
            }
        } else {
            return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(WARP_BLOCK, 4) k_trace_hero_warp(SceneDev S, RunDev R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = hero_warp_layout(S.B, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS_<true, false> m{S, sm};
    constexpr unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const unsigned lower = (1u << lane) - 1u;
    HQueue q;
    {
        unsigned char *base = smem_raw + L.queue_off_bytes;
        float *f = reinterpret_cast<float *>(base) + warp * HQ_CAP * HQ_WORDS;
        q.x = f;
        q.y = q.x + HQ_CAP;
        q.z = q.y + HQ_CAP;
        q.w = q.z + HQ_CAP;
        q.q0 = q.w + HQ_CAP;
        q.q1 = q.q0 + HQ_CAP;
        q.q2 = q.q1 + HQ_CAP;
        q.q3 = q.q2 + HQ_CAP;
        q.bins = reinterpret_cast<uint32_t *>(q.q3 + HQ_CAP);
        q.nhl = q.bins + HQ_CAP;
        q.pid_lo = q.nhl + HQ_CAP;
        q.pid_hi = q.pid_lo + HQ_CAP;
        q.step = q.pid_hi + HQ_CAP;
        q.head_tail = reinterpret_cast<int *>(base + (size_t)nwarps * HQ_CAP * HQ_WORDS * 4) + 2 * warp;
        if (lane == 0) { q.head_tail[0] = 0; q.head_tail[1] = 0; }
    }
    __syncwarp();
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    Path p;
    p.alive = false;
    HeroSet h;
    bool exhausted = false;
    while (true) {
        const bool spawn_now = __popc(__ballot_sync(FULL, !p.alive && !exhausted)) >= SPAWN_MIN ||
                               __ballot_sync(FULL, p.alive) == 0u;
        if (!p.alive) {
            if (!exhausted && spawn_now) {
                const unsigned long long i = atomicAdd(R.work_counter, 1ull);
                if (i >= R.n_paths) {
                    exhausted = true;
                } else {
                    int k = 0;
                    const Conn c = spawn(m, R, sm, R.path_offset + i, p, &k);
                    hero_lines(m, S, k, R.hero, h);
                    if (c.valid) hq_push(q, c, h);
                }
            }
        } else {
            const Conn c = track_step_hero(m, R, sm, p, h, rc);
            if (c.valid) hq_push(q, c, h);
        }
        __syncwarp();
        const bool any = __any_sync(FULL, p.alive || !exhausted);
        const int avail = q.head_tail[1];
        if (avail >= HQ_DRAIN || (!any && avail > 0)) {
            HMarch hm;
            bool active = false;
            int claimed = 0;
            for (;;) {
                const unsigned need = __ballot_sync(FULL, !active);
                if (need != 0u && !active) {
                    const int k = claimed + __popc(need & lower);
                    if (k < avail) active = hero_march_begin(S, R, sm, q, k, hm, rc);
                }
                claimed += __popc(need);
                if (active) active = hero_march_step(S, R, sm, hm, rc);
                if (!__any_sync(FULL, active) && claimed >= avail) break;
            }
            __syncwarp();
            if (lane == 0) q.head_tail[1] = 0;
            __syncwarp();
        }
        if (!any) break;
    }
    block_epilogue(S, R, sm, rc);
}

// ---------------------------------------------------------------------------------------------
// Camera-side estimator of the paper's single-inelastic model (Sec. 4.1-4.3, Eq. 12). A path
// starts at the sensor (pixel = path id mod W*H, a point uniform in it) at an emission bin drawn
// from the mixture (1/D) sum_d p_d of the dyes' emission pmfs, and walks the medium at that bin by
// delta tracking: isotropic scattering continues it, Lambertian walls reflect it, an absorption
// ends it (a dye absorption would be a second inelastic event). At every real collision x one
// light sample (Eq. 12: a line in proportion to its power, a point on it) estimates the uncollided
// excitation fluence (Eq. 4-6), and the collision adds
//     beta * sum_d QY_d p_d(lambda) sigma_a,d(x, lambda_x) fluence / (4 pi sigma_t(x, lambda) p(lambda))
// to its pixel: collisions occur with density sigma_t T, so the sum estimates the integral of the
// emission (Eq. 10) times the transmittance along the walk.
constexpr uint32_t STEP_CAM_SPAWN = 0xFFFFFFFEu;

// p_d(b) as the fp32 CDF table realises it (the pmf the light tracer samples)
__device__ __forceinline__ float emission_pmf(const Smem &sm, int B, int d, int b)
{
    const float *c = sm.cdf + d * B;
    return c[b] - (b > 0 ? c[b - 1] : 0.0f);
}

// One light sample for the uncollided excitation fluence at x (Eq. 4-6), per unit total source
// power: the line u0 picks (p(lambda_x) of Eq. 12) and, on a Lambertian line, the point (u1, u2)
// (p(x_n)). The fluence is geom * T(start -> start + len dir) at the line's bin bx.
struct LightGeom {
    float3 start, dir;
    float len, geom;
    int bx;
    bool ok;
};

__device__ __forceinline__ LightGeom light_geometry(const SceneDev &S, float3 x, float u0, float u1, float u2)
{
    LightGeom g;
    g.ok = false;
    int k = 0;
    while (k < S.n_emitters - 1 && !(S.em_cdf[k] > u0)) ++k;
    const EmitterDev &e = S.em[k];
    g.bx = e.bin;
    if (e.kind == FLR_SOURCE_LAMBERTIAN) {
        const float3 xn = make_float3(e.origin[0] + u1 * e.eu[0] + u2 * e.ev[0],
                                      e.origin[1] + u1 * e.eu[1] + u2 * e.ev[1],
                                      e.origin[2] + u1 * e.eu[2] + u2 * e.ev[2]);
        const float3 v = make_float3(x.x - xn.x, x.y - xn.y, x.z - xn.z);
        const float r2 = v.x * v.x + v.y * v.y + v.z * v.z;
        if (!(r2 > 0.0f)) return g;
        const float ir = rsqrtf(r2);
        const float cn = e.sign * comp(v, e.axis) * ir;
        if (!(cn > 0.0f)) return g;
        g.start = xn;
        g.dir = make_float3(v.x * ir, v.y * ir, v.z * ir);
        g.len = r2 * ir;
        g.geom = cn * INV_PI / r2;   // Lambertian radiance 1/(pi A) x cos / r^2 x A
        g.ok = true;
        return g;
    }
    // collimated parallelogram: the point q of the source with x = q + l dir, l >= 0
    const float dl = rsqrtf(e.dir[0] * e.dir[0] + e.dir[1] * e.dir[1] + e.dir[2] * e.dir[2]);
    const float3 dir = make_float3(e.dir[0] * dl, e.dir[1] * dl, e.dir[2] * dl);
    const float3 eu = make_float3(e.eu[0], e.eu[1], e.eu[2]), ev = make_float3(e.ev[0], e.ev[1], e.ev[2]);
    const float3 n = make_float3(eu.y * ev.z - eu.z * ev.y, eu.z * ev.x - eu.x * ev.z, eu.x * ev.y - eu.y * ev.x);
    const float nn = n.x * n.x + n.y * n.y + n.z * n.z;
    const float dnd = dir.x * n.x + dir.y * n.y + dir.z * n.z;
    if (!(nn > 0.0f) || dnd == 0.0f) return g;
    const float3 xo = make_float3(x.x - e.origin[0], x.y - e.origin[1], x.z - e.origin[2]);
    const float l = (xo.x * n.x + xo.y * n.y + xo.z * n.z) / dnd;
    if (!(l >= 0.0f)) return g;
    const float3 q = make_float3(xo.x - l * dir.x, xo.y - l * dir.y, xo.z - l * dir.z);
    const float3 c1 = make_float3(q.y * ev.z - q.z * ev.y, q.z * ev.x - q.x * ev.z, q.x * ev.y - q.y * ev.x);
    const float3 c2 = make_float3(eu.y * q.z - eu.z * q.y, eu.z * q.x - eu.x * q.z, eu.x * q.y - eu.y * q.x);
    const float a = (c1.x * n.x + c1.y * n.y + c1.z * n.z) / nn;
    const float b = (c2.x * n.x + c2.y * n.y + c2.z * n.z) / nn;
    if (!(a >= 0.0f && a < 1.0f && b >= 0.0f && b < 1.0f)) return g;
    g.start = make_float3(e.origin[0] + q.x, e.origin[1] + q.y, e.origin[2] + q.z);
    g.dir = dir;
    g.len = l;
    g.geom = 1.0f / fabsf(dnd);   // the beam's cross-section is |eu x ev| |cos(normal, dir)|
    g.ok = true;
    return g;
}

// The emission (Eq. 10) a collision at x sends into `bin` per unit excitation fluence at bx,
// divided by sigma_t(x, bin) and by the bin's sampling probability (the collision estimator).
__device__ __forceinline__ float emission_weight(const SceneDev &S, const Smem &sm, float3 x, int bin,
                                                 int bx, float sigma_t, float pb)
{
    const Coeffs kx = coeffs_at(MedS_<false>{S, sm}, x, bx);
    float src = 0.0f;
    for (int d = 0; d < S.D; ++d) src += sm.qy[d] * emission_pmf(sm, S.B, d, bin) * kx.dye[d];
    return src * INV_4PI / (sigma_t * pb);
}

// A camera path's start: its pixel, emission bin and sampling probability, and the ray into the
// box (false: the ray misses the box or enters through a wall).
struct CamStart {
    float3 x, w;
    int pix, bin;
    float pb;
};

__device__ __forceinline__ bool camera_start(const SceneDev &S, const RunDev &R, const Smem &sm,
                                             uint64_t pid, CamStart &cs)
{
    const uint64_t npix = (uint64_t)S.W * (uint64_t)S.H;
    cs.pix = (int)(pid % npix);
    const int px = cs.pix % S.W, py = cs.pix / S.W;
    const U4 s0 = draw_rk(R, pid, STEP_CAM_SPAWN, 0u);
    const float fx = ((float)px + s0.a) / (float)S.W, fy = ((float)py + s0.b) / (float)S.H;
    const int dsel = min((int)(s0.c * (float)S.D), S.D - 1);
    cs.bin = sample_cdf(sm.cdf + dsel * S.B, S.B, s0.d);
    float pb = 0.0f;
    for (int d = 0; d < S.D; ++d) pb += emission_pmf(sm, S.B, d, cs.bin);
    cs.pb = pb * (1.0f / (float)S.D);
    if (!(cs.pb > 0.0f)) return false;
    float3 o, w;
    if (S.sensor_kind == FLR_SENSOR_ORTHO) {
        const float vl = rsqrtf(S.s_view[0] * S.s_view[0] + S.s_view[1] * S.s_view[1] + S.s_view[2] * S.s_view[2]);
        o = make_float3(S.s_origin[0] + fx * S.cam_U[0] + fy * S.cam_V[0],
                        S.s_origin[1] + fx * S.cam_U[1] + fy * S.cam_V[1],
                        S.s_origin[2] + fx * S.cam_U[2] + fy * S.cam_V[2]);
        w = make_float3(-S.s_view[0] * vl, -S.s_view[1] * vl, -S.s_view[2] * vl);
    } else {
        const float X = (2.0f * fx - 1.0f) * S.tan_x, Y = (2.0f * fy - 1.0f) * S.tan_y;
        const float3 d = make_float3(S.s_view[0] + X * S.s_U[0] + Y * S.s_V[0],
                                     S.s_view[1] + X * S.s_U[1] + Y * S.s_V[1],
                                     S.s_view[2] + X * S.s_U[2] + Y * S.s_V[2]);
        const float dl = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
        o = make_float3(S.s_origin[0], S.s_origin[1], S.s_origin[2]);
        w = make_float3(d.x * dl, d.y * dl, d.z * dl);
    }
    // enter the box; the entry face must be open (walls are opaque from outside)
    float t_in = -FLT_MAX, t_out = FLT_MAX;
    int f_in = -1;
    const float os[3] = {o.x, o.y, o.z}, ws[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (ws[k] == 0.0f) {
            if (os[k] < S.lo[k] || os[k] > S.hi[k]) return false;
            continue;
        }
        float ta = (S.lo[k] - os[k]) / ws[k], tb = (S.hi[k] - os[k]) / ws[k];
        int fa = 2 * k, fb = 2 * k + 1;
        if (ta > tb) {
            const float tt = ta; ta = tb; tb = tt;
            const int ff = fa; fa = fb; fb = ff;
        }
        if (ta > t_in) { t_in = ta; f_in = fa; }
        if (tb < t_out) t_out = tb;
    }
    if (!(t_out > t_in) || !(t_out > 0.0f)) return false;
    cs.x = o;
    if (t_in > 0.0f) {
        if (S.wall_mask & (1 << f_in)) return false;
        cs.x = make_float3(o.x + t_in * w.x, o.y + t_in * w.y, o.z + t_in * w.z);
    }
    cs.w = w;
    return true;
}

// A camera walk between collisions: the state one lane carries.
struct CamPath {
    float3 x, w, iw;
    float beta, pb;
    int pix, bin;
    uint64_t pid;
    uint32_t step;
    long long n_events;
    bool alive;
};

// What one walk step asks for at a real collision: a light sample (its geometry and weight).
struct CamRec {
    LightGeom g;
    float wt;
    bool valid;
};

// One step of a camera walk (free flight, then a wall bounce, an escape or a collision). At a
// real collision it returns the light sample whose transmittance completes the contribution
// wt * T, wt including film_scale.
__device__ __forceinline__ CamRec camera_step(const SceneDev &S, const RunDev &R, const Smem &sm,
                                              CamPath &cp, RegCnt &rc)
{
    const MedS_<false> m{S, sm};
    CamRec out;
    out.valid = false;
    if ((long long)cp.step >= R.max_steps) { cnt_add(sm, FLR_C_STEP_BUDGET); cp.alive = false; return out; }
    rc.steps++;
    const uint32_t step = cp.step;
    cp.step++;
    const U4 b0 = draw_rk(R, cp.pid, step, 0u);
    const U4 b1 = draw_rk(R, cp.pid, step, 1u);
    int face;
    const float te = exit_distance(m, cp.x, cp.w, cp.iw, face);
    const float sb = sm.maj[cp.bin];
    const float tf = sb > 0.0f ? -__logf(1.0f - b0.a) * sm.inv_maj[cp.bin] : FLT_MAX;
    if (tf >= te) {
        cp.x = make_float3(cp.x.x + te * cp.w.x, cp.x.y + te * cp.w.y, cp.x.z + te * cp.w.z);
        if (face >= 0 && (S.wall_mask & (1 << face))) {
            if (cp.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); cp.alive = false; return out; }
            cp.n_events++;
            rc.events++;
            cnt_add(sm, FLR_C_WALL_BOUNCES);
            const U4 b2 = draw_rk(R, cp.pid, step, 2u);
            if (R.analog) {
                if (!(b2.a < S.wall_albedo)) { cnt_add(sm, FLR_C_ABSORBED_DEAD); cp.alive = false; return out; }
            } else {
                cp.beta *= S.wall_albedo;
                if (cp.beta == 0.0f) { cnt_add(sm, FLR_C_ABSORBED_DEAD); cp.alive = false; return out; }
            }
            const int ax = face >> 1;
            const float sg = (face & 1) ? -1.0f : 1.0f;
            if (ax == 0) cp.x.x = (face & 1) ? S.hi[0] : S.lo[0];
            else if (ax == 1) cp.x.y = (face & 1) ? S.hi[1] : S.lo[1];
            else cp.x.z = (face & 1) ? S.hi[2] : S.lo[2];
            cp.w = cosine_dir(b0.d, b1.a, ax, sg);
            cp.iw = inv_dir(cp.w);
            if (cp.n_events >= R.n_rr) {
                const float q = fminf(cp.beta, 1.0f);
                if (!(b2.b < q)) { cnt_add(sm, FLR_C_RR_KILLS); cp.alive = false; return out; }
                cp.beta = cp.beta < 1.0f ? 1.0f : cp.beta;   // beta / min(beta, 1), exactly
            }
            return out;
        }
        cnt_add(sm, FLR_C_ESCAPES);
        cp.alive = false;
        return out;
    }
    cp.x = make_float3(cp.x.x + tf * cp.w.x, cp.x.y + tf * cp.w.y, cp.x.z + tf * cp.w.z);
    const Coeffs k = coeffs_at(m, cp.x, cp.bin);
    if (k.total > sb) cnt_add(sm, FLR_C_MAJORANT_VIOLATIONS);
    if (!(b0.b * sb < k.total)) { rc.nulls++; return out; }
    if (cp.n_events == R.max_events) { cnt_add(sm, FLR_C_CAP_HITS); cp.alive = false; return out; }
    cp.n_events++;
    rc.events++;
    // emission at this collision through one light sample
    out.g = light_geometry(S, cp.x, b1.b, b1.c, b1.d);
    if (out.g.ok) {
        out.wt = cp.beta * out.g.geom * emission_weight(S, sm, cp.x, cp.bin, out.g.bx, k.total, cp.pb) *
                 R.film_scale;
        out.valid = out.wt != 0.0f;
    }
    // the event at the emission wavelength: scattering continues, an absorption ends the walk
    if (!(b0.c * k.total < k.scat)) {
        cnt_add(sm, b0.c * k.total < k.total - k.bg ? FLR_C_VF_REJECTED : FLR_C_ABSORBED_DEAD);
        cp.alive = false;
        return out;
    }
    rc.scatters++;
    {
        const float z = 1.0f - 2.0f * b0.d;
        float sn, cs;
        __sincosf(TWO_PI * b1.a, &sn, &cs);
        const float r = sqrt_approx(fmaxf(0.0f, 1.0f - z * z));
        cp.w = make_float3(r * cs, r * sn, z);
    }
    cp.iw = inv_dir(cp.w);
    if (cp.n_events >= R.n_rr) {
        const float q = fminf(cp.beta, 1.0f);
        const U4 b2 = draw_rk(R, cp.pid, step, 2u);
        if (!(b2.b < q)) { cnt_add(sm, FLR_C_RR_KILLS); cp.alive = false; return out; }
        cp.beta = cp.beta < 1.0f ? 1.0f : cp.beta;
    }
    return out;
}

// Plain form: one thread per camera path, the light sample's transmittance marched inline
// (ratio tracking with the uniforms of slots 3.. of its collision step).
__global__ void __launch_bounds__(256) k_trace_camera(SceneDev S, RunDev R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_PLAIN, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R.n_paths; i += stride) {
        CamPath cp;
        cp.pid = R.path_offset + i;
        cnt_add(sm, FLR_C_PATHS);
        CamStart cs;
        if (!camera_start(S, R, sm, cp.pid, cs)) continue;
        cp.x = cs.x;
        cp.w = cs.w;
        cp.iw = inv_dir(cp.w);
        cp.pix = cs.pix;
        cp.bin = cs.bin;
        cp.pb = cs.pb;
        cp.beta = 1.0f;
        cp.step = 0;
        cp.n_events = 0;
        cp.alive = true;
        while (cp.alive) {
            const uint32_t step = cp.step;
            const CamRec r = camera_step(S, R, sm, cp, rc);
            if (!r.valid) continue;
            const float T = transmittance<NoSink, false, false, false, 3u>(S, R, sm, r.g.start, r.g.dir, r.g.len,
                                                                           r.g.bx, cp.pid, step, rc, NoSink{});
            const float val = r.wt * T;
            if (val != 0.0f) {
                film_add(S, R, (size_t)cp.pix * S.B + cp.bin, val);
                rc.connections++;
            }
        }
    }
    block_epilogue(S, R, sm, rc);
}

// Warp-regrouped form: the lanes' light samples go to a per-warp shared-memory queue and are
// marched by whole warps, one march per lane, with pull-based claims as in the light tracer's warp
// form. The marches draw the same uniforms as transmittance(), so both forms give the same film up
// to the order of fp32 additions.
constexpr int CQ_CAP = 160;
constexpr int CQ_DRAIN = 128;
constexpr int CQ_WORDS = 13;   // start 3, dir 3, len, weight, pixel, bins, pid lo/hi, step
static_assert(CQ_DRAIN + 31 < CQ_CAP, "camera queue overflow");

__host__ __device__ inline int camera_queue_offset(int B, int block)
{
    return ((smem_layout(B, FLR_FORM_PLAIN, block).total_bytes + 15) / 16) * 16;
}

__host__ __device__ inline int camera_smem_bytes(int B, int block)
{
    return camera_queue_offset(B, block) + (block / 32) * (CQ_CAP * CQ_WORDS * 4 + 8);
}

__global__ void __launch_bounds__(256, 2) k_trace_camera_warp(SceneDev S, RunDev R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_PLAIN, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, R.tallies);
    const MedS_<false> m{S, sm};
    constexpr unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const unsigned lower = (1u << lane) - 1u;
    float *qf = reinterpret_cast<float *>(smem_raw + camera_queue_offset(S.B, blockDim.x)) + warp * CQ_CAP * CQ_WORDS;
    int *tail = reinterpret_cast<int *>(smem_raw + camera_queue_offset(S.B, blockDim.x) +
                                        (size_t)nwarps * CQ_CAP * CQ_WORDS * 4) + 2 * warp;
    if (lane == 0) *tail = 0;
    __syncwarp();
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    CamPath cp;
    cp.alive = false;
    bool exhausted = false;
    while (true) {
        const bool spawn_now = __popc(__ballot_sync(FULL, !cp.alive && !exhausted)) >= SPAWN_MIN ||
                               __ballot_sync(FULL, cp.alive) == 0u;
        if (!cp.alive) {
            if (!exhausted && spawn_now) {
                const unsigned long long i = atomicAdd(R.work_counter, 1ull);
                if (i >= R.n_paths) {
                    exhausted = true;
                } else {
                    cp.pid = R.path_offset + i;
                    cnt_add(sm, FLR_C_PATHS);
                    CamStart cs;
                    if (camera_start(S, R, sm, cp.pid, cs)) {
                        cp.x = cs.x;
                        cp.w = cs.w;
                        cp.iw = inv_dir(cp.w);
                        cp.pix = cs.pix;
                        cp.bin = cs.bin;
                        cp.pb = cs.pb;
                        cp.beta = 1.0f;
                        cp.step = 0;
                        cp.n_events = 0;
                        cp.alive = true;
                    }
                }
            }
        } else {
            const uint32_t step = cp.step;
            const CamRec r = camera_step(S, R, sm, cp, rc);
            if (r.valid) {
                const int slot = atomicAdd(tail, 1);
                float *f = qf + (FLR_CHK(slot < CQ_CAP, CK_QUEUE, slot) ? slot : CQ_CAP - 1);
                f[0 * CQ_CAP] = r.g.start.x;
                f[1 * CQ_CAP] = r.g.start.y;
                f[2 * CQ_CAP] = r.g.start.z;
                f[3 * CQ_CAP] = r.g.dir.x;
                f[4 * CQ_CAP] = r.g.dir.y;
                f[5 * CQ_CAP] = r.g.dir.z;
                f[6 * CQ_CAP] = r.g.len;
                f[7 * CQ_CAP] = r.wt;
                f[8 * CQ_CAP] = __int_as_float(cp.pix);
                f[9 * CQ_CAP] = __int_as_float(cp.bin | (r.g.bx << 16));
                f[10 * CQ_CAP] = __uint_as_float((uint32_t)cp.pid);
                f[11 * CQ_CAP] = __uint_as_float((uint32_t)(cp.pid >> 32));
                f[12 * CQ_CAP] = __uint_as_float(step);
            }
        }
        __syncwarp();
        const bool any = __any_sync(FULL, cp.alive || !exhausted);
        const int avail = *tail;
        if (avail >= CQ_DRAIN || (!any && avail > 0)) {
            // pull-based drain; claims every second iteration (see the light tracer's warp form)
            float3 x0, dir;
            float tl = 0.0f, t = 0.0f, T = 1.0f, isb = 0.0f, wt = 0.0f;
            int pix = 0, bin = 0, bx = 0, it = 0;
            uint32_t mstep = 0;
            uint64_t pid = 0;
            MarchRng rg{0u, 0u, 0u, 0u};
            bool active = false;
            int claimed = 0;
            for (;;) {
                const unsigned need = __ballot_sync(FULL, !active);
                if (need != 0u && !active) {
                    const int k = claimed + __popc(need & lower);
                    if (k < avail) {
                        const float *f = qf + k;
                        x0 = make_float3(f[0 * CQ_CAP], f[1 * CQ_CAP], f[2 * CQ_CAP]);
                        dir = make_float3(f[3 * CQ_CAP], f[4 * CQ_CAP], f[5 * CQ_CAP]);
                        tl = f[6 * CQ_CAP];
                        wt = f[7 * CQ_CAP];
                        pix = __float_as_int(f[8 * CQ_CAP]);
                        const int bb = __float_as_int(f[9 * CQ_CAP]);
                        bin = bb & 0xFFFF;
                        bx = bb >> 16;
                        pid = ((uint64_t)__float_as_uint(f[11 * CQ_CAP]) << 32) | __float_as_uint(f[10 * CQ_CAP]);
                        mstep = __float_as_uint(f[12 * CQ_CAP]);
                        const float sb = sm.maj[bx];
                        if (!(sb > 0.0f) || S.homogeneous) {
                            const float Tc = !(sb > 0.0f) ? 1.0f : __expf(-sigma_t_at(m, x0, bx) * tl);
                            const float val = wt * Tc;
                            if (val != 0.0f) {
                                film_add(S, R, (size_t)pix * S.B + bin, val);
                                rc.connections++;
                            }
                        } else {
                            t = 0.0f;
                            T = 1.0f;
                            isb = sm.inv_maj[bx];
                            rg = march_rng(R, pid, mstep, 3u);
                            it = 0;
                            active = true;
                        }
                    }
                }
                claimed += __popc(need);
                if (active) {
                    // one ratio-tracking step (the body of transmittance()'s loop; the stream
                    // seeded by slot 3)
                    if (it >= MAX_CONNECT_STEPS) {
                        cnt_add(sm, FLR_C_CONNECT_BUDGET);
                        active = false;
                    } else {
                        ++it;
                        const float u = march_next(rg);
                        t -= __logf(1.0f - u) * isb;
                        if (t >= tl) {
                            const float val = wt * T;
                            if (val != 0.0f) {
                                film_add(S, R, (size_t)pix * S.B + bin, val);
                                rc.connections++;
                            }
                            active = false;
                        } else {
                            rc.connect_steps++;
                            const float3 pnt = make_float3(x0.x + t * dir.x, x0.y + t * dir.y, x0.z + t * dir.z);
                            const float st = sigma_t_at(m, pnt, bx);
                            T *= fmaxf(0.0f, 1.0f - st * isb);
                            if (T < RT_RR_THRESHOLD) {
                                const float u2 = march_next(rg);
                                if (u2 * RT_RR_THRESHOLD < T) T = RT_RR_THRESHOLD;
                                else active = false;
                            }
                        }
                    }
                }
                if (!__any_sync(FULL, active) && claimed >= avail) break;
            }
            __syncwarp();
            if (lane == 0) *tail = 0;
            __syncwarp();
        }
        if (!any) break;
    }
    block_epilogue(S, R, sm, rc);
}

// ---------------------------------------------------------------------------------------------
// Batched persistent form: independent media in one launch. A device queue holds chunks of
// consecutive path ids of one medium (ordered longest expected paths first). Each warp owns one
// chunk at a time and hands its path ids to lanes as their paths end (regeneration), so a lane
// never waits for the rest of its warp; lanes of one warp may be in different media. Face,
// absorption and emission tallies go to each medium's own fixed-point arrays.
__device__ __forceinline__ void counters_epilogue(const RunDev &R, const Smem &sm, const RegCnt &rc)
{
    const unsigned vals[7] = {rc.steps, rc.nulls, rc.events, rc.scatters, rc.connections,
                              rc.connect_steps, rc.cell_walks};
    const int idx[7] = {FLR_C_STEPS, FLR_C_NULLS, FLR_C_EVENTS, FLR_C_SCATTERS, FLR_C_CONNECTIONS,
                        FLR_C_CONNECT_STEPS, FLR_C_CELL_WALKS};
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        unsigned long long v = vals[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sm.cnt[idx[i]], v);
    }
    __syncthreads();
    budget_flag(R, sm);
    for (int i = threadIdx.x; i < FLR_NCOUNTERS; i += blockDim.x)
        if (sm.cnt[i]) atomicAdd(&R.counters[i], sm.cnt[i]);
}

__global__ void __launch_bounds__(256) k_trace_batch(BatchDev Bt, RunDev R)
{
    __shared__ unsigned long long s_cnt[FLR_NCOUNTERS];
    for (int i = threadIdx.x; i < FLR_NCOUNTERS; i += blockDim.x) s_cnt[i] = 0ull;
    __syncthreads();
    Smem sm;
    sm.sig_a = sm.cdf = sm.maj = sm.inv_maj = sm.qy = nullptr;
    sm.tal = nullptr;
    sm.cnt = s_cnt;
    RegCnt rc = {0, 0, 0, 0, 0, 0, 0};
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    Path p;
    p.alive = false;
    int mi = 0;                                        // medium of this lane's path
    int cm = 0;                                        // warp's current chunk (warp-uniform)
    unsigned long long cnext = 0ull, cend = 0ull;
    bool done = false;
    while (true) {
        unsigned need = __ballot_sync(FULL, !p.alive);
        while (need != 0u && !done) {
            if (cnext >= cend) {
                unsigned long long ci = 0ull;
                if (lane == 0) ci = atomicAdd(Bt.head, 1ull);
                ci = __shfl_sync(FULL, ci, 0);
                if (ci >= (unsigned long long)Bt.n_chunks) {
                    done = true;
                    break;
                }
                const ChunkDev c = Bt.chunks[ci];
                cm = c.medium;
                cnext = c.start;
                cend = c.start + c.count;
            }
            const unsigned long long avail = cend - cnext;
            const int rank = __popc(need & lower);
            if (((need >> lane) & 1u) && (unsigned long long)rank < avail) {
                mi = cm;
                const MedB m{Bt.media + cm, Bt.B};
                spawn(m, R, sm, cnext + (unsigned long long)rank, p);
            }
            const unsigned long long n_need = (unsigned long long)__popc(need);
            cnext += n_need < avail ? n_need : avail;
            need = __ballot_sync(FULL, !p.alive);
        }
        if (__ballot_sync(FULL, p.alive) == 0u && done) break;
        if (p.alive) {
            const MedB m{Bt.media + mi, Bt.B};
            track_step(m, R, sm, p, rc);
        }
    }
    counters_epilogue(R, sm, rc);
}

// ---------------------------------------------------------------------------------------------
// Utility kernels.
__global__ void k_grid_max(const float *__restrict__ g, long long n, unsigned int *out_bits,
                           int *neg_flag)
{
    float m = 0.0f;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = g[i];
        if (!(v >= 0.0f) || !isfinite(v)) bad = true; else m = fmaxf(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(m));
    if (bad) atomicOr(neg_flag, 1);
}

// Per-cell maxima (cell plus a one-voxel halo) of each dye's concentration and of the solvent
// mask; one thread per cell.
__global__ void k_build_macro(const float4 *__restrict__ grid, float4 uniform,
                              const uint8_t *__restrict__ solvent, int nx, int ny, int nz, int cell,
                              int mx, int my, int mz, float4 *__restrict__ out_c,
                              float *__restrict__ out_s)
{
    const long long ncell = (long long)mx * my * mz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(c % mx), cy = (int)((c / mx) % my), cz = (int)(c / ((long long)mx * my));
        const int dims[3] = {nx, ny, nz};
        const int bd[3] = {grid_bricks(dims[0]), grid_bricks(dims[1]), grid_bricks(dims[2])};
        const int x0 = max(cx * cell - 1, 0), x1 = min((cx + 1) * cell, nx - 1);
        const int y0 = max(cy * cell - 1, 0), y1 = min((cy + 1) * cell, ny - 1);
        const int z0 = max(cz * cell - 1, 0), z1 = min((cz + 1) * cell, nz - 1);
        float4 m = grid ? make_float4(0.f, 0.f, 0.f, 0.f) : uniform;
        float sm = solvent ? 0.0f : 1.0f;
        for (int z = z0; z <= z1; ++z)
            for (int y = y0; y <= y1; ++y)
                for (int x = x0; x <= x1; ++x) {
                    const long long v = ((long long)z * ny + y) * nx + x;
                    if (grid) {
                        const float4 g = grid[packed_index(x, y, z, bd)];
                        m.x = fmaxf(m.x, g.x);
                        m.y = fmaxf(m.y, g.y);
                        m.z = fmaxf(m.z, g.z);
                        m.w = fmaxf(m.w, g.w);
                    }
                    if (solvent && solvent[v]) sm = 1.0f;
                }
        out_c[c] = m;
        out_s[c] = sm;
    }
}

// Empty-space distances on the cell grid: a cell holds matter if its maxima (cell plus halo) show
// solvent (with sigma_s + sigma_a0 > 0) or any positive concentration; k_dist_init marks those 0
// and the others `cap`. The Chebyshev distance to matter, min over matter cells q of
// max(|dx|, |dy|, |dz|), is separable: one pass per axis, each taking
//     g'(p) = min over |k| <= cap of max(|k|, g(p + k e_axis)),
// gives it exactly, capped at `cap` (k_dist_axis; three launches instead of `cap` 26-neighbour
// dilation steps, which took about 1 ms of every medium upload on the Cornell box).
__global__ void k_dist_init(const float4 *__restrict__ mc, const float *__restrict__ ms, long long n,
                            int solvent_matter, int cap, uint8_t *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 c = mc[i];
        const bool matter = (solvent_matter && ms[i] > 0.0f) || c.x > 0.0f || c.y > 0.0f ||
                            c.z > 0.0f || c.w > 0.0f;
        out[i] = matter ? 0 : (uint8_t)cap;
    }
}

__global__ void k_dist_axis(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int mx, int my,
                            int mz, int axis, int cap)
{
    const long long n = (long long)mx * my * mz;
    const int len = axis == 0 ? mx : (axis == 1 ? my : mz);
    const long long stride = axis == 0 ? 1 : (axis == 1 ? mx : (long long)mx * my);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = axis == 0 ? (int)(i % mx) : (axis == 1 ? (int)((i / mx) % my) : (int)(i / ((long long)mx * my)));
        int best = in[i];
        const int lo = max(-cap, -c), hi = min(cap, len - 1 - c);
        for (int k = lo; k <= hi; ++k) {
            const int a = k < 0 ? -k : k;
            if (a >= best) continue;   // max(|k|, .) cannot beat the best so far
            best = min(best, max(a, (int)in[i + k * stride]));
        }
        out[i] = (uint8_t)min(best, cap);
    }
}

struct PackArgs {
    const float *conc[MAXD];
    float uniform[MAXD];
    int D;
    int dims[3], bdims[3];
};

// Reads the caller's row-major grids and writes the interleaved voxels into their bricks; the
// padding voxels of partial bricks are never read (lookups clamp to the grid).
__global__ void k_pack_grid(PackArgs a, long long n, float4 *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int d = 0; d < MAXD; ++d)
            if (d < a.D) v[d] = a.conc[d] ? a.conc[d][i] : a.uniform[d];
        const int ix = (int)(i % a.dims[0]), iy = (int)((i / a.dims[0]) % a.dims[1]);
        const int iz = (int)(i / ((long long)a.dims[0] * a.dims[1]));
        out[packed_index(ix, iy, iz, a.bdims)] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

__global__ void k_solvent_any(const uint8_t *__restrict__ s, long long n, unsigned int *out)
{
    unsigned any = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        any |= s[i] ? 1u : 0u;
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(out, 1u);
}

__global__ void k_philox(uint32_t seed, uint32_t medium, const uint4 *__restrict__ ctr, long long n,
                         uint4 *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = philox(ctr[i], seed, medium);
}

__global__ void k_sample_emission(const float *__restrict__ cdf, int B, const float *__restrict__ u,
                                  long long n, int32_t *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = sample_cdf(cdf, B, u[i]);
}

// Folds a launch's fixed-point film sums into the fp32 film: film[j] = fx[j] 2^-32, or
// film[j] + fx[j] 2^-32 when the launch adds to the film (one fp32 rounding per value and launch).
// Two values per thread and iteration as 16-byte loads of the sums when both buffers allow it.
__global__ void __launch_bounds__(256) k_film_fold(float *__restrict__ film,
                                                   const unsigned long long *__restrict__ fx,
                                                   long long n, int add)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(film) & 7) | (reinterpret_cast<uintptr_t>(fx) & 15)) == 0;
    long long done = 0;
    if (vec) {
        const long long pairs = n / 2;
        for (long long i = first; i < pairs; i += stride) {
            const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2 *>(fx) + i);
            float2 f = make_float2((float)((double)v.x * FILM_FX_INV), (float)((double)v.y * FILM_FX_INV));
            float2 *o = reinterpret_cast<float2 *>(film) + i;
            if (add) {
                const float2 g = *o;
                f.x = g.x + f.x;
                f.y = g.y + f.y;
            }
            *o = f;
        }
        done = pairs * 2;
    }
    for (long long j = done + first; j < n; j += stride) {
        const float f = (float)((double)fx[j] * FILM_FX_INV);
        film[j] = add ? film[j] + f : f;
    }
}

// sigma_t(x, bin) of the current medium at points [n][3] by the lookup the tracking uses
// (coeffs_at: nearest voxel, Sec. 4.1), and the row-major index of the voxel read (-1 without grids).
__global__ void __launch_bounds__(256) k_debug_sigma_t(SceneDev S, const float *__restrict__ pts, long long n,
                                                       int bin, float *__restrict__ out,
                                                       int32_t *__restrict__ vox)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(S.B, FLR_FORM_PLAIN, blockDim.x);
    const Smem sm = block_prologue(S, smem_raw, L, nullptr);
    const MedS_<false> m{S, sm};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float3 x = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        out[i] = coeffs_at(m, x, bin).total;
        if (vox) vox[i] = S.homogeneous ? -1 : voxel_of(m, x);
    }
}

}  // namespace

int device_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

namespace {
int num_sms() { return device_sms(); }
}  // namespace

// ---------------------------------------------------------------------------------------------
// Launchers.
int trace_block_default() { return 256; }

namespace {
__global__ void k_debug_check(long long index, long long bound)
{
    (void)FLR_CHK(index >= 0 && index < bound, CK_DEBUG, index);
}
}  // namespace

int checked_build()
{
#ifdef FLR_CHECKED
    return 1;
#else
    return 0;
#endif
}

cudaError_t check_word_take(unsigned long long *word)
{
    *word = 0ull;
#ifdef FLR_CHECKED
    cudaError_t e = cudaMemcpyFromSymbol(word, g_check_word, sizeof(*word));
    if (e != cudaSuccess || *word == 0ull) return e;
    const unsigned long long zero = 0ull;
    return cudaMemcpyToSymbol(g_check_word, &zero, sizeof(zero));
#else
    return cudaSuccess;
#endif
}

cudaError_t launch_debug_check(long long index, long long bound, cudaStream_t st)
{
    k_debug_check<<<1, 1, 0, st>>>(index, bound);
    return cudaGetLastError();
}

int trace_smem_bytes(int B, int form, int block) { return smem_layout(B, form, block).total_bytes; }

cudaError_t launch_hero_warp(const SceneDev &S, const RunDev &R, int block, int blocks_per_sm,
                             cudaStream_t st)
{
    block = WARP_BLOCK;
    const int smem = hero_warp_layout(S.B, block).total_bytes;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_trace_hero_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_hero_warp, block, smem);
    if (occ < 1) occ = 1;
    if (blocks_per_sm <= 0 || blocks_per_sm > occ) blocks_per_sm = occ;
    const long long grid = (long long)num_sms() * blocks_per_sm;
    k_trace_hero_warp<<<(unsigned)grid, block, smem, st>>>(S, R);
    return cudaGetLastError();
}

namespace {
// Opts a trace kernel into dynamic shared memory above the default 48 KB (the warp-regrouped
// form's queues reach about 59 KB at 128 bins and 256 threads).
cudaError_t allow_smem(int form, int smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    if (form == FLR_FORM_WAVEFRONT)
        return cudaFuncSetAttribute(k_trace_wavefront, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (form == FLR_FORM_WAVEFRONT_WARP) {
        void (*const ks[])(SceneDev, RunDev, AdjDev) = {
            k_trace_wavefront_warp<WM_RENDER, false, false>, k_trace_wavefront_warp<WM_RENDER, false, true>,
            k_trace_wavefront_warp<WM_RENDER, false, false, true>, k_trace_wavefront_warp<WM_RENDER, true>,
            k_trace_wavefront_warp<WM_ADJ_WEIGHTS, false>, k_trace_wavefront_warp<WM_ADJ_WEIGHTS, true>,
            k_trace_wavefront_warp<WM_ADJ_GRAD, false>, k_trace_wavefront_warp<WM_ADJ_GRAD, true>};
        for (auto k : ks) {
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    void (*const kp[])(SceneDev, RunDev) = {k_trace_plain<true, true>, k_trace_plain<false, true>,
                                             k_trace_plain<false, false>, k_trace_plain<false, false, true>};
    for (auto k : kp) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

int occupancy_blocks_per_sm(int B, int form, int block)
{
    int n = 0;
    const int smem = trace_smem_bytes(B, form, block);
    if (allow_smem(form, smem) != cudaSuccess) return 1;
    if (form == FLR_FORM_WAVEFRONT)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_wavefront, block, smem);
    else if (form == FLR_FORM_WAVEFRONT_WARP)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_wavefront_warp<WM_RENDER, false, false>, block, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_plain<true, true>, block, smem);
    return n > 0 ? n : 1;
}

cudaError_t launch_pool(const SceneDev &S, const RunDev &R, int blocks_per_sm, cudaStream_t st)
{
    const int block = WARP_BLOCK;
    const int smem = trace_smem_bytes(S.B, FLR_FORM_WAVEFRONT_POOL, block);
    void (*const k)(SceneDev, RunDev) = S.iface ? k_trace_pool<true> : k_trace_pool<false>;
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, smem);
    if (occ < 1) occ = 1;
    if (blocks_per_sm <= 0 || blocks_per_sm > occ) blocks_per_sm = occ;
    k<<<(unsigned)(num_sms() * blocks_per_sm), block, smem, st>>>(S, R);
    return cudaGetLastError();
}

cudaError_t launch_trace(const SceneDev &S, const RunDev &R, int form, int block, int blocks_per_sm,
                         cudaStream_t st)
{
    if (form == FLR_FORM_WAVEFRONT_POOL) return launch_pool(S, R, blocks_per_sm, st);
    if (R.hero > 0 && form == FLR_FORM_WAVEFRONT_WARP) return launch_hero_warp(S, R, block, blocks_per_sm, st);
    if (block <= 0) block = trace_block_default();
    if (form == FLR_FORM_WAVEFRONT_WARP) block = std::min(block, WARP_BLOCK);
    const int smem = trace_smem_bytes(S.B, form, block);
    const cudaError_t ea = allow_smem(form, smem);
    if (ea != cudaSuccess) return ea;
    const int occ = occupancy_blocks_per_sm(S.B, form, block);
    if (blocks_per_sm <= 0 || blocks_per_sm > occ) blocks_per_sm = occ;
    long long grid = (long long)num_sms() * blocks_per_sm;
    if (form == FLR_FORM_PLAIN) {
        const long long need = ((long long)R.n_paths + block - 1) / block;
        if (need < grid) grid = need;
    }
    if (grid < 1) grid = 1;
    // the instances that take decisions without a grid read where a bound settles them
    // (minorant_known), for the media where the bounds decide most steps (SceneDev::lazy)
    const bool lazy = S.lazy != 0 && !S.homogeneous && S.solvent == nullptr;
    if (form == FLR_FORM_WAVEFRONT)
        k_trace_wavefront<<<(unsigned)grid, block, smem, st>>>(S, R);
    else if (form == FLR_FORM_WAVEFRONT_WARP)
    {
        if (S.mc > 0)
            k_trace_wavefront_warp<WM_RENDER, true><<<(unsigned)grid, block, smem, st>>>(S, R, AdjDev{});
        else if (S.iface)
            k_trace_wavefront_warp<WM_RENDER, false, true><<<(unsigned)grid, block, smem, st>>>(S, R, AdjDev{});
        else if (lazy)
            k_trace_wavefront_warp<WM_RENDER, false, false, true><<<(unsigned)grid, block, smem, st>>>(S, R, AdjDev{});
        else
            k_trace_wavefront_warp<WM_RENDER, false, false><<<(unsigned)grid, block, smem, st>>>(S, R, AdjDev{});
    }
    else if (R.hero > 0)
        k_trace_hero<<<(unsigned)grid, block, smem, st>>>(S, R);
    else if (S.mc > 0 || S.sk > 0)
        k_trace_plain<true, true><<<(unsigned)grid, block, smem, st>>>(S, R);
    else if (S.iface)
        k_trace_plain<false, true><<<(unsigned)grid, block, smem, st>>>(S, R);
    else if (lazy)
        k_trace_plain<false, false, true><<<(unsigned)grid, block, smem, st>>>(S, R);
    else
        k_trace_plain<false, false><<<(unsigned)grid, block, smem, st>>>(S, R);
    return cudaGetLastError();
}

int batch_occupancy_blocks_per_sm(int block)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_batch, block, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_batch(const BatchDev &Bt, const RunDev &R, int block, int blocks_per_sm,
                         cudaStream_t st)
{
    if (block <= 0) block = trace_block_default();
    const int occ = batch_occupancy_blocks_per_sm(block);
    if (blocks_per_sm <= 0 || blocks_per_sm > occ) blocks_per_sm = occ;
    const long long grid = (long long)num_sms() * blocks_per_sm;
    k_trace_batch<<<(unsigned)grid, block, 0, st>>>(Bt, R);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const SceneDev &S, const RunDev &R, const AdjDev &A, int block,
                           int blocks_per_sm, cudaStream_t st)
{
    if (block <= 0) block = trace_block_default();
    const int smem = trace_smem_bytes(S.B, FLR_FORM_PLAIN, block);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint, block, smem);
    if (occ < 1) occ = 1;
    if (blocks_per_sm <= 0 || blocks_per_sm > occ) blocks_per_sm = occ;
    long long grid = (long long)num_sms() * blocks_per_sm;
    const long long need = ((long long)R.n_paths + block - 1) / block;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    k_adjoint<<<(unsigned)grid, block, smem, st>>>(S, R, A);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_warp(const SceneDev &S, const RunDev &R, const AdjDev &A, int pass,
                                int block, int blocks_per_sm, cudaStream_t st)
{
    if (block <= 0) block = trace_block_default();
    block = std::min(block, WARP_BLOCK);
    const int smem = trace_smem_bytes(S.B, FLR_FORM_WAVEFRONT_WARP, block);
    const cudaError_t ea = allow_smem(FLR_FORM_WAVEFRONT_WARP, smem);
    if (ea != cudaSuccess) return ea;
    int occ = 0;
    void (*k)(SceneDev, RunDev, AdjDev);
    if (pass == 1)
        k = S.mc > 0 ? k_trace_wavefront_warp<WM_ADJ_WEIGHTS, true> : k_trace_wavefront_warp<WM_ADJ_WEIGHTS, false>;
    else
        k = S.mc > 0 ? k_trace_wavefront_warp<WM_ADJ_GRAD, true> : k_trace_wavefront_warp<WM_ADJ_GRAD, false>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, smem);
    if (occ < 1) occ = 1;
    if (blocks_per_sm <= 0 || blocks_per_sm > occ) blocks_per_sm = occ;
    const long long grid = (long long)num_sms() * blocks_per_sm;
    k<<<(unsigned)grid, block, smem, st>>>(S, R, A);
    return cudaGetLastError();
}

cudaError_t launch_camera(const SceneDev &S, const RunDev &R, int form, int block, cudaStream_t st)
{
    if (block <= 0) block = trace_block_default();
    if (form != FLR_FORM_PLAIN) {
        const int smem = camera_smem_bytes(S.B, block);
        cudaError_t e = cudaFuncSetAttribute(k_trace_camera_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_camera_warp, block, smem);
        if (occ < 1) occ = 1;
        k_trace_camera_warp<<<(unsigned)(num_sms() * occ), block, smem, st>>>(S, R);
        return cudaGetLastError();
    }
    const int smem = trace_smem_bytes(S.B, FLR_FORM_PLAIN, block);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_camera, block, smem);
    if (occ < 1) occ = 1;
    long long grid = (long long)num_sms() * occ;
    const long long need = ((long long)R.n_paths + block - 1) / block;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    k_trace_camera<<<(unsigned)grid, block, smem, st>>>(S, R);
    return cudaGetLastError();
}

cudaError_t launch_build_macro(const float4 *grid, float4 uniform, const uint8_t *solvent,
                               const int dims[3], int cell, const int mdims[3], float4 *out_c,
                               float *out_s, cudaStream_t st)
{
    const long long ncell = (long long)mdims[0] * mdims[1] * mdims[2];
    long long blocks = (ncell + 127) / 128;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_build_macro<<<(unsigned)blocks, 128, 0, st>>>(grid, uniform, solvent, dims[0], dims[1], dims[2],
                                                     cell, mdims[0], mdims[1], mdims[2], out_c, out_s);
    return cudaGetLastError();
}

cudaError_t launch_empty_distance(const float4 *mc, const float *ms, const int mdims[3],
                                  int solvent_matter, int cap, uint8_t *out, uint8_t *tmp,
                                  cudaStream_t st)
{
    const long long n = (long long)mdims[0] * mdims[1] * mdims[2];
    long long blocks = (n + 255) / 256;
    const long long lim = (long long)num_sms() * 16;
    if (blocks > lim) blocks = lim;
    if (blocks < 1) blocks = 1;
    k_dist_init<<<(unsigned)blocks, 256, 0, st>>>(mc, ms, n, solvent_matter, cap, tmp);
    k_dist_axis<<<(unsigned)blocks, 256, 0, st>>>(tmp, out, mdims[0], mdims[1], mdims[2], 0, cap);
    k_dist_axis<<<(unsigned)blocks, 256, 0, st>>>(out, tmp, mdims[0], mdims[1], mdims[2], 1, cap);
    k_dist_axis<<<(unsigned)blocks, 256, 0, st>>>(tmp, out, mdims[0], mdims[1], mdims[2], 2, cap);
    return cudaGetLastError();
}


cudaError_t launch_grid_max(const float *g, long long n, unsigned int *out_bits, int *neg_flag,
                            cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_grid_max<<<(unsigned)blocks, 256, 0, st>>>(g, n, out_bits, neg_flag);
    return cudaGetLastError();
}

cudaError_t launch_pack_grid(const float *const *conc, const float *uniform, int D, const int dims[3],
                             float4 *out, cudaStream_t st)
{
    const long long n = (long long)dims[0] * dims[1] * dims[2];
    PackArgs a;
    for (int k = 0; k < 3; ++k) {
        a.dims[k] = dims[k];
        a.bdims[k] = grid_bricks(dims[k]);
    }
    for (int d = 0; d < MAXD; ++d) {
        a.conc[d] = d < D ? conc[d] : nullptr;
        a.uniform[d] = d < D ? uniform[d] : 0.0f;
    }
    a.D = D;
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_pack_grid<<<(unsigned)blocks, 256, 0, st>>>(a, n, out);
    return cudaGetLastError();
}

cudaError_t launch_solvent_any(const uint8_t *s, long long n, unsigned int *out, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_solvent_any<<<(unsigned)blocks, 256, 0, st>>>(s, n, out);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t seed, uint32_t medium, const uint32_t *ctr, long long n,
                          uint32_t *out, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_philox<<<(unsigned)blocks, 256, 0, st>>>(seed, medium, reinterpret_cast<const uint4 *>(ctr), n,
                                                reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_frozen_sums(const SceneDev &S, const RunDev &R, int pert_dye, long long pert_voxel,
                               float pert_delta, float pert_dsig, const float *adj, double *out,
                               cudaStream_t st)
{
    const int block = 256;
    const int smem = trace_smem_bytes(S.B, FLR_FORM_PLAIN, block);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_frozen_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_frozen_sums, block, smem);
    if (occ < 1) occ = 1;
    long long grid = (long long)num_sms() * occ;
    const long long need = ((long long)R.n_paths + block - 1) / block;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    PertDev P{pert_dye, pert_voxel, pert_delta, pert_dsig, adj, out};
    k_frozen_sums<<<(unsigned)grid, block, smem, st>>>(S, R, P);
    return cudaGetLastError();
}

cudaError_t launch_debug_sigma_t(const SceneDev &S, const float *pts, long long n, int bin, float *out,
                                 int32_t *vox, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const int smem = trace_smem_bytes(S.B, FLR_FORM_PLAIN, 256);
    k_debug_sigma_t<<<(unsigned)blocks, 256, smem, st>>>(S, pts, n, bin, out, vox);
    return cudaGetLastError();
}

cudaError_t launch_film_fold(float *film, const unsigned long long *fx, size_t n, int add, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    long long blocks = ((long long)n / 2 + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_film_fold<<<(unsigned)blocks, 256, 0, st>>>(film, fx, (long long)n, add);
    return cudaGetLastError();
}

cudaError_t launch_sample_emission(const SceneDev &S, int dye, const float *u, long long n,
                                   int32_t *out, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_sample_emission<<<(unsigned)blocks, 256, 0, st>>>(S.tables + tab_cdf(S.B) + dye * S.B, S.B, u,
                                                         n, out);
    return cudaGetLastError();
}

}  // namespace flr
