// pair.cu -- pair kernels of the soft and hard forces (Eq. 2 split by Eq. 7-10).
//
// The walk gives every sink group three lists:
//   cells and far particles: K = 0 for every pair (the walk's R2 + b_max
//     test), so they only add F to the soft force ("far" kernel);
//   near particles: the only pairs where K can be non-zero; one pass adds
//     F (1 - K) to the soft force and F K to the hard force ("near" kernel).
//
// FP32 form. Work item = (group, run of at most item_len consecutive entries
// of one of the group's lists), written by the walk and pulled from a global
// counter. One warp per work item: sources are staged, 64 at a time, into the
// warp's shared-memory tile relative to the group's reference point (the hi
// part of its first sink: on the hi grid, so hi - c is exact), as {x, y, z, m}
// or, for far sources, in the expanded form of body_exp2; the gathers run
// ahead of their use (see the staging ring). A group of n sinks uses
// lpc = ceil(n / KS) lanes per copy with KS sinks per lane in registers, and
// copies = 32 / lpc copies of the group split the sources (source j goes to
// copy j mod copies) and are added at the end. In the far kernel, when that
// leaves many lanes idle (e.g. 72 sinks, KS = 4: 18 lanes, one copy), the
// sinks are taken in rounds whose lanes per copy are a power of two (64
// sinks on 2 copies of 16 lanes, then 8 sinks on 16 copies of 2 lanes):
// each round streams the item's sources again, but no lane idles. A group
// with one chunk stores its sums; a group with several adds them atomically
// into zeroed outputs.
// rsqrtf runs on the CUDA cores: the pair sum is not a dense contraction.
//
// FP64 form (the plain form): one warp per group, one sink per lane, plain
// FP64 differences and 1/sqrt.
#include "hy_internal.cuh"

namespace hy {

namespace {

constexpr int PAIR_THREADS = 128;
constexpr int FAR_SPLIT_PCT = 75;   // far kernel: a round below this fill of its sink slots is split (see below)
constexpr int PAIR_WARPS = PAIR_THREADS / 32;
constexpr int NEAR_MIN_BLOCKS = 4;  // near kernels: resident blocks of PAIR_THREADS per SM (see k_pair_f32)
constexpr int TILE = 64;

struct PairArgs {
    const int64_t *ngroups;
    const uint32_t *gfirst, *gcount, *gsys;
    const SysParams *sp;
    const uint64_t *off;    // [3 * ng + 1] list offsets: cells, far particles, near particles
    const uint32_t *list;
    const float4 *phi, *plo, *nA, *nB;
    const double4_32a *pd, *nD;
    void *as[3], *ah[3];    // soft / hard accelerations (float or double)
    unsigned long long *counter;
    unsigned long long *inter_soft, *inter_hard;   // pairs of the far kernel / of the near kernel
    const Status *st;
    // FP32 work items (see WorkItem) and their number
    const WorkItem *items;
    const uint64_t *nwork;
    int want_soft, want_hard;
};

struct HardC {
    float eps2, R2, R2sq, R2sqlo, invdR;
};

// ---- FP32 bodies ----------------------------------------------------------
// weight 1 (cells, far particles). GUARD: r^2 + eps^2 may be 0 (eps = 0 and a
// self pair, only possible without a hard part).
template <bool GUARD>
__device__ __forceinline__ void body_far(const float4 q, float sx, float sy, float sz, float eps2, float &ax, float &ay,
                                         float &az)
{
    const float dx = q.x - sx, dy = q.y - sy, dz = q.z - sz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float ri = rsqrtf(r2);
    if (GUARD) ri = r2 > 0.0f ? ri : 0.0f;
    const float mr = q.w * ri;
    const float f = mr * (ri * ri);
    ax = fmaf(dx, f, ax);
    ay = fmaf(dy, f, ay);
    az = fmaf(dz, f, az);
}

// Eq. (10) with Y from D = R2^2 - r^2: Y = D / ((R2 + r)(R2 - R1)), clamped
// to [0, 1]; K = Y^6 (10 + Y^2 (-15 + 6 Y^2)), exactly 1 at Y = 1 and 0 at Y = 0.
// D is rebuilt in double-float arithmetic from the grid-aligned hi parts
// (whose differences are exact) and the lo parts: near R2, K ~ 10 Y^6
// magnifies any error of R2 - r.
__device__ __forceinline__ float dll_K_precise(float r2u, float hx, float hy, float hz, float lx, float ly, float lz,
                                               const HardC &H)
{
    const float px = __fmul_rn(hx, hx), py = __fmul_rn(hy, hy), pz = __fmul_rn(hz, hz);
    const float ex = __fmaf_rn(hx, hx, -px), ey = __fmaf_rn(hy, hy, -py), ez = __fmaf_rn(hz, hz, -pz);
    // R2^2 - px - py - pz keeping every rounding error (|R2^2| >= px, d1 >= py, d2 >= pz inside R2)
    const float d1 = __fsub_rn(H.R2sq, px), e1 = __fsub_rn(__fsub_rn(H.R2sq, d1), px);
    const float d2 = __fsub_rn(d1, py), e2 = __fsub_rn(__fsub_rn(d1, d2), py);
    const float d3 = __fsub_rn(d2, pz), e3 = __fsub_rn(__fsub_rn(d2, d3), pz);
    // (h + l)^2 = h^2 + (2h + l) l: the lo parts are up to half a grid step, so l^2 counts too
    const float cross = fmaf(2.0f * hx + lx, lx, fmaf(2.0f * hy + ly, ly, (2.0f * hz + lz) * lz));
    const float corr = ((e1 + e2) + e3) + (H.R2sqlo - ((ex + ey) + ez)) - cross;
    const float D = d3 + corr;
    const float r = sqrtf(r2u);
    const float Y = __saturatef(D * H.invdR / (H.R2 + r));
    const float Y2 = Y * Y;
    return (Y2 * Y2 * Y2) * fmaf(Y2, fmaf(6.0f, Y2, -15.0f), 10.0f);
}

// near particle: soft += F (1 - K), hard += F K. (dx, dy, dz) = source - sink
// and r2u = |.|^2 are computed by the caller; hh/ll are the source's raw hi
// and lo parts and (shx, ..), (slx, ..) the sink's: hi differences are exact.
template <bool SOFT, bool HARD>
__device__ __forceinline__ void near_finish(float w, float dx, float dy, float dz, float r2u, const float4 &hh,
                                            const float4 &ll, float shx, float shy, float shz, float slx, float sly,
                                            float slz, const HardC &H, float &sax, float &say, float &saz, float &hax,
                                            float &hay, float &haz)
{
    const bool inside = r2u < H.R2sq;
    if (!SOFT && !inside) return;
    const float r2 = r2u + H.eps2;
    const float ri = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    const float f = w * ri * (ri * ri);
    float K = 0.0f;
    if (inside)
        K = dll_K_precise(r2u, __fsub_rn(hh.x, shx), __fsub_rn(hh.y, shy), __fsub_rn(hh.z, shz),
                          __fsub_rn(ll.x, slx), __fsub_rn(ll.y, sly), __fsub_rn(ll.z, slz), H);
    if (SOFT) {
        const float fs = f * (1.0f - K);
        sax = fmaf(dx, fs, sax);
        say = fmaf(dy, fs, say);
        saz = fmaf(dz, fs, saz);
    }
    if (HARD) {
        const float fh = f * K;
        hax = fmaf(dx, fh, hax);
        hay = fmaf(dy, fh, hay);
        haz = fmaf(dz, fh, haz);
    }
}

// ---- FP64 bodies ----------------------------------------------------------
__device__ __forceinline__ double dll_K64(double r, double R1, double R2)
{
    const double Y = (R2 - r) / (R2 - R1);
    if (Y >= 1.0) return 1.0;
    if (Y <= 0.0) return 0.0;
    const double Y2 = Y * Y;
    return (Y2 * Y2 * Y2) * (10.0 + Y2 * (-15.0 + 6.0 * Y2));
}

__device__ __forceinline__ int64_t next_item(unsigned long long *counter, int lane)
{
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(counter, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, g, 0);
}

// ---------------------------------------------------------------------------
// FP32 work items and source staging
// ---------------------------------------------------------------------------
constexpr uint32_t MULTI = ITEM_MULTI;

// Raw sources (hi, lo float4 pairs of cells or particles) are gathered into a
// ring of NST shared-memory stages (the staging depth, 2 to 4; the near
// kernel uses 3) with 16-byte cp.async copies issued NST - 1 tiles ahead,
// from list indices loaded one tile before that; only the rebasing to the
// group's reference point (one pass per staged entry, by the lane that copied
// it) stands between a landed stage and its use.
constexpr int PER = TILE / 32;

// Rebased sources: the near kernel keeps {x, y, z, m} in tile[0, TILE); the
// far kernel keeps each source twice over, {x, x, y, y} {z, z, m, m}, for the
// packed two-sink arithmetic, or in the expanded form of exp_tile, two float4
// per entry, in tile[0, 2 PADT): entries from nt up to PADT = TILE + 32 are
// zero-mass sources (all zero in either form).
constexpr int PADT = TILE + 32;
static_assert(2 * PADT >= 3 * TILE, "the near filter keeps three float4 rows of TILE entries");
template <int NST>
struct WarpStage {
    float4 tile[2 * PADT];
    float4 rh[NST][TILE];     // raw hi parts (cells: nA, particles: phi)
    float4 rl[NST][TILE];     // raw lo parts (cells: nB, particles: plo)
};

__device__ __forceinline__ void cp16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct ItemSrc {
    uint64_t cbase, pbase;
    uint32_t Lc, e0, e1;

    __device__ __forceinline__ void load_idx(const PairArgs &a, int t, int lane, uint32_t (&idx)[PER]) const
    {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const uint32_t e = e0 + (uint32_t)(t * TILE + u * 32 + lane);
            idx[u] = e < e1 ? a.list[(e < Lc ? cbase : pbase) + e] : 0u;
        }
    }
    // gathers of tile t into stage t % NST; always closes one cp.async group
    template <int NST, typename Stage>
    __device__ __forceinline__ void issue(const PairArgs &a, Stage &S, int t, int lane,
                                          const uint32_t (&idx)[PER]) const
    {
        const int st = t % NST;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const uint32_t e = e0 + (uint32_t)(t * TILE + u * 32 + lane);
            if (e < e1) {
                const bool cell = e < Lc;
                cp16(&S.rh[st][u * 32 + lane], (cell ? a.nA : a.phi) + idx[u]);
                cp16(&S.rl[st][u * 32 + lane], (cell ? a.nB : a.plo) + idx[u]);
            }
        }
        cp_commit();
    }
};

// Runs the staging pipeline over the item's entries and calls
// body(stage, nt) once per tile, after the tile has been rebased into S.tile.
// Box of a warp's sinks (group-relative FP32) for the near filter.
struct SinkBox {
    float lo[3], hi[3], R2sq;
};

// Staging modes: FAR_PACKED writes every source twice over for the packed far
// sweep and calls body(stage, nt); FAR_EXP writes the expanded form of
// exp_tile and calls body(stage, nt). NEAR_FILTER keeps a source for the near
// body only when its distance to the sinks' box is below R2 (computed like the
// pair distance, so no pair with r < R2 is dropped): kept sources go to
// tile[0, n_in) with their rebased hi part at tile[TILE + j] and raw lo part at
// tile[2 TILE + j]; the others (K = 0 for every sink) to tile[TILE - n_out,
// TILE); then body(n_in, n_out).
enum { FAR_PACKED = 0, NEAR_FILTER = 1, FAR_EXP = 2 };

template <int SMODE, int NST, typename Stage, typename Body>
__device__ __forceinline__ void pipeline(const PairArgs &a, const ItemSrc &src, Stage &S, int lane,
                                         float crx, float cry, float crz, const SinkBox &sb, Body &&body)
{
    static_assert(NST >= 2 && NST <= 4, "staging depth");
    const uint32_t ne = src.e1 - src.e0;
    const int ntile = (int)((ne + TILE - 1) / TILE);
    if (ntile == 0) return;
    {   // prologue: the indices of tiles 0 .. NST-2 are loaded together, then their gathers issued
        uint32_t ip[NST - 1][PER];
#pragma unroll
        for (int t = 0; t < NST - 1; ++t) src.load_idx(a, t, lane, ip[t]);
#pragma unroll
        for (int t = 0; t < NST - 1; ++t) src.issue<NST>(a, S, t, lane, ip[t]);
    }
    uint32_t i0[PER];
    src.load_idx(a, NST - 1, lane, i0);
    for (int t = 0; t < ntile; ++t) {
        src.issue<NST>(a, S, t + NST - 1, lane, i0);   // no copies past the end, but one group per tile
        if (t + NST < ntile) src.load_idx(a, t + NST, lane, i0);
        cp_wait<NST - 1>();                       // this lane's copies of tile t have landed
        const int st = t % NST;
        const int nt = (int)min((uint32_t)TILE, ne - (uint32_t)(t * TILE));
        if (SMODE == FAR_PACKED || SMODE == FAR_EXP) {
#pragma unroll
            for (int u = 0; u < PER; ++u) {   // entries past nt become zero-mass sources
                const int el = u * 32 + lane;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (el < nt) {
                    const float4 h = S.rh[st][el], l = S.rl[st][el];
                    v = make_float4((h.x - crx) + l.x, (h.y - cry) + l.y, (h.z - crz) + l.z, h.w);
                }
                if (SMODE == FAR_PACKED) {
                    S.tile[2 * el] = make_float4(v.x, v.x, v.y, v.y);
                    S.tile[2 * el + 1] = make_float4(v.z, v.z, v.w, v.w);
                } else {
                    const float c = fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
                    S.tile[2 * el] = make_float4(-2.0f * v.x, -2.0f * v.y, -2.0f * v.z, c);
                    S.tile[2 * el + 1] = make_float4(v.w * v.x, v.w * v.y, v.w * v.z, v.w);
                }
            }
            __syncwarp();
            body(st, nt);
        } else {
            float4 v[PER], vh[PER], vl[PER];
            bool keep[PER], out[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int el = u * 32 + lane;
                keep[u] = out[u] = false;
                if (el < nt) {
                    const float4 h = S.rh[st][el], l = S.rl[st][el];
                    vh[u] = make_float4(h.x - crx, h.y - cry, h.z - crz, 0.0f);
                    vl[u] = l;
                    v[u] = make_float4(vh[u].x + l.x, vh[u].y + l.y, vh[u].z + l.z, h.w);
                    const float gx = fmaxf(fmaxf(sb.lo[0] - v[u].x, v[u].x - sb.hi[0]), 0.0f);
                    const float gy = fmaxf(fmaxf(sb.lo[1] - v[u].y, v[u].y - sb.hi[1]), 0.0f);
                    const float gz = fmaxf(fmaxf(sb.lo[2] - v[u].z, v[u].z - sb.hi[2]), 0.0f);
                    keep[u] = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < sb.R2sq;
                    out[u] = !keep[u];
                }
            }
            const unsigned ltm = (1u << lane) - 1u;
            const unsigned k0 = __ballot_sync(0xffffffffu, keep[0]), k1 = __ballot_sync(0xffffffffu, keep[1]);
            const unsigned o0 = __ballot_sync(0xffffffffu, out[0]), o1 = __ballot_sync(0xffffffffu, out[1]);
            const int n_in = __popc(k0) + __popc(k1), n_out = __popc(o0) + __popc(o1);
#pragma unroll
            for (int u = 0; u < PER; ++u) {   // order kept within each part
                if (keep[u]) {
                    const int j = u == 0 ? __popc(k0 & ltm) : __popc(k0) + __popc(k1 & ltm);
                    S.tile[j] = v[u];
                    S.tile[TILE + j] = vh[u];
                    S.tile[2 * TILE + j] = vl[u];
                } else if (out[u]) {
                    const int j = u == 0 ? __popc(o0 & ltm) : __popc(o0) + __popc(o1 & ltm);
                    S.tile[TILE - n_out + j] = v[u];
                }
            }
            __syncwarp();
            body(n_in, n_out);
        }
        __syncwarp();
    }
}

// sums of the copies into copy 0: a butterfly over the copies when they fill the warp (lpc a power of
// two), else in copy order
template <int KS>
__device__ __forceinline__ void reduce_copies(int lane, int copy, int copies, int lpc, float (&x)[KS], float (&y)[KS],
                                              float (&z)[KS])
{
    if (copies > 1 && copies * lpc == 32) {
        for (int o = lpc; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < KS; ++k) {
                x[k] += __shfl_xor_sync(0xffffffffu, x[k], o);
                y[k] += __shfl_xor_sync(0xffffffffu, y[k], o);
                z[k] += __shfl_xor_sync(0xffffffffu, z[k], o);
            }
        }
        return;
    }
    for (int cc = 1; cc < copies; ++cc) {
        const int src = (copy == 0) ? lane + cc * lpc : lane;
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const float vx = __shfl_sync(0xffffffffu, x[k], src);
            const float vy = __shfl_sync(0xffffffffu, y[k], src);
            const float vz = __shfl_sync(0xffffffffu, z[k], src);
            if (copy == 0) {
                x[k] += vx;
                y[k] += vy;
                z[k] += vz;
            }
        }
    }
}

// ---- packed two-sink arithmetic (f32x2: one instruction, two FP32 lanes) ----
__device__ __forceinline__ uint64_t pk2(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// the body of body_far for two sinks (S*) against one source given twice
// over (X2 = {x, x}, ..): the same roundings per lane
template <bool GUARD>
__device__ __forceinline__ void body_far2(uint64_t X2, uint64_t Y2, uint64_t Z2, uint64_t M2, uint64_t SX, uint64_t SY,
                                          uint64_t SZ, uint64_t E2, uint64_t &AX, uint64_t &AY, uint64_t &AZ)
{
    const uint64_t dx = sub2(X2, SX), dy = sub2(Y2, SY), dz = sub2(Z2, SZ);
    const uint64_t r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, E2)));
    float ra, rb;
    upk2(r2, ra, rb);
    float ia = rsqrtf(ra), ib = rsqrtf(rb);
    if (GUARD) {
        ia = ra > 0.0f ? ia : 0.0f;
        ib = rb > 0.0f ? ib : 0.0f;
    }
    const uint64_t ri = pk2(ia, ib);
    const uint64_t f = mul2(mul2(M2, ri), mul2(ri, ri));
    AX = fma2(dx, f, AX);
    AY = fma2(dy, f, AY);
    AZ = fma2(dz, f, AZ);
}

// The far sweep of one tile: copy c takes sources c, c + copies, ... Every
// lane runs the same number of rounds of two sources (entries from nt to
// PADT are zero-mass sources), so the loop has no divergence; lanes outside
// the copies compute sums that are never used. KP sink pairs per lane.
template <int KP, bool GUARD, typename Stage>
__device__ __forceinline__ void far_tile(const Stage &S, int nt, int copy, int copies, uint64_t E2,
                                         const uint64_t (&SX)[KP], const uint64_t (&SY)[KP], const uint64_t (&SZ)[KP],
                                         uint64_t (&AX)[KP], uint64_t (&AY)[KP], uint64_t (&AZ)[KP])
{
    const int rounds = (nt + 2 * copies - 1) / (2 * copies);
    uint32_t q = (uint32_t)__cvta_generic_to_shared(S.tile) + 32u * (uint32_t)copy;
    const uint32_t step = 32u * (uint32_t)copies;
    for (int m = 0; m < rounds; ++m, q += 2 * step) {
        uint64_t X0, Y0, Z0, M0, X1, Y1, Z1, M1;
        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(X0), "=l"(Y0) : "r"(q));
        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(Z0), "=l"(M0) : "r"(q + 16));
        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(X1), "=l"(Y1) : "r"(q + step));
        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(Z1), "=l"(M1) : "r"(q + step + 16));
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            body_far2<GUARD>(X0, Y0, Z0, M0, SX[k], SY[k], SZ[k], E2, AX[k], AY[k], AZ[k]);
            body_far2<GUARD>(X1, Y1, Z1, M1, SX[k], SY[k], SZ[k], E2, AX[k], AY[k], AZ[k]);
        }
    }
}

// Far sources in expanded form. With the source at s and a sink at k
// (both group-relative), r^2 = |s|^2 + (|k|^2 + eps^2) - 2 s.k and
// sum_j m_j r_j^-3 (s_j - k) = sum_j r_j^-3 (m_j s_j) - k sum_j r_j^-3 m_j, so
// a source stages {-2s, |s|^2, m s, m} and a pair costs the sum c + Q, three
// fma for r^2, rsqrt, two mul for r^-3 and four fma: 10 FP32 lane operations
// against 12 for body_far. The rounding of r^2 is at most about
// 4 u (|s| + |k|)^2 <= 4 u (r + 2 |k|)^2 (u = 2^-24). With a hard part the walk
// takes a cell only beyond R2 + b_max (and beyond its opening radius) and a far
// particle only beyond R2 of the sinks' box, so r >= R2, and with every sink
// within 64 R2 of the reference point the rounding stays below ~4e-3 of r^2
// (r^2 cannot change sign; typical pairs sit far from that bound). Other items
// keep body_far: without a hard part a cell of one or a few particles can be
// taken right next to the sinks, and a very large group in sparse outskirts
// can have far sources at R2 from its edge.
// Q = |k|^2 + eps^2 per sink; the caller subtracts k FM from A at the end.
__device__ __forceinline__ void body_exp2(uint64_t NX, uint64_t NY, uint64_t NZ, uint64_t C2, uint64_t MX, uint64_t MY,
                                           uint64_t MZ, uint64_t M2, uint64_t SX, uint64_t SY, uint64_t SZ, uint64_t Q,
                                           uint64_t &AX, uint64_t &AY, uint64_t &AZ, uint64_t &FM)
{
    const uint64_t r2 = fma2(NX, SX, fma2(NY, SY, fma2(NZ, SZ, add2(C2, Q))));
    float ra, rb;
    upk2(r2, ra, rb);
    const uint64_t ri = pk2(rsqrtf(ra), rsqrtf(rb));
    const uint64_t t = mul2(mul2(ri, ri), ri);
    AX = fma2(MX, t, AX);
    AY = fma2(MY, t, AY);
    AZ = fma2(MZ, t, AZ);
    FM = fma2(M2, t, FM);
}

// The expanded sweep of one tile (same rounds and copies as far_tile); each
// source is stored once, {-2s, |s|^2} {m s, m}, and every value is paired
// with itself in registers for the packed arithmetic.
template <int KP, typename Stage>
__device__ __forceinline__ void exp_tile(const Stage &S, int nt, int copy, int copies, const uint64_t (&SX)[KP],
                                          const uint64_t (&SY)[KP], const uint64_t (&SZ)[KP], const uint64_t (&Q)[KP],
                                          uint64_t (&AX)[KP], uint64_t (&AY)[KP], uint64_t (&AZ)[KP],
                                          uint64_t (&FM)[KP])
{
    const int rounds = (nt + 2 * copies - 1) / (2 * copies);
    uint32_t q = (uint32_t)__cvta_generic_to_shared(S.tile) + 32u * (uint32_t)copy;
    const uint32_t step = 32u * (uint32_t)copies;
    for (int m = 0; m < rounds; ++m, q += 2 * step) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t qa = q + (h ? step : 0u);
            float nx, ny, nz, c, mx, my, mz, ms;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(nx), "=f"(ny), "=f"(nz), "=f"(c) : "r"(qa));
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(mx), "=f"(my), "=f"(mz), "=f"(ms) : "r"(qa + 16));
            const uint64_t NX = pk2(nx, nx), NY = pk2(ny, ny), NZ = pk2(nz, nz), C2 = pk2(c, c);
            const uint64_t MX = pk2(mx, mx), MY = pk2(my, my), MZ = pk2(mz, mz), M2 = pk2(ms, ms);
#pragma unroll
            for (int k = 0; k < KP; ++k)
                body_exp2(NX, NY, NZ, C2, MX, MY, MZ, M2, SX[k], SY[k], SZ[k], Q[k], AX[k], AY[k], AZ[k], FM[k]);
        }
    }
}

// NEAR = false: cells + far particles -> soft. NEAR = true: near particles ->
// soft (1 - K) and/or hard (K), by SOFT/HARD.
// The near kernels wait on the latency of their loads (work items, sinks, list
// entries): they are held to 4 blocks of 128 threads per SM (at most 128
// registers), one block more than they would use freely.
template <int KS, bool NEAR, bool SOFT, bool HARD, int NST>
__global__ void __launch_bounds__(PAIR_THREADS, NEAR ? NEAR_MIN_BLOCKS : 0) k_pair_f32(PairArgs a)
{
    using Stage = WarpStage<NST>;
    __shared__ Stage stages[PAIR_WARPS];
    if (a.st->code) return;
    const int lane = threadIdx.x & 31;
    Stage &S = stages[threadIdx.x >> 5];
    for (int e = 2 * TILE + lane; e < 2 * PADT; e += 32) S.tile[e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const int64_t W = (int64_t)*a.nwork;
    unsigned long long inter = 0;
    int64_t w = next_item(a.counter, lane);
    while (w < W) {
        const int64_t wn = next_item(a.counter, lane);   // the next item's number arrives while this one runs
        // the near kernel takes its items from the last written to the first, which shortens the end of its
        // launch (fewer SMs idle while the last items run: 0.353 -> 0.338 ms per soft step at N = 2^17; the same
        // at 2^24); the far kernel is faster in the walk's order
        const WorkItem d = a.items[NEAR ? W - 1 - w : w];
        const SysParams &P = a.sp[d.sys];
        HardC H;
        H.eps2 = P.eps2f;
        H.R2 = P.R2f;
        H.R2sq = P.R2sqf;
        H.R2sqlo = P.R2sqlo;
        H.invdR = P.invdRf;
        const ItemSrc src = {d.cbase, d.pbase, d.Lc, d.e0, d.e1};
        const uint32_t first = d.first;
        const int n = (int)(d.n & ~MULTI);
        const bool multi = (d.n & MULTI) != 0;
        const float4 cref = a.phi[first];
        const float crx = cref.x, cry = cref.y, crz = cref.z;
        inter += (unsigned long long)n * (d.e1 - d.e0);
        for (int r0 = 0, per_round = 0; r0 < n; r0 += per_round) {
            const int rem = n - r0;
            int lpc = rem <= 32 * KS ? (rem + KS - 1) / KS : 32;
            // far kernel: when the copies would leave many sink slots idle (rem * copies below
            // FAR_SPLIT_PCT % of 32 KS), this round takes a power of two of lanes per copy, which keeps
            // every slot busy, and leaves the other sinks to the next round
            if (!NEAR && rem * (32 / lpc) * 100 < FAR_SPLIT_PCT * 32 * KS) lpc = 1 << (31 - __clz(lpc));
            const int copies = 32 / lpc;
            const int copy = lane / lpc, slot = lane - copy * lpc;
            const bool active = copy < copies;
            per_round = lpc * KS;
            float sx[KS], sy[KS], sz[KS], ax[KS], ay[KS], az[KS], bx[KS], by[KS], bz[KS];
            float shx[KS], shy[KS], shz[KS], slx[KS], sly[KS], slz[KS];
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                int si = r0 + kk * lpc + slot;
                si = si < n ? si : n - 1;
                const float4 h = a.phi[first + si], l = a.plo[first + si];
                shx[kk] = h.x - crx;   // rebased hi (exact): differences with the staged sources' are exact
                shy[kk] = h.y - cry;
                shz[kk] = h.z - crz;
                slx[kk] = l.x;
                sly[kk] = l.y;
                slz[kk] = l.z;
                sx[kk] = (h.x - crx) + l.x;
                sy[kk] = (h.y - cry) + l.y;
                sz[kk] = (h.z - crz) + l.z;
                ax[kk] = ay[kk] = az[kk] = 0.0f;
                bx[kk] = by[kk] = bz[kk] = 0.0f;
            }
            if (!NEAR) {
                constexpr int KP = (KS + 1) / 2;
                uint64_t SX[KP], SY[KP], SZ[KP], AX[KP], AY[KP], AZ[KP];
#pragma unroll
                for (int p = 0; p < KP; ++p) {
                    const int k1 = 2 * p + 1 < KS ? 2 * p + 1 : 2 * p;
                    SX[p] = pk2(sx[2 * p], sx[k1]);
                    SY[p] = pk2(sy[2 * p], sy[k1]);
                    SZ[p] = pk2(sz[2 * p], sz[k1]);
                    AX[p] = AY[p] = AZ[p] = 0ull;
                }
                const uint64_t E2 = pk2(H.eps2, H.eps2);
                // the expanded form only with a hard part (then every far source is at least R2 from the sinks'
                // box; without one, cells and particles can sit next to the sinks) and for sinks within 64 R2
                // of the reference point: the rounding of r^2 stays below 4 u (1 + 2 * 64)^2 ~ 4e-3 of r^2
                float k2 = 0.0f;
#pragma unroll
                for (int kk = 0; kk < KS; ++kk) k2 = fmaxf(k2, fmaf(sx[kk], sx[kk], fmaf(sy[kk], sy[kk], sz[kk] * sz[kk])));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) k2 = fmaxf(k2, __shfl_xor_sync(0xffffffffu, k2, o));
                if (H.eps2 > 0.0f && P.has_hard && k2 <= 4096.0f * H.R2sq) {
                    uint64_t Q[KP], FM[KP];
#pragma unroll
                    for (int p = 0; p < KP; ++p) {
                        const int k1 = 2 * p + 1 < KS ? 2 * p + 1 : 2 * p;
                        Q[p] = pk2(fmaf(sx[2 * p], sx[2 * p], fmaf(sy[2 * p], sy[2 * p], fmaf(sz[2 * p], sz[2 * p], H.eps2))),
                                   fmaf(sx[k1], sx[k1], fmaf(sy[k1], sy[k1], fmaf(sz[k1], sz[k1], H.eps2))));
                        FM[p] = 0ull;
                    }
                    pipeline<FAR_EXP, NST>(a, src, S, lane, crx, cry, crz, SinkBox(), [&](int, int nt) {
                        exp_tile<KP>(S, nt, copy, copies, SX, SY, SZ, Q, AX, AY, AZ, FM);
                    });
#pragma unroll
                    for (int p = 0; p < KP; ++p) {   // A - k FM
                        const int k1 = 2 * p + 1 < KS ? 2 * p + 1 : 2 * p;
                        AX[p] = fma2(pk2(-sx[2 * p], -sx[k1]), FM[p], AX[p]);
                        AY[p] = fma2(pk2(-sy[2 * p], -sy[k1]), FM[p], AY[p]);
                        AZ[p] = fma2(pk2(-sz[2 * p], -sz[k1]), FM[p], AZ[p]);
                    }
                } else {
                    if (H.eps2 > 0.0f)
                        pipeline<FAR_PACKED, NST>(a, src, S, lane, crx, cry, crz, SinkBox(), [&](int, int nt) {
                            far_tile<KP, false>(S, nt, copy, copies, E2, SX, SY, SZ, AX, AY, AZ);
                        });
                    else   // eps = 0 without a hard part: a sink meets itself in its far particles
                        pipeline<FAR_PACKED, NST>(a, src, S, lane, crx, cry, crz, SinkBox(), [&](int, int nt) {
                            far_tile<KP, true>(S, nt, copy, copies, E2, SX, SY, SZ, AX, AY, AZ);
                        });
                }
#pragma unroll
                for (int p = 0; p < KP; ++p) {
                    float t0, t1;
                    upk2(AX[p], t0, t1);
                    ax[2 * p] = t0;
                    if (2 * p + 1 < KS) ax[2 * p + 1] = t1;
                    upk2(AY[p], t0, t1);
                    ay[2 * p] = t0;
                    if (2 * p + 1 < KS) ay[2 * p + 1] = t1;
                    upk2(AZ[p], t0, t1);
                    az[2 * p] = t0;
                    if (2 * p + 1 < KS) az[2 * p + 1] = t1;
                }
            } else {
                // the box of this round's sinks: sources farther than R2 from it have K = 0 for every sink
                SinkBox sb;
                sb.R2sq = H.R2sq;
                {
                    float lo0 = sx[0], lo1 = sy[0], lo2 = sz[0], hi0 = sx[0], hi1 = sy[0], hi2 = sz[0];
#pragma unroll
                    for (int k = 1; k < KS; ++k) {
                        lo0 = fminf(lo0, sx[k]);
                        lo1 = fminf(lo1, sy[k]);
                        lo2 = fminf(lo2, sz[k]);
                        hi0 = fmaxf(hi0, sx[k]);
                        hi1 = fmaxf(hi1, sy[k]);
                        hi2 = fmaxf(hi2, sz[k]);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
                        lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
                        lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
                        hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
                        hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
                        hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
                    }
                    sb.lo[0] = lo0;
                    sb.lo[1] = lo1;
                    sb.lo[2] = lo2;
                    sb.hi[0] = hi0;
                    sb.hi[1] = hi1;
                    sb.hi[2] = hi2;
                }
                pipeline<NEAR_FILTER, NST>(a, src, S, lane, crx, cry, crz, sb, [&](int n_in, int n_out) {
                    if (!active) return;
                    for (int j = copy; j < n_in; j += copies) {   // sources within R2 of the box
                        const float4 q = S.tile[j];
                        float dx[KS], dy[KS], dz[KS], r2u[KS];
                        bool any_in = false;
#pragma unroll
                        for (int k = 0; k < KS; ++k) {
                            dx[k] = q.x - sx[k];
                            dy[k] = q.y - sy[k];
                            dz[k] = q.z - sz[k];
                            r2u[k] = fmaf(dx[k], dx[k], fmaf(dy[k], dy[k], dz[k] * dz[k]));
                            any_in |= r2u[k] < H.R2sq;
                        }
                        float4 hh = make_float4(0.0f, 0.0f, 0.0f, 0.0f), ll = hh;
                        if (any_in) {
                            hh = S.tile[TILE + j];
                            ll = S.tile[2 * TILE + j];
                        }
#pragma unroll
                        for (int k = 0; k < KS; ++k)
                            near_finish<SOFT, HARD>(q.w, dx[k], dy[k], dz[k], r2u[k], hh, ll, shx[k], shy[k], shz[k],
                                                    slx[k], sly[k], slz[k], H, ax[k], ay[k], az[k], bx[k], by[k],
                                                    bz[k]);
                    }
                    if (SOFT)   // the rest: K = 0 for every sink, weight 1 on the soft force
                        for (int j = TILE - n_out + copy; j < TILE; j += copies) {
                            const float4 q = S.tile[j];
#pragma unroll
                            for (int k = 0; k < KS; ++k) body_far<false>(q, sx[k], sy[k], sz[k], H.eps2, ax[k], ay[k], az[k]);
                        }
                });
            }
            if (SOFT) reduce_copies<KS>(lane, copy, copies, lpc, ax, ay, az);
            if (HARD) reduce_copies<KS>(lane, copy, copies, lpc, bx, by, bz);
            if (copy == 0) {
                const float Gf = P.Gf;
#pragma unroll
                for (int kk = 0; kk < KS; ++kk) {
                    const int si = r0 + kk * lpc + slot;
                    if (si < n) {
                        const uint32_t i = first + si;
                        if (SOFT) {
                            float *ox = (float *)a.as[0], *oy = (float *)a.as[1], *oz = (float *)a.as[2];
                            if (!NEAR && !multi) {
                                ox[i] = Gf * ax[kk];
                                oy[i] = Gf * ay[kk];
                                oz[i] = Gf * az[kk];
                            } else {   // several items, or the near part added to the far part
                                atomicAdd(ox + i, Gf * ax[kk]);
                                atomicAdd(oy + i, Gf * ay[kk]);
                                atomicAdd(oz + i, Gf * az[kk]);
                            }
                        }
                        if (HARD) {
                            float *ox = (float *)a.ah[0], *oy = (float *)a.ah[1], *oz = (float *)a.ah[2];
                            if (!multi) {
                                ox[i] = Gf * bx[kk];
                                oy[i] = Gf * by[kk];
                                oz[i] = Gf * bz[kk];
                            } else {
                                atomicAdd(ox + i, Gf * bx[kk]);
                                atomicAdd(oy + i, Gf * by[kk]);
                                atomicAdd(oz + i, Gf * bz[kk]);
                            }
                        }
                    }
                }
            }
        }
        w = wn;
    }
    cp_wait<0>();   // nothing may stay in flight into shared memory at exit
    if (lane == 0) atomicAdd(NEAR ? a.inter_hard : a.inter_soft, inter);
}

// ---------------------------------------------------------------------------
// FP64 kernel: one warp per group, one lane per sink (rounds of 32 sinks),
// sources staged as double4 in shared memory.
// ---------------------------------------------------------------------------
template <bool NEAR>
__global__ void __launch_bounds__(PAIR_THREADS) k_pair_f64(PairArgs a)
{
    __shared__ double4_32a tiles[PAIR_WARPS][TILE];
    if (a.st->code) return;
    const int lane = threadIdx.x & 31;
    double4_32a *tile = tiles[threadIdx.x >> 5];
    const int64_t ng = *a.ngroups;
    unsigned long long inter = 0;
    for (;;) {
        const int64_t g = next_item(a.counter, lane);
        if (g >= ng) break;
        const uint32_t first = a.gfirst[g];
        const int n = (int)a.gcount[g];
        const SysParams P = a.sp[a.gsys[g]];
        uint64_t c0, c1, p0, p1;
        if (!NEAR) {
            c0 = a.off[g];
            c1 = a.off[g + 1];
            p0 = a.off[ng + g];
            p1 = a.off[ng + g + 1];
        } else {
            c0 = c1 = 0;
            p0 = a.off[2 * ng + g];
            p1 = a.off[2 * ng + g + 1];
        }
        inter += (unsigned long long)n * ((c1 - c0) + (p1 - p0));
        for (int r0 = 0; r0 < n; r0 += 32) {
            const int si = r0 + lane;
            const double4_32a s = a.pd[first + (si < n ? si : n - 1)];
            double ax = 0.0, ay = 0.0, az = 0.0, bx = 0.0, by = 0.0, bz = 0.0;
            for (int part = 0; part < 2; ++part) {
                const uint64_t q0 = part ? p0 : c0, q1 = part ? p1 : c1;
                for (uint64_t t0 = q0; t0 < q1; t0 += TILE) {
                    const int nt = (int)min((uint64_t)TILE, q1 - t0);
                    for (int e = lane; e < nt; e += 32) {
                        const uint32_t idx = a.list[t0 + e];
                        tile[e] = part ? a.pd[idx] : a.nD[idx];
                    }
                    __syncwarp();
                    for (int j = 0; j < nt; ++j) {
                        const double4_32a q = tile[j];
                        const double dx = q.x - s.x, dy = q.y - s.y, dz = q.z - s.z;
                        const double r2u = dx * dx + dy * dy + dz * dz;
                        const double r2 = r2u + P.eps2;
                        const double ri = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
                        const double f = q.w * ri * ri * ri;
                        if (!NEAR) {
                            ax += f * dx;
                            ay += f * dy;
                            az += f * dz;
                        } else {
                            const double K = r2u < P.R2sq ? dll_K64(sqrt(r2u), P.R1, P.R2) : 0.0;
                            const double fs = f * (1.0 - K);
                            ax += fs * dx;
                            ay += fs * dy;
                            az += fs * dz;
                            const double fh = f * K;
                            bx += fh * dx;
                            by += fh * dy;
                            bz += fh * dz;
                        }
                    }
                    __syncwarp();
                }
            }
            if (si < n) {
                const uint32_t i = first + si;
                if (!NEAR) {
                    ((double *)a.as[0])[i] = P.G * ax;
                    ((double *)a.as[1])[i] = P.G * ay;
                    ((double *)a.as[2])[i] = P.G * az;
                } else {
                    if (a.want_soft) {   // the far kernel ran first on the same stream
                        ((double *)a.as[0])[i] += P.G * ax;
                        ((double *)a.as[1])[i] += P.G * ay;
                        ((double *)a.as[2])[i] += P.G * az;
                    }
                    if (a.want_hard) {
                        ((double *)a.ah[0])[i] = P.G * bx;
                        ((double *)a.ah[1])[i] = P.G * by;
                        ((double *)a.ah[2])[i] = P.G * bz;
                    }
                }
            }
        }
    }
    if (lane == 0) atomicAdd(NEAR ? a.inter_hard : a.inter_soft, inter);
}

void fill_args(hybrid_ctx *c, PairArgs &a)
{
    a.ngroups = (const int64_t *)c->ngroups_dev.p;
    a.gfirst = (const uint32_t *)c->gfirst.p;
    a.gcount = (const uint32_t *)c->gcount.p;
    a.gsys = (const uint32_t *)c->gsys.p;
    a.sp = (const SysParams *)c->sp_dev.p;
    a.off = (const uint64_t *)c->lcnt.p;
    a.list = (const uint32_t *)c->list.p;
    a.phi = (const float4 *)c->phi.p;
    a.plo = (const float4 *)c->plo.p;
    a.nA = (const float4 *)c->nA.p;
    a.nB = (const float4 *)c->nB.p;
    a.pd = (const double4_32a *)c->pd.p;
    a.nD = (const double4_32a *)c->nD.p;
    for (int d = 0; d < 3; ++d) {
        a.as[d] = c->acc_s[d].p;
        a.ah[d] = c->acc_h[d].p;
    }
    unsigned long long *ctr = (unsigned long long *)c->counter.p;
    a.counter = ctr + 2;
    a.inter_soft = ctr + 6;
    a.inter_hard = ctr + 7;
    a.st = status_dev(c);
    a.items = nullptr;
    a.nwork = nullptr;
    a.want_soft = a.want_hard = 0;
}

// staging depth: tile_depth (2, 3 or 4; 0 = 3) for the far kernel, 3 for the near kernel
template <int KS, bool NEAR, bool SOFT, bool HARD>
void go_f32(hybrid_ctx *c, const PairArgs &a)
{
    const int depth = NEAR || c->p.tile_depth == 0 ? 3 : c->p.tile_depth;
    if (!NEAR && depth == 2) k_pair_f32<KS, NEAR, SOFT, HARD, 2><<<c->nsm * 16, PAIR_THREADS, 0, c->st>>>(a);
    else if (!NEAR && depth == 4) k_pair_f32<KS, NEAR, SOFT, HARD, 4><<<c->nsm * 16, PAIR_THREADS, 0, c->st>>>(a);
    else k_pair_f32<KS, NEAR, SOFT, HARD, 3><<<c->nsm * 16, PAIR_THREADS, 0, c->st>>>(a);
}

// Sinks per lane KS = ceil(n_crit / threads_per_group): 1, 2, 4 or (far
// kernel only) 8; the default is 4 (one shared-memory read feeds 4
// interactions; the far kernel runs them as packed sink pairs).
template <bool NEAR, bool SOFT, bool HARD>
void go_ks(hybrid_ctx *c, const PairArgs &a)
{
    int ks;
    if (c->p.threads_per_group > 0) ks = (c->p.n_crit + c->p.threads_per_group - 1) / c->p.threads_per_group;
    else ks = 4;
    ks = ks <= 1 ? 1 : (ks <= 2 ? 2 : (ks <= 4 || NEAR ? 4 : 8));   // 8 sinks per lane: far kernel only
    if (ks == 1) go_f32<1, NEAR, SOFT, HARD>(c, a);
    else if (ks == 2) go_f32<2, NEAR, SOFT, HARD>(c, a);
    else if (ks == 4) go_f32<4, NEAR, SOFT, HARD>(c, a);
    else if constexpr (!NEAR) go_f32<8, NEAR, SOFT, HARD>(c, a);
}

// near = false: cells and far particles (soft); near = true: near particles
// (soft and/or hard per mode bits)
void launch_pairs(hybrid_ctx *c, bool near, int mode)
{
    PairArgs a;
    fill_args(c, a);
    a.want_soft = mode & 1;
    a.want_hard = (mode >> 1) & 1;
    Status *st = status_dev(c);
    unsigned long long *ctr = (unsigned long long *)c->counter.p;
    cudaMemsetAsync(ctr + 2, 0, sizeof(unsigned long long), c->st);
    cudaMemsetAsync(ctr + (near ? 7 : 6), 0, sizeof(unsigned long long), c->st);
    const int kind = near ? PROF_HARD : PROF_SOFT;
    cudaEvent_t e0 = nullptr;
    prof_begin(c, kind, &e0);
    if (c->p.precision == 0) {
        if (near) k_pair_f64<true><<<c->nsm * 12, PAIR_THREADS, 0, c->st>>>(a);
        else k_pair_f64<false><<<c->nsm * 12, PAIR_THREADS, 0, c->st>>>(a);
        c->launches++;
    } else {
        // work items written by the one-pass walk: far ones in wmap, near ones in wnear
        a.items = (const WorkItem *)(near ? c->wnear.p : c->wmap.p);
        a.nwork = (const uint64_t *)c->counter.p + (near ? 12 : 11);
        if (!near)
            for (int d = 0; d < 3; ++d) cudaMemsetAsync(c->acc_s[d].p, 0, (size_t)c->N * sizeof(float), c->st);
        if (near && a.want_hard)
            for (int d = 0; d < 3; ++d) cudaMemsetAsync(c->acc_h[d].p, 0, (size_t)c->N * sizeof(float), c->st);
        if (!near) go_ks<false, true, false>(c, a);
        else if (a.want_soft && a.want_hard) go_ks<true, true, true>(c, a);
        else if (a.want_soft) go_ks<true, true, false>(c, a);
        else go_ks<true, false, true>(c, a);
        c->launches += 1;
    }
    prof_end(c, kind, e0);
}

}  // namespace

void launch_pair_far(hybrid_ctx *c) { launch_pairs(c, false, 1); }

namespace {
template <int KS, bool NEAR, bool SOFT, bool HARD, int NST>
cudaError_t prefer_shared()
{
    return cudaFuncSetAttribute(k_pair_f32<KS, NEAR, SOFT, HARD, NST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}
}  // namespace

// The pair kernels are limited by registers and by shared memory per block:
// the whole carveout goes to shared memory (they read nothing through L1
// twice), so shared memory never limits their blocks per SM below registers.
cudaError_t init_pair_kernels()
{
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {prefer_shared<1, false, true, false, 2>(), prefer_shared<1, false, true, false, 3>(),
                          prefer_shared<1, false, true, false, 4>(), prefer_shared<2, false, true, false, 2>(),
                          prefer_shared<2, false, true, false, 3>(), prefer_shared<2, false, true, false, 4>(),
                          prefer_shared<4, false, true, false, 2>(), prefer_shared<4, false, true, false, 3>(),
                          prefer_shared<4, false, true, false, 4>(), prefer_shared<8, false, true, false, 2>(),
                          prefer_shared<8, false, true, false, 3>(), prefer_shared<8, false, true, false, 4>(),
                          prefer_shared<1, true, true, true, 3>(), prefer_shared<2, true, true, true, 3>(),
                          prefer_shared<4, true, true, true, 3>(), prefer_shared<1, true, true, false, 3>(),
                          prefer_shared<2, true, true, false, 3>(), prefer_shared<4, true, true, false, 3>(),
                          prefer_shared<1, true, false, true, 3>(), prefer_shared<2, true, false, true, 3>(),
                          prefer_shared<4, true, false, true, 3>()})
        if (e == cudaSuccess) e = r;
    return e;
}
void launch_pair_near(hybrid_ctx *c, int mode) { launch_pairs(c, true, mode); }

}  // namespace hy
