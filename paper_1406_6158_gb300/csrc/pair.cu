// pair.cu -- pair kernels of the soft and hard forces (Eq. 2 split by Eq. 7-10).
//
// The walk gives every sink group three lists:
//   cells and far particles: K = 0 for every pair (the walk's R2 + b_max
//     test), so they only add F to the soft force ("far" kernel);
//   near particles: the only pairs where K can be non-zero; one pass adds
//     F (1 - K) to the soft force and F K to the hard force ("near" kernel).
//
// FP32 form. Work item = (group, chunk of at most lch consecutive entries of
// one of the group's lists), pulled from a global counter. One warp per work
// item: sources are staged, 64 at a time, into the warp's shared-memory tile
// as float4 {x, y, z, m} relative to the group's reference point (the hi part
// of its first sink: on the hi grid, so hi - c is exact); the next tile's
// gathers are issued before the current tile is used. A group of n sinks uses
// lpc = ceil(n / KS) lanes per copy with KS sinks per lane in registers, and
// copies = 32 / lpc copies of the group split the sources (source j goes to
// copy j mod copies) and are added at the end. A group with one chunk stores
// its sums; a group with several adds them atomically into zeroed outputs.
// rsqrtf runs on the CUDA cores: the pair sum is not a dense contraction.
//
// FP64 form (the plain form): one warp per group, one sink per lane, plain
// FP64 differences and 1/sqrt.
#include "hy_internal.cuh"

namespace hy {

namespace {

constexpr int PAIR_THREADS = 128;
constexpr int PAIR_WARPS = PAIR_THREADS / 32;
constexpr int TILE = 64;
constexpr int LCH_FAR = 512, LCH_NEAR = 256;

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
    // work items: chunks of at most lch list entries of one group
    const uint32_t *wstart;   // [ng + 1]
    const uint32_t *wmap;     // work item -> group
    const uint64_t *nwork;
    int lch;
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

// near particle: soft += F (1 - K), hard += F K
template <bool SOFT, bool HARD>
__device__ __forceinline__ void body_near(const float4 t, const float4 th, const float4 tl, float sx, float sy,
                                          float sz, float shx, float shy, float shz, float slx, float sly, float slz,
                                          const HardC &H, float &sax, float &say, float &saz, float &hax, float &hay,
                                          float &haz)
{
    const float dx = t.x - sx, dy = t.y - sy, dz = t.z - sz;
    const float r2u = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool inside = r2u < H.R2sq;
    if (!SOFT && !inside) return;
    const float r2 = r2u + H.eps2;
    const float ri = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    const float f = t.w * ri * (ri * ri);
    float K = 0.0f;
    if (inside)
        K = dll_K_precise(r2u, __fsub_rn(th.x, shx), __fsub_rn(th.y, shy), __fsub_rn(th.z, shz),
                          __fsub_rn(tl.x, slx), __fsub_rn(tl.y, sly), __fsub_rn(tl.z, slz), H);
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
// FP32 staging
// ---------------------------------------------------------------------------
struct SrcCell {
    __device__ __forceinline__ static void load(const PairArgs &a, uint32_t idx, float crx, float cry, float crz,
                                                float4 &t, float4 &th, float4 &tl)
    {
        const float4 A = a.nA[idx], B = a.nB[idx];
        t = make_float4((A.x - crx) + B.x, (A.y - cry) + B.y, (A.z - crz) + B.z, A.w);
        th = tl = t;
    }
};
struct SrcPart {
    __device__ __forceinline__ static void load(const PairArgs &a, uint32_t idx, float crx, float cry, float crz,
                                                float4 &t, float4 &th, float4 &tl)
    {
        const float4 h = a.phi[idx], l = a.plo[idx];
        const float hx = h.x - crx, hy = h.y - cry, hz = h.z - crz;
        t = make_float4(hx + l.x, hy + l.y, hz + l.z, h.w);
        th = make_float4(hx, hy, hz, 0.0f);
        tl = l;
    }
};

// One list range [q0, q1) against the lane's KS sinks.
// MODE 0: far (weight 1, no guard), 1: far with the r = 0 guard, 2: near.
template <int KS, int MODE, bool SOFT, bool HARD, typename SRC>
__device__ __forceinline__ void sweep(const PairArgs &a, uint64_t q0, uint64_t q1, float4 *tile, float4 *tile_h,
                                      float4 *tile_l, int lane, int copy, int copies, bool active, float crx, float cry,
                                      float crz, const float (&sx)[KS], const float (&sy)[KS], const float (&sz)[KS],
                                      const float (&shx)[KS], const float (&shy)[KS], const float (&shz)[KS],
                                      const float (&slx)[KS], const float (&sly)[KS], const float (&slz)[KS],
                                      const HardC &H, float (&ax)[KS], float (&ay)[KS], float (&az)[KS],
                                      float (&bx)[KS], float (&by)[KS], float (&bz)[KS])
{
    constexpr int PER = TILE / 32;
    constexpr bool NEAR = (MODE == 2);
    float4 rt[PER], rh[PER], rl[PER];
    auto fetch = [&](uint64_t t0) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const uint64_t e = t0 + (uint64_t)(u * 32 + lane);
            if (e < q1) SRC::load(a, a.list[e], crx, cry, crz, rt[u], rh[u], rl[u]);
        }
    };
    if (q0 < q1) fetch(q0);
    for (uint64_t t0 = q0; t0 < q1; t0 += TILE) {
        const int nt = (int)min((uint64_t)TILE, q1 - t0);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = u * 32 + lane;
            if (e < nt) {
                tile[e] = rt[u];
                if (NEAR) {
                    tile_h[e] = rh[u];
                    tile_l[e] = rl[u];
                }
            }
        }
        __syncwarp();
        if (t0 + TILE < q1) fetch(t0 + TILE);   // next tile's loads overlap this tile's arithmetic
        if (active) {
            int j = copy;
            if (!NEAR) {   // two sources per round: one loop overhead per 2 KS interactions
                for (; j + copies < nt; j += 2 * copies) {
                    const float4 q0 = tile[j], q1 = tile[j + copies];
#pragma unroll
                    for (int k = 0; k < KS; ++k) {
                        body_far<MODE == 1>(q0, sx[k], sy[k], sz[k], H.eps2, ax[k], ay[k], az[k]);
                        body_far<MODE == 1>(q1, sx[k], sy[k], sz[k], H.eps2, ax[k], ay[k], az[k]);
                    }
                }
            }
            for (; j < nt; j += copies) {
                const float4 q = tile[j];
                if (!NEAR) {
#pragma unroll
                    for (int k = 0; k < KS; ++k) body_far<MODE == 1>(q, sx[k], sy[k], sz[k], H.eps2, ax[k], ay[k], az[k]);
                } else {
                    const float4 qh = tile_h[j], ql = tile_l[j];
#pragma unroll
                    for (int k = 0; k < KS; ++k)
                        body_near<SOFT, HARD>(q, qh, ql, sx[k], sy[k], sz[k], shx[k], shy[k], shz[k], slx[k], sly[k],
                                              slz[k], H, ax[k], ay[k], az[k], bx[k], by[k], bz[k]);
                }
            }
        }
        __syncwarp();
    }
}

// sums of the copies into copy 0, in copy order
template <int KS>
__device__ __forceinline__ void reduce_copies(int lane, int copy, int copies, int lpc, float (&x)[KS], float (&y)[KS],
                                              float (&z)[KS])
{
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

// NEAR = false: cells + far particles -> soft. NEAR = true: near particles ->
// soft (1 - K) and/or hard (K), by SOFT/HARD.
template <int KS, bool NEAR, bool SOFT, bool HARD>
__global__ void __launch_bounds__(PAIR_THREADS) k_pair_f32(PairArgs a)
{
    constexpr int HT = NEAR ? TILE : 1;
    __shared__ float4 tiles[PAIR_WARPS][TILE];
    __shared__ float4 tiles_h[PAIR_WARPS][HT];
    __shared__ float4 tiles_l[PAIR_WARPS][HT];
    if (a.st->code) return;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    float4 *tile = tiles[wid];
    float4 *tile_h = tiles_h[wid];
    float4 *tile_l = tiles_l[wid];
    const int64_t ng = *a.ngroups;
    const int64_t W = (int64_t)*a.nwork;
    unsigned long long inter = 0;
    for (;;) {
        const int64_t w = next_item(a.counter, lane);
        if (w >= W) break;
        const uint32_t g = a.wmap[w];
        const uint32_t ws0 = a.wstart[g];
        const int nchunk = (int)(a.wstart[g + 1] - ws0);
        const uint64_t k = (uint64_t)(w - ws0);
        const uint32_t first = a.gfirst[g];
        const int n = (int)a.gcount[g];
        const SysParams &P = a.sp[a.gsys[g]];
        HardC H;
        H.eps2 = P.eps2f;
        H.R2 = P.R2f;
        H.R2sq = P.R2sqf;
        H.R2sqlo = P.R2sqlo;
        H.invdR = P.invdRf;
        const float4 cref = a.phi[first];
        const float crx = cref.x, cry = cref.y, crz = cref.z;
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
        const uint64_t Lc = c1 - c0, L = Lc + (p1 - p0);
        const uint64_t e0 = k * (uint64_t)a.lch, e1 = min(L, e0 + (uint64_t)a.lch);
        const uint64_t qc0 = c0 + min(e0, Lc), qc1 = c0 + min(e1, Lc);
        const uint64_t qp0 = p0 + (e0 > Lc ? e0 - Lc : 0), qp1 = p0 + (e1 > Lc ? e1 - Lc : 0);
        inter += (unsigned long long)n * (e1 > e0 ? e1 - e0 : 0);
        const int lpc = n <= 32 * KS ? (n + KS - 1) / KS : 32;
        const int copies = 32 / lpc;
        const int copy = lane / lpc, slot = lane - copy * lpc;
        const bool active = copy < copies;
        const int per_round = lpc * KS;
        for (int r0 = 0; r0 < n; r0 += per_round) {
            float sx[KS], sy[KS], sz[KS], ax[KS], ay[KS], az[KS], bx[KS], by[KS], bz[KS];
            float shx[KS], shy[KS], shz[KS], slx[KS], sly[KS], slz[KS];
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                int si = r0 + kk * lpc + slot;
                si = si < n ? si : n - 1;
                const float4 h = a.phi[first + si], l = a.plo[first + si];
                shx[kk] = h.x - crx;
                shy[kk] = h.y - cry;
                shz[kk] = h.z - crz;
                slx[kk] = l.x;
                sly[kk] = l.y;
                slz[kk] = l.z;
                sx[kk] = shx[kk] + l.x;
                sy[kk] = shy[kk] + l.y;
                sz[kk] = shz[kk] + l.z;
                ax[kk] = ay[kk] = az[kk] = 0.0f;
                bx[kk] = by[kk] = bz[kk] = 0.0f;
            }
            if (!NEAR) {
                sweep<KS, 0, true, false, SrcCell>(a, qc0, qc1, tile, tile_h, tile_l, lane, copy, copies, active, crx,
                                                    cry, crz, sx, sy, sz, shx, shy, shz, slx, sly, slz, H, ax, ay, az,
                                                    bx, by, bz);
                if (H.eps2 > 0.0f)
                    sweep<KS, 0, true, false, SrcPart>(a, qp0, qp1, tile, tile_h, tile_l, lane, copy, copies, active,
                                                        crx, cry, crz, sx, sy, sz, shx, shy, shz, slx, sly, slz, H, ax,
                                                        ay, az, bx, by, bz);
                else
                    sweep<KS, 1, true, false, SrcPart>(a, qp0, qp1, tile, tile_h, tile_l, lane, copy, copies, active,
                                                        crx, cry, crz, sx, sy, sz, shx, shy, shz, slx, sly, slz, H, ax,
                                                        ay, az, bx, by, bz);
            } else {
                sweep<KS, 2, SOFT, HARD, SrcPart>(a, qp0, qp1, tile, tile_h, tile_l, lane, copy, copies, active, crx,
                                                   cry, crz, sx, sy, sz, shx, shy, shz, slx, sly, slz, H, ax, ay, az, bx,
                                                   by, bz);
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
                            if (!NEAR && nchunk == 1) {
                                ox[i] = Gf * ax[kk];
                                oy[i] = Gf * ay[kk];
                                oz[i] = Gf * az[kk];
                            } else {   // several chunks, or the near part added to the far part
                                atomicAdd(ox + i, Gf * ax[kk]);
                                atomicAdd(oy + i, Gf * ay[kk]);
                                atomicAdd(oz + i, Gf * az[kk]);
                            }
                        }
                        if (HARD) {
                            float *ox = (float *)a.ah[0], *oy = (float *)a.ah[1], *oz = (float *)a.ah[2];
                            if (nchunk == 1) {
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
    }
    if (lane == 0) atomicAdd(NEAR ? a.inter_hard : a.inter_soft, inter);
}

// work items per group: max(1, ceil(list length / lch))
__global__ void __launch_bounds__(256) k_pair_plan(const int64_t *__restrict__ ngroups,
                                                   const uint64_t *__restrict__ off, int near, int lch,
                                                   uint32_t *__restrict__ wcount, const Status *st)
{
    if (st->code) return;
    const int64_t ng = *ngroups;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t L = near ? (off[2 * ng + g + 1] - off[2 * ng + g])
                                : (off[g + 1] - off[g]) + (off[ng + g + 1] - off[ng + g]);
        wcount[g] = (uint32_t)max((uint64_t)1, (L + lch - 1) / (uint64_t)lch);
    }
}

__global__ void __launch_bounds__(256) k_pair_map(const int64_t *__restrict__ ngroups, uint32_t *__restrict__ wstart,
                                                  const uint64_t *__restrict__ total, uint32_t *__restrict__ wmap,
                                                  const Status *st)
{
    if (st->code) return;
    const int64_t ng = *ngroups;
    const uint32_t T = (uint32_t)*total;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s0 = wstart[g];
        const uint32_t s1 = (g + 1 < ng) ? wstart[g + 1] : T;
        for (uint32_t w = s0; w < s1; ++w) wmap[w] = (uint32_t)g;
        if (g == ng - 1) wstart[ng] = T;
    }
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
    a.wstart = nullptr;
    a.wmap = nullptr;
    a.nwork = nullptr;
    a.lch = 0;
    a.want_soft = a.want_hard = 0;
}

template <int KS, bool NEAR, bool SOFT, bool HARD>
void go_f32(hybrid_ctx *c, const PairArgs &a)
{
    k_pair_f32<KS, NEAR, SOFT, HARD><<<c->nsm * 16, PAIR_THREADS, 0, c->st>>>(a);
}

// Sinks per lane KS = ceil(n_crit / threads_per_group), from 1 to 4; the
// default is 4 for the far kernel (one shared-memory read feeds 4
// interactions) and 2 for the near kernel (it also keeps hi/lo offsets per sink).
template <bool NEAR, bool SOFT, bool HARD>
void go_ks(hybrid_ctx *c, const PairArgs &a)
{
    int ks;
    if (c->p.threads_per_group > 0) ks = (c->p.n_crit + c->p.threads_per_group - 1) / c->p.threads_per_group;
    else ks = NEAR ? (c->p.n_crit > 64 ? 4 : 2) : 4;
    ks = ks <= 1 ? 1 : (ks <= 2 ? 2 : 4);
    if (ks == 1) go_f32<1, NEAR, SOFT, HARD>(c, a);
    else if (ks == 2) go_f32<2, NEAR, SOFT, HARD>(c, a);
    else go_f32<4, NEAR, SOFT, HARD>(c, a);
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
        const int lch = near ? LCH_NEAR : LCH_FAR;
        uint32_t *wstart = (uint32_t *)c->wstart.p;
        uint64_t *d_total = (uint64_t *)c->counter.p + 8;
        const int gridg = (int)std::max<int64_t>(1, std::min<int64_t>((c->capGroups + 255) / 256, c->nsm * 8));
        k_pair_plan<<<gridg, 256, 0, c->st>>>(a.ngroups, a.off, near ? 1 : 0, lch, wstart, st);
        scan_u32(c, wstart, 0, a.ngroups, c->capGroups, d_total);
        k_pair_map<<<gridg, 256, 0, c->st>>>(a.ngroups, wstart, d_total, (uint32_t *)c->wmap.p, st);
        a.wstart = wstart;
        a.wmap = (const uint32_t *)c->wmap.p;
        a.nwork = d_total;
        a.lch = lch;
        if (!near)
            for (int d = 0; d < 3; ++d) cudaMemsetAsync(c->acc_s[d].p, 0, (size_t)c->N * sizeof(float), c->st);
        if (near && a.want_hard)
            for (int d = 0; d < 3; ++d) cudaMemsetAsync(c->acc_h[d].p, 0, (size_t)c->N * sizeof(float), c->st);
        if (!near) go_ks<false, true, false>(c, a);
        else if (a.want_soft && a.want_hard) go_ks<true, true, true>(c, a);
        else if (a.want_soft) go_ks<true, true, false>(c, a);
        else go_ks<true, false, true>(c, a);
        c->launches += 3;
    }
    prof_end(c, kind, e0);
}

}  // namespace

void launch_pair_far(hybrid_ctx *c) { launch_pairs(c, false, 1); }
void launch_pair_near(hybrid_ctx *c, int mode) { launch_pairs(c, true, mode); }

}  // namespace hy
