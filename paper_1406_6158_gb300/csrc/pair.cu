// pair.cu -- soft and hard pair kernels (Eq. 2 split by Eq. 7-10).
//
// One warp takes one sink group at a time (dynamic queue) and sums over the
// group's interaction list. Sources are staged, 64 at a time, into the warp's
// own shared-memory tile as float4 {x, y, z, m} relative to the group centre
// (FP32 form), so every source is rebased once per group and then reused by
// every sink of the group from shared memory.
//
// Lane layout: a group of n sinks uses lpc = ceil(n / KS) lanes per copy, each
// lane holding KS sinks in registers; copies = 32 / lpc copies of the group
// split the sources between them (source j goes to copy j mod copies) and are
// added up at the end, so small groups still keep most lanes busy.
//
// FP32 form: positions relative to the group centre from the hi/lo split
// (x = hi + lo), so the subtraction of two nearby coordinates loses nothing;
// rsqrtf on the CUDA cores (the pair sum is not a dense contraction).
// FP64 form: plain FP64 differences and 1/sqrt.
#include "hy_internal.cuh"

namespace hy {

namespace {

constexpr int PAIR_THREADS = 128;
constexpr int PAIR_WARPS = PAIR_THREADS / 32;
constexpr int TILE = 64;

struct PairArgs {
    const int64_t *ngroups;
    const uint32_t *gfirst, *gcount, *gsys;
    const GroupF *gF;
    const SysParams *sp;
    const uint64_t *off;    // [3 * ng + 1] list offsets (cells, particles, hard particles)
    const uint32_t *list;
    const float4 *phi, *plo, *nA, *nB;
    const double4_32a *pd, *nD;
    void *ax, *ay, *az;
    unsigned long long *counter;
    unsigned long long *inter;
    const Status *st;
};

// ---- FP32 bodies ----------------------------------------------------------
// far cell: F only (K = 0 is guaranteed by the walk's cutoff test)
__device__ __forceinline__ void body_cell(const float4 q, float sx, float sy, float sz, float eps2, float &ax,
                                          float &ay, float &az)
{
    const float dx = q.x - sx, dy = q.y - sy, dz = q.z - sz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float ri = rsqrtf(r2);
    const float mr = q.w * ri;
    const float f = mr * (ri * ri);
    ax = fmaf(dx, f, ax);
    ay = fmaf(dy, f, ay);
    az = fmaf(dz, f, az);
}

// DLL kernel, Eq. (10), from r^2: Y = clamp((R2 - r)/(R2 - R1), 0, 1),
// K = Y^6 (10 + Y^2 (-15 + 6 Y^2)); exact 1 at Y = 1 and 0 at Y = 0.
__device__ __forceinline__ float dll_K(float r2u, float R2, float invdR)
{
    const float r = sqrtf(r2u);
    const float Y = __saturatef((R2 - r) * invdR);
    const float Y2 = Y * Y;
    return (Y2 * Y2 * Y2) * fmaf(Y2, fmaf(6.0f, Y2, -15.0f), 10.0f);
}

// particle in the soft list: F * (1 - K)
__device__ __forceinline__ void body_soft_part(const float4 q, float sx, float sy, float sz, float eps2, float R2,
                                               float R2sq, float invdR, float &ax, float &ay, float &az)
{
    const float dx = q.x - sx, dy = q.y - sy, dz = q.z - sz;
    const float r2u = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float r2 = r2u + eps2;
    const float ri = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    float w = 1.0f;
    if (r2u < R2sq) w = 1.0f - dll_K(r2u, R2, invdR);
    const float f = q.w * w * ri * (ri * ri);
    ax = fmaf(dx, f, ax);
    ay = fmaf(dy, f, ay);
    az = fmaf(dz, f, az);
}

// particle in the hard list: F * K, zero beyond R2. Near R2, K ~ 10 Y^6
// magnifies any error of R2 - r, so for pairs inside R2 the kernel rebuilds
// D = R2^2 - r^2 in double-float arithmetic from the grid-aligned hi parts
// (whose differences are exact) and the lo parts, and takes
// Y = D / ((R2 + r)(R2 - R1)).
struct HardC {
    float eps2, R2, R2sq, R2sqlo, invdR;
};

__device__ __forceinline__ void body_hard(const float4 t, const float4 th, const float4 tl, float sx, float sy,
                                          float sz, float shx, float shy, float shz, float slx, float sly, float slz,
                                          const HardC &H, float &ax, float &ay, float &az)
{
    const float dx = t.x - sx, dy = t.y - sy, dz = t.z - sz;
    const float r2u = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2u < H.R2sq) {
        const float hx = __fsub_rn(th.x, shx), hy = __fsub_rn(th.y, shy), hz = __fsub_rn(th.z, shz);
        const float lx = __fsub_rn(tl.x, slx), ly = __fsub_rn(tl.y, sly), lz = __fsub_rn(tl.z, slz);
        const float px = __fmul_rn(hx, hx), py = __fmul_rn(hy, hy), pz = __fmul_rn(hz, hz);
        const float ex = __fmaf_rn(hx, hx, -px), ey = __fmaf_rn(hy, hy, -py), ez = __fmaf_rn(hz, hz, -pz);
        // R2^2 - px - py - pz with the rounding errors kept (|R2^2| >= px, d1 >= py, d2 >= pz inside R2)
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
        const float K = (Y2 * Y2 * Y2) * fmaf(Y2, fmaf(6.0f, Y2, -15.0f), 10.0f);
        const float r2 = r2u + H.eps2;
        const float ri = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
        const float f = t.w * K * ri * (ri * ri);
        ax = fmaf(dx, f, ax);
        ay = fmaf(dy, f, ay);
        az = fmaf(dz, f, az);
    }
}

// ---- FP64 bodies ----------------------------------------------------------
__device__ __forceinline__ double dll_K64(double r, double R1, double R2)
{
    double Y = (R2 - r) / (R2 - R1);
    if (Y >= 1.0) return 1.0;
    if (Y <= 0.0) return 0.0;
    const double Y2 = Y * Y;
    return (Y2 * Y2 * Y2) * (10.0 + Y2 * (-15.0 + 6.0 * Y2));
}

// kind 0: far cell (w = 1), 1: soft particle (w = 1 - K), 2: hard (w = K)
template <int KIND>
__device__ __forceinline__ void body64(const double4_32a q, double sx, double sy, double sz, const SysParams &P,
                                       double &ax, double &ay, double &az)
{
    const double dx = q.x - sx, dy = q.y - sy, dz = q.z - sz;
    const double r2u = dx * dx + dy * dy + dz * dz;
    if (KIND == 2 && !(r2u < P.R2sq)) return;
    const double r2 = r2u + P.eps2;
    const double ri = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
    double w = 1.0;
    if (KIND == 1 && r2u < P.R2sq) w = 1.0 - dll_K64(sqrt(r2u), P.R1, P.R2);
    if (KIND == 2) w = dll_K64(sqrt(r2u), P.R1, P.R2);
    const double f = q.w * w * ri * ri * ri;
    ax += f * dx;
    ay += f * dy;
    az += f * dz;
}

__device__ __forceinline__ int64_t next_group(unsigned long long *counter, int lane)
{
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(counter, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, g, 0);
}

// ---------------------------------------------------------------------------
// FP32 kernel. SOFT: cells then particles with (1-K); else hard list with K.
// Coordinates are taken relative to the group's reference point c = the hi
// part of its first sink (on the hi grid, so hi - c is exact).
// ---------------------------------------------------------------------------
template <int KS, bool SOFT>
__global__ void __launch_bounds__(PAIR_THREADS) k_pair_f32(PairArgs a)
{
    constexpr int HT = SOFT ? 1 : TILE;
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
    unsigned long long inter = 0;
    for (;;) {
        const int64_t g = next_group(a.counter, lane);
        if (g >= ng) break;
        const uint32_t first = a.gfirst[g];
        const int n = (int)a.gcount[g];
        const SysParams &P = a.sp[a.gsys[g]];
        const float eps2 = P.eps2f, R2 = P.R2f, R2sq = P.R2sqf, invdR = P.invdRf;
        HardC H;
        H.eps2 = eps2;
        H.R2 = R2;
        H.R2sq = R2sq;
        H.R2sqlo = P.R2sqlo;
        H.invdR = invdR;
        const float4 cref = a.phi[first];
        const float crx = cref.x, cry = cref.y, crz = cref.z;
        uint64_t c0, c1, p0, p1;
        if (SOFT) {
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
        const int lpc = n <= 32 * KS ? (n + KS - 1) / KS : 32;
        const int copies = 32 / lpc;
        const int copy = lane / lpc, slot = lane - copy * lpc;
        const bool active = copy < copies;
        const int per_round = lpc * KS;
        for (int r0 = 0; r0 < n; r0 += per_round) {
            float sx[KS], sy[KS], sz[KS], ax[KS], ay[KS], az[KS];
            float shx[KS], shy[KS], shz[KS], slx[KS], sly[KS], slz[KS];
#pragma unroll
            for (int k = 0; k < KS; ++k) {
                int si = r0 + k * lpc + slot;
                si = si < n ? si : n - 1;
                const float4 h = a.phi[first + si], l = a.plo[first + si];
                shx[k] = h.x - crx;
                shy[k] = h.y - cry;
                shz[k] = h.z - crz;
                slx[k] = l.x;
                sly[k] = l.y;
                slz[k] = l.z;
                sx[k] = shx[k] + l.x;
                sy[k] = shy[k] + l.y;
                sz[k] = shz[k] + l.z;
                ax[k] = ay[k] = az[k] = 0.0f;
            }
            if (SOFT) {
                for (uint64_t t0 = c0; t0 < c1; t0 += TILE) {
                    const int nt = (int)min((uint64_t)TILE, c1 - t0);
                    for (int e = lane; e < nt; e += 32) {
                        const uint32_t cc = a.list[t0 + e];
                        const float4 A = a.nA[cc], B = a.nB[cc];
                        tile[e] = make_float4((A.x - crx) + B.x, (A.y - cry) + B.y, (A.z - crz) + B.z, A.w);
                    }
                    __syncwarp();
                    if (active) {
                        for (int j = copy; j < nt; j += copies) {
                            const float4 q = tile[j];
#pragma unroll
                            for (int k = 0; k < KS; ++k) body_cell(q, sx[k], sy[k], sz[k], eps2, ax[k], ay[k], az[k]);
                        }
                    }
                    __syncwarp();
                }
            }
            for (uint64_t t0 = p0; t0 < p1; t0 += TILE) {
                const int nt = (int)min((uint64_t)TILE, p1 - t0);
                for (int e = lane; e < nt; e += 32) {
                    const uint32_t j = a.list[t0 + e];
                    const float4 h = a.phi[j], l = a.plo[j];
                    const float hx = h.x - crx, hy = h.y - cry, hz = h.z - crz;
                    tile[e] = make_float4(hx + l.x, hy + l.y, hz + l.z, h.w);
                    if (!SOFT) {
                        tile_h[e] = make_float4(hx, hy, hz, 0.0f);
                        tile_l[e] = l;
                    }
                }
                __syncwarp();
                if (active) {
                    for (int j = copy; j < nt; j += copies) {
                        const float4 q = tile[j];
                        if (SOFT) {
#pragma unroll
                            for (int k = 0; k < KS; ++k)
                                body_soft_part(q, sx[k], sy[k], sz[k], eps2, R2, R2sq, invdR, ax[k], ay[k], az[k]);
                        } else {
                            const float4 qh = tile_h[j], ql = tile_l[j];
#pragma unroll
                            for (int k = 0; k < KS; ++k)
                                body_hard(q, qh, ql, sx[k], sy[k], sz[k], shx[k], shy[k], shz[k], slx[k], sly[k],
                                          slz[k], H, ax[k], ay[k], az[k]);
                        }
                    }
                }
                __syncwarp();
            }
            // add the copies into copy 0, in copy order
            for (int cc = 1; cc < copies; ++cc) {
                const int src = (copy == 0) ? lane + cc * lpc : lane;
#pragma unroll
                for (int k = 0; k < KS; ++k) {
                    const float vx = __shfl_sync(0xffffffffu, ax[k], src);
                    const float vy = __shfl_sync(0xffffffffu, ay[k], src);
                    const float vz = __shfl_sync(0xffffffffu, az[k], src);
                    if (copy == 0) {
                        ax[k] += vx;
                        ay[k] += vy;
                        az[k] += vz;
                    }
                }
            }
            if (copy == 0) {
                const float Gf = P.Gf;
#pragma unroll
                for (int k = 0; k < KS; ++k) {
                    const int si = r0 + k * lpc + slot;
                    if (si < n) {
                        const uint32_t i = first + si;
                        ((float *)a.ax)[i] = Gf * ax[k];
                        ((float *)a.ay)[i] = Gf * ay[k];
                        ((float *)a.az)[i] = Gf * az[k];
                    }
                }
            }
        }
    }
    if (lane == 0) atomicAdd(a.inter, inter);
}

// ---------------------------------------------------------------------------
// FP64 kernel: one lane per sink (rounds of 32 sinks), sources staged as
// double4_32a in shared memory.
// ---------------------------------------------------------------------------
template <bool SOFT>
__global__ void __launch_bounds__(PAIR_THREADS) k_pair_f64(PairArgs a)
{
    __shared__ double4_32a tiles[PAIR_WARPS][TILE];
    if (a.st->code) return;
    const int lane = threadIdx.x & 31;
    double4_32a *tile = tiles[threadIdx.x >> 5];
    const int64_t ng = *a.ngroups;
    unsigned long long inter = 0;
    for (;;) {
        const int64_t g = next_group(a.counter, lane);
        if (g >= ng) break;
        const uint32_t first = a.gfirst[g];
        const int n = (int)a.gcount[g];
        const SysParams P = a.sp[a.gsys[g]];
        uint64_t c0, c1, p0, p1;
        if (SOFT) {
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
            double ax = 0.0, ay = 0.0, az = 0.0;
            if (SOFT) {
                for (uint64_t t0 = c0; t0 < c1; t0 += TILE) {
                    const int nt = (int)min((uint64_t)TILE, c1 - t0);
                    for (int e = lane; e < nt; e += 32) tile[e] = a.nD[a.list[t0 + e]];
                    __syncwarp();
                    for (int j = 0; j < nt; ++j) body64<0>(tile[j], s.x, s.y, s.z, P, ax, ay, az);
                    __syncwarp();
                }
            }
            for (uint64_t t0 = p0; t0 < p1; t0 += TILE) {
                const int nt = (int)min((uint64_t)TILE, p1 - t0);
                for (int e = lane; e < nt; e += 32) tile[e] = a.pd[a.list[t0 + e]];
                __syncwarp();
                for (int j = 0; j < nt; ++j) {
                    if (SOFT) body64<1>(tile[j], s.x, s.y, s.z, P, ax, ay, az);
                    else body64<2>(tile[j], s.x, s.y, s.z, P, ax, ay, az);
                }
                __syncwarp();
            }
            if (si < n) {
                const uint32_t i = first + si;
                ((double *)a.ax)[i] = P.G * ax;
                ((double *)a.ay)[i] = P.G * ay;
                ((double *)a.az)[i] = P.G * az;
            }
        }
    }
    if (lane == 0) atomicAdd(a.inter, inter);
}

void fill_args(hybrid_ctx *c, PairArgs &a, bool soft)
{
    a.ngroups = (const int64_t *)c->ngroups_dev.p;
    a.gfirst = (const uint32_t *)c->gfirst.p;
    a.gcount = (const uint32_t *)c->gcount.p;
    a.gsys = (const uint32_t *)c->gsys.p;
    a.gF = (const GroupF *)c->gF.p;
    a.sp = (const SysParams *)c->sp_dev.p;
    a.off = (const uint64_t *)c->lcnt.p;
    a.list = (const uint32_t *)c->list.p;
    a.phi = (const float4 *)c->phi.p;
    a.plo = (const float4 *)c->plo.p;
    a.nA = (const float4 *)c->nA.p;
    a.nB = (const float4 *)c->nB.p;
    a.pd = (const double4_32a *)c->pd.p;
    a.nD = (const double4_32a *)c->nD.p;
    hy::Buf *acc = soft ? c->acc_s : c->acc_h;
    a.ax = acc[0].p;
    a.ay = acc[1].p;
    a.az = acc[2].p;
    unsigned long long *ctr = (unsigned long long *)c->counter.p;
    a.counter = ctr + (soft ? 2 : 3);
    a.inter = ctr + (soft ? 6 : 7);
    a.st = status_dev(c);
}

template <bool SOFT>
void launch_pair(hybrid_ctx *c)
{
    PairArgs a;
    fill_args(c, a, SOFT);
    unsigned long long *ctr = (unsigned long long *)c->counter.p;
    cudaMemsetAsync(ctr + (SOFT ? 2 : 3), 0, sizeof(unsigned long long), c->st);
    cudaMemsetAsync(ctr + (SOFT ? 6 : 7), 0, sizeof(unsigned long long), c->st);
    const int grid = c->nsm * 12;
    cudaEvent_t e0 = nullptr;
    prof_begin(c, SOFT ? PROF_SOFT : PROF_HARD, &e0);
    if (c->p.precision == 0) {
        k_pair_f64<SOFT><<<grid, PAIR_THREADS, 0, c->st>>>(a);
    } else {
        const int ks = c->p.n_crit <= 32 ? 1 : (c->p.n_crit <= 64 ? 2 : 4);
        if (ks == 1) k_pair_f32<1, SOFT><<<grid, PAIR_THREADS, 0, c->st>>>(a);
        else if (ks == 2) k_pair_f32<2, SOFT><<<grid, PAIR_THREADS, 0, c->st>>>(a);
        else k_pair_f32<4, SOFT><<<grid, PAIR_THREADS, 0, c->st>>>(a);
    }
    prof_end(c, SOFT ? PROF_SOFT : PROF_HARD, e0);
    c->launches++;
}

}  // namespace

void launch_pair_soft(hybrid_ctx *c) { launch_pair<true>(c); }
void launch_pair_hard(hybrid_ctx *c) { launch_pair<false>(c); }

}  // namespace hy
