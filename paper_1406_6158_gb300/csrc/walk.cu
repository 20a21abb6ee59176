// walk.cu -- grouped tree walk that emits interaction lists (Sec. II-B
// traversal rule; Eq. 11 with the box of a sink group in place of the n_vec
// sinks; Eq. 15 for the hard neighbours and for the cutoff test).
//
// One warp walks one group at a time, starting at its system's root. Each
// iteration pops up to 32 pending cells (one per lane) from a per-warp stack,
// tests them, and with warp ballots/scans appends:
//   cells           taken whole: r >= r_b and r >= R2 + b_max (K = 0 for
//                   every pair, weight 1),
//   far particles   members of leaves the soft walk opens with
//                   r >= R2 + b_max (K = 0 for every pair, weight 1),
//   near particles  members of leaves with r < R2 + b_max, reached by the
//                   soft or the hard walk: the only pairs where K can be
//                   non-zero (soft weight 1 - K, hard weight K),
// and pushes the children of opened cells. r is the distance from the cell's
// centre of mass to the group box.
//
// FP32 form (one pass): each warp writes the three kinds of entries into
// regions of the list buffer it claims with an atomic add (at least
// WALK_REGION entries per kind at a time), so a group's entries of one kind
// are contiguous until a region runs out; every contiguous run becomes pair
// work items of at most item_len entries, appended to the far (cells, far
// particles) or near item array, which the pair kernels consume directly.
// FP64 form (two passes): the count pass sizes every list, a scan turns
// counts into offsets, and the fill pass writes them (one list per group and
// kind, for the deterministic FP64 pair kernel).
#include "hy_internal.cuh"

namespace hy {

namespace {

constexpr int WALK_THREADS = 128;

struct WalkArgs {
    const int64_t *ngroups;
    const uint32_t *gnode, *gsys;
    const GroupF *gF;
    const double *glo, *ghi;
    const uint32_t *sysroot;
    const SysParams *sp;
    const uint4 *topo;
    const float4 *nA, *nB;
    const float2 *crit;
    const double4_32a *nD;
    const double *rb, *hr;
    uint64_t *cnt;          // count pass: counts; fill pass: offsets ([3][ng] + total)
    int64_t *d_n3;
    const uint64_t *list_total;
    uint32_t *list;
    int64_t cap_list;
    uint32_t *stack;
    int64_t cap_stack;
    unsigned long long *counter;
    int mode;
    Status *st;
    int where;
    // one-pass form
    const uint32_t *gfirst, *gcount;
    unsigned long long *list_cursor;     // next free list entry
    unsigned long long *item_count;      // [0] far items, [1] near items
    WorkItem *items_far, *items_near;
    int64_t cap_items;
    int lch_far, lch_near;               // base lengths of far and near work items
};

constexpr uint32_t WALK_REGION = 2048;
constexpr int WALK_SSTK = 1024;   // entries of a warp's stack kept in shared memory (one walk iteration pushes <= 256)

__device__ __forceinline__ void fail(Status *st, int code, int where)
{
    // the first failure wins and keeps its op index: later kernels of the same sequence may fail too (a build
    // after an unsorted one), and the sequence resumes at the first
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t &total)
{
    const int lane = threadIdx.x & 31;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

// distance from p to the box [lo, hi], per axis max(lo - p, 0, p - hi)
__device__ __forceinline__ double dist_box_f64(double p0, double p1, double p2, const double *lo, const double *hi)
{
    const double p[3] = {p0, p1, p2};
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        const double a = lo[d] - p[d];
        const double b = p[d] - hi[d];
        if (a > g) g = a;
        if (b > g) g = b;
        s += g * g;
    }
    return sqrt(s);
}

template <bool F64, bool FILL>
__global__ void __launch_bounds__(WALK_THREADS) k_walk(WalkArgs a)
{
    Status *st = a.st;
    if (st->code) return;
    const int lane = threadIdx.x & 31;
    const unsigned ltmask = (1u << lane) - 1u;
    const int64_t ng = *a.ngroups;
    if (!FILL && blockIdx.x == 0 && threadIdx.x == 0) *a.d_n3 = 3 * ng;
    if (FILL) {
        const uint64_t total = *a.list_total;
        if ((int64_t)total > a.cap_list) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                fail(st, HYBRID_ECAPACITY, a.where);
                st->need[1] = (int64_t)total;
            }
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[3 * ng] = total;
    }
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t *stk = a.stack + gw * a.cap_stack;
    const bool want_soft = a.mode & 1, want_hard = (a.mode >> 1) & 1;

    for (;;) {
        unsigned long long gg = 0;
        if (lane == 0) gg = atomicAdd(a.counter, 1ull);
        const int64_t g = (int64_t)__shfl_sync(0xffffffffu, gg, 0);
        if (g >= ng) break;
        const uint32_t s = a.gsys[g];
        const bool has_hard = a.sp[s].has_hard != 0;
        const bool wh0 = want_hard && has_hard;
        float cx = 0, cy = 0, cz = 0, lx = 0, ly = 0, lz = 0, hx = 0, hy = 0, hz = 0;
        double blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
        if (F64) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                blo[d] = a.glo[3 * g + d];
                bhi[d] = a.ghi[3 * g + d];
            }
        } else {
            const GroupF G = a.gF[g];
            cx = G.c_hi.x;
            cy = G.c_hi.y;
            cz = G.c_hi.z;
            hx = G.c_hi.w;
            lx = G.c_lo.x;
            ly = G.c_lo.y;
            lz = G.c_lo.z;
            hy = G.c_lo.w;
            hz = G.hz_root.x;
        }
        uint64_t nc = 0, np = 0, nh = 0, oc = 0, op = 0, oh = 0;
        if (FILL) {
            oc = a.cnt[g];
            op = a.cnt[ng + g];
            oh = a.cnt[2 * ng + g];
        }
        int64_t sp = 0;
        if (want_soft || wh0) {
            if (lane == 0) stk[0] = a.sysroot[s] | ((uint32_t)want_soft << 30) | ((uint32_t)wh0 << 31);
            sp = 1;
        }
        __syncwarp();
        bool overflow = false;
        while (sp > 0) {
            const int take = (int)(sp < 32 ? sp : 32);
            uint32_t e = 0;
            if (lane < take) e = stk[sp - take + lane];
            sp -= take;
            __syncwarp();
            const bool valid = lane < take;
            const uint32_t c = e & 0x3fffffffu;
            const bool ws = (e >> 30) & 1u, wh = (e >> 31) & 1u;
            bool accept = false, near = false;
            uint4 T = make_uint4(NONE, 0, 0, 0);
            if (valid) {
                T = a.topo[c];
                if (F64) {
                    const double4_32a D = a.nD[c];
                    const double d = dist_box_f64(D.x, D.y, D.z, blo, bhi);
                    const double hr = a.hr[c];
                    accept = (d >= a.rb[c]) && (d >= hr);
                    near = has_hard && (d < hr);
                } else {
                    const float4 A = a.nA[c], B = a.nB[c];
                    const float2 cr = a.crit[c];
                    const float rx = fmaxf(fabsf((A.x - cx) + (B.x - lx)) - hx, 0.0f);
                    const float ry = fmaxf(fabsf((A.y - cy) + (B.y - ly)) - hy, 0.0f);
                    const float rz = fmaxf(fabsf((A.z - cz) + (B.z - lz)) - hz, 0.0f);
                    const float d2 = rx * rx + ry * ry + rz * rz;
                    accept = d2 >= cr.x;
                    near = has_hard && (d2 < cr.y);
                }
            }
            const bool leaf = (T.y == 0);
            const bool open_s = ws && !accept;             // the soft walk goes on below c
            const bool open_h = wh && near;                // the hard walk goes on below c
            const bool take_cell = valid && ws && accept;
            const bool soft_leaf = valid && leaf && open_s && !near;        // far particles
            const bool hard_leaf = valid && leaf && (open_s || open_h) && near;   // near particles
            const bool open = valid && !leaf && (open_s || open_h);
            // taken cells
            const unsigned bm = __ballot_sync(0xffffffffu, take_cell);
            if (FILL && take_cell) a.list[oc + nc + __popc(bm & ltmask)] = c;
            nc += (uint64_t)__popc(bm);
            // soft particles
            {
                uint32_t tot;
                const uint32_t k = soft_leaf ? T.w : 0u;
                const uint32_t ex = warp_excl_scan(k, tot);
                if (FILL && soft_leaf) {
                    uint32_t *dst = a.list + op + np + ex;
                    for (uint32_t j = 0; j < k; ++j) dst[j] = T.z + j;
                }
                np += tot;
            }
            // hard particles
            {
                uint32_t tot;
                const uint32_t k = hard_leaf ? T.w : 0u;
                const uint32_t ex = warp_excl_scan(k, tot);
                if (FILL && hard_leaf) {
                    uint32_t *dst = a.list + oh + nh + ex;
                    for (uint32_t j = 0; j < k; ++j) dst[j] = T.z + j;
                }
                nh += tot;
            }
            // children of opened cells
            {
                uint32_t tot;
                const uint32_t k = open ? T.y : 0u;
                const uint32_t ex = warp_excl_scan(k, tot);
                if (sp + (int64_t)tot > a.cap_stack) {
                    overflow = true;
                    break;
                }
                if (open) {
                    const uint32_t fl = ((uint32_t)open_s << 30) | ((uint32_t)open_h << 31);
                    for (uint32_t j = 0; j < k; ++j) stk[sp + ex + j] = (T.x + j) | fl;
                }
                sp += tot;
            }
            __syncwarp();
        }
        if (overflow) {
            if (lane == 0) {
                fail(st, HYBRID_ECAPACITY, a.where);
                st->need[2] = 2 * a.cap_stack;
            }
            break;
        }
        if (!FILL && lane == 0) {
            a.cnt[g] = nc;
            a.cnt[ng + g] = np;
            a.cnt[2 * ng + g] = nh;
        }
    }
}

// Work items of one contiguous run [start, start + len) of a group's entries
// of kind t (0 cells, 1 far particles, 2 near particles); all lanes call it.
__device__ __forceinline__ bool emit_items(const WalkArgs &a, int t, uint64_t start, uint64_t len, uint32_t first,
                                           uint32_t n, uint32_t sys, bool multi, int lane)
{
    const int cls = t == 2 ? 1 : 0;
    const uint64_t per = item_len(n, t == 2 ? a.lch_near : a.lch_far);
    const uint64_t m = (len + per - 1) / per;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.item_count + cls, (unsigned long long)m);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)(base + m) > a.cap_items) return false;
    WorkItem *dst = (cls ? a.items_near : a.items_far) + base;
    for (uint64_t j = lane; j < m; j += 32) {
        WorkItem d;
        d.cbase = t == 0 ? start : 0;
        d.pbase = t == 0 ? 0 : start;
        d.Lc = t == 0 ? (uint32_t)len : 0u;
        d.e0 = (uint32_t)(j * per);
        d.e1 = (uint32_t)min(len, (j + 1) * per);
        d.first = first;
        d.n = n | (multi ? ITEM_MULTI : 0u);
        d.sys = sys;
        dst[j] = d;
    }
    return true;
}

// FP32 form of the walk in one pass (see the top of the file). The warp's
// region and open-run state of kind t (0 cells, 1 far, 2 near particles)
// lives on lane t and is broadcast when needed.
// MINB blocks per SM: 6 (80 registers) for batches of at most 2^20 particles, whose groups are fewer than the
// resident warps; 8 (64 registers, a few spilled) above, where more warps hide more of the node loads.
template <int MINB>
__global__ void __launch_bounds__(WALK_THREADS, MINB) k_walk1(WalkArgs a)
{
    Status *st = a.st;
    if (st->code) return;
    const int lane = threadIdx.x & 31;
    const int64_t ng = *a.ngroups;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t *stk = a.stack + gw * a.cap_stack;   // overflow part of the stack (older entries)
    __shared__ uint32_t sstk_all[WALK_THREADS / 32][WALK_SSTK];
    uint32_t *sstk = sstk_all[threadIdx.x >> 5];    // top part of the stack
    const bool want_soft = a.mode & 1, want_hard = (a.mode >> 1) & 1;
    uint64_t my_cur = 0, my_end = 0, my_start = 0, my_len = 0;   // kind = lane (lanes 0..2)
    bool fail_list = false, fail_items = false, overflow = false;

    for (;;) {
        unsigned long long gg = 0;
        if (lane == 0) gg = atomicAdd(a.counter, 1ull);
        const int64_t g = (int64_t)__shfl_sync(0xffffffffu, gg, 0);
        if (g >= ng) break;
        const uint32_t s = a.gsys[g];
        const bool has_hard = a.sp[s].has_hard != 0;
        const bool wh0 = want_hard && has_hard;
        const uint32_t gfirst = a.gfirst[g], gn = a.gcount[g];
        const GroupF G = a.gF[g];
        const float cx = G.c_hi.x, cy = G.c_hi.y, cz = G.c_hi.z, hx = G.c_hi.w;
        const float lx = G.c_lo.x, ly = G.c_lo.y, lz = G.c_lo.z, hy = G.c_lo.w, hz = G.hz_root.x;
        my_start = my_cur;
        my_len = 0;
        uint32_t early_far = 0, early_near = 0;   // items already emitted for this group
        int sp = 0;        // entries in the shared-memory part
        int64_t gp = 0;    // entries in the global part
        if (want_soft || wh0) {
            if (lane == 0) sstk[0] = a.sysroot[s] | ((uint32_t)want_soft << 30) | ((uint32_t)wh0 << 31);
            sp = 1;
        }
        __syncwarp();
        // position for tot more entries of kind t, or ~0 on failure; closes the open run and claims a
        // new region when the current one is too small
        auto reserve = [&](int t, uint64_t tot) -> uint64_t {
            const uint64_t cur = __shfl_sync(0xffffffffu, my_cur, t), end = __shfl_sync(0xffffffffu, my_end, t);
            if (cur + tot <= end) return cur;
            const uint64_t len = __shfl_sync(0xffffffffu, my_len, t), st0 = __shfl_sync(0xffffffffu, my_start, t);
            if (len > 0) {
                if (!emit_items(a, t, st0, len, gfirst, gn, s, true, lane)) {
                    fail_items = true;
                    return ~0ull;
                }
                const uint64_t per = item_len(gn, t == 2 ? a.lch_near : a.lch_far);
                (t == 2 ? early_near : early_far) += (uint32_t)((len + per - 1) / per);
            }
            const uint64_t size = tot > WALK_REGION ? tot : WALK_REGION;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.list_cursor, (unsigned long long)size);
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((int64_t)(base + size) > a.cap_list) {
                fail_list = true;
                return ~0ull;
            }
            if (lane == t) {
                my_cur = base;
                my_end = base + size;
                my_start = base;
                my_len = 0;
            }
            return base;
        };
        while (sp > 0 || gp > 0) {
            if (sp == 0) {   // refill the shared part from the top of the global part
                const int m = (int)(gp < WALK_SSTK / 2 ? gp : WALK_SSTK / 2);
                for (int j = lane; j < m; j += 32) sstk[j] = stk[gp - m + j];
                gp -= m;
                sp = m;
                __syncwarp();
            }
            const int take = sp < 32 ? sp : 32;
            uint32_t e = 0;
            if (lane < take) e = sstk[sp - take + lane];
            sp -= take;
            __syncwarp();
            const bool valid = lane < take;
            const uint32_t c = e & 0x3fffffffu;
            const bool ws = (e >> 30) & 1u, wh = (e >> 31) & 1u;
            bool accept = false, near = false;
            uint4 T = make_uint4(NONE, 0, 0, 0);
            if (valid) {
                T = a.topo[c];
                const float4 A = a.nA[c], B = a.nB[c];
                const float2 cr = a.crit[c];
                const float rx = fmaxf(fabsf((A.x - cx) + (B.x - lx)) - hx, 0.0f);
                const float ry = fmaxf(fabsf((A.y - cy) + (B.y - ly)) - hy, 0.0f);
                const float rz = fmaxf(fabsf((A.z - cz) + (B.z - lz)) - hz, 0.0f);
                const float d2 = rx * rx + ry * ry + rz * rz;
                accept = d2 >= cr.x;
                near = has_hard && (d2 < cr.y);
            }
            const bool leaf = (T.y == 0);
            const bool open_s = ws && !accept;
            const bool open_h = wh && near;
            const bool take_cell = valid && ws && accept;
            const bool soft_leaf = valid && leaf && open_s && !near;
            const bool hard_leaf = valid && leaf && (open_s || open_h) && near;
            const bool open = valid && !leaf && (open_s || open_h);
            // per-lane counts of far particles, near particles and children, packed 10 bits each when every
            // count is below 32 (one scan instead of three); cells take one ballot
            const uint32_t kf = soft_leaf ? T.w : 0u, kn = hard_leaf ? T.w : 0u, kc = open ? T.y : 0u;
            const bool small = __all_sync(0xffffffffu, kf < 32u && kn < 32u);
            uint32_t exf, exn, exc, totf, totn, totc;
            if (small) {
                uint32_t tp;
                const uint32_t ep = warp_excl_scan(kf | (kn << 10) | (kc << 20), tp);
                exf = ep & 1023u;
                exn = (ep >> 10) & 1023u;
                exc = ep >> 20;
                totf = tp & 1023u;
                totn = (tp >> 10) & 1023u;
                totc = tp >> 20;
            } else {
                exf = warp_excl_scan(kf, totf);
                exn = warp_excl_scan(kn, totn);
                exc = warp_excl_scan(kc, totc);
            }
            {
                const unsigned bm = __ballot_sync(0xffffffffu, take_cell);
                const uint32_t totk[3] = {(uint32_t)__popc(bm), totf, totn};
#pragma unroll
                for (int t = 0; t < 3; ++t) {   // cells, far particles, near particles
                    const uint32_t tot = totk[t];
                    if (tot) {
                        const uint64_t pos = reserve(t, tot);
                        if (pos == ~0ull) break;
                        if (t == 0) {
                            if (take_cell) a.list[pos + __popc(bm & ((1u << lane) - 1u))] = c;
                        } else {
                            const uint32_t k = t == 1 ? kf : kn;
                            uint32_t *dst = a.list + pos + (t == 1 ? exf : exn);
                            for (uint32_t j = 0; j < k; ++j) dst[j] = T.z + j;
                        }
                        if (lane == t) {
                            my_cur = pos + tot;
                            my_len += tot;
                        }
                    }
                }
            }
            if (fail_list || fail_items) break;
            {   // children of opened cells
                const uint32_t tot = totc, k = kc, ex = exc;
                if (sp + (int)tot > WALK_SSTK) {   // move the shared part under the global part
                    if (gp + sp > a.cap_stack) {
                        overflow = true;
                        break;
                    }
                    for (int j = lane; j < sp; j += 32) stk[gp + j] = sstk[j];
                    gp += sp;
                    sp = 0;
                    __syncwarp();
                }
                if (open) {
                    const uint32_t fl = ((uint32_t)open_s << 30) | ((uint32_t)open_h << 31);
                    for (uint32_t j = 0; j < k; ++j) sstk[sp + ex + j] = (T.x + j) | fl;
                }
                sp += (int)tot;
            }
            __syncwarp();
        }
        if (overflow || fail_list || fail_items) break;
        // the group's final runs: several items of one kind add atomically, a single one stores
        uint64_t len3[3], st3[3];
        uint32_t fin_far = early_far, fin_near = early_near;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            len3[t] = __shfl_sync(0xffffffffu, my_len, t);
            st3[t] = __shfl_sync(0xffffffffu, my_start, t);
            const uint64_t per = item_len(gn, t == 2 ? a.lch_near : a.lch_far);
            (t == 2 ? fin_near : fin_far) += (uint32_t)((len3[t] + per - 1) / per);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (len3[t] > 0 && !fail_items)
                if (!emit_items(a, t, st3[t], len3[t], gfirst, gn, s, (t == 2 ? fin_near : fin_far) > 1, lane))
                    fail_items = true;
        if (fail_items) break;
    }
    if (lane == 0) {
        if (overflow) {
            fail(st, HYBRID_ECAPACITY, a.where);
            st->need[2] = 2 * a.cap_stack;
        }
        if (fail_list) {
            fail(st, HYBRID_ECAPACITY, a.where);
            atomicMax((unsigned long long *)&st->need[1], (unsigned long long)(2 * a.cap_list));
        }
        if (fail_items) {
            fail(st, HYBRID_ECAPACITY, a.where);
            atomicMax((unsigned long long *)&st->need[3], (unsigned long long)(2 * a.cap_items));
        }
    }
}

}  // namespace

void launch_walk(hybrid_ctx *c, int mode)
{
    Status *st = status_dev(c);
    WalkArgs a;
    a.ngroups = (const int64_t *)c->ngroups_dev.p;
    a.gnode = (const uint32_t *)c->gnode.p;
    a.gsys = (const uint32_t *)c->gsys.p;
    a.gF = (const GroupF *)c->gF.p;
    a.glo = (const double *)c->glo.p;
    a.ghi = (const double *)c->ghi.p;
    a.sysroot = (const uint32_t *)c->sysroot.p;
    a.sp = (const SysParams *)c->sp_dev.p;
    a.topo = (const uint4 *)c->ntopo.p;
    a.nA = (const float4 *)c->nA.p;
    a.nB = (const float4 *)c->nB.p;
    a.crit = (const float2 *)c->ncrit.p;
    a.nD = (const double4_32a *)c->nD.p;
    a.rb = (const double *)c->nrb.p;
    a.hr = (const double *)c->nhr.p;
    a.cnt = (uint64_t *)c->lcnt.p;
    int64_t *d_n3 = (int64_t *)c->counter.p + 4;
    uint64_t *d_total = (uint64_t *)c->counter.p + 5;
    a.d_n3 = d_n3;
    a.list_total = d_total;
    a.list = (uint32_t *)c->list.p;
    a.cap_list = c->capList;
    a.stack = (uint32_t *)c->stack.p;
    a.cap_stack = c->capStack;
    a.mode = mode;
    a.st = st;
    a.where = c->op;
    a.gfirst = (const uint32_t *)c->gfirst.p;
    a.gcount = (const uint32_t *)c->gcount.p;
    a.list_cursor = (unsigned long long *)c->counter.p + 10;
    a.item_count = (unsigned long long *)c->counter.p + 11;
    a.items_far = (WorkItem *)c->wmap.p;
    a.items_near = (WorkItem *)c->wnear.p;
    a.cap_items = c->capWork;
    // near items: the near kernel's time per tile is mostly latency, so short items spread a small job over more
    // warps; on large jobs every warp has items anyway and longer ones save the per-item set-up. Far items: on a
    // small job short items even out the warps' ends; on a large job long ones hide the set-up of each item (its
    // descriptor, sinks and first gathers) behind more tiles
    const bool small_job = c->N <= (int64_t)1 << 20;
    a.lch_near = small_job ? LCH_NEAR_SMALL : LCH_NEAR;
    a.lch_far = small_job ? LCH_FAR_SMALL : LCH_FAR;
    const int grid = c->walk_warps * 32 / WALK_THREADS;
    cudaEvent_t e0 = nullptr;
    prof_begin(c, PROF_WALK, &e0);
    if (c->p.precision == 1) {   // one pass: the group counter, the list cursor and the item counts start at 0
        cudaMemsetAsync(c->counter.p, 0, sizeof(unsigned long long), c->st);
        cudaMemsetAsync((unsigned long long *)c->counter.p + 10, 0, 3 * sizeof(unsigned long long), c->st);
        a.counter = (unsigned long long *)c->counter.p;
        if (small_job) k_walk1<6><<<grid, WALK_THREADS, 0, c->st>>>(a);
        else k_walk1<8><<<grid, WALK_THREADS, 0, c->st>>>(a);
        prof_end(c, PROF_WALK, e0);
        c->launches += 1;
        c->last_walk_mode = mode;
        return;
    }
    // count pass
    cudaMemsetAsync(c->counter.p, 0, 2 * sizeof(unsigned long long), c->st);
    a.counter = (unsigned long long *)c->counter.p;
    k_walk<true, false><<<grid, WALK_THREADS, 0, c->st>>>(a);
    scan_u64(c, (uint64_t *)c->lcnt.p, 0, d_n3, 3 * c->capGroups, d_total);
    // fill pass
    a.counter = (unsigned long long *)c->counter.p + 1;
    k_walk<true, true><<<grid, WALK_THREADS, 0, c->st>>>(a);
    prof_end(c, PROF_WALK, e0);
    c->launches += 2;
    c->last_walk_mode = mode;
}

}  // namespace hy
