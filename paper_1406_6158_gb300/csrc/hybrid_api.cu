// hybrid_api.cu -- the C-ABI of include/hybrid.h: context, device memory,
// and the step driver that enqueues the hybrid scheme (Sec. II-C) as a
// sequence of ops on the context's stream.
//
// Recovery from capacity overflow: every kernel returns at once when the
// device status word holds a failure, so after a failed op nothing later in
// the sequence has touched the state. The driver then grows the buffer that
// overflowed and resumes at the tree build of the failed force evaluation
// (a build re-sorts already sorted particles into the same order, so it can
// be repeated).
#include <cmath>
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "hy_internal.cuh"

using hy::Buf;

namespace hy {

bool ensure(hybrid_ctx *c, Buf &b, size_t bytes)
{
    if (b.p && b.bytes >= bytes) return true;
    if (c->capturing) {   // no allocation inside a graph capture: every buffer is sized beforehand
        set_err(c, "buffer growth requested during graph capture");
        return false;
    }
    c->gen++;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    const size_t nb = std::max<size_t>(bytes, 256);
    if (cudaMalloc(&b.p, nb) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        set_err(c, "cudaMalloc of %zu bytes failed", nb);
        return false;
    }
    b.bytes = nb;
    return true;
}

void set_err(hybrid_ctx *c, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
}

// A profiling timestamp. Inside a stream capture a plain event record only
// marks a dependency; the external flag makes it a record node of the graph.
void prof_record(hybrid_ctx *c, cudaEvent_t e)
{
    if (c->capturing) cudaEventRecordWithFlags(e, c->st, cudaEventRecordExternal);
    else cudaEventRecord(e, c->st);
}

void prof_begin(hybrid_ctx *c, int kind, cudaEvent_t *e0)
{
    *e0 = nullptr;
    if (!c->prof) return;
    if (c->prof == 1 && kind != PROF_SOFT && kind != PROF_HARD) return;   // level 1: the pair kernels only
    if (c->ev_pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    *e0 = c->ev_pool.back();
    c->ev_pool.pop_back();
    prof_record(c, *e0);
}

void prof_end(hybrid_ctx *c, int kind, cudaEvent_t e0)
{
    if (!c->prof || !e0) return;
    if (c->ev_pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    cudaEvent_t e1 = c->ev_pool.back();
    c->ev_pool.pop_back();
    prof_record(c, e1);
    c->ev_used.push_back({kind, {e0, e1}});
}

}  // namespace hy

namespace {

using namespace hy;

bool params_ok(const hybrid_params *p, std::string *why)
{
    auto bad = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (!std::isfinite(p->G)) return bad("G must be finite");
    if (!(p->eps >= 0.0) || !std::isfinite(p->eps)) return bad("eps must be >= 0");
    if (!(p->theta >= 0.0) || !std::isfinite(p->theta)) return bad("theta must be >= 0");
    const bool no_hard = (p->R1 == 0.0 && p->R2 == 0.0);
    if (!no_hard && !(p->R1 >= 0.0 && p->R2 > p->R1 && std::isfinite(p->R2)))
        return bad("need 0 <= R1 < R2, or R1 = R2 = 0");
    if (!std::isfinite(p->dt_soft)) return bad("dt_soft must be finite");
    if (p->n_hard < 1) return bad("n_hard must be >= 1");
    if (p->n_leaf < 1) return bad("n_leaf must be >= 1");
    if (p->n_crit < 1) return bad("n_crit must be >= 1");
    if (p->precision != 0 && p->precision != 1) return bad("precision must be 0 or 1");
    if (p->mac != 0 && p->mac != 1) return bad("mac must be 0 or 1");
    if (p->mac == 1 && !(p->a_err > 0.0)) return bad("a_err must be > 0 for the absolute MAC");
    if (p->threads_per_group < 0) return bad("threads_per_group must be >= 0");
    if (p->tile_depth != 0 && (p->tile_depth < 2 || p->tile_depth > 4)) return bad("tile_depth must be 0, 2, 3 or 4");
    if (!(p->skin >= 0.0) || !std::isfinite(p->skin)) return bad("skin must be >= 0");
    if (p->skin > 0.0 && (p->precision != 1 || no_hard))
        return bad("skin > 0 needs the FP32 form (precision 1) and a hard part (R2 > 0)");
    return true;
}

SysParams make_sp(const hybrid_params &p)
{
    SysParams s;
    memset(&s, 0, sizeof(s));
    s.G = p.G;
    s.eps2 = p.eps * p.eps;
    s.theta = p.theta;
    s.R1 = p.R1;
    s.R2 = p.R2;
    s.dt_soft = p.dt_soft;
    s.a_err = p.a_err;
    s.h_soft = 0.5 * p.dt_soft;
    s.dt_hard = p.dt_soft / (double)p.n_hard;
    s.h_hard = 0.5 * s.dt_hard;
    s.skin = p.R2 > 0.0 ? p.skin : 0.0;
    s.skinf = (float)s.skin;
    s.half_skinf = (float)(0.5 * s.skin);
    s.has_hard = p.R2 > 0.0 ? 1 : 0;
    s.R2sq = s.has_hard ? p.R2 * p.R2 : 0.0;
    s.invdR = s.has_hard ? 1.0 / (p.R2 - p.R1) : 0.0;
    s.Gf = (float)p.G;
    s.eps2f = (float)s.eps2;
    s.R2f = (float)p.R2;
    s.R2sqf = (float)s.R2sq;
    s.R2sqlo = (float)(s.R2sq - (double)s.R2sqf);
    s.invdRf = (float)s.invdR;
    s.mac = p.mac;
    return s;
}

hybrid_status cuda_fail(hybrid_ctx *c, cudaError_t e, const char *what)
{
    set_err(c, "%s: %s", what, cudaGetErrorString(e));
    return HYBRID_ECUDA;
}

// Node-capacity dependent buffers.
bool alloc_nodes(hybrid_ctx *c, int64_t cap)
{
    const size_t n = (size_t)cap;
    bool ok = true;
    for (Buf *b : {&c->nfirst, &c->ncount, &c->nchild, &c->nnch, &c->nparent, &c->nlevel, &c->ndone, &c->rb2d,
                   &c->rd2b})
        ok = ok && ensure(c, *b, n * 4);
    ok = ok && ensure(c, c->rec, n * 8) && ensure(c, c->nbig, n * 4) && ensure(c, c->nbmax32, n * 4);
    ok = ok && ensure(c, c->rhist, (size_t)(LEVELS + 1) * ((n + 1023) / 1024) * 4);
    for (Buf *b : {&c->nM, &c->ncx, &c->ncy, &c->ncz, &c->nB2, &c->nbmax, &c->nrb, &c->nhr, &c->ndelta, &c->nside})
        ok = ok && ensure(c, *b, n * 8);
    ok = ok && ensure(c, c->norg, n * 24);
    ok = ok && ensure(c, c->nA, n * 16) && ensure(c, c->nB, n * 16) && ensure(c, c->ncrit, n * 8);
    ok = ok && ensure(c, c->ntopo, n * 16) && ensure(c, c->nD, n * 32);
    if (ok) c->capNodes = cap;
    return ok;
}

// FP32 pair work items (40 B each), far (wmap) and near (wnear)
bool ensure_items(hybrid_ctx *c, int64_t n)
{
    if (n <= c->capWork) return true;
    const bool ok = ensure(c, c->wmap, (size_t)n * sizeof(WorkItem)) && ensure(c, c->wnear, (size_t)n * sizeof(WorkItem));
    if (ok) c->capWork = n;
    return ok;
}

bool reserve(hybrid_ctx *c)
{
    const int64_t N = c->N, S = c->S;
    bool ok = true;
    if (N > c->capN) {
        const size_t n = (size_t)N;
        for (int f = 0; f < 7; ++f) ok = ok && ensure(c, c->x[f], n * 8) && ensure(c, c->xa[f], n * 8);
        for (Buf *b : {&c->id, &c->ida, &c->orig, &c->origa, &c->psys, &c->leafof, &c->gflag, &c->gscan, &c->gnode,
                       &c->gfirst, &c->gcount, &c->gsys, &c->pn})
            ok = ok && ensure(c, *b, n * 4);
        ok = ok && ensure(c, c->pc, n) && ensure(c, c->pD, n);
        const size_t asz = c->p.precision == 1 ? 4 : 8;
        for (int d = 0; d < 3; ++d) ok = ok && ensure(c, c->acc_s[d], n * asz) && ensure(c, c->acc_h[d], n * asz);
        if (c->p.precision == 1) ok = ok && ensure(c, c->phi, n * 16) && ensure(c, c->plo, n * 16);
        else ok = ok && ensure(c, c->pd, n * 32);
        if (c->p.skin > 0.0) ok = ok && ensure(c, c->disp, n * 4);
        ok = ok && ensure(c, c->keys[0], n * 8) && ensure(c, c->keys[1], n * 8);
        ok = ok && ensure(c, c->vals[0], n * 4) && ensure(c, c->vals[1], n * 4);
        ok = ok && ensure(c, c->gF, n * sizeof(GroupF)) && ensure(c, c->glo, n * 24) && ensure(c, c->ghi, n * 24);
        ok = ok && ensure(c, c->lcnt, (3 * n + 2) * 8) && ensure(c, c->wstart, (n + 2) * 4);
        // chunks of 128 particles of the large cells: at most 2 N / 128 per level
        const size_t items = 44 * n / 128 + 4096;
        ok = ok && ensure(c, c->mitems, items * 4) && ensure(c, c->mpart, items * 40);
        if (ok) c->capItems = (int64_t)items;
        if (ok) {
            c->capN = N;
            c->capGroups = N;
        }
    }
    if (S > c->capS) {
        const size_t s = (size_t)S;
        ok = ok && ensure(c, c->off_dev, (s + 1) * 8) && ensure(c, c->sp_dev, s * sizeof(SysParams));
        ok = ok && ensure(c, c->boxmin, s * 24) && ensure(c, c->boxmax, s * 24) && ensure(c, c->box, s * sizeof(SysBox));
        ok = ok && ensure(c, c->sysroot, s * 4) && ensure(c, c->io_dev, s * sizeof(SysIO));
        ok = ok && ensure(c, c->energy_dev, s * 16);
        if (ok) c->capS = S;
    }
    if (c->nchunks > c->capChunks) {
        ok = ok && ensure(c, c->chunks_dev, (size_t)c->nchunks * sizeof(Chunk));
        if (ok) c->capChunks = c->nchunks;
    }
    // sample sort: a system table, splitters and bucket counts, starts and cursors, each key's bucket
    ok = ok && ensure(c, c->ss_sys, (size_t)S * sizeof(SSys)) && ensure(c, c->ss_flag, 256) &&
         ensure(c, c->ss_pb, (size_t)std::max<int64_t>(N, 1) * 4);
    if (c->nbk > c->capBk) {
        const size_t nb = (size_t)c->nbk;
        ok = ok && ensure(c, c->ss_spk, nb * 8) && ensure(c, c->ss_spv, nb * 4) && ensure(c, c->ss_cnt, nb * 4) &&
             ensure(c, c->ss_start, nb * 4) && ensure(c, c->ss_cur, nb * 4);
        if (ok) c->capBk = c->nbk;
    }
    // radix sort scratch: 64 tickets, digit counts [S][8][256], look-back words [8][chunks][256]
    ok = ok && ensure(c, c->hist, ((size_t)64 + (size_t)2048 * (S + c->nchunks)) * 4);
    if (c->capNodes < std::max<int64_t>(4096, N)) ok = ok && alloc_nodes(c, std::max<int64_t>(4096, N));
    // list entries: ~128 per particle, plus the unused tails of the regions the walking warps
    // claim (three kinds of at most 2048 entries per warp)
    const int64_t list0 = std::max<int64_t>(1 << 20, 128 * N) + (int64_t)3 * 2048 * c->walk_warps;
    if (c->capList < list0) {
        ok = ok && ensure(c, c->list, (size_t)list0 * 4);
        if (ok) c->capList = list0;
    }
    ok = ok && ensure_items(c, 2 * c->capGroups + c->capList / 256 + 1024);
    if (c->capStack == 0) c->capStack = 4096;
    ok = ok && ensure(c, c->stack, (size_t)c->walk_warps * c->capStack * 4);
    // scratch of the scans: the longest scan is over max(N, nodes, 3 groups + 1, tiles x 256)
    const int64_t longest = std::max<int64_t>({N, c->capNodes, 3 * c->capGroups + 2, (int64_t)c->nchunks * 256});
    ok = ok && ensure(c, c->blocksum, (size_t)((longest + SCAN_SEG - 1) / SCAN_SEG + 1) * 8);
    return ok;
}

// Validates the systems, lays them out back to back, builds the radix tiles
// and the per-system parameter table, and reserves every buffer.
hybrid_status setup_batch(hybrid_ctx *c, const hybrid_system *sys, int S, bool need_acc)
{
    if (!sys || S < 1) {
        set_err(c, "no systems");
        return HYBRID_EINVAL;
    }
    c->h_off.assign(S + 1, 0);
    c->h_sp.resize(S);
    for (int s = 0; s < S; ++s) {
        const hybrid_system &y = sys[s];
        if (y.n < 1) {
            set_err(c, "system %d: n must be >= 1", s);
            return HYBRID_EINVAL;
        }
        if (!y.x || !y.y || !y.z || !y.vx || !y.vy || !y.vz || !y.m) {
            set_err(c, "system %d: null state pointer", s);
            return HYBRID_EINVAL;
        }
        if (need_acc && (!y.ax_s || !y.ay_s || !y.az_s || !y.ax_h || !y.ay_h || !y.az_h)) {
            set_err(c, "system %d: null acceleration pointer", s);
            return HYBRID_EINVAL;
        }
        hybrid_params p = c->p;
        if (y.params) {
            const hybrid_params &q = *y.params;
            p.G = q.G;
            p.eps = q.eps;
            p.theta = q.theta;
            p.R1 = q.R1;
            p.R2 = q.R2;
            p.dt_soft = q.dt_soft;
            p.a_err = q.a_err;
            p.mac = q.mac;
            std::string why;
            if (!params_ok(&p, &why)) {
                set_err(c, "system %d: %s", s, why.c_str());
                return HYBRID_EINVAL;
            }
        }
        c->h_sp[s] = make_sp(p);
        c->h_off[s + 1] = c->h_off[s] + y.n;
    }
    if (c->h_off[S] >= (int64_t)0x7fffffff) {
        set_err(c, "too many particles (%lld)", (long long)c->h_off[S]);
        return HYBRID_EINVAL;
    }
    c->S = S;
    c->N = c->h_off[S];
    // radix tiles: the largest of 512..2048 keys that still gives about 4 tiles per SM
    c->ipt = RS_IPT_MAX;
    while (c->ipt > 2 && c->N / (RS_WARPS * 32 * c->ipt) < 4 * c->nsm) c->ipt >>= 1;
    c->tile = RS_WARPS * 32 * c->ipt;
    const int tile = c->tile;
    c->h_chunks.clear();
    for (int s = 0; s < S; ++s) {
        const int first = (int)c->h_chunks.size();
        const int64_t n = c->h_off[s + 1] - c->h_off[s];
        const int nch = (int)((n + tile - 1) / tile);
        for (int k = 0; k < nch; ++k) {
            Chunk ch;
            ch.start = c->h_off[s] + (int64_t)k * tile;
            ch.len = (int)std::min<int64_t>(tile, n - (int64_t)k * tile);
            ch.sys = s;
            ch.first_chunk = first;
            ch.nchunk = nch;
            c->h_chunks.push_back(ch);
        }
    }
    c->nchunks = (int)c->h_chunks.size();
    // sample sort layout: about SS_BUCKET keys per bucket, half that on batches of at most 2^20 particles (more
    // blocks for the bucket sort when the whole batch is a few tens of buckets)
    c->h_ss.resize(S);
    c->nbk = 0;
    c->ss_ok = true;
    const int64_t bucket = c->N <= ((int64_t)1 << 20) ? SS_BUCKET / 2 : SS_BUCKET;
    for (int s = 0; s < S; ++s) {
        const int64_t n = c->h_off[s + 1] - c->h_off[s];
        SSys &y = c->h_ss[s];
        y.nb = (int32_t)((n + bucket - 1) / bucket);
        y.bbase = c->nbk;
        c->nbk += y.nb;
    }
    if (!reserve(c)) return HYBRID_ENOMEM;
    c->h_io.resize(S);
    for (int s = 0; s < S; ++s) {
        const hybrid_system &y = sys[s];
        SysIO &o = c->h_io[s];
        o.x[0] = y.x;
        o.x[1] = y.y;
        o.x[2] = y.z;
        o.x[3] = y.vx;
        o.x[4] = y.vy;
        o.x[5] = y.vz;
        o.x[6] = y.m;
        o.id = y.id;
        o.as[0] = y.ax_s;
        o.as[1] = y.ay_s;
        o.as[2] = y.az_s;
        o.ah[0] = y.ax_h;
        o.ah[1] = y.ay_h;
        o.ah[2] = y.az_h;
        o.n = y.n;
        o.off = c->h_off[s];
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->off_dev.p, c->h_off.data(), (S + 1) * 8, cudaMemcpyHostToDevice, c->st)) ||
        (e = cudaMemcpyAsync(c->sp_dev.p, c->h_sp.data(), S * sizeof(SysParams), cudaMemcpyHostToDevice, c->st)) ||
        (e = cudaMemcpyAsync(c->chunks_dev.p, c->h_chunks.data(), c->nchunks * sizeof(Chunk),
                             cudaMemcpyHostToDevice, c->st)) ||
        (e = cudaMemcpyAsync(c->io_dev.p, c->h_io.data(), S * sizeof(SysIO), cudaMemcpyHostToDevice, c->st)) ||
        (e = cudaMemcpyAsync(c->ss_sys.p, c->h_ss.data(), S * sizeof(SSys), cudaMemcpyHostToDevice, c->st)))
        return cuda_fail(c, e, "upload of the batch tables");
    c->tree_valid = false;
    return HYBRID_OK;
}

// ---- ops ----
enum OpKind { OP_KICKS, OP_BUILD, OP_WALK, OP_PAIR_FAR, OP_PAIR_NEAR };
struct Op {
    int kind = OP_BUILD;
    int mode = 0;
    int nk = 0;
    int which[4] = {0, 0, 0, 0};
    int kmode[4] = {0, 0, 0, 0};
    double val[4] = {0, 0, 0, 0};
    int dmode = -1;
    double dval = 0.0;
};

void enqueue(hybrid_ctx *c, const Op &o, int idx)
{
    c->op = idx;
    switch (o.kind) {
    case OP_KICKS:   // mode 1: the drift of a hard step that reuses the neighbour lists
        launch_kick_seq(c, o.nk, o.which, o.kmode, o.val, o.dmode, o.dval, o.mode == 1);
        break;
    case OP_BUILD: {
        // The build as a two-branch DAG: after the key sort, the topology (keys only) and then the group
        // table run beside the permutation of the state; the moments need the topology and the permuted
        // state (not the groups), the group boxes the group table and the permuted state.
        cudaEvent_t e0 = nullptr;
        prof_begin(c, PROF_TREE, &e0);
        cudaEvent_t e1 = nullptr;
        prof_begin(c, PROF_SORT, &e1);
        launch_box(c);
        launch_keys_sort(c);
        prof_end(c, PROF_SORT, e1);
        cudaStream_t main = c->st;
        cudaEventRecord(c->ev_fork[0], main);
        cudaStreamWaitEvent(c->st2, c->ev_fork[0], 0);
        c->st = c->st2;
        prof_begin(c, PROF_TOPO, &e1);
        launch_build_levels(c);
        prof_end(c, PROF_TOPO, e1);
        cudaEventRecord(c->ev_join[0], c->st2);   // topology done
        prof_begin(c, PROF_GROUPS, &e1);
        launch_groups(c);
        prof_end(c, PROF_GROUPS, e1);
        c->st = main;
        launch_permute(c);
        cudaEventRecord(c->ev_fork[1], main);      // permuted state done
        cudaStreamWaitEvent(main, c->ev_join[0], 0);
        prof_begin(c, PROF_MOM, &e1);
        launch_moments(c);
        prof_end(c, PROF_MOM, e1);
        c->st = c->st2;
        cudaStreamWaitEvent(c->st2, c->ev_fork[1], 0);
        launch_group_boxes(c);
        cudaEventRecord(c->ev_join[1], c->st2);
        c->st = main;
        cudaStreamWaitEvent(main, c->ev_join[1], 0);
        prof_end(c, PROF_TREE, e0);
        break;
    }
    case OP_WALK:
        launch_walk(c, o.mode);
        break;
    case OP_PAIR_FAR:
        launch_pair_far(c);
        break;
    case OP_PAIR_NEAR:
        launch_pair_near(c, o.mode);
        break;
    }
}

hybrid_status read_status(hybrid_ctx *c, Status *out)
{
    cudaError_t e = cudaMemcpyAsync(c->h_status, c->status.p, sizeof(Status), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronisation");
    *out = *c->h_status;
    return HYBRID_OK;
}

hybrid_status clear_status(hybrid_ctx *c)
{
    cudaError_t e = cudaMemsetAsync(c->status.p, 0, sizeof(Status), c->st);
    return e == cudaSuccess ? HYBRID_OK : cuda_fail(c, e, "status reset");
}

void swap_state(hybrid_ctx *c)
{
    for (int f = 0; f < 7; ++f) std::swap(c->x[f], c->xa[f]);
    std::swap(c->id, c->ida);
    std::swap(c->orig, c->origa);
    c->swaps ^= 1;
}

// Adds the elapsed times of recorded (kind, start, end) event pairs; the
// stream has been synchronised by the caller.
void prof_collect(hybrid_ctx *c, const std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> &ev)
{
    for (auto &u : ev) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, u.second.first, u.second.second) == cudaSuccess) {
            c->prof_ms[u.first] += t;
            c->prof_n[u.first] += 1;
        }
    }
    cudaGetLastError();
}

void drop_graphs(hybrid_ctx *c)
{
    for (auto &g : c->graphs) {
        cudaGraphExecDestroy(g.exec);
        for (auto &u : g.events) {
            c->ev_pool.push_back(u.second.first);
            c->ev_pool.push_back(u.second.second);
        }
    }
    c->graphs.clear();
}

uint64_t ops_signature(const hybrid_ctx *c, const std::vector<Op> &ops)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix((uint64_t)c->N);
    mix((uint64_t)c->S);
    mix((uint64_t)c->nchunks);
    mix((uint64_t)c->ipt);
    mix((uint64_t)c->nbk);
    mix((uint64_t)c->ss_ok);
    mix((uint64_t)c->prof);
    for (const Op &o : ops) {
        mix((uint64_t)o.kind);
        mix((uint64_t)o.mode);
        mix((uint64_t)o.nk);
        mix((uint64_t)o.dmode);
        for (int k = 0; k < o.nk; ++k) mix((uint64_t)(o.which[k] * 4 + o.kmode[k]));
    }
    return h;
}

// Captures ops as a CUDA graph (or finds the cached one) and launches it.
// Returns false when graphs cannot be used; the ops are then not enqueued.
bool launch_as_graph(hybrid_ctx *c, const std::vector<Op> &ops, std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> **events)
{
    if (!c->use_graphs || c->st == nullptr) return false;
    const uint64_t sig = ops_signature(c, ops);
    for (auto &g : c->graphs) {
        if (g.sig == sig && g.parity == c->swaps && g.gen == c->gen) {
            if (cudaGraphLaunch(g.exec, c->st) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            if (g.net_swaps) swap_state(c);
            c->launches += g.nlaunch;
            *events = &g.events;
            return true;
        }
    }
    // make sure the profiling events exist before capturing
    if (c->prof)
        while (c->ev_pool.size() < 4 * ops.size() + 64) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->ev_pool.push_back(e);
        }
    const int parity0 = c->swaps;
    const int64_t gen0 = c->gen, l0 = c->launches;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> saved;
    saved.swap(c->ev_used);
    cudaGraph_t graph = nullptr;
    c->capturing = true;
    cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (size_t i = 0; i < ops.size(); ++i) enqueue(c, ops[i], (int)i);
        e = cudaStreamEndCapture(c->st, &graph);
    }
    c->capturing = false;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && c->gen == gen0) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || c->gen != gen0 || !exec) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (c->swaps != parity0) swap_state(c);   // undo the host side of the capture
        for (auto &u : c->ev_used) {
            c->ev_pool.push_back(u.second.first);
            c->ev_pool.push_back(u.second.second);
        }
        c->ev_used.swap(saved);
        c->launches = l0;
        c->use_graphs = false;
        return false;
    }
    hybrid_ctx::GraphEntry g;
    g.sig = sig;
    g.parity = parity0;
    g.net_swaps = c->swaps != parity0;
    g.gen = gen0;
    g.nlaunch = c->launches - l0;
    g.exec = exec;
    g.events.swap(c->ev_used);
    c->ev_used.swap(saved);
    // the capture already moved the host-side pointers to their post-graph state
    if (cudaGraphLaunch(exec, c->st) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(exec);
        if (g.net_swaps) swap_state(c);
        c->launches = l0;
        c->use_graphs = false;
        return false;
    }
    c->graphs.push_back(std::move(g));
    *events = &c->graphs.back().events;
    return true;
}

Op simple(int kind, int mode = 0);

hybrid_status run_ops(hybrid_ctx *c, const std::vector<Op> &ops_in)
{
    std::vector<Op> ops = ops_in;
    size_t start = 0;
    bool skin_recovered = false;
    c->sort_fallback = false;
    struct SortMode {   // the radix sort of a fallback lasts for this sequence only
        hybrid_ctx *c;
        ~SortMode() { c->sort_fallback = false; }
    } sort_mode{c};
    for (int attempt = 0; attempt < 12; ++attempt) {
        std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> *gev = nullptr;
        if (!(attempt == 0 && !skin_recovered && !c->sort_fallback && launch_as_graph(c, ops, &gev)))
            for (size_t i = start; i < ops.size(); ++i) enqueue(c, ops[i], (int)i);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return cuda_fail(c, le, "kernel launch");
        Status s;
        hybrid_status r = read_status(c, &s);
        if (r != HYBRID_OK) return r;
        if (c->prof) {
            if (gev) prof_collect(c, *gev);
            prof_collect(c, c->ev_used);
            for (auto &u : c->ev_used) {
                c->ev_pool.push_back(u.second.first);
                c->ev_pool.push_back(u.second.second);
            }
            c->ev_used.clear();
        }
        if (s.code == 0) return HYBRID_OK;
        if (s.code == ST_SORT && !c->sort_fallback && s.where >= 0 && (size_t)s.where < ops.size()) {
            // a sample-sort bucket overflowed (a state far from key order): that build left the order as it was
            // and skipped the rest; repeat from it with the radix sort (eagerly; the captured graphs stay)
            c->sort_fallback = true;
            c->sort_fallbacks++;
            start = (size_t)s.where;
            while (start > 0 && ops[start].kind != OP_BUILD) --start;
            --attempt;
            if ((r = clear_status(c)) != HYBRID_OK) return r;
            continue;
        }
        drop_graphs(c);
        if (s.code == ST_SKIN && !skin_recovered && s.where >= 0 && (size_t)s.where < ops.size()) {
            // a particle moved more than skin / 2 in the drift of op `where`: that hard step and every later
            // one in this call rebuild the tree and the lists (the drift itself is done)
            std::vector<Op> rest;
            rest.push_back(simple(OP_BUILD));
            rest.push_back(simple(OP_WALK, 2));
            for (size_t i = (size_t)s.where + 1; i < ops.size(); ++i) {
                Op o = ops[i];
                const bool reused = o.kind == OP_KICKS && o.mode == 1;
                o.mode = reused ? 0 : o.mode;
                rest.push_back(o);
                if (reused) {
                    rest.push_back(simple(OP_BUILD));
                    rest.push_back(simple(OP_WALK, 2));
                }
            }
            ops.swap(rest);
            start = 0;
            skin_recovered = true;
            --attempt;   // not a capacity attempt; the rest runs eagerly
            if ((r = clear_status(c)) != HYBRID_OK) return r;
            continue;
        }
        if (s.code != HYBRID_ECAPACITY) {
            set_err(c, "device failure %d at op %d", s.code, s.where);
            clear_status(c);
            return (hybrid_status)s.code;
        }
        // grow what overflowed, then resume at the build of the failed evaluation
        bool ok = true;
        if (s.need[0] > c->capNodes) ok = ok && alloc_nodes(c, s.need[0]);
        if (s.need[1] > c->capList) {
            const int64_t cap = s.need[1] + s.need[1] / 4 + 1024;
            ok = ok && ensure(c, c->list, (size_t)cap * 4);
            if (ok) c->capList = cap;
            ok = ok && ensure_items(c, 2 * c->capGroups + c->capList / 256 + 1024);
        }
        if (s.need[3] > c->capWork) ok = ok && ensure_items(c, s.need[3]);
        if (s.need[2] > c->capStack) {
            ok = ok && ensure(c, c->stack, (size_t)c->walk_warps * s.need[2] * 4);
            if (ok) c->capStack = s.need[2];
        }
        const int64_t longest = std::max<int64_t>({c->N, c->capNodes, 3 * c->capGroups + 2, (int64_t)c->nchunks * 256});
        ok = ok && ensure(c, c->blocksum, (size_t)((longest + SCAN_SEG - 1) / SCAN_SEG + 1) * 8);
        if (!ok) return HYBRID_ENOMEM;
        if ((r = clear_status(c)) != HYBRID_OK) return r;
        start = (size_t)std::max(0, s.where);
        while (start > 0 && ops[start].kind != OP_BUILD) --start;
    }
    set_err(c, "capacity could not be grown enough");
    return HYBRID_ECAPACITY;
}

Op kicks(int nk, const int *which, const int *kmode, int dmode)
{
    Op o;
    o.kind = OP_KICKS;
    o.nk = nk;
    for (int k = 0; k < nk; ++k) {
        o.which[k] = which[k];
        o.kmode[k] = kmode[k];
    }
    o.dmode = dmode;
    return o;
}

Op simple(int kind, int mode)
{
    Op o;
    o.kind = kind;
    o.mode = mode;
    return o;
}

// The op sequence of n_steps soft steps (Sec. II-C, kick-drift-kick):
// K_s(dt_s/2); n x [K_h(dt_h/2); D(dt_h); build; hard (+ soft at the last);
// K_h(dt_h/2)]; K_s(dt_s/2). Adjacent kicks share one launch (same order).
// With a skin (reused lists, not part of the method) the hard steps 1..n-1
// skip the build and the walk when the lists of the last build still hold:
// their drift also refreshes the FP32 positions and the distance bound.
std::vector<Op> step_ops(const hybrid_ctx *c, int n_steps, bool valid, bool lists_ok)
{
    const bool reuse = c->p.skin > 0.0;
    std::vector<Op> ops;
    if (!valid) {
        ops.push_back(simple(OP_BUILD));
        ops.push_back(simple(OP_WALK, 3));
        ops.push_back(simple(OP_PAIR_FAR));
        ops.push_back(simple(OP_PAIR_NEAR, 3));
        lists_ok = true;
    }
    int pw[8], pm[8], np = 0;
    auto add = [&](int which, int mode) {
        pw[np] = which;
        pm[np] = mode;
        ++np;
    };
    const int nh = c->p.n_hard;
    for (int s = 0; s < n_steps; ++s) {
        add(0, 1);
        for (int k = 1; k <= nh; ++k) {
            add(1, 2);
            Op kd = kicks(np, pw, pm, 2);
            np = 0;
            if (reuse && k < nh && lists_ok) {
                kd.mode = 1;
                ops.push_back(kd);
                ops.push_back(simple(OP_PAIR_NEAR, 2));
            } else {
                ops.push_back(kd);
                ops.push_back(simple(OP_BUILD));
                ops.push_back(simple(OP_WALK, k == nh ? 3 : 2));
                if (k == nh) ops.push_back(simple(OP_PAIR_FAR));
                ops.push_back(simple(OP_PAIR_NEAR, k == nh ? 3 : 2));
                lists_ok = true;
            }
            add(1, 2);
        }
        add(0, 1);
    }
    if (np) ops.push_back(kicks(np, pw, pm, -1));
    return ops;
}

hybrid_status finish(hybrid_ctx *c, hybrid_status r)
{
    if (r == HYBRID_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    }
    return r;
}

template <typename T>
bool d2h(hybrid_ctx *c, std::vector<T> &v, const Buf &b, size_t n)
{
    v.resize(n);
    if (n == 0) return true;
    return cudaMemcpyAsync(v.data(), b.p, n * sizeof(T), cudaMemcpyDeviceToHost, c->st) == cudaSuccess;
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

hybrid_status hybrid_create(hybrid_ctx **out, const hybrid_params *p, void *stream)
{
    if (!out || !p) return HYBRID_EINVAL;
    *out = nullptr;
    if (!params_ok(p, nullptr)) return HYBRID_EINVAL;
    hybrid_ctx *c = new hybrid_ctx();
    c->p = *p;
    c->st = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev);
    if (e == cudaSuccess) e = init_pair_kernels();
    if (e == cudaSuccess) e = init_tree_kernels();
    if (e != cudaSuccess) {
        delete c;
        return HYBRID_ECUDA;
    }
    c->walk_warps = c->nsm * 32;
    if (cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return HYBRID_ECUDA;
    }
    for (int k = 0; k < 2; ++k) {
        cudaEventCreateWithFlags(&c->ev_fork[k], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming);
    }
    {   // HYBRID_GRAPHS=0 enqueues every op directly instead of replaying captured CUDA graphs
        const char *g = getenv("HYBRID_GRAPHS");
        if (g && g[0] == '0') c->use_graphs = false;
    }
    bool ok = ensure(c, c->status, sizeof(Status)) && ensure(c, c->counter, 16 * 8) && ensure(c, c->lvl, 1024) &&
              ensure(c, c->ngroups_dev, 64);
    if (!ok) {
        hybrid_destroy(c);
        return HYBRID_ENOMEM;
    }
    if (cudaMallocHost((void **)&c->h_status, sizeof(Status)) != cudaSuccess) {
        hybrid_destroy(c);
        return HYBRID_ENOMEM;
    }
    cudaMemsetAsync(c->status.p, 0, sizeof(Status), c->st);
    cudaMemsetAsync(c->counter.p, 0, 16 * 8, c->st);
    cudaMemsetAsync(c->ngroups_dev.p, 0, 64, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) {
        hybrid_destroy(c);
        return HYBRID_ECUDA;
    }
    *out = c;
    return HYBRID_OK;
}

hybrid_status hybrid_destroy(hybrid_ctx *c)
{
    if (!c) return HYBRID_OK;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    Buf *all[] = {&c->id, &c->ida, &c->orig, &c->origa, &c->psys, &c->phi, &c->plo, &c->pd, &c->disp, &c->keys[0], &c->keys[1],
                  &c->vals[0], &c->vals[1], &c->hist, &c->blocksum, &c->off_dev, &c->sp_dev, &c->chunks_dev,
                  &c->ss_sys, &c->ss_spk, &c->ss_spv, &c->ss_cnt, &c->ss_start, &c->ss_cur, &c->ss_pb, &c->ss_flag,
                  &c->boxmin, &c->boxmax, &c->box, &c->sysroot, &c->status, &c->lvl, &c->nfirst, &c->ncount,
                  &c->nchild, &c->nnch, &c->nparent, &c->nlevel, &c->ndone, &c->leafof, &c->pc, &c->pD, &c->pn, &c->rec,
                  &c->rb2d, &c->rd2b, &c->rhist, &c->nM, &c->ncx,
                  &c->ncy, &c->ncz, &c->nB2, &c->nbmax, &c->nA, &c->nB, &c->ncrit, &c->ntopo, &c->nD, &c->nrb,
                  &c->nhr, &c->ndelta, &c->nside, &c->norg, &c->gflag, &c->gscan, &c->gnode, &c->gfirst, &c->gcount,
                  &c->gsys, &c->gF, &c->glo, &c->ghi, &c->ngroups_dev, &c->lcnt, &c->list, &c->stack, &c->counter,
                  &c->io_dev, &c->energy_dev, &c->wstart, &c->wmap, &c->nbig, &c->mitems, &c->mpart, &c->nbmax32, &c->wnear};
    for (Buf *b : all)
        if (b->p) cudaFree(b->p);
    for (int f = 0; f < 7; ++f) {
        if (c->x[f].p) cudaFree(c->x[f].p);
        if (c->xa[f].p) cudaFree(c->xa[f].p);
    }
    for (int d = 0; d < 3; ++d) {
        if (c->acc_s[d].p) cudaFree(c->acc_s[d].p);
        if (c->acc_h[d].p) cudaFree(c->acc_h[d].p);
    }
    drop_graphs(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (auto &u : c->ev_used) {
        cudaEventDestroy(u.second.first);
        cudaEventDestroy(u.second.second);
    }
    if (c->h_status) cudaFreeHost(c->h_status);
    for (int k = 0; k < 2; ++k) {
        if (c->ev_fork[k]) cudaEventDestroy(c->ev_fork[k]);
        if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
    }
    if (c->st2) {
        cudaStreamSynchronize(c->st2);
        cudaStreamDestroy(c->st2);
    }
    delete c;
    return HYBRID_OK;
}

hybrid_status hybrid_build_tree(hybrid_ctx *c, hybrid_system *sys)
{
    if (!c || !sys) return HYBRID_EINVAL;
    hybrid_status r = setup_batch(c, sys, 1, false);
    if (r != HYBRID_OK) return r;
    launch_copy_in(c, (const SysIO *)c->io_dev.p, false);
    c->lists_fresh = false;
    r = run_ops(c, {simple(OP_BUILD)});
    if (r != HYBRID_OK) return r;
    launch_copy_out(c, (const SysIO *)c->io_dev.p, true, false, false);
    sys->forces_valid = 0;
    c->tree_valid = true;
    c->have_soft = c->have_hard = false;
    return finish(c, HYBRID_OK);
}

hybrid_status force_call(hybrid_ctx *c, hybrid_system *sys, bool soft)
{
    if (!c || !sys) return HYBRID_EINVAL;
    if (!c->tree_valid || c->S != 1 || c->N != sys->n) {
        set_err(c, "no tree for this system: call hybrid_build_tree first");
        return HYBRID_EINVAL;
    }
    void *a[3] = {soft ? sys->ax_s : sys->ax_h, soft ? sys->ay_s : sys->ay_h, soft ? sys->az_s : sys->az_h};
    if (!a[0] || !a[1] || !a[2]) {
        set_err(c, "null acceleration pointer");
        return HYBRID_EINVAL;
    }
    // the output arrays may differ from the ones of the build call
    SysIO &o = c->h_io[0];
    for (int d = 0; d < 3; ++d) (soft ? o.as : o.ah)[d] = a[d];
    cudaError_t e = cudaMemcpyAsync(c->io_dev.p, &o, sizeof(SysIO), cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload");
    c->lists_fresh = false;
    std::vector<Op> ops = {simple(OP_WALK, soft ? 1 : 2)};
    if (soft) ops.push_back(simple(OP_PAIR_FAR));
    ops.push_back(simple(OP_PAIR_NEAR, soft ? 1 : 2));
    hybrid_status r = run_ops(c, ops);
    if (r != HYBRID_OK) return r;
    launch_copy_out(c, (const SysIO *)c->io_dev.p, false, soft, !soft);
    (soft ? c->have_soft : c->have_hard) = true;
    sys->forces_valid = (c->have_soft && c->have_hard) ? 1 : 0;
    return finish(c, HYBRID_OK);
}

hybrid_status hybrid_soft_force(hybrid_ctx *c, hybrid_system *sys) { return force_call(c, sys, true); }
hybrid_status hybrid_hard_force(hybrid_ctx *c, hybrid_system *sys) { return force_call(c, sys, false); }

hybrid_status hybrid_kick(hybrid_ctx *c, hybrid_system *sys, int which, double dt)
{
    if (!c || !sys || (which != 0 && which != 1) || sys->n < 1 || !sys->vx || !sys->vy || !sys->vz) return HYBRID_EINVAL;
    if (which == 0 && (!sys->ax_s || !sys->ay_s || !sys->az_s)) return HYBRID_EINVAL;
    if (which == 1 && (!sys->ax_h || !sys->ay_h || !sys->az_h)) return HYBRID_EINVAL;
    launch_kick_ext(c, sys, which, dt);
    return finish(c, HYBRID_OK);
}

hybrid_status hybrid_drift(hybrid_ctx *c, hybrid_system *sys, double dt)
{
    if (!c || !sys || sys->n < 1 || !sys->x || !sys->y || !sys->z || !sys->vx || !sys->vy || !sys->vz)
        return HYBRID_EINVAL;
    launch_drift_ext(c, sys, dt);
    sys->forces_valid = 0;
    return finish(c, HYBRID_OK);
}

hybrid_status hybrid_step_batched(hybrid_ctx *c, hybrid_system *sys, int n_sys, int n_soft_steps)
{
    if (!c || !sys || n_sys < 1 || n_soft_steps < 0) return HYBRID_EINVAL;
    hybrid_status r = setup_batch(c, sys, n_sys, true);
    if (r != HYBRID_OK) return r;
    bool valid = true;
    for (int s = 0; s < n_sys; ++s) valid = valid && sys[s].forces_valid;
    // the lists of the previous call hold when the same arrays come back unchanged (forces_valid)
    uint64_t sig = 1469598103934665603ull;
    auto mixs = [&](uint64_t v) { sig = (sig ^ v) * 1099511628211ull; };
    mixs((uint64_t)n_sys);
    for (int s = 0; s < n_sys; ++s) {
        mixs((uint64_t)sys[s].n);
        mixs((uint64_t)(uintptr_t)sys[s].x);
    }
    const bool lists_ok = valid && c->lists_fresh && c->lists_sig == sig;
    c->lists_fresh = false;
    launch_copy_in(c, (const SysIO *)c->io_dev.p, valid);
    r = run_ops(c, step_ops(c, n_soft_steps, valid, lists_ok));
    if (r != HYBRID_OK) return r;
    c->lists_fresh = c->p.skin > 0.0;
    c->lists_sig = sig;
    launch_copy_out(c, (const SysIO *)c->io_dev.p, true, true, true);
    Status s;
    if ((r = read_status(c, &s)) != HYBRID_OK) return r;
    for (int k = 0; k < n_sys; ++k) sys[k].forces_valid = 1;
    c->tree_valid = (n_sys == 1);
    c->have_soft = c->have_hard = true;
    return finish(c, HYBRID_OK);
}

hybrid_status hybrid_step(hybrid_ctx *c, hybrid_system *sys, int n_soft_steps)
{
    return hybrid_step_batched(c, sys, 1, n_soft_steps);
}

hybrid_status hybrid_autotune(hybrid_ctx *c, hybrid_system *sys, int n_sys, const int32_t *cand, int n_cand,
                              double *ms_out, int32_t *best_out)
{
    static const int32_t defaults[][3] = {
        {16, 4, 0},  {16, 8, 0},  {32, 8, 0},  {32, 16, 0}, {64, 16, 0},  {64, 32, 0}, {128, 32, 0}, {128, 64, 0},
        {32, 8, 2},  {32, 8, 4},  {64, 16, 2}, {64, 16, 4}, {128, 32, 2}, {128, 32, 4}, {256, 64, 0},
        {256, 64, 2}, {128, 16, 0}, {256, 32, 0}};
    if (!c || !sys || n_sys < 1 || n_cand < 0 || (n_cand > 0 && !cand)) return HYBRID_EINVAL;
    c->lists_fresh = false;
    const int32_t *cv = n_cand > 0 ? cand : &defaults[0][0];
    const int nc = n_cand > 0 ? n_cand : (int)(sizeof(defaults) / sizeof(defaults[0]));
    const hybrid_params saved = c->p;
    for (int i = 0; i < nc; ++i) {
        hybrid_params q = saved;
        q.n_crit = cv[3 * i];
        q.threads_per_group = cv[3 * i + 1];
        q.tile_depth = cv[3 * i + 2];
        std::string why;
        if (!params_ok(&q, &why)) {
            set_err(c, "candidate %d: %s", i, why.c_str());
            return HYBRID_EINVAL;
        }
    }
    hybrid_status r = setup_batch(c, sys, n_sys, true);
    if (r != HYBRID_OK) return r;
    // the systems' own arrays are only read (copy-in); every candidate runs on the working copy
    launch_copy_in(c, (const SysIO *)c->io_dev.p, false);
    const std::vector<Op> soft = {simple(OP_BUILD), simple(OP_WALK, 3), simple(OP_PAIR_FAR), simple(OP_PAIR_NEAR, 3)};
    const std::vector<Op> hard = {simple(OP_BUILD), simple(OP_WALK, 2), simple(OP_PAIR_NEAR, 2)};
    cudaEvent_t ev[3];
    for (int k = 0; k < 3; ++k)
        if (cudaEventCreate(&ev[k]) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "event creation");
    int best = -1;
    double best_ms = 0.0;
    for (int i = 0; i < nc && r == HYBRID_OK; ++i) {
        c->p.n_crit = cv[3 * i];
        c->p.threads_per_group = cv[3 * i + 1];
        c->p.tile_depth = cv[3 * i + 2];
        drop_graphs(c);   // captured launches carry the old choice
        if ((r = run_ops(c, soft)) != HYBRID_OK || (r = run_ops(c, hard)) != HYBRID_OK) break;   // warm-up
        cudaEventRecord(ev[0], c->st);
        if ((r = run_ops(c, soft)) != HYBRID_OK) break;
        cudaEventRecord(ev[1], c->st);
        if ((r = run_ops(c, hard)) != HYBRID_OK) break;
        cudaEventRecord(ev[2], c->st);
        float t1 = 0.0f, t2 = 0.0f;
        cudaError_t e = cudaEventSynchronize(ev[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t2, ev[1], ev[2]);
        if (e != cudaSuccess) {
            r = cuda_fail(c, e, "autotune timing");
            break;
        }
        // one soft step = one soft evaluation + (n_hard - 1) hard evaluations (kicks do not depend on the choice)
        const double ms = (double)t1 + (double)(c->p.n_hard - 1) * (double)t2;
        if (ms_out) ms_out[i] = ms;
        if (best < 0 || ms < best_ms) {
            best = i;
            best_ms = ms;
        }
    }
    for (int k = 0; k < 3; ++k) cudaEventDestroy(ev[k]);
    c->p = saved;
    if (r == HYBRID_OK && best >= 0) {
        c->p.n_crit = cv[3 * best];
        c->p.threads_per_group = cv[3 * best + 1];
        c->p.tile_depth = cv[3 * best + 2];
    }
    drop_graphs(c);
    c->tree_valid = false;
    c->have_soft = c->have_hard = false;
    if (best_out) *best_out = best;
    return finish(c, r);
}

hybrid_status hybrid_selftest_wait(hybrid_ctx *c, int32_t max_polls)
{
    if (!c || max_polls < 1) return HYBRID_EINVAL;
    launch_wait_selftest(c, max_polls);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    return hybrid_sync(c);
}

hybrid_status hybrid_get_perm(hybrid_ctx *c, int32_t *dev_perm)
{
    if (!c || !dev_perm || c->N == 0) return HYBRID_EINVAL;
    cudaError_t e = cudaMemcpyAsync(dev_perm, c->orig.p, (size_t)c->N * 4, cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return e == cudaSuccess ? HYBRID_OK : cuda_fail(c, e, "perm copy");
}

hybrid_status hybrid_sync(hybrid_ctx *c)
{
    if (!c) return HYBRID_EINVAL;
    Status s;
    hybrid_status r = read_status(c, &s);
    if (r != HYBRID_OK) return r;
    if (s.code) {
        set_err(c, "device failure %d at op %d", s.code, s.where);
        clear_status(c);
        return (hybrid_status)s.code;
    }
    return HYBRID_OK;
}

const char *hybrid_last_error(hybrid_ctx *c) { return c ? c->err.c_str() : "null context"; }

hybrid_status hybrid_tree_info(hybrid_ctx *c, int64_t *n_nodes, int64_t *n_groups)
{
    if (!c || !c->tree_valid) return HYBRID_EINVAL;
    uint32_t lv[LEVELS + 3];
    int64_t ng = 0;
    cudaError_t e = cudaMemcpyAsync(lv, c->lvl.p, sizeof(lv), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ng, c->ngroups_dev.p, 8, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "tree info");
    if (n_nodes) *n_nodes = lv[LEVELS + 1];
    if (n_groups) *n_groups = ng;
    return HYBRID_OK;
}

hybrid_status hybrid_tree_copy(hybrid_ctx *c, uint64_t *keys, int32_t *level, int64_t *first, int64_t *count,
                               int64_t *child, int32_t *nchild, int64_t *parent, double *moments, int64_t *group_node,
                               double *group_lo, double *group_hi)
{
    int64_t nn = 0, ng = 0;
    hybrid_status r = hybrid_tree_info(c, &nn, &ng);
    if (r != HYBRID_OK) return r;
    std::vector<uint32_t> f, cn, ch, nc, pa, lv, gn;
    std::vector<double> M, cx, cy, cz, bm, B2, de, sd, og, rb, glo, ghi;
    std::vector<uint64_t> k;
    bool ok = d2h(c, f, c->nfirst, nn) && d2h(c, cn, c->ncount, nn) && d2h(c, ch, c->nchild, nn) &&
              d2h(c, nc, c->nnch, nn) && d2h(c, pa, c->nparent, nn) && d2h(c, lv, c->nlevel, nn) &&
              d2h(c, gn, c->gnode, ng) && d2h(c, M, c->nM, nn) && d2h(c, cx, c->ncx, nn) && d2h(c, cy, c->ncy, nn) &&
              d2h(c, cz, c->ncz, nn) && d2h(c, bm, c->nbmax, nn) && d2h(c, B2, c->nB2, nn) &&
              d2h(c, de, c->ndelta, nn) && d2h(c, sd, c->nside, nn) && d2h(c, og, c->norg, 3 * nn) &&
              d2h(c, rb, c->nrb, nn) && d2h(c, glo, c->glo, 3 * ng) && d2h(c, ghi, c->ghi, 3 * ng) &&
              d2h(c, k, c->keys[0], c->N);
    if (!ok || cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "tree copy");
    for (int64_t i = 0; i < nn; ++i) {
        if (level) level[i] = (int32_t)lv[i];
        if (first) first[i] = f[i];
        if (count) count[i] = cn[i];
        if (child) child[i] = nc[i] ? (int64_t)ch[i] : -1;
        if (nchild) nchild[i] = (int32_t)nc[i];
        if (parent) parent[i] = pa[i] == NONE ? -1 : (int64_t)pa[i];
        if (moments) {
            double *o = moments + 13 * i;
            o[0] = M[i];
            o[1] = cx[i];
            o[2] = cy[i];
            o[3] = cz[i];
            o[4] = bm[i];
            o[5] = B2[i];
            o[6] = de[i];
            o[7] = sd[i];
            o[8] = og[3 * i];
            o[9] = og[3 * i + 1];
            o[10] = og[3 * i + 2];
            o[11] = rb[i];
            o[12] = 0.0;
        }
    }
    for (int64_t g = 0; g < ng; ++g) {
        if (group_node) group_node[g] = gn[g];
        for (int d = 0; d < 3; ++d) {
            if (group_lo) group_lo[3 * g + d] = glo[3 * g + d];
            if (group_hi) group_hi[3 * g + d] = ghi[3 * g + d];
        }
    }
    if (keys) memcpy(keys, k.data(), (size_t)c->N * 8);
    return HYBRID_OK;
}

hybrid_status hybrid_lists_copy(hybrid_ctx *c, int64_t *counts, int64_t *entries, int64_t cap_entries)
{
    int64_t nn = 0, ng = 0;
    hybrid_status r = hybrid_tree_info(c, &nn, &ng);
    if (r != HYBRID_OK) return r;
    const bool soft = c->last_walk_mode & 1, hard = (c->last_walk_mode >> 1) & 1;
    if (c->p.precision == 1) {
        // one-pass walk: a group's entries of each kind are the runs of its work items, in item order
        uint64_t ctr[16];
        if (cudaMemcpyAsync(ctr, c->counter.p, sizeof ctr, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
            cudaStreamSynchronize(c->st) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "list copy");
        std::vector<WorkItem> itf, itn;
        std::vector<uint32_t> gf, L;
        if (!d2h(c, itf, c->wmap, (size_t)ctr[11]) || !d2h(c, itn, c->wnear, (size_t)ctr[12]) ||
            !d2h(c, gf, c->gfirst, (size_t)ng) || !d2h(c, L, c->list, (size_t)ctr[10]) ||
            cudaStreamSynchronize(c->st) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "list copy");
        auto group_of = [&](uint32_t first) {
            return (int64_t)(std::lower_bound(gf.begin(), gf.end(), first) - gf.begin());
        };
        std::vector<std::vector<uint32_t>> K[3];
        for (auto &k : K) k.assign((size_t)ng, {});
        for (const WorkItem &d : itf) {
            const int64_t g = group_of(d.first);
            for (uint32_t e = d.e0; e < d.e1; ++e)
                K[e < d.Lc ? 0 : 1][(size_t)g].push_back(L[(e < d.Lc ? d.cbase : d.pbase) + e]);
        }
        for (const WorkItem &d : itn) {
            const int64_t g = group_of(d.first);
            for (uint32_t e = d.e0; e < d.e1; ++e) K[2][(size_t)g].push_back(L[d.pbase + e]);
        }
        int64_t need = 0;
        for (int64_t g = 0; g < ng; ++g) {
            counts[3 * g + 0] = soft ? (int64_t)K[0][g].size() : 0;
            counts[3 * g + 1] = soft ? (int64_t)(K[1][g].size() + K[2][g].size()) : 0;
            counts[3 * g + 2] = hard ? (int64_t)K[2][g].size() : 0;
            need += counts[3 * g] + counts[3 * g + 1] + counts[3 * g + 2];
        }
        if (!entries) return HYBRID_OK;
        if (need > cap_entries) return HYBRID_EINVAL;
        int64_t o = 0;
        for (int64_t g = 0; g < ng; ++g) {
            if (soft)
                for (int k = 0; k < 3; ++k)
                    for (uint32_t v : K[k][g]) entries[o++] = v;
            if (hard)
                for (uint32_t v : K[2][g]) entries[o++] = v;
        }
        return HYBRID_OK;
    }
    std::vector<uint64_t> off;
    if (!d2h(c, off, c->lcnt, 3 * ng + 1) || cudaStreamSynchronize(c->st) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "list copy");
    // stored as cells, far particles, near particles; reported as cells, soft
    // particles (far then near) and hard particles (near, when the walk asked for them)
    const uint64_t total = off[3 * ng];
    int64_t need = 0;
    for (int64_t g = 0; g < ng; ++g) {
        const int64_t nc = (int64_t)(off[g + 1] - off[g]), nf = (int64_t)(off[ng + g + 1] - off[ng + g]),
                      nn = (int64_t)(off[2 * ng + g + 1] - off[2 * ng + g]);
        counts[3 * g + 0] = soft ? nc : 0;
        counts[3 * g + 1] = soft ? nf + nn : 0;
        counts[3 * g + 2] = hard ? nn : 0;
        need += counts[3 * g] + counts[3 * g + 1] + counts[3 * g + 2];
    }
    if (!entries) return HYBRID_OK;
    if (need > cap_entries) return HYBRID_EINVAL;
    std::vector<uint32_t> L;
    if (!d2h(c, L, c->list, total) || cudaStreamSynchronize(c->st) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "list copy");
    int64_t o = 0;
    for (int64_t g = 0; g < ng; ++g) {
        if (soft) {
            for (uint64_t j = off[g]; j < off[g + 1]; ++j) entries[o++] = L[j];
            for (uint64_t j = off[ng + g]; j < off[ng + g + 1]; ++j) entries[o++] = L[j];
            for (uint64_t j = off[2 * ng + g]; j < off[2 * ng + g + 1]; ++j) entries[o++] = L[j];
        }
        if (hard)
            for (uint64_t j = off[2 * ng + g]; j < off[2 * ng + g + 1]; ++j) entries[o++] = L[j];
    }
    return HYBRID_OK;
}

hybrid_status hybrid_interactions(hybrid_ctx *c, int64_t *soft, int64_t *hard)
{
    if (!c) return HYBRID_EINVAL;
    uint64_t v[16];
    cudaError_t e = cudaMemcpyAsync(v, c->counter.p, sizeof(v), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "counters");
    if (soft) *soft = (int64_t)v[6];
    if (hard) *hard = (int64_t)v[7];
    return HYBRID_OK;
}

hybrid_status hybrid_profile(hybrid_ctx *c, int enable)
{
    if (!c) return HYBRID_EINVAL;
    const int level = enable == 0 ? 0 : (enable == 1 ? 1 : 2);
    if (c->prof != level) drop_graphs(c);   // the brackets are part of the captured graphs
    c->prof = level;
    return HYBRID_OK;
}

hybrid_status hybrid_profile_read(hybrid_ctx *c, int kind, double *ms, int64_t *launches, int reset)
{
    if (!c || kind < 0 || kind >= PROF_KINDS) return HYBRID_EINVAL;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "profile sync");
    prof_collect(c, c->ev_used);
    for (auto &u : c->ev_used) {
        c->ev_pool.push_back(u.second.first);
        c->ev_pool.push_back(u.second.second);
    }
    c->ev_used.clear();
    if (ms) *ms = c->prof_ms[kind];
    if (launches) *launches = c->prof_n[kind];
    if (reset)
        for (int k = 0; k < PROF_KINDS; ++k) {
            c->prof_ms[k] = 0.0;
            c->prof_n[k] = 0;
        }
    return HYBRID_OK;
}

int64_t hybrid_launch_count(hybrid_ctx *c) { return c ? c->launches : 0; }

int64_t hybrid_sort_fallbacks(hybrid_ctx *c) { return c ? c->sort_fallbacks : 0; }

hybrid_status hybrid_energy(hybrid_ctx *c, hybrid_system *sys, double *kinetic, double *potential)
{
    if (!c || !sys || !kinetic || !potential) return HYBRID_EINVAL;
    hybrid_status r = setup_batch(c, sys, 1, false);
    if (r != HYBRID_OK) return r;
    launch_copy_in(c, (const SysIO *)c->io_dev.p, false);
    launch_energy(c, (double *)c->energy_dev.p);
    double v[2];
    cudaError_t e = cudaMemcpyAsync(v, c->energy_dev.p, 16, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "energy");
    *kinetic = v[0];
    *potential = v[1];
    return HYBRID_OK;
}

}  // extern "C"
