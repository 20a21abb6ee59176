// hy_internal.cuh -- internal definitions of the CUDA library (context, device
// tables, kernel launchers). Not a public header; see include/hybrid.h.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hybrid.h"

namespace hy {

constexpr int LEVELS = 21;                 // 3 x 21 = 63 Morton key bits
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr int RS_WARPS = 8;                // radix sort: 8 warps x 32 lanes x ipt items per tile
constexpr int RS_IPT_MAX = 8;
constexpr int RS_TILE_MAX = RS_WARPS * 32 * RS_IPT_MAX;   // 2048 keys per tile at most
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_SEG = SCAN_THREADS * SCAN_IPT; // 2048 elements per scan segment

// Per-system parameters on the device (FP64 for the tree/integrator, FP32
// copies for the pair kernels).
struct SysParams {
    double G, eps2, theta, R1, R2, dt_soft, a_err;
    double R2sq, invdR;            // R2^2, 1/(R2-R1) (0 when there is no hard part)
    double h_soft, dt_hard, h_hard;   // dt_soft/2, dt_soft/n_hard, dt_hard/2 (each correctly rounded)
    double skin;                      // Verlet skin of reused neighbour lists (0: rebuild every hard step)
    float Gf, eps2f, R2f, R2sqf, invdRf, R2sqlo;   // R2sqf + R2sqlo = R2^2 to ~2^-48
    float skinf, half_skinf;       // skin and skin / 2 in FP32
    int32_t mac, has_hard;
};

// Root cube of one system: origin lo, side L (a power of two), scale = 2^21/L.
// The FP32 copies of positions are taken relative to lo and split as
// x - lo = hi + lo_part with hi on the grid of step u = L / 2^20, so hi is
// exact in FP32 and the difference of two hi values is exact too.
struct SysBox {
    double lo[3];
    double L;
    double scale;
    double u, inv_u;
    float uf, inv_uf;   // u and 1/u in FP32 (powers of two: exact)
};

// FP32 hi/lo copy of a coordinate relative to the root corner: hi = the
// nearest multiple of u (at most 2^20 steps: exact in FP32), lo = the rest
// (exact in FP64, then rounded to FP32, |lo| <= u/2).
__device__ __forceinline__ void grid_split(double x, double lo0, const SysBox &b, float &h, float &l)
{
    const double xp = __dsub_rn(x, lo0);
    const double hh = __dmul_rn(rint(__dmul_rn(xp, b.inv_u)), b.u);
    h = (float)hh;
    l = (float)__dsub_rn(xp, hh);
}

// Internal status code (never returned to the caller): a particle moved more
// than skin / 2 since the last build; the step resumes with a rebuild.
constexpr int32_t ST_SKIN = 100;
// Internal status code: a bucket of the sample sort held more keys than a
// block sorts in shared memory; the build left the order unchanged and is
// repeated with the radix sort.
constexpr int32_t ST_SORT = 101;

// Sample sort of the keys (the usual path once the state is close to key
// order): per system, nb buckets of about SS_BUCKET keys split by keys taken
// at regular positions; a bucket of at most SS_CAP keys (twice the target:
// the splitters are the last build's quantiles, and only the particles that
// crossed a coarse cell boundary since move between buckets) is sorted in one
// block.
constexpr int SS_BUCKET = 2048;
constexpr int SS_CAP = 4096;
struct SSys {
    int32_t nb;      // buckets of the system
    int32_t bbase;   // index of its first bucket
};

// Device status block: first failure wins (atomicCAS on code).
struct Status {
    int32_t code;        // hybrid_status of the first failure, 0 = none
    int32_t where;       // op index at which it happened
    int64_t need[6];     // [0] nodes, [1] list entries, [2] walk stack entries
    int64_t counters[4]; // [0] soft interactions, [1] hard interactions
};

// A tile of at most ctx->tile consecutive particles inside one system.
struct Chunk {
    int64_t start;
    int32_t len;
    int32_t sys;
    int32_t first_chunk;   // first chunk of this chunk's system
    int32_t nchunk;        // chunks of this chunk's system
};

// Per-group data for the walk and pair kernels.
// FP32 pair work item: the entry range [e0, e1) of one group's list, that
// list being a cell run (entries e < Lc, at list[cbase + e]) followed by a
// particle run (entries e >= Lc, at list[pbase + e]; pbase = start of the
// particle run - Lc, modulo 2^64). Written by the single-pass walk.
struct WorkItem {
    uint64_t cbase, pbase;
    uint32_t Lc, e0, e1, first;
    uint32_t n;     // group size; bit 31 set when the group has several work items of this kind
    uint32_t sys;
};
static_assert(sizeof(WorkItem) == 40, "WorkItem layout");
constexpr uint32_t ITEM_MULTI = 0x80000000u;
constexpr int LCH_FAR = 2048, LCH_FAR_SMALL = 256, LCH_NEAR = 512, LCH_NEAR_SMALL = 64;

// Entries per work item of a group of n sinks: lch for n >= 64, longer runs
// (up to 8 lch) for smaller groups, so that items cost about the same
// n x entries and a small group pays the per-item set-up less often.
__host__ __device__ __forceinline__ uint64_t item_len(uint32_t n, int lch)
{
    const uint32_t f = n >= 64 ? 1u : (64u / (n > 0 ? n : 1u) < 8u ? 64u / (n > 0 ? n : 1u) : 8u);
    return (uint64_t)lch * f;
}

struct GroupF {
    float4 c_hi;       // centre of the member box, hi part; w = half extent x
    float4 c_lo;       // centre lo part; w = half extent y
    float2 hz_root;    // x = half extent z; y unused
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Caller arrays of one system (device pointers) and its offset in the batch.
struct SysIO {
    double *x[7];
    int32_t *id;
    void *as[3], *ah[3];
    int64_t n, off;
};

enum ProfKind {
    PROF_SOFT = 0, PROF_HARD = 1, PROF_WALK = 2, PROF_TREE = 3, PROF_INTEG = 4,
    PROF_SORT = 5, PROF_TOPO = 6, PROF_MOM = 7, PROF_GROUPS = 8, PROF_KINDS = 9
};

}  // namespace hy

struct hybrid_ctx {
    hybrid_params p{};
    cudaStream_t st = nullptr;
    cudaStream_t st2 = nullptr;          // second branch of the tree build
    cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr};
    int dev = 0, nsm = 0;
    std::string err;
    int64_t launches = 0;
    int op = 0;   // index of the op being enqueued (for failure reports)

    // batch layout of the current call
    int S = 0;
    int64_t N = 0;
    std::vector<int64_t> h_off;                // S + 1
    std::vector<hy::SysParams> h_sp;
    std::vector<hy::Chunk> h_chunks;
    std::vector<hy::SysIO> h_io;
    int nchunks = 0;
    int ipt = hy::RS_IPT_MAX, tile = hy::RS_TILE_MAX;   // radix tile: 8 warps x 32 lanes x ipt keys, sized to fill the GPU
    // sample sort layout of the batch (buckets over all systems) and whether the current call repeats a build
    // with the radix sort after a bucket overflowed
    std::vector<hy::SSys> h_ss;
    int nbk = 0;
    bool ss_ok = false, sort_fallback = false;
    int64_t sort_fallbacks = 0;
    bool tree_valid = false, have_soft = false, have_hard = false;
    // reused neighbour lists (skin > 0): the lists of the last walk still hold for the working state of the
    // batch with this signature (set at the end of a step, cleared by anything else that builds or walks)
    bool lists_fresh = false;
    uint64_t lists_sig = 0;

    // capacities
    int64_t capN = 0, capS = 0, capChunks = 0, capNodes = 0, capGroups = 0, capList = 0, capStack = 0;
    int walk_warps = 0;

    // device buffers: state (two copies each for the permutation), ids
    hy::Buf x[7], xa[7], id, ida, orig, origa, psys;
    hy::Buf acc_s[3], acc_h[3];            // float or double
    hy::Buf phi, plo, pd;                  // float4 hi/lo (precision 1), double4_32a (precision 0)
    hy::Buf disp;                          // float: bound of the distance moved since the last build (skin > 0)
    hy::Buf keys[2], vals[2], hist, blocksum;
    hy::Buf ss_sys, ss_spk, ss_spv, ss_cnt, ss_start, ss_cur, ss_pb, ss_flag;   // sample sort
    int64_t capBk = 0;
    hy::Buf off_dev, sp_dev, chunks_dev, boxmin, boxmax, box, sysroot;
    hy::Buf status;
    // tree
    hy::Buf lvl, nfirst, ncount, nchild, nnch, nparent, nlevel, ndone, leafof;
    hy::Buf pc, pD, pn, rec, rb2d, rd2b, rhist;     // topology build scratch
    hy::Buf nbig, mitems, mpart;                  // moments of large cells: chunk items and sums
    hy::Buf nbmax32;                              // b_max as FP32 bits (FP32 form)
    int64_t capItems = 0;
    hy::Buf nM, ncx, ncy, ncz, nB2, nbmax;     // FP64 moments
    hy::Buf nA, nB, ncrit, ntopo;              // FP32 walk/pair node data
    hy::Buf nD, nrb, nhr;                      // FP64 walk/pair node data (precision 0)
    hy::Buf ndelta, nside, norg;               // geometry (inspection + finalize)
    hy::Buf gflag, gscan, gnode, gfirst, gcount, gsys, gF, glo, ghi, ngroups_dev;
    // lists
    hy::Buf lcnt, loff, list, stack, counter, io_dev, energy_dev, wstart, wmap;
    hy::Buf wnear;                                 // near-pair work items (wmap holds the far ones)
    int64_t capWork = 0;                           // work items per kind
    int last_walk_mode = 0;

    // profiling
    int prof = 0;                          // 0 off, 1 pair kernels, 2 every stage
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    double prof_ms[hy::PROF_KINDS] = {0};
    int64_t prof_n[hy::PROF_KINDS] = {0};

    // host pinned status
    hy::Status *h_status = nullptr;

    // CUDA graphs of op sequences (one per sequence, buffer generation and
    // parity of the state-buffer swaps done by the tree builds)
    int swaps = 0;          // parity of x <-> xa swaps so far
    int64_t gen = 0;        // bumped by every (re)allocation
    bool use_graphs = true;
    struct GraphEntry {
        uint64_t sig;
        int parity, net_swaps;
        int64_t gen, nlaunch;
        cudaGraphExec_t exec;
        std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
    };
    std::vector<GraphEntry> graphs;
    bool capturing = false;
};

namespace hy {

// ---- memory / errors (hybrid_api.cu) ----
bool ensure(hybrid_ctx *c, Buf &b, size_t bytes);
void set_err(hybrid_ctx *c, const char *fmt, ...);
inline Status *status_dev(hybrid_ctx *c) { return (Status *)c->status.p; }
void prof_begin(hybrid_ctx *c, int kind, cudaEvent_t *e0);
void prof_end(hybrid_ctx *c, int kind, cudaEvent_t e0);

// ---- scans (scan.cu) ----
// Exclusive scan of n uint32 values (n from *d_n when d_n != null, else n_host),
// in place; *d_total (optional) receives the sum. n_max bounds the grid.
// always = true: runs even after a recorded failure (the sort's scans).
void scan_u32(hybrid_ctx *c, uint32_t *data, int64_t n_host, const int64_t *d_n, int64_t n_max, uint64_t *d_total,
              bool always = false);
void scan_u64(hybrid_ctx *c, uint64_t *data, int64_t n_host, const int64_t *d_n, int64_t n_max, uint64_t *d_total,
              bool always = false);

// ---- tree (tree.cu) ----
void launch_box(hybrid_ctx *c);
void launch_keys_sort(hybrid_ctx *c);      // keys and their stable sort (keys[0], vals[0])
void launch_permute(hybrid_ctx *c);        // state into key order, pair-kernel copies of the positions
bool launch_build_levels(hybrid_ctx *c);   // topology from the sorted keys
void launch_moments(hybrid_ctx *c);        // needs topology and the permuted state
void launch_groups(hybrid_ctx *c);         // group table from the topology
void launch_group_boxes(hybrid_ctx *c);    // needs the group table and the permuted state
void launch_wait_selftest(hybrid_ctx *c, int max_polls);   // a bounded wait on a flag nothing sets

// ---- walk (walk.cu) ----
void launch_walk(hybrid_ctx *c, int mode);   // mode bit 0 soft, bit 1 hard

// ---- pair kernels (pair.cu) ----
// cells and far particles of the last walk -> soft accelerations (zeroed first)
void launch_pair_far(hybrid_ctx *c);
// near particles of the last walk: mode bit 0 adds F (1 - K) to the soft
// accelerations (after launch_pair_far), bit 1 writes F K as the hard ones
void launch_pair_near(hybrid_ctx *c, int mode);
// shared-memory attributes of the far kernels (once per device, before any launch or capture)
cudaError_t init_pair_kernels();
// shared-memory attribute of the sample sort's splitter kernel
cudaError_t init_tree_kernels();

// ---- integrator and io (integrate.cu) ----
void launch_copy_in(hybrid_ctx *c, const SysIO *d_io, bool with_acc);
void launch_copy_out(hybrid_ctx *c, const SysIO *d_io, bool state, bool acc_s, bool acc_h);
// Applies n <= 4 kicks v <- v + h a_which in order (which 0 soft, 1 hard;
// mode 0: h = val, 1: h = dt_soft/2, 2: h = (dt_soft/n_hard)/2, per system),
// then a drift x <- x + dt v (dmode -1: none, 0: dt = dval, 2: dt_soft/n_hard).
void launch_kick_seq(hybrid_ctx *c, int n, const int *which, const int *mode, const double *val, int dmode,
                     double dval, bool resplit = false);
void launch_kick_ext(hybrid_ctx *c, const hybrid_system *s, int which, double h);
void launch_drift_ext(hybrid_ctx *c, const hybrid_system *s, double dt);
void launch_energy(hybrid_ctx *c, double *d_out /* 2*S */);

}  // namespace hy

// kernel launch bookkeeping
#define HY_LAUNCHED(c) ((c)->launches++)
