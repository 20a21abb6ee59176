/*
 * hybrid.h -- C-ABI of the GB300 hybrid tree force path.
 *
 * The method (Watanabe & Nakasato, "GPU accelerated Hybrid Tree Algorithm for
 * Collision-less N-body Simulations") splits softened gravity, Eq. (1)-(2),
 * into a hard part F*K(r) and a soft part F*(1-K(r)) with the DLL kernel K of
 * Eq. (10) (Eq. 7-9). The soft part comes from a Barnes-Hut octree
 * (Sec. II-B), the hard part from direct summation over neighbours within R2
 * (found with the test of Eq. 15), and each part is advanced by its own
 * leap-frog, Eq. (3)-(4), with dt_soft = n_hard * dt_hard (Sec. II-C).
 *
 * Conventions for every call:
 *  - All particle arrays are DEVICE pointers owned by the caller (CUDA
 *    allocations, e.g. torch tensors), structure-of-arrays, length n.
 *  - Work is enqueued on the context's stream and is asynchronous unless a
 *    call says otherwise. Device-side failures (capacity, timeout) are
 *    reported by the next call that synchronises (hybrid_step,
 *    hybrid_step_batched, hybrid_sync).
 *  - Argument errors return HYBRID_EINVAL before anything is enqueued.
 *  - Nothing throws across this boundary; hybrid_last_error() gives the text
 *    of the last failure on a context.
 *  - The state is kept in Morton (key) order: a tree build re-sorts x, v, m
 *    and id in place (the particle sort of Sec. III-A1).
 */
#ifndef HYBRID_H
#define HYBRID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYBRID_OK = 0,
    HYBRID_EINVAL = 1,     /* bad argument: nothing was enqueued */
    HYBRID_ENOMEM = 2,     /* device allocation failed */
    HYBRID_ECUDA = 3,      /* a CUDA runtime call failed */
    HYBRID_ECAPACITY = 4,  /* an internal buffer overflowed and could not be regrown */
    HYBRID_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
    HYBRID_ETOOLARGE = 6   /* input larger than a fixed-size scratch buffer holds */
} hybrid_status;

/* Method parameters (Sec. II; Sec. IV-A gives the paper's values).
 * G        gravitational constant (Eq. 2)
 * eps      softening length (Eq. 2), >= 0
 * theta    opening angle for mac = 0: a cell is opened when r < l/theta + delta
 *          (l cell side, delta offset of the centre of mass from the cell
 *          centre); theta = 0 opens every cell (direct summation)
 * R1, R2   transition radii of K (Eq. 10); 0 <= R1 < R2, or R1 = R2 = 0 for
 *          no hard part (K = 0)
 * dt_soft  soft time step dt_s; the hard step is dt_soft / n_hard (Sec. II-C)
 * a_err    accuracy parameter of the absolute MAC (Eq. 5), used when mac = 1
 * n_hard   n >= 1: hard sub-steps per soft step
 * n_leaf   a cell splits while it holds more than n_leaf particles (Sec. II-B)
 * n_crit   sink groups are the first cells holding <= n_crit particles (or
 *          leaves): the grouped form of the n_vec sinks of Sec. III-A2, Eq. (11)
 * precision 0: all pair arithmetic in FP64; 1: FP32 pair arithmetic on
 *          coordinates relative to each sink group (state stays FP64)
 * mac      0: opening angle theta; 1: absolute MAC with a_err (Eq. 5-6)
 * threads_per_group: lanes that share one copy of a sink group in the FP32
 *          pair kernels; each lane then keeps ceil(n_crit / threads_per_group)
 *          sinks in registers (1, 2, 4 or 8; 4 at most in the near kernel).
 *          0 = built-in default.
 * tile_depth: shared-memory staging depth of the FP32 far pair kernel: source
 *          gathers run tile_depth - 1 tiles of 64 list entries ahead of their
 *          use; 2, 3 or 4, 0 = built-in default (3).
 * n_crit, threads_per_group and tile_depth change speed, not results beyond
 * FP32 rounding order (n_crit also changes the groups and thus the lists);
 * hybrid_autotune chooses them.
 * skin:    Verlet skin for reusing the tree and the neighbour lists across
 *          hard steps. The paper rebuilds the tree at every hard step (Sec.
 *          II-C, IV-C); this option is not part of the method and 0 (the
 *          default) keeps the paper's scheme. With skin > 0 (FP32 form,
 *          precision 1, with a hard part, R2 > 0) the walk of each soft-force
 *          evaluation treats R2 + skin as the cutoff radius of Eq. (15): a
 *          cell is taken whole only beyond R2 + skin + b_max and every leaf
 *          within that radius lists its particles as neighbours (pairs beyond
 *          R2 get K = 0, so the forces are those of the method with that
 *          slightly more accurate tree opening). The n - 1 hard steps that
 *          follow reuse that tree, its groups and its neighbour lists: their
 *          hard force is the same sum over the current positions of the
 *          listed neighbours. Each drift adds the distance it moved a
 *          particle (rounded up) to a per-particle bound since the last
 *          build; when one exceeds skin / 2 a pair within R2 could be
 *          missing, and that hard step and the later ones of the same call
 *          rebuild the tree and the lists first. EINVAL when skin < 0, or
 *          skin > 0 without precision 1 and a hard part. */
typedef struct {
    double G, eps, theta, R1, R2, dt_soft, a_err;
    int32_t n_hard, n_leaf, n_crit;
    int32_t precision;
    int32_t mac;
    int32_t threads_per_group;
    int32_t tile_depth;
    double skin;
} hybrid_params;

/* One independent system. Arrays are device pointers of length n.
 * x..m      FP64 state (positions, velocities, masses), caller-owned
 * id        optional int32 labels permuted together with the state (NULL ok)
 * ax_s..az_h accelerations: soft (s) and hard (h); float when the context's
 *          precision is 1, double when 0. hybrid_step reads them as the
 *          forces at the current positions when forces_valid != 0 and writes
 *          the forces at the final positions.
 * params   optional per-system override of G, eps, theta, R1, R2, dt_soft,
 *          a_err and mac (the other fields are taken from the context); NULL
 *          uses the context's parameters.
 * forces_valid in/out: set to 1 by every call that leaves the accelerations
 *          consistent with the positions, to 0 by hybrid_build_tree.
 * n        particles, n >= 1: a call given an empty system (n < 1), alone or
 *          in a batch, returns HYBRID_EINVAL before anything is enqueued. */
typedef struct {
    int64_t n;
    double *x, *y, *z, *vx, *vy, *vz, *m;
    int32_t *id;
    void *ax_s, *ay_s, *az_s, *ax_h, *ay_h, *az_h;
    const hybrid_params *params;
    int32_t forces_valid;
} hybrid_system;

typedef struct hybrid_ctx hybrid_ctx;

/* Creates a context bound to the current CUDA device and to `stream`
 * (a cudaStream_t; NULL = the legacy default stream). Validates p (EINVAL). */
hybrid_status hybrid_create(hybrid_ctx **ctx, const hybrid_params *p, void *stream);

/* Frees every device buffer the context owns. NULL is accepted. */
hybrid_status hybrid_destroy(hybrid_ctx *ctx);

/* Sec. III-A1: root cell, Morton keys, stable key sort, the particle data
 * gathered into key order, level-wise octree split (n_leaf), cell mass and
 * centre of mass (Sec. II-B), b_max, B2 and the MAC radius (Eq. 5-6), and the
 * sink groups. Re-sorts x, v, m and id of `sys` in place and keeps the tree
 * in the context for the force calls; sets sys->forces_valid = 0. */
hybrid_status hybrid_build_tree(hybrid_ctx *ctx, hybrid_system *sys);

/* Soft force (Eq. 9): for every sink group, a tree walk from the root
 * (Sec. II-B traversal; Eq. 11 distance to the group box) that takes a cell
 * whole when r >= r_b and r >= R2 + b_max (Eq. 15), else opens it; then
 * a_soft = sum over taken cells of F + sum over listed particles of
 * F*(1 - K). Uses the tree and positions of the last hybrid_build_tree on
 * this context; writes ax_s, ay_s, az_s. */
hybrid_status hybrid_soft_force(hybrid_ctx *ctx, hybrid_system *sys);

/* Hard force (Eq. 8): neighbour walk keeping cells with r < R2 + b_max
 * (Eq. 15), then a_hard = sum over their particles of F*K(r) (Eq. 10).
 * Same tree as hybrid_soft_force; writes ax_h, ay_h, az_h. */
hybrid_status hybrid_hard_force(hybrid_ctx *ctx, hybrid_system *sys);

/* Kick, Eq. (3): v <- v + dt * a, with a the soft (which = 0) or the hard
 * (which = 1) acceleration of sys. */
hybrid_status hybrid_kick(hybrid_ctx *ctx, hybrid_system *sys, int which, double dt);

/* Drift, Eq. (4): x <- x + dt * v. */
hybrid_status hybrid_drift(hybrid_ctx *ctx, hybrid_system *sys, double dt);

/* n_soft_steps soft steps of the hybrid scheme (Sec. II-C), each
 *   K_s(dt_s/2); n_hard x [K_h(dt_h/2); D(dt_h); tree build; hard force
 *   (and at the last sub-step also the soft force); K_h(dt_h/2)]; K_s(dt_s/2)
 * i.e. one soft-step and n_hard - 1 hard-steps per dt_s. Forces at the start
 * are computed first when sys->forces_valid == 0. Synchronises the stream at
 * the end and returns any device-side failure. */
hybrid_status hybrid_step(hybrid_ctx *ctx, hybrid_system *sys, int n_soft_steps);

/* The same for n_sys independent systems of uneven size, processed together:
 * every kernel launch covers all systems. All systems share n_hard, n_leaf,
 * n_crit and precision; their other parameters may differ (params). */
hybrid_status hybrid_step_batched(hybrid_ctx *ctx, hybrid_system *sys, int n_sys, int n_soft_steps);

/* Autotuner (an implementation choice, not part of the method): for each
 * candidate (n_crit, threads_per_group, tile_depth) -- cand holds n_cand
 * triples; cand = NULL, n_cand = 0 uses a built-in list of 18 -- times one
 * soft evaluation (tree build, walk, far and near pairs) and one hard
 * evaluation (build, hard walk, near pairs) of the given systems with CUDA
 * events after one untimed run, and estimates the time of a soft step as
 * soft + (n_hard - 1) x hard. The fastest candidate becomes the context's
 * setting for later calls. ms_out (optional, host, n_cand doubles) receives
 * the estimates, best_out (optional) the index of the choice. The systems'
 * arrays are read, not written. EINVAL for an invalid candidate. With a
 * skin (see hybrid_params) the estimate still counts a build and a walk per
 * hard step, which reused lists skip. */
hybrid_status hybrid_autotune(hybrid_ctx *ctx, hybrid_system *sys, int n_sys, const int32_t *cand, int n_cand,
                              double *ms_out, int32_t *best_out);

/* Copies the permutation of the last call into dev_perm (device int32, length
 * = total particles of that call): dev_perm[k] = index, in that call's input
 * order within its system, of the particle now at position k. */
hybrid_status hybrid_get_perm(hybrid_ctx *ctx, int32_t *dev_perm);

/* Self-test of failure detection (not part of the method): the library's one
 * device-side wait (the key sort's look-back) is bounded, records
 * HYBRID_ETIMEOUT when its polls run out and lets the kernel finish. This call
 * runs that wait, with max_polls polls, on a flag that nothing sets, then
 * returns what hybrid_sync returns: HYBRID_ETIMEOUT, with the context still
 * usable. EINVAL for max_polls < 1. */
hybrid_status hybrid_selftest_wait(hybrid_ctx *ctx, int32_t max_polls);

/* Waits for the context's stream and returns the first device-side failure
 * recorded since the last check (and clears it). */
hybrid_status hybrid_sync(hybrid_ctx *ctx);

/* Text of the last failure on ctx ("" if none). Valid until the next call. */
const char *hybrid_last_error(hybrid_ctx *ctx);

/* ---- inspection (tests and tuning; not needed to run a simulation) ---- */

/* Tree of the last build: node count, group count, and host copies.
 * Sizes: the caller passes arrays of length >= the counts; any pointer may be
 * NULL. Nodes are in breadth-first order over all systems: by level, then
 * system, then key. Groups are in particle order. level/nchild are int32,
 * first/count/child/parent int64 (child = -1 for a leaf, parent = -1 for a
 * root); moments are 13 doubles per node (M, cx, cy, cz, b_max, B2, delta,
 * side, ox, oy, oz, r_b, 0). keys (uint64) are in sorted order. */
hybrid_status hybrid_tree_info(hybrid_ctx *ctx, int64_t *n_nodes, int64_t *n_groups);
hybrid_status hybrid_tree_copy(hybrid_ctx *ctx, uint64_t *keys, int32_t *level, int64_t *first, int64_t *count,
                               int64_t *child, int32_t *nchild, int64_t *parent, double *moments,
                               int64_t *group_node, double *group_lo, double *group_hi);

/* Interaction lists of the last force walk, host copies. mode bit 0: the
 * soft lists (cells, particles), bit 1: the hard list. counts: 3 int64 per
 * group (soft cells, soft particles, hard particles); entries (int64, node or
 * sorted particle index) back to back per group in that order. Pass
 * entries = NULL to get the counts only. */
hybrid_status hybrid_lists_copy(hybrid_ctx *ctx, int64_t *counts, int64_t *entries, int64_t cap_entries);

/* Sink-source pairs (sum over groups of |group| x list length) of the last
 * force evaluation: far = pairs with K = 0 for certain (taken cells and far
 * particles, soft force only); near = near-particle pairs (soft force with
 * weight 1 - K and hard force with weight K). The soft force sums far + near
 * pairs, the hard force the near pairs. */
hybrid_status hybrid_interactions(hybrid_ctx *ctx, int64_t *far, int64_t *near);

/* Profiling: enable = 1 brackets the pair kernels (kinds 0 and 1) with CUDA
 * events on the context stream, enable = 2 every stage; 0 turns it off. In a
 * replayed CUDA graph the brackets are event-record nodes of the graph. The
 * tree-build parts run on two branches (topology and groups beside the
 * permutation and the moments), so kinds 5-8 can overlap. hybrid_profile_read
 * synchronises and returns, per kind (0 far pair kernel, 1 near pair kernel,
 * 2 walk, 3 tree build, 4 kick/drift, 5 key sort, 6 tree topology, 7 moments,
 * 8 groups; 5-8 are parts of 3), the summed milliseconds and number of
 * brackets since the last reset. */
hybrid_status hybrid_profile(hybrid_ctx *ctx, int enable);
hybrid_status hybrid_profile_read(hybrid_ctx *ctx, int kind, double *ms, int64_t *launches, int reset);

/* Number of kernels this context has launched so far (all kinds). */
int64_t hybrid_launch_count(hybrid_ctx *ctx);

/* Number of tree builds this context has repeated with the radix sort. The
 * key sort of Sec. III-A1 is first tried as a sample sort, which assumes the
 * state is close to key order (as it is from one build to the next: the state
 * stays in key order and moves by one drift); when a bucket overflows, the
 * build leaves the order unchanged and is repeated with the radix sort. Both
 * give the same stable order. A diagnostic; not part of the method. */
int64_t hybrid_sort_fallbacks(hybrid_ctx *ctx);

/* Softened energies (Sec. IV-A "total energy") of a system by direct
 * summation on the device: kinetic and potential, returned to the host
 * (synchronises). Uses the context's eps and G (or sys->params). */
hybrid_status hybrid_energy(hybrid_ctx *ctx, hybrid_system *sys, double *kinetic, double *potential);

/* ---- serving: continuous batching of independent simulations ----
 *
 * Not part of the method: the paper advances one simulation at a time. A
 * server owns one context (created with p; p->precision selects the form) and
 * serves requests, each an independent system with its own parameters and
 * number of soft steps:
 *  - hybrid_server_submit copies a request's host state (FP64 arrays of
 *    length n) and queues it under the caller's tag (>= 0); ETOOLARGE if
 *    n x HYBRID_SERVER_BYTES_PER_PARTICLE exceeds the budget.
 *  - hybrid_server_step admits queued requests in arrival order while the bytes
 *    charged for the admitted ones (HYBRID_SERVER_BYTES_PER_PARTICLE per
 *    particle: the request's device arrays and its share of the context's
 *    working buffers) stay within budget_bytes; computes the first forces of
 *    the newly admitted requests; advances every admitted request by one soft
 *    step in one batched call (hybrid_step_batched); and retires the requests
 *    whose steps are done (state back to host memory held by the server,
 *    device arrays freed). It synchronises the stream; the counts returned are
 *    those after the step.
 *  - hybrid_server_next reports the oldest finished request: with all seven
 *    arrays NULL it only sets tag and n (tag = -1 when none has finished);
 *    with seven host arrays of length n it copies the final state, in the
 *    request's input order, and forgets the request.
 * A request's result does not depend on the other requests: bitwise in the
 * FP64 form, to FP32 summation order in the FP32 form. One server is driven
 * by one host thread. */
#define HYBRID_SERVER_BYTES_PER_PARTICLE 1536
typedef struct hybrid_server hybrid_server;
hybrid_status hybrid_server_create(hybrid_server **srv, const hybrid_params *p, double budget_bytes, void *stream);
hybrid_status hybrid_server_destroy(hybrid_server *srv);
hybrid_status hybrid_server_submit(hybrid_server *srv, int64_t tag, int64_t n, const double *x, const double *y,
                                   const double *z, const double *vx, const double *vy, const double *vz,
                                   const double *m, const hybrid_params *params, int32_t n_steps);
hybrid_status hybrid_server_step(hybrid_server *srv, int32_t *n_active, int32_t *n_queued, int32_t *n_finished);
hybrid_status hybrid_server_next(hybrid_server *srv, int64_t *tag, int64_t *n, double *x, double *y, double *z,
                                 double *vx, double *vy, double *vz, double *m);
/* Bytes currently charged for admitted requests; text of the last failure. */
double hybrid_server_used_bytes(hybrid_server *srv);
const char *hybrid_server_last_error(hybrid_server *srv);

/* ---- allocation-free entry point ----
 *
 * The paper has no counterpart to this call: it is an interface addition for
 * callers that cannot allocate device memory (no cudaMalloc/cudaFree or any
 * allocating library call, torch's included) -- code that runs when the
 * device has no free memory left (an out-of-memory handler, a process whose
 * caching allocator holds the whole device) or a latency-sensitive loop that
 * must not pay the implicit device synchronisation of cudaFree. Every other
 * call here allocates through its context, so they cannot use those.
 *
 * hybrid_energy_noalloc computes what hybrid_energy does -- softened kinetic
 * and potential energy by direct FP64 summation (Sec. IV-A total energy,
 * potential of Eq. 2 with eps) -- for one system of n particles given as
 * caller-owned DEVICE arrays (FP64, length n, any order), with G and eps
 * passed directly and no context. Results are written to the two HOST
 * doubles; the call enqueues two kernels and one 16-byte device-to-host copy
 * on `stream` (a cudaStream_t; NULL = legacy default stream) and synchronises
 * that stream before returning.
 *
 * Scratch is a fixed device array inside the library, sized for
 * n <= HYBRID_ENERGY_NOALLOC_MAX_N (256 KB of FP64 partial sums); larger n returns
 * HYBRID_ETOOLARGE before anything is enqueued. Its address is looked up once
 * per device, on the first call made with that device current, which also
 * loads the call's two kernels (so that a lazily loaded module does not take
 * device memory at a later call): make a first call (n = 0 is enough: it only
 * does this set-up and returns zeros) before any stream capture. The scratch is shared by all calls on a device, so
 * calls that overlap in time (two streams or two host threads) race on it and
 * must be serialised by the caller. Nothing in the scratch has to start at
 * zero: each call writes every slot it reads.
 *
 * Errors: HYBRID_EINVAL (n < 0, eps < 0, a NULL array with n > 0 or a NULL
 * result pointer), HYBRID_ETOOLARGE, HYBRID_ECUDA (a failed launch, copy or
 * look-up). */
#define HYBRID_ENERGY_NOALLOC_MAX_N 4194304
hybrid_status hybrid_energy_noalloc(int64_t n, const double *x, const double *y, const double *z, const double *vx,
                                    const double *vy, const double *vz, const double *m, double G, double eps,
                                    void *stream, double *kinetic, double *potential);

#ifdef __cplusplus
}
#endif

#endif /* HYBRID_H */
