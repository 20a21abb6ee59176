// tree.cu -- octree construction on the device (Sec. III-A1 of the paper,
// done on the GPU instead of the host): root cube, Morton keys, a stable LSD
// radix sort of the keys with the particle data gathered into key order, a
// level-wise split (a cell with more than n_leaf particles splits into its
// non-empty octants), cell moments (Sec. II-B: mass, centre of mass; Eq. 5-6:
// b_max, B2, MAC radius) and the sink groups.
//
// All systems of a batch are processed by the same launches; every node,
// particle range and radix tile stays inside one system.
#include "hy_internal.cuh"

#include <cuda/atomic>
#include <cstdio>
#include <type_traits>

namespace hy {

namespace {

__device__ __forceinline__ void fail(Status *st, int code, int where)
{
    // the first failure wins and keeps its op index: later kernels of the same sequence may fail too (a build
    // after an unsorted one), and the sequence resumes at the first
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

// order-preserving map of doubles to unsigned integers (for atomic min/max)
__device__ __forceinline__ unsigned long long ord_dbl(double v)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord_dbl(unsigned long long u)
{
    return __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
}

// ---------------------------------------------------------------------------
// Root cube: per-axis minimum lo; side L = smallest power of two >= the
// largest extent (1 when all particles coincide); scale = 2^21 / L.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_box(const double *__restrict__ x, const double *__restrict__ y,
                                             const double *__restrict__ z, const Chunk *__restrict__ chunks,
                                             int nchunks, unsigned long long *bmin, unsigned long long *bmax,
                                             const Status *st)
{
    (void)st;   // the sort always runs: later kernels rely on a consistent permutation
    // min/max of the order-preserving integer images: exact, and no FP64 pipe work
    __shared__ unsigned long long sh[6][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const Chunk ch = chunks[c];
        unsigned long long v[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
        for (int i = threadIdx.x; i < ch.len; i += blockDim.x) {
            const int64_t k = ch.start + i;
            const unsigned long long p0 = ord_dbl(x[k]), p1 = ord_dbl(y[k]), p2 = ord_dbl(z[k]);
            v[0] = min(v[0], p0);
            v[1] = min(v[1], p1);
            v[2] = min(v[2], p2);
            v[3] = max(v[3], p0);
            v[4] = max(v[4], p1);
            v[5] = max(v[5], p2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int j = 0; j < 3; ++j) v[j] = min(v[j], __shfl_xor_sync(0xffffffffu, v[j], o));
#pragma unroll
            for (int j = 3; j < 6; ++j) v[j] = max(v[j], __shfl_xor_sync(0xffffffffu, v[j], o));
        }
        if (lane == 0)
            for (int j = 0; j < 6; ++j) sh[j][w] = v[j];
        __syncthreads();
        if (threadIdx.x < 6) {
            const int j = threadIdx.x;
            unsigned long long r = sh[j][0];
            for (int k = 1; k < 8; ++k) r = (j < 3) ? min(r, sh[j][k]) : max(r, sh[j][k]);
            if (j < 3) atomicMin(&bmin[3 * ch.sys + j], r);
            else atomicMax(&bmax[3 * ch.sys + j - 3], r);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ SysBox make_box(const unsigned long long *bmin, const unsigned long long *bmax, int s)
{
    double lo[3], ext = 0.0;
    for (int d = 0; d < 3; ++d) {
        lo[d] = unord_dbl(bmin[3 * s + d]);
        const double e = __dsub_rn(unord_dbl(bmax[3 * s + d]), lo[d]);
        if (e > ext) ext = e;
    }
    double L = 1.0;
    if (ext > 0.0) {
        int e2;
        const double f = frexp(ext, &e2);
        L = (f == 0.5) ? ext : ldexp(1.0, e2);
    }
    SysBox b;
    b.lo[0] = lo[0];
    b.lo[1] = lo[1];
    b.lo[2] = lo[2];
    b.L = L;
    b.scale = ldexp(1.0, LEVELS) / L;   // ratio of powers of two: exact
    b.u = ldexp(L, -20);
    b.inv_u = ldexp(1.0, 20) / L;
    b.uf = (float)b.u;
    b.inv_uf = (float)b.inv_u;
    return b;
}

// ---------------------------------------------------------------------------
// Morton keys: q = clamp(floor((x - lo) * scale), 0, 2^21 - 1) per axis, bits
// interleaved from the top, x first. Only the subtraction rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// d = p - lo rounds once (FP64); the scale is a power of two 2^s, so
// floor(d 2^s) is taken from the bits of d (d = m 2^e with an integer m):
// m shifted by e + s, which keeps the FP64 pipe to one operation per axis.
__device__ __forceinline__ uint32_t cell_coord(double p, double lo, int s)
{
    const double d = __dsub_rn(p, lo);
    if (!(d > 0.0)) return 0u;   // zero, or below the root corner
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const int E = (int)((bits >> 52) & 0x7ffu);
    const unsigned long long frac = bits & ((1ull << 52) - 1ull);
    const unsigned long long m = E ? (frac | (1ull << 52)) : frac;
    const int sh = (E ? E : 1) - 1075 + s;   // d 2^s = m 2^sh
    constexpr unsigned long long QMAX = (1ull << LEVELS) - 1ull;
    unsigned long long q;
    if (sh >= 0) q = sh >= 11 ? QMAX : min(m << sh, QMAX);   // m >= 2^52 when normal: past the clamp
    else q = -sh >= 64 ? 0ull : (m >> -sh);
    return (uint32_t)min(q, QMAX);
}

// exponent s of a scale that is an exact power of two (normal)
__device__ __forceinline__ int pow2_exponent(double scale)
{
    return (int)(((unsigned long long)__double_as_longlong(scale) >> 52) & 0x7ffu) - 1023;
}

// Also finishes the root cubes (from the atomic min/max) and stores them.
__global__ void __launch_bounds__(256) k_keys(int64_t N, const double *__restrict__ x, const double *__restrict__ y,
                                              const double *__restrict__ z, const int32_t *__restrict__ psys, int S,
                                              const unsigned long long *__restrict__ bmin,
                                              const unsigned long long *__restrict__ bmax, SysBox *__restrict__ boxout,
                                              uint64_t *__restrict__ key, uint32_t *__restrict__ val, const Status *st)
{
    if (blockIdx.x == 0)
        for (int s = threadIdx.x; s < S; s += blockDim.x) boxout[s] = make_box(bmin, bmax, s);
    __shared__ SysBox b1;   // single-system batches: the cube computed once per block
    if (S == 1) {
        if (threadIdx.x == 0) b1 = make_box(bmin, bmax, 0);
        __syncthreads();
    }
    (void)st;   // the sort always runs: later kernels rely on a consistent permutation
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const SysBox b = S == 1 ? b1 : make_box(bmin, bmax, psys[i]);
        const int es = pow2_exponent(b.scale);
        const uint32_t qx = cell_coord(x[i], b.lo[0], es);
        const uint32_t qy = cell_coord(y[i], b.lo[1], es);
        const uint32_t qz = cell_coord(z[i], b.lo[2], es);
        key[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
        val[i] = (uint32_t)i;
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits, one launch per digit.
// k_digit_counts counts, per system, the digits of all eight passes. Pass p
// runs k_onesweep: tiles (chunks of at most ctx->tile keys inside one system)
// are claimed in order from a ticket counter; a tile ranks its keys (stable:
// warp-striped input order), publishes its per-digit counts, then adds up
// the counts of the earlier tiles of its system by reading their published
// words backwards until it meets an inclusive prefix (a chained scan with
// look-back), and publishes its own inclusive prefix. A key's destination is
// the system's start + the system's count of smaller digits + the earlier
// tiles' count of its digit + its rank in the tile; the tile is reordered in
// shared memory by (digit, rank) first, so that consecutive threads write
// consecutive addresses of one digit's run. Tiles only wait on tiles
// with smaller tickets, which were claimed by running blocks and publish
// their counts before they wait on anything; every wait is bounded.
// ---------------------------------------------------------------------------
constexpr uint32_t LB_AGG = 1u << 30, LB_INC = 2u << 30, LB_CNT = (1u << 30) - 1u;
constexpr int LB_SPIN_MAX = 1 << 22;
// sort scratch layout (u32): [0, 64) tickets, then counts[S][8][256], then look[8][nchunks][256]
constexpr int RS_HDR = 64;

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Polls *q until one of the flag bits is set, at most max_polls times with a
// short sleep in between; when the polls run out it records HYBRID_ETIMEOUT in
// the status block and returns dflt, so the caller finishes without waiting.
__device__ __forceinline__ uint32_t wait_flagged(const uint32_t *q, uint32_t flags, int max_polls, Status *st,
                                                 uint32_t dflt)
{
    uint32_t v = ld_relaxed_u32(q);
    for (int spins = 0; (v & flags) == 0u; ++spins) {
        if (spins >= max_polls) {
            fail(st, HYBRID_ETIMEOUT, -1);
            return dflt;
        }
        __nanosleep(64);
        v = ld_relaxed_u32(q);
    }
    return v;
}

// Self-test of the bounded wait: one thread waits for a flag that nothing sets.
__global__ void k_wait_selftest(const uint32_t *word, int max_polls, Status *st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)wait_flagged(word, 1u, max_polls, st, 0u);
}

__global__ void __launch_bounds__(256) k_digit_counts(const uint64_t *__restrict__ key, const Chunk *__restrict__ chunks,
                                                      int nchunks, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t h[8][256];
    const int lane = threadIdx.x & 31;
    const unsigned ltmask = (1u << lane) - 1u;
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const Chunk ch = chunks[c];
        for (int t = threadIdx.x; t < 8 * 256; t += blockDim.x) (&h[0][0])[t] = 0;
        __syncthreads();
        for (int i0 = 0; i0 < ch.len; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            const bool ok = i < ch.len;
            const uint64_t k = ok ? key[ch.start + i] : 0ull;
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const uint32_t d = ok ? (uint32_t)(k >> (8 * p)) & 0xffu : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                if (ok && (peers & ltmask) == 0u) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        uint32_t *dst = counts + (size_t)ch.sys * 2048;
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
            const uint32_t v = (&h[0][0])[t];
            if (v) atomicAdd(dst + t, v);
        }
        __syncthreads();
    }
}

template <int IPT>
__global__ void __launch_bounds__(256) k_onesweep(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                  uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                  const Chunk *__restrict__ chunks, int nchunks, int pass,
                                                  const uint32_t *__restrict__ counts, uint32_t *look,
                                                  uint32_t *ticket, int64_t ntotal, Status *st)
{
    // the sort always runs (later kernels rely on a consistent permutation); st only records a timeout
    constexpr int TILE_K = RS_WARPS * 32 * IPT;
    __shared__ uint32_t whist[RS_WARPS][256];
    __shared__ uint32_t base[256];    // global position of the tile's first key of digit d
    __shared__ uint32_t tloc[256];    // position in the tile's sorted order of its first key of digit d
    __shared__ uint64_t wsum[RS_WARPS];
    __shared__ uint64_t skey[TILE_K];
    __shared__ uint32_t sval[TILE_K];
    __shared__ int cid;
    const int shift = 8 * pass;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned ltmask = (1u << lane) - 1u;
    for (;;) {
        if (threadIdx.x == 0) cid = (int)atomicAdd(ticket, 1u);
        for (int t = threadIdx.x; t < RS_WARPS * 256; t += blockDim.x) (&whist[0][0])[t] = 0;
        __syncthreads();
        const int c = cid;
        if (c >= nchunks) break;
        const Chunk ch = chunks[c];
        uint64_t k[IPT];
        uint32_t v[IPT], r[IPT];
        const int wbase = w * 32 * IPT;
#pragma unroll
        for (int it = 0; it < IPT; ++it) {   // every load in flight before the ranking starts
            const int li = wbase + it * 32 + lane;   // warp-striped: (it, lane) is input order
            const bool ok = li < ch.len;
            k[it] = ok ? kin[ch.start + li] : 0ull;
            v[it] = ok ? vin[ch.start + li] : 0u;
        }
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            const int li = wbase + it * 32 + lane;
            const bool ok = li < ch.len;
            const uint32_t d = ok ? (uint32_t)(k[it] >> shift) & 0xffu : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = ok ? whist[w][d] : 0u;
            __syncwarp();
            if (ok && (peers & ltmask) == 0u) whist[w][d] = before + (uint32_t)__popc(peers);
            __syncwarp();
            r[it] = before + (uint32_t)__popc(peers & ltmask);
        }
        __syncthreads();
        const int d = threadIdx.x;
        // loads that do not depend on the look-back go out before it
        const uint32_t cd = counts[(size_t)ch.sys * 2048 + pass * 256 + d];
        const int64_t s0 = chunks[ch.first_chunk].start;
        uint32_t run = 0;   // tile count of digit d; whist becomes the exclusive prefix over the warps
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            const uint32_t cnt = whist[ww][d];
            whist[ww][d] = run;
            run += cnt;
        }
        uint32_t *mine = look + (size_t)c * 256 + d;
        const bool first = (c == ch.first_chunk);
        st_relaxed_u32(mine, (first ? LB_INC : LB_AGG) | run);
        uint32_t excl = 0;
        if (!first) {
            for (int j = c - 1; j >= ch.first_chunk; --j) {
                const uint32_t *q = look + (size_t)j * 256 + d;
                const uint32_t vq = wait_flagged(q, LB_AGG | LB_INC, LB_SPIN_MAX, st, LB_INC);
                excl += vq & LB_CNT;
                if (vq & LB_INC) break;
            }
            st_relaxed_u32(mine, LB_INC | (excl + run));
        }
        // exclusive prefixes over digits, in one block scan: the system's counts (high 32 bits) and the
        // tile's counts (low 32 bits; at most 2048, so no carry crosses over)
        const uint64_t both = ((uint64_t)cd << 32) | run;
        uint64_t incl = both;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        uint64_t wpre = 0;
        for (int ww = 0; ww < w; ++ww) wpre += wsum[ww];
        const uint64_t ex = wpre + incl - both;
        tloc[d] = (uint32_t)ex;
        base[d] = (uint32_t)(ex >> 32) + excl;
        __syncthreads();
        // reorder the tile in shared memory by (digit, rank), then write runs of equal digits
        // with consecutive threads on consecutive addresses
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            const int li = wbase + it * 32 + lane;
            if (li < ch.len) {
                const uint32_t dd = (uint32_t)(k[it] >> shift) & 0xffu;
                const uint32_t lp = tloc[dd] + whist[w][dd] + r[it];
                skey[lp] = k[it];
                sval[lp] = v[it];
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < IPT; ++it) {
            const int lp = it * 256 + threadIdx.x;
            if (lp < ch.len) {
                const uint64_t kk = skey[lp];
                const uint32_t dd = (uint32_t)(kk >> shift) & 0xffu;
                const int64_t dst = s0 + (int64_t)(base[dd] + ((uint32_t)lp - tloc[dd]));
                if (dst < ntotal) {   // always true unless a look-back timed out (recorded in st)
                    kout[dst] = kk;
                    vout[dst] = sval[lp];
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Sample sort of the keys, for a state that is close to key order (the state
// stays in the order of the last build and moves by one drift in between).
// The stable order is the order of the composite (key, current index), so
// per system: nb - 1 non-decreasing splitters are taken from the last
// build's sorted keys at regular positions (k_ss_split); each key goes to the
// bucket of the number of splitters at or below its composite; buckets are laid out back to back
// (counts, then a scan) and each is sorted by composite in shared memory by
// one block. Keys end sorted in keys[0] with their source positions in
// vals[0], exactly as the radix sort leaves them. A bucket of more than
// SS_CAP keys (a state far from key order) makes the build leave the order
// unchanged and record ST_SORT; the build is then repeated with the radix
// sort.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool comp_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb)
{
    return ka < kb || (ka == kb && va < vb);
}

// Block-wide stable LSD radix sort of n keys (with their positions) in shared
// memory, over the key bits that differ between the smallest and the largest
// key, 8 bits per pass; equal keys are then put in order of their positions
// (ties are rare: particles in one cell of the finest level). blockDim.x =
// SSB_THREADS; whist holds SSB_WARPS x 256 counters; n <= SSB_THREADS * EPT.
constexpr int SSB_THREADS = 512, SSB_WARPS = SSB_THREADS / 32;

template <int EPT>
__device__ __forceinline__ void block_radix_sort(uint64_t *sk, uint32_t *sv, int n, uint32_t (*whist)[256],
                                                 uint32_t *tloc, uint64_t *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned ltmask = (1u << lane) - 1u;
    // the bits that vary: highest set bit of (min key ^ max key)
    uint64_t mn = ~0ull, mx = 0ull;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        mn = min(mn, sk[j]);
        mx = max(mx, sk[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        red[w] = mn;
        red[SSB_WARPS + w] = mx;
    }
    __syncthreads();
    mn = red[0];
    mx = red[SSB_WARPS];
    for (int k = 1; k < SSB_WARPS; ++k) {
        mn = min(mn, red[k]);
        mx = max(mx, red[SSB_WARPS + k]);
    }
    const int vbits = (mn == mx) ? 0 : 64 - __clzll((long long)(mn ^ mx));
    const int E = (n + SSB_THREADS - 1) / SSB_THREADS;   // slots per thread: every warp holds a share of the keys
    const int wbase = w * 32 * E;
    for (int shift = 0; shift < vbits; shift += 8) {
        uint64_t k[EPT];
        uint32_t v[EPT], r[EPT], d[EPT];
        for (int t = threadIdx.x; t < SSB_WARPS * 256; t += blockDim.x) (&whist[0][0])[t] = 0u;
#pragma unroll
        for (int it = 0; it < EPT; ++it) {   // warp-striped: (warp, it, lane) is the current order
            const int e = wbase + it * 32 + lane;
            const bool ok = it < E && e < n;
            k[it] = ok ? sk[e] : 0ull;
            v[it] = ok ? sv[e] : 0u;
            d[it] = ok ? (uint32_t)(k[it] >> shift) & 0xffu : 256u;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < EPT; ++it) {
            if (it >= E || wbase + it * 32 >= n) break;   // the rest of this warp's slots are empty
            const unsigned peers = __match_any_sync(0xffffffffu, d[it]);
            const uint32_t before = d[it] < 256u ? whist[w][d[it]] : 0u;
            __syncwarp();
            if (d[it] < 256u && (peers & ltmask) == 0u) whist[w][d[it]] = before + (uint32_t)__popc(peers);
            __syncwarp();
            r[it] = before + (uint32_t)__popc(peers & ltmask);
        }
        __syncthreads();
        if (threadIdx.x < 256) {   // per digit: exclusive prefix over the warps, then over the digits
            const int dd = threadIdx.x;
            uint32_t run = 0;
            for (int ww = 0; ww < SSB_WARPS; ++ww) {
                const uint32_t c = whist[ww][dd];
                whist[ww][dd] = run;
                run += c;
            }
            uint32_t inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) red[w] = inc;   // the 8 digit warps' totals (red is free here)
            tloc[dd] = inc - run;
        }
        __syncthreads();
        if (threadIdx.x < 256) {
            uint32_t pre = 0;
            for (int ww = 0; ww < w; ++ww) pre += (uint32_t)red[ww];
            tloc[threadIdx.x] += pre;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < EPT; ++it)
            if (d[it] < 256u) {
                const uint32_t pos = tloc[d[it]] + whist[w][d[it]] + r[it];
                sk[pos] = k[it];
                sv[pos] = v[it];
            }
        __syncthreads();
    }
    // runs of equal keys: in order of their positions (insertion sort by the run's first thread)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (j + 1 < n && sk[j + 1] == sk[j] && (j == 0 || sk[j - 1] != sk[j])) {
            int e = j + 1;
            while (e < n && sk[e] == sk[j]) ++e;
            for (int a = j + 1; a < e; ++a) {
                const uint32_t x = sv[a];
                int b = a - 1;
                while (b >= j && sv[b] > x) {
                    sv[b + 1] = sv[b];
                    --b;
                }
                sv[b + 1] = x;
            }
        }
    }
    __syncthreads();
}

// One block per system: its nb - 1 splitters and cleared bucket counts. It
// runs before the new keys are computed, on the keys of the last build: the
// state is still in that build's order and its sorted keys are still in the
// key buffer, so the composite (old key, position) at position j n / nb is the
// j-th nb-quantile of the last build, and the particles have moved little
// since. A running maximum over j makes the splitters non-decreasing whatever
// the buffer holds (another batch, a first build): buckets may then be empty
// or large, and a large one sends the build to the radix sort.
__device__ __forceinline__ void comp_max(uint64_t &k, uint32_t &v, uint64_t k2, uint32_t v2)
{
    if (comp_less(k, v, k2, v2)) {
        k = k2;
        v = v2;
    }
}

__global__ void __launch_bounds__(SSB_THREADS) k_ss_split(const uint64_t *__restrict__ key,
                                                          const int64_t *__restrict__ off, const SSys *__restrict__ ss,
                                                          int S, uint64_t *__restrict__ spk, uint32_t *__restrict__ spv,
                                                          uint32_t *__restrict__ cnt)
{
    __shared__ uint64_t wk[SSB_WARPS];
    __shared__ uint32_t wv[SSB_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int s = blockIdx.x; s < S; s += gridDim.x) {
        const SSys y = ss[s];
        const int64_t o = off[s], n = off[s + 1] - off[s];
        for (int b = threadIdx.x; b < y.nb; b += blockDim.x) cnt[y.bbase + b] = 0u;
        const int m = y.nb - 1;   // splitters
        if (m > 0) {
            // thread t takes candidates [t per, (t + 1) per) and keeps their running maximum
            const int per = (m + blockDim.x - 1) / blockDim.x;
            const int j0 = threadIdx.x * per, j1 = min(m, j0 + per);
            uint64_t rk = 0ull;
            uint32_t rv = 0u;
            for (int j = j0; j < j1; ++j) {
                const int64_t p = o + ((int64_t)(j + 1) * n) / y.nb;   // 1 <= p - o <= n - 1
                const uint64_t mk = key[p];
                const uint32_t mv = (uint32_t)p;
                if (j == j0) {
                    rk = mk;
                    rv = mv;
                } else {
                    comp_max(rk, rv, mk, mv);
                }
                spk[y.bbase + j] = rk;
                spv[y.bbase + j] = rv;
            }
            // exclusive running maximum of the threads' maxima (empty ranges carry the zero composite)
            uint64_t ik = rk;
            uint32_t iv = rv;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const uint64_t k2 = __shfl_up_sync(0xffffffffu, ik, o2);
                const uint32_t v2 = __shfl_up_sync(0xffffffffu, iv, o2);
                if (lane >= o2) comp_max(ik, iv, k2, v2);
            }
            if (lane == 31) {
                wk[w] = ik;
                wv[w] = iv;
            }
            __syncthreads();
            uint64_t pk = 0ull;
            uint32_t pv = 0u;
            for (int ww = 0; ww < w; ++ww) comp_max(pk, pv, wk[ww], wv[ww]);
            {
                const uint64_t k2 = __shfl_up_sync(0xffffffffu, ik, 1);
                const uint32_t v2 = __shfl_up_sync(0xffffffffu, iv, 1);
                if (lane >= 1) comp_max(pk, pv, k2, v2);
            }
            for (int j = j0; j < j1; ++j) {   // apply the maximum of everything before this thread's range
                uint64_t k2 = spk[y.bbase + j];
                uint32_t v2 = spv[y.bbase + j];
                comp_max(k2, v2, pk, pv);
                spk[y.bbase + j] = k2;
                spv[y.bbase + j] = v2;
            }
        }
        __syncthreads();
    }
}

// The sample sort's keys: the key of every particle as k_keys, its bucket (the
// number of its system's splitters, taken before the keys were replaced, at
// or below its composite (key, position)), and the bucket counts.
__global__ void __launch_bounds__(256) k_keys_count(int64_t N, const double *__restrict__ x,
                                                    const double *__restrict__ y, const double *__restrict__ z,
                                                    const int32_t *__restrict__ psys, int S,
                                                    const unsigned long long *__restrict__ bmin,
                                                    const unsigned long long *__restrict__ bmax,
                                                    SysBox *__restrict__ boxout, uint64_t *__restrict__ key,
                                                    uint32_t *__restrict__ val, const SSys *__restrict__ ss,
                                                    const uint64_t *__restrict__ spk, const uint32_t *__restrict__ spv,
                                                    uint32_t *__restrict__ pb, uint32_t *__restrict__ cnt)
{
    if (blockIdx.x == 0)
        for (int s = threadIdx.x; s < S; s += blockDim.x) boxout[s] = make_box(bmin, bmax, s);
    __shared__ SysBox b1;   // single-system batches: the cube computed once per block
    if (S == 1) {
        if (threadIdx.x == 0) b1 = make_box(bmin, bmax, 0);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < N; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        uint32_t b = ~0u;
        if (i < N) {
            const int sy = S == 1 ? 0 : psys[i];
            const SysBox bx = S == 1 ? b1 : make_box(bmin, bmax, sy);
            const int es = pow2_exponent(bx.scale);
            const uint32_t qx = cell_coord(x[i], bx.lo[0], es);
            const uint32_t qy = cell_coord(y[i], bx.lo[1], es);
            const uint32_t qz = cell_coord(z[i], bx.lo[2], es);
            const uint64_t k = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
            key[i] = k;
            val[i] = (uint32_t)i;
            const SSys yy = ss[sy];
            int lo = 0, hi = yy.nb - 1;   // upper bound over the splitters [0, nb - 1)
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (comp_less(k, (uint32_t)i, spk[yy.bbase + mid], spv[yy.bbase + mid])) hi = mid;
                else lo = mid + 1;
            }
            b = (uint32_t)(yy.bbase + lo);
            pb[i] = b;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        if (b != ~0u && lane == __ffs(peers) - 1) atomicAdd(cnt + b, (uint32_t)__popc(peers));
    }
}

// One block per system: bucket starts (exclusive scan of the counts from the
// system's first position) and the overflow check.
__global__ void __launch_bounds__(256) k_ss_scan(const int64_t *__restrict__ off, const SSys *__restrict__ ss, int S,
                                                 const uint32_t *__restrict__ cnt, uint32_t *__restrict__ start,
                                                 uint32_t *__restrict__ cur, uint32_t *flag, Status *st, int where)
{
    __shared__ uint32_t part[256];
    for (int s = blockIdx.x; s < S; s += gridDim.x) {
        const SSys y = ss[s];
        const int per = (y.nb + blockDim.x - 1) / blockDim.x;
        const int b0 = threadIdx.x * per, b1 = min(y.nb, b0 + per);
        uint32_t sum = 0, mx = 0;
        for (int b = b0; b < b1; ++b) {
            const uint32_t v = cnt[y.bbase + b];
            sum += v;
            mx = max(mx, v);
        }
        part[threadIdx.x] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t run = (uint32_t)off[s];
            for (int t = 0; t < (int)blockDim.x; ++t) {
                const uint32_t v = part[t];
                part[t] = run;
                run += v;
            }
        }
        __syncthreads();
        uint32_t run = part[threadIdx.x];
        for (int b = b0; b < b1; ++b) {
            start[y.bbase + b] = run;
            cur[y.bbase + b] = 0u;
            run += cnt[y.bbase + b];
        }
        if (mx > (uint32_t)SS_CAP) {
            atomicExch(flag, 1u);
            fail(st, ST_SORT, where);
        }
        __syncthreads();
    }
}

// Every key and its position into its bucket's range (any order inside).
__global__ void __launch_bounds__(256) k_ss_scatter(int64_t N, const uint64_t *__restrict__ k0,
                                                    const uint32_t *__restrict__ pb, const uint32_t *__restrict__ start,
                                                    uint32_t *__restrict__ cur, uint64_t *__restrict__ k1,
                                                    uint32_t *__restrict__ v1, const uint32_t *flag)
{
    if (*flag) return;
    const int lane = threadIdx.x & 31;
    const unsigned ltmask = (1u << lane) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < N; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const uint32_t b = i < N ? pb[i] : ~0u;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (b != ~0u && lane == leader) base = atomicAdd(cur + b, (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b != ~0u) {
            const uint32_t pos = start[b] + base + (uint32_t)__popc(peers & ltmask);
            k1[pos] = k0[i];
            v1[pos] = (uint32_t)i;
        }
    }
}

// One block per bucket: its keys sorted by composite in shared memory, written
// to their final positions.
__global__ void __launch_bounds__(SSB_THREADS, 2) k_ss_sort(int nbk, const uint32_t *__restrict__ cnt,
                                                         const uint32_t *__restrict__ start,
                                                         const uint64_t *__restrict__ k1, const uint32_t *__restrict__ v1,
                                                         uint64_t *__restrict__ k0, uint32_t *__restrict__ v0,
                                                         const uint32_t *flag)
{
    extern __shared__ uint64_t ss_smem[];   // SS_CAP keys, then SS_CAP positions
    __shared__ uint32_t whist[SSB_WARPS][256];
    __shared__ uint32_t tloc[256];
    __shared__ uint64_t red[2 * SSB_WARPS];
    uint64_t *sk = ss_smem;
    uint32_t *sv = reinterpret_cast<uint32_t *>(ss_smem + SS_CAP);
    if (*flag) return;
    for (int b = blockIdx.x; b < nbk; b += gridDim.x) {
        const int n = (int)cnt[b];
        const uint32_t s0 = start[b];
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            sk[j] = k1[s0 + j];
            sv[j] = v1[s0 + j];
        }
        __syncthreads();
        block_radix_sort<SS_CAP / SSB_THREADS>(sk, sv, n, whist, tloc, red);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            k0[s0 + j] = sk[j];
            v0[s0 + j] = sv[j];
        }
        __syncthreads();
    }
}

// Gather of the state into key order; also writes the pair-kernel copies of
// the positions: FP32 hi/lo split (x = hi + lo to ~2^-48) or FP64 double4_32a.
struct PermArgs {
    const double *xin[7];
    double *xout[7];
    const int32_t *id_in;
    int32_t *id_out;
    const int32_t *orig_in;
    int32_t *orig_out;
    const uint32_t *src;
    float4 *phi, *plo;
    double4_32a *pd;
    float *disp;          // zeroed: distance moved since this build (reused lists), or null
    const int32_t *psys;
    const SysBox *box;
    int64_t N;
};

__global__ void __launch_bounds__(256) k_permute(PermArgs a, const Status *st)
{
    (void)st;   // the sort always runs: later kernels rely on a consistent permutation
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = a.src[i];
        double v[7];
#pragma unroll
        for (int f = 0; f < 7; ++f) {
            v[f] = a.xin[f][j];
            a.xout[f][i] = v[f];
        }
        if (a.id_in) a.id_out[i] = a.id_in[j];
        a.orig_out[i] = a.orig_in[j];
        if (a.phi) {
            const SysBox b = a.box[a.psys[i]];
            float h[3], l[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) grid_split(v[d], b.lo[d], b, h[d], l[d]);
            a.phi[i] = make_float4(h[0], h[1], h[2], (float)v[6]);
            a.plo[i] = make_float4(l[0], l[1], l[2], 0.0f);
        }
        if (a.pd) a.pd[i] = make_double4_32a(v[0], v[1], v[2], v[6]);
        if (a.disp) a.disp[i] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Octree topology from the sorted keys, all levels at once.
//
// c(i) = number of leading octal digits keys i-1 and i share (-1 at the first
// particle of a system): particle i starts a cell at every level l > c(i).
// The level-l cell around particle p spans positions up to the nearest
// starts on either side, so its size is known from c in a window of n_leaf
// positions whenever it is at most n_leaf. The leaf depth D(p) is the first
// level whose cell holds <= n_leaf particles (21 at most): cells exist down to
// D(p). Particle i therefore owns the nodes (l, first = i) for
// c(i) < l <= D(i). These records are written in particle order (a scan
// gives each particle its slot), then stably sorted by level: the result is
// the breadth-first order (level, system, key) of the split rule.
// ---------------------------------------------------------------------------
// c(i): common leading octal digits of keys i-1 and i; -1 at a system's first particle
__device__ __forceinline__ int prefix_c(const uint64_t *__restrict__ key, const int32_t *__restrict__ psys, int64_t i)
{
    if (i == 0 || psys[i] != psys[i - 1]) return -1;
    const unsigned long long x = key[i - 1] ^ key[i];
    return x == 0ull ? LEVELS : (__clzll((long long)x) - 1) / 3;   // keys use bits 0..62
}

constexpr int LD_T = 256;

// Leaf depth D(p) and the number of nodes particle p starts, max(0, D - c).
__global__ void __launch_bounds__(LD_T) k_leaf_depth(int64_t N, const uint64_t *__restrict__ key,
                                                     const int32_t *__restrict__ psys, int8_t *__restrict__ pc,
                                                     int n_leaf, uint8_t *__restrict__ pD, uint32_t *__restrict__ pn,
                                                     const Status *st)
{
    if (st->code) return;
    extern __shared__ int8_t sc[];   // LD_T + 2 n_leaf values of c
    const int win = LD_T + 2 * n_leaf;
    for (int64_t base = (int64_t)blockIdx.x * LD_T; base < N; base += (int64_t)gridDim.x * LD_T) {
        __syncthreads();
        for (int k = threadIdx.x; k < win; k += blockDim.x) {
            const int64_t j = base - n_leaf + k;
            const int cj = (j < 0 || j >= N) ? -1 : prefix_c(key, psys, j);
            sc[k] = (int8_t)cj;
            if (k >= n_leaf && k < n_leaf + LD_T && j < N) pc[j] = (int8_t)cj;
        }
        __syncthreads();
        const int64_t p = base + threadIdx.x;
        if (p < N) {
            const int w = threadIdx.x + n_leaf;
            // size of the level-lev cell around p, capped at n_leaf + 1 on each side
            auto count_at = [&](int lev) {
                int kl = 0;
                while (kl <= n_leaf && sc[w - kl] >= lev) ++kl;
                int kr = 1;
                while (kr <= n_leaf && sc[w + kr] >= lev) ++kr;
                return kl + kr;
            };
            int D;
            if (count_at(LEVELS) > n_leaf) {
                D = LEVELS;
            } else {
                int lo = 0, hi = LEVELS;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (count_at(mid) <= n_leaf) hi = mid;
                    else lo = mid + 1;
                }
                D = lo;
            }
            const int c = sc[w];
            pD[p] = (uint8_t)D;
            pn[p] = D > c ? (uint32_t)(D - c) : 0u;
        }
    }
}

// records (level << 32 | first) in particle order
__global__ void __launch_bounds__(256) k_records(int64_t N, const int8_t *__restrict__ pc,
                                                 const uint8_t *__restrict__ pD, const uint32_t *__restrict__ poff,
                                                 const uint64_t *__restrict__ total, int64_t cap,
                                                 unsigned long long *__restrict__ rec, Status *st, int where)
{
    if (st->code) return;
    if ((int64_t)*total > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            fail(st, HYBRID_ECAPACITY, where);
            st->need[0] = (int64_t)*total + (int64_t)(*total >> 3) + 1024;
        }
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = pc[i], D = pD[i];
        uint32_t o = poff[i];
        for (int l = c + 1; l <= D; ++l) rec[o++] = ((unsigned long long)l << 32) | (unsigned long long)i;
    }
}

constexpr int REC_IPT = 4;
constexpr int REC_TILE = RS_WARPS * 32 * REC_IPT;   // 1024 records per tile
constexpr int NLEV = LEVELS + 1;    // levels 0..21

__global__ void __launch_bounds__(256) k_rec_hist(const unsigned long long *__restrict__ rec,
                                                  const uint64_t *__restrict__ total, int ntiles,
                                                  uint32_t *__restrict__ hist, const Status *st)
{
    if (st->code) return;
    __shared__ uint32_t h[NLEV];
    const uint64_t T = *total;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (threadIdx.x < NLEV) h[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t b0 = (uint64_t)t * REC_TILE;
        for (int k = threadIdx.x; k < REC_TILE; k += blockDim.x)
            if (b0 + k < T) atomicAdd(&h[(uint32_t)(rec[b0 + k] >> 32)], 1u);
        __syncthreads();
        if (threadIdx.x < NLEV) hist[(size_t)threadIdx.x * ntiles + t] = h[threadIdx.x];
        __syncthreads();
    }
}

// stable scatter by level; also the level starts lvl[0..23]
__global__ void __launch_bounds__(256) k_rec_scatter(const unsigned long long *__restrict__ rec,
                                                     const uint64_t *__restrict__ total, int ntiles,
                                                     const uint32_t *__restrict__ hoff, uint32_t *__restrict__ bfs2dfs,
                                                     uint32_t *__restrict__ dfs2bfs, uint32_t *__restrict__ lvl,
                                                     const Status *st)
{
    if (st->code) return;
    __shared__ uint32_t whist[RS_WARPS][NLEV];
    __shared__ uint32_t base[NLEV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned ltmask = (1u << lane) - 1u;
    const uint64_t T = *total;
    if (blockIdx.x == 0 && threadIdx.x <= NLEV + 1)
        lvl[threadIdx.x] = threadIdx.x < NLEV ? hoff[(size_t)threadIdx.x * ntiles] : (uint32_t)T;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t b0 = (uint64_t)t * REC_TILE;
        if (b0 >= T) break;
        for (int k = threadIdx.x; k < RS_WARPS * NLEV; k += blockDim.x) (&whist[0][0])[k] = 0;
        if (threadIdx.x < NLEV) base[threadIdx.x] = hoff[(size_t)threadIdx.x * ntiles + t];
        __syncthreads();
        uint32_t lv[REC_IPT], r[REC_IPT];
        const int wbase = w * 32 * REC_IPT;
#pragma unroll
        for (int it = 0; it < REC_IPT; ++it) {
            const uint64_t li = b0 + wbase + it * 32 + lane;
            const bool ok = li < T;
            const uint32_t d = ok ? (uint32_t)(rec[li] >> 32) : 32u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = ok ? whist[w][d] : 0u;
            __syncwarp();
            if (ok && (peers & ltmask) == 0u) whist[w][d] = before + (uint32_t)__popc(peers);
            __syncwarp();
            r[it] = before + (uint32_t)__popc(peers & ltmask);
            lv[it] = d;
        }
        __syncthreads();
        if (threadIdx.x < NLEV) {
            uint32_t run = 0;
            for (int ww = 0; ww < RS_WARPS; ++ww) {
                const uint32_t cnt = whist[ww][threadIdx.x];
                whist[ww][threadIdx.x] = run;
                run += cnt;
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < REC_IPT; ++it) {
            const uint64_t li = b0 + wbase + it * 32 + lane;
            if (li < T) {
                const uint32_t dst = base[lv[it]] + whist[w][lv[it]] + r[it];
                bfs2dfs[dst] = (uint32_t)li;
                dfs2bfs[li] = dst;
            }
        }
        __syncthreads();
    }
}

// per node: level, first, count (end of the key-prefix run, exponential then
// binary search), first child, parent of the roots, system roots
__global__ void __launch_bounds__(256) k_nodes_a(const uint64_t *__restrict__ total,
                                                 const uint32_t *__restrict__ bfs2dfs,
                                                 const uint32_t *__restrict__ dfs2bfs,
                                                 const unsigned long long *__restrict__ rec,
                                                 const uint8_t *__restrict__ pD, const uint64_t *__restrict__ key,
                                                 const int32_t *__restrict__ psys, const int64_t *__restrict__ off,
                                                 uint32_t *nfirst, uint32_t *ncount, uint32_t *nlevel, uint32_t *nchild,
                                                 uint32_t *nparent, uint32_t *sysroot, const Status *st)
{
    if (st->code) return;
    const uint64_t T = *total;
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < T; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = bfs2dfs[b];
        const unsigned long long R = rec[r];
        const int lev = (int)(R >> 32);
        const uint32_t f = (uint32_t)R;
        const int s = psys[f];
        const uint32_t send = (uint32_t)off[s + 1];
        uint32_t end;
        if (lev == 0) {
            end = send;
            nparent[b] = NONE;
            sysroot[s] = (uint32_t)b;
        } else {
            const int sh = 3 * (LEVELS - lev);
            const uint64_t pre = key[f] >> sh;
            uint32_t step = 1, lo = f;   // key[lo] has the prefix
            while (f + step < send && (key[f + step] >> sh) == pre) {
                lo = f + step;
                step <<= 1;
            }
            uint32_t hi = min(f + step, send);   // first index known not to have it (or the end)
            while (hi - lo > 1) {
                const uint32_t mid = lo + ((hi - lo) >> 1);
                if ((key[mid] >> sh) == pre) lo = mid;
                else hi = mid;
            }
            end = hi;
        }
        nfirst[b] = f;
        ncount[b] = end - f;
        nlevel[b] = (uint32_t)lev;
        nchild[b] = (lev < (int)pD[f]) ? dfs2bfs[r + 1] : NONE;
    }
}

// children: the level l+1 nodes that start inside the parent's range
__global__ void __launch_bounds__(256) k_nodes_b(const uint64_t *__restrict__ total, const uint32_t *__restrict__ lvl,
                                                 const uint32_t *__restrict__ nfirst,
                                                 const uint32_t *__restrict__ ncount,
                                                 const uint32_t *__restrict__ nlevel,
                                                 const uint32_t *__restrict__ nchild, uint32_t *nnch,
                                                 uint32_t *nparent, const Status *st)
{
    if (st->code) return;
    const uint64_t T = *total;
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < T; b += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t ch = nchild[b];
        uint32_t k = 0;
        if (ch != NONE) {
            const uint32_t end = nfirst[b] + ncount[b];
            const uint32_t lend = lvl[nlevel[b] + 2];
            while (k < 8 && ch + k < lend && nfirst[ch + k] < end) {
                nparent[ch + k] = (uint32_t)b;
                ++k;
            }
        }
        nnch[b] = k;
    }
}

// ---------------------------------------------------------------------------
// Moments. A cell of at most MOM_CH particles sums its own particle range
// (one warp): M, centre of mass, B2 and b_max, with no wait on other cells.
// A larger cell is combined from its children by the last of them to finish
// (counted with an atomic; no wait anywhere): M = sum M_j, COM = sum M_j
// COM_j / M, B2 = sum_j [B2_j + M_j |COM_j - COM|^2] (parallel axis, no
// cancellation), in a fixed order. b_max of a larger cell is the largest
// distance of its particles to its centre of mass, taken afterwards over
// chunks of BM_CH particles with one atomic max per chunk.
// ---------------------------------------------------------------------------
struct MomArgs {
    const uint32_t *lvl, *nfirst, *ncount, *nnch, *nchild, *nparent, *nlevel;
    const double *x, *y, *z, *m;
    const uint64_t *key;
    const int32_t *psys;
    const SysBox *box;
    double *M, *cx, *cy, *cz, *B2;
    float4 *nA, *nB;
    uint32_t *done;
    const float4 *phi, *plo;
    unsigned long long *bmax64;   // FP64 form: b_max as FP64 bits
    unsigned int *bmax32;         // FP32 form: b_max as FP32 bits
};

__device__ __forceinline__ uint32_t digit_at(uint64_t key, int lev)
{
    return (uint32_t)(key >> (3 * (LEVELS - lev))) & 7u;
}

__device__ __forceinline__ void cell_geom(const SysBox &b, uint64_t key, uint32_t lev, double o[3], double *side)
{
    const double sd = ldexp(b.L, -(int)lev);
    // integer cell coordinate of the key prefix along each axis
    uint32_t q[3] = {0, 0, 0};
    for (uint32_t l = 1; l <= lev; ++l) {
        const uint32_t d = digit_at(key, (int)l);
        q[0] = (q[0] << 1) | ((d >> 2) & 1u);
        q[1] = (q[1] << 1) | ((d >> 1) & 1u);
        q[2] = (q[2] << 1) | (d & 1u);
    }
    for (int k = 0; k < 3; ++k) o[k] = __dadd_rn(b.lo[k], __dmul_rn((double)q[k], sd));
    *side = sd;
}

__device__ __forceinline__ void store_com(const MomArgs &a, uint32_t c, double M, double c0, double c1, double c2,
                                          double B2)
{
    a.M[c] = M;
    a.cx[c] = c0;
    a.cy[c] = c1;
    a.cz[c] = c2;
    a.B2[c] = B2;
    const SysBox b = a.box[a.psys[a.nfirst[c]]];
    float h[3], l[3];
    grid_split(c0, b.lo[0], b, h[0], l[0]);
    grid_split(c1, b.lo[1], b, h[1], l[1]);
    grid_split(c2, b.lo[2], b, h[2], l[2]);
    a.nA[c] = make_float4(h[0], h[1], h[2], (float)M);
    a.nB[c] = make_float4(l[0], l[1], l[2], 0.0f);
}

// Moments straight from each cell's particle range, with no wait on the
// children: M, sum m (x - o) and Q = sum m |x - o|^2 with o = the cell's first
// particle; COM = o + sum m (x - o) / M and B2 = Q - M |COM - o|^2 (o lies
// inside the cell, so the subtraction loses little). Cells of at most MOM_CH
// particles: one warp each (at most 4 rounds of loads per lane). Larger cells: chunks of MOM_CH particles, one warp
// per chunk, then one warp per cell adds the chunk sums in chunk order.
constexpr uint32_t MOM_CH = 128;

struct MomSums {
    double M, sx, sy, sz, Q;
};

// FP32 form: offsets from the first particle from the hi/lo copies (hi parts
// on a common grid, so hi_i - hi_f is exact), sums of at most MOM_CH terms in
// FP32; the chunk sums of larger cells are added in FP64.
struct MomSumsF {
    float M, sx, sy, sz, Q;
};

// G lanes (a whole warp, G = 32, or an aligned group of G = 8 lanes with
// member mask gm; sl = lane within the group) sum a particle range.
template <int G>
__device__ __forceinline__ MomSumsF mom_range_f32(const float4 *__restrict__ phi, const float4 *__restrict__ plo,
                                                  uint32_t f, uint32_t n, uint32_t ref, int sl, unsigned gm)
{
    const float4 hr = phi[ref], lr = plo[ref];
    MomSumsF r = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 4
    for (uint32_t i = f + sl; i < f + n; i += G) {
        const float4 h = phi[i], l = plo[i];
        const float d0 = (h.x - hr.x) + (l.x - lr.x), d1 = (h.y - hr.y) + (l.y - lr.y), d2 = (h.z - hr.z) + (l.z - lr.z);
        const float mi = h.w;
        r.M += mi;
        r.sx = fmaf(mi, d0, r.sx);
        r.sy = fmaf(mi, d1, r.sy);
        r.sz = fmaf(mi, d2, r.sz);
        r.Q = fmaf(mi, fmaf(d0, d0, fmaf(d1, d1, d2 * d2)), r.Q);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        r.M += __shfl_xor_sync(gm, r.M, o, G);
        r.sx += __shfl_xor_sync(gm, r.sx, o, G);
        r.sy += __shfl_xor_sync(gm, r.sy, o, G);
        r.sz += __shfl_xor_sync(gm, r.sz, o, G);
        r.Q += __shfl_xor_sync(gm, r.Q, o, G);
    }
    return r;
}

// FP32 form: centre of mass as offsets e from the first particle f, stored
// as the grid-aligned hi/lo pair; B2 goes to nB.w. No FP64 instruction here:
// a single-lane FP64 instruction costs a full warp's FP64 pipe time.
__device__ __forceinline__ void mom_store_f32(const MomArgs &a, uint32_t c, uint32_t f, float M, float e0, float e1,
                                              float e2, float B2)
{
    const SysBox &b = a.box[a.psys[f]];
    const float4 h = a.phi[f], l = a.plo[f];
    const float t0 = l.x + e0, t1 = l.y + e1, t2 = l.z + e2;
    const float g0 = rintf(t0 * b.inv_uf) * b.uf, g1 = rintf(t1 * b.inv_uf) * b.uf, g2 = rintf(t2 * b.inv_uf) * b.uf;
    a.nA[c] = make_float4(h.x + g0, h.y + g1, h.z + g2, M);
    a.nB[c] = make_float4(t0 - g0, t1 - g1, t2 - g2, B2);
}

// B2 of a small cell about its centre of mass e (offsets from particle ref),
// summed directly so that no M|e|^2 cancels against the second moment, and
// b_max, the largest distance of its particles to e (G lanes as above).
template <int G>
__device__ __forceinline__ void mom_b2_f32(const float4 *__restrict__ phi, const float4 *__restrict__ plo, uint32_t f,
                                           uint32_t n, uint32_t ref, float e0, float e1, float e2, int sl, unsigned gm,
                                           float &B2, float &bmax)
{
    const float4 hr = phi[ref], lr = plo[ref];
    float q = 0.0f, d2max = 0.0f;
    for (uint32_t i = f + sl; i < f + n; i += G) {
        const float4 h = phi[i], l = plo[i];
        const float d0 = ((h.x - hr.x) + (l.x - lr.x)) - e0, d1 = ((h.y - hr.y) + (l.y - lr.y)) - e1,
                    d2 = ((h.z - hr.z) + (l.z - lr.z)) - e2;
        const float r2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        q = fmaf(h.w, r2, q);
        d2max = fmaxf(d2max, r2);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        q += __shfl_xor_sync(gm, q, o, G);
        d2max = fmaxf(d2max, __shfl_xor_sync(gm, d2max, o, G));
    }
    B2 = q;
    bmax = sqrtf(d2max);
}

__device__ __forceinline__ MomSums mom_range(const MomArgs &a, uint32_t f, uint32_t n, double o0, double o1, double o2,
                                             int lane)
{
    MomSums r = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (uint32_t i = f + lane; i < f + n; i += 32) {
        const double mi = a.m[i];
        const double d0 = a.x[i] - o0, d1 = a.y[i] - o1, d2 = a.z[i] - o2;
        r.M += mi;
        r.sx += mi * d0;
        r.sy += mi * d1;
        r.sz += mi * d2;
        r.Q += mi * (d0 * d0 + d1 * d1 + d2 * d2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {   // fixed butterfly: the same order every run
        r.M += __shfl_xor_sync(0xffffffffu, r.M, o);
        r.sx += __shfl_xor_sync(0xffffffffu, r.sx, o);
        r.sy += __shfl_xor_sync(0xffffffffu, r.sy, o);
        r.sz += __shfl_xor_sync(0xffffffffu, r.sz, o);
        r.Q += __shfl_xor_sync(0xffffffffu, r.Q, o);
    }
    return r;
}

__device__ __forceinline__ void mom_store(const MomArgs &a, uint32_t c, const MomSums &r, double o0, double o1,
                                          double o2)
{
    double c0, c1, c2, B2 = 0.0;
    if (r.M > 0.0) {
        const double e0 = r.sx / r.M, e1 = r.sy / r.M, e2 = r.sz / r.M;
        c0 = o0 + e0;
        c1 = o1 + e1;
        c2 = o2 + e2;
        B2 = fmax(r.Q - r.M * (e0 * e0 + e1 * e1 + e2 * e2), 0.0);
    } else {   // massless cell: its geometric centre
        double o[3], sd;
        const uint32_t f = a.nfirst[c];
        cell_geom(a.box[a.psys[f]], a.key[f], a.nlevel[c], o, &sd);
        c0 = o[0] + 0.5 * sd;
        c1 = o[1] + 0.5 * sd;
        c2 = o[2] + 0.5 * sd;
    }
    store_com(a, c, r.M, c0, c1, c2, B2);
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A larger cell from its (at most 8) children, one per lane, in a fixed order.
// FP64 form in FP64 (a whole warp). FP32 form in FP32 on offsets from the
// first child's hi/lo centre of mass (hi differences exact), stored like a
// small cell's, by G lanes (a warp or an aligned group of 8 with mask gm).
__device__ void mom_combine_f64(const MomArgs &a, uint32_t c, int lane)
{
    const uint32_t ch0 = a.nchild[c], k = a.nnch[c];
    const uint32_t f = a.nfirst[c];
    const SysBox &b = a.box[a.psys[f]];
    const bool on = (uint32_t)lane < k;
    double M = 0.0, x = 0.0, y = 0.0, z = 0.0, B2 = 0.0;
    if (on) {
        const uint32_t j = ch0 + lane;
        M = __ldcg(a.M + j);
        x = __ldcg(a.cx + j);
        y = __ldcg(a.cy + j);
        z = __ldcg(a.cz + j);
        B2 = __ldcg(a.B2 + j);
    }
    const double rx = __shfl_sync(0xffffffffu, x, 0), ry = __shfl_sync(0xffffffffu, y, 0),
                 rz = __shfl_sync(0xffffffffu, z, 0);
    const double dx = x - rx, dy = y - ry, dz = z - rz;
    const double Mt = warp_sum_d(M);
    double c0, c1, c2, B2t = 0.0;
    if (Mt > 0.0) {
        const double ex = warp_sum_d(M * dx) / Mt, ey = warp_sum_d(M * dy) / Mt, ez = warp_sum_d(M * dz) / Mt;
        c0 = rx + ex;
        c1 = ry + ey;
        c2 = rz + ez;
        const double qx = dx - ex, qy = dy - ey, qz = dz - ez;
        B2t = warp_sum_d(on ? B2 + M * (qx * qx + qy * qy + qz * qz) : 0.0);
    } else {   // massless cell: its geometric centre
        double o[3], sd;
        cell_geom(b, a.key[f], a.nlevel[c], o, &sd);
        c0 = o[0] + 0.5 * sd;
        c1 = o[1] + 0.5 * sd;
        c2 = o[2] + 0.5 * sd;
    }
    if (lane == 0) store_com(a, c, Mt, c0, c1, c2, B2t);
}

template <int G>
__device__ void mom_combine_f32(const MomArgs &a, uint32_t c, int lane, unsigned gm)
{
    const uint32_t ch0 = a.nchild[c], k = a.nnch[c];
    const uint32_t f = a.nfirst[c];
    const SysBox &b = a.box[a.psys[f]];
    const bool on = (uint32_t)lane < k;
    float4 A = make_float4(0.0f, 0.0f, 0.0f, 0.0f), B = A;
    if (on) {
        A = __ldcg(a.nA + ch0 + lane);
        B = __ldcg(a.nB + ch0 + lane);
    }
    const float hx = __shfl_sync(gm, A.x, 0, G), hy = __shfl_sync(gm, A.y, 0, G),
                hz = __shfl_sync(gm, A.z, 0, G);
    const float lx = __shfl_sync(gm, B.x, 0, G), ly = __shfl_sync(gm, B.y, 0, G),
                lz = __shfl_sync(gm, B.z, 0, G);
    const float M = A.w, dx = (A.x - hx) + (B.x - lx), dy = (A.y - hy) + (B.y - ly), dz = (A.z - hz) + (B.z - lz);
    float Mt = M, sx = M * dx, sy = M * dy, sz = M * dz;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        Mt += __shfl_xor_sync(gm, Mt, o, G);
        sx += __shfl_xor_sync(gm, sx, o, G);
        sy += __shfl_xor_sync(gm, sy, o, G);
        sz += __shfl_xor_sync(gm, sz, o, G);
    }
    float e0, e1, e2, B2t = 0.0f;
    if (Mt > 0.0f) {
        e0 = sx / Mt;
        e1 = sy / Mt;
        e2 = sz / Mt;
        const float qx = dx - e0, qy = dy - e1, qz = dz - e2;
        B2t = on ? fmaf(M, qx * qx + qy * qy + qz * qz, B.w) : 0.0f;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) B2t += __shfl_xor_sync(gm, B2t, o, G);
    } else {   // massless cell: its geometric centre, relative to the first child's centre
        double o[3], sd;
        cell_geom(b, a.key[f], a.nlevel[c], o, &sd);
        e0 = (float)((o[0] + 0.5 * sd - b.lo[0]) - ((double)hx + (double)lx));
        e1 = (float)((o[1] + 0.5 * sd - b.lo[1]) - ((double)hy + (double)ly));
        e2 = (float)((o[2] + 0.5 * sd - b.lo[2]) - ((double)hz + (double)lz));
    }
    if (lane == 0) {
        const float t0 = lx + e0, t1 = ly + e1, t2 = lz + e2;
        const float g0 = rintf(t0 * b.inv_uf) * b.uf, g1 = rintf(t1 * b.inv_uf) * b.uf,
                    g2 = rintf(t2 * b.inv_uf) * b.uf;
        a.nA[c] = make_float4(hx + g0, hy + g1, hz + g2, Mt);
        a.nB[c] = make_float4(t0 - g0, t1 - g1, t2 - g2, B2t);
    }
}

// After cell c is final: if its parent is a larger cell and c is the last of
// its children to finish, combine the parent, and so on upwards. G lanes (a
// warp, or an aligned group of 8 with mask gm; lane = lane within the group).
template <bool F64, int G>
__device__ void mom_climb(const MomArgs &a, uint32_t c, int lane, unsigned gm)
{
    for (;;) {
        const uint32_t p = a.nparent[c];
        if (p == NONE || a.ncount[p] <= MOM_CH) return;
        __syncwarp(gm);
        unsigned int old = 0;
        if (lane == 0) {   // release: c's moments (stored by this lane) before the count; acquire: the others' after
            cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(a.done[p]);
            old = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
        }
        old = __shfl_sync(gm, old, 0, G);
        if (old + 1u != a.nnch[p]) return;
        __syncwarp(gm);
        if (F64) mom_combine_f64(a, p, lane);
        else mom_combine_f32<G>(a, p, lane, gm);
        c = p;
    }
}

constexpr uint32_t BM_CH = 256;

// every cell of at most MOM_CH particles, and every leaf (a leaf holds more
// only when its particles share one level-21 cell): moments and b_max from its
// particles, then the climb; larger cells get their b_max chunk items
template <bool F64>
__global__ void __launch_bounds__(256) k_mom_small(MomArgs a, unsigned long long *nitems, uint32_t *bigbase,
                                                   uint32_t *items, uint32_t cap_items, Status *st, int where)
{
    if (st->code) return;
    const uint32_t total = a.lvl[LEVELS + 1];
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (F64) {   // one warp per cell
        for (uint32_t c = warp; c < total; c += nw) {
            const uint32_t f = a.nfirst[c], n = a.ncount[c];
            if (n <= MOM_CH || a.nnch[c] == 0) {
                const double o0 = a.x[f], o1 = a.y[f], o2 = a.z[f];
                const MomSums r = mom_range(a, f, n, o0, o1, o2, lane);
                if (lane == 0) mom_store(a, c, r, o0, o1, o2);
                __syncwarp();
                const double c0 = __shfl_sync(0xffffffffu, lane == 0 ? a.cx[c] : 0.0, 0);
                const double c1 = __shfl_sync(0xffffffffu, lane == 0 ? a.cy[c] : 0.0, 0);
                const double c2 = __shfl_sync(0xffffffffu, lane == 0 ? a.cz[c] : 0.0, 0);
                double dm = 0.0;
                for (uint32_t i = f + lane; i < f + n; i += 32) {
                    const double d0 = a.x[i] - c0, d1 = a.y[i] - c1, d2 = a.z[i] - c2;
                    dm = fmax(dm, sqrt(d0 * d0 + d1 * d1 + d2 * d2));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
                if (lane == 0) a.bmax64[c] = (unsigned long long)__double_as_longlong(dm);
                mom_climb<true, 32>(a, c, lane, 0xffffffffu);
            } else if (lane == 0) {
                const uint32_t nch = (n + BM_CH - 1) / BM_CH;
                const unsigned long long base = atomicAdd(nitems, (unsigned long long)nch);
                if (base + nch > cap_items) {
                    fail(st, HYBRID_ECAPACITY, where);
                    continue;
                }
                bigbase[c] = (uint32_t)base;
                for (uint32_t k = 0; k < nch; ++k) items[base + k] = c;
            }
        }
    } else {   // FP32 form: four cells per warp, eight lanes each (most cells are leaves of a few particles)
        const int sub = lane >> 3, sl = lane & 7;
        const unsigned gm = 0xFFu << (8 * sub);
        const uint32_t nq = (total + 3) / 4;
        for (uint32_t q = warp; q < nq; q += nw) {
            const uint32_t c = 4 * q + sub;
            if (c >= total) continue;
            const uint32_t f = a.nfirst[c], n = a.ncount[c];
            if (n <= MOM_CH || a.nnch[c] == 0) {
                const MomSumsF r = mom_range_f32<8>(a.phi, a.plo, f, n, f, sl, gm);
                const float iM = r.M > 0.0f ? 1.0f / r.M : 0.0f;
                const float e0 = r.sx * iM, e1 = r.sy * iM, e2 = r.sz * iM;
                float B2, bm;
                mom_b2_f32<8>(a.phi, a.plo, f, n, f, e0, e1, e2, sl, gm, B2, bm);
                if (sl == 0) {
                    mom_store_f32(a, c, f, r.M, e0, e1, e2, B2);
                    a.bmax32[c] = __float_as_uint(bm);
                }
                mom_climb<false, 8>(a, c, sl, gm);
            } else if (sl == 0) {
                const uint32_t nch = (n + BM_CH - 1) / BM_CH;
                const unsigned long long base = atomicAdd(nitems, (unsigned long long)nch);
                if (base + nch > cap_items) {
                    fail(st, HYBRID_ECAPACITY, where);
                    continue;
                }
                bigbase[c] = (uint32_t)base;
                for (uint32_t k = 0; k < nch; ++k) items[base + k] = c;
            }
        }
    }
}

// b_max of the larger cells: one warp per chunk of BM_CH particles, one atomic
// max per chunk (non-negative floats order as their bit patterns)
template <bool F64>
__global__ void __launch_bounds__(256) k_bmax_big(MomArgs a, const unsigned long long *nitems,
                                                  const uint32_t *bigbase, const uint32_t *items, const Status *st)
{
    if (st->code) return;
    const uint32_t T = (uint32_t)*nitems;
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < T; w += nw) {
        const uint32_t c = items[w];
        const uint32_t k = w - bigbase[c];
        const uint32_t f = a.nfirst[c], n = a.ncount[c];
        const uint32_t f0 = f + k * BM_CH, n0 = min(BM_CH, f + n - f0);
        if (F64) {
            const double c0 = a.cx[c], c1 = a.cy[c], c2 = a.cz[c];
            double dm = 0.0;
            for (uint32_t i = f0 + lane; i < f0 + n0; i += 32) {
                const double d0 = a.x[i] - c0, d1 = a.y[i] - c1, d2 = a.z[i] - c2;
                dm = fmax(dm, sqrt(d0 * d0 + d1 * d1 + d2 * d2));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
            if (lane == 0) atomicMax(a.bmax64 + c, (unsigned long long)__double_as_longlong(dm));
        } else {
            const float4 A = a.nA[c], B = a.nB[c];
            float dm = 0.0f;
            for (uint32_t i = f0 + lane; i < f0 + n0; i += 32) {
                const float4 h = a.phi[i], l = a.plo[i];
                const float d0 = (h.x - A.x) + (l.x - B.x);
                const float d1 = (h.y - A.y) + (l.y - B.y);
                const float d2 = (h.z - A.z) + (l.z - B.z);
                dm = fmaxf(dm, d0 * d0 + d1 * d1 + d2 * d2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
            if (lane == 0) atomicMax(a.bmax32 + c, __float_as_uint(sqrtf(dm)));
        }
    }
}

// Per node: geometry, delta, MAC radius, walk criteria and packed topology.
struct FinArgs {
    const uint32_t *lvl, *nfirst, *ncount, *nnch, *nchild, *nlevel;
    const uint64_t *key;
    const int32_t *psys;
    const SysBox *box;
    const SysParams *sp;
    double *M, *cx, *cy, *cz, *B2;
    unsigned long long *bmax;
    const unsigned int *bmax32;
    const float4 *nA, *nB;
    float2 *crit;
    uint4 *topo;
    double4_32a *nD;
    double *rb, *hr, *delta, *side, *org;
};

__device__ __forceinline__ void prefix_q(uint64_t key, uint32_t lev, uint32_t q[3])
{
    q[0] = q[1] = q[2] = 0;
    for (uint32_t l = 1; l <= lev; ++l) {
        const uint32_t d = digit_at(key, (int)l);
        q[0] = (q[0] << 1) | ((d >> 2) & 1u);
        q[1] = (q[1] << 1) | ((d >> 1) & 1u);
        q[2] = (q[2] << 1) | (d & 1u);
    }
}

// Per node: geometry, delta, MAC radius, walk criteria and packed topology.
// F64: from the FP64 moments. FP32 form: delta, r_b and the criteria in FP32
// from the hi/lo centre of mass (cell centres are exact in FP32 on the hi
// grid), then the FP64 copies of the moments for inspection.
template <bool F64>
__global__ void __launch_bounds__(256) k_finalize(FinArgs a, const Status *st)
{
    if (st->code) return;
    const uint32_t total = a.lvl[LEVELS + 1];
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x) {
        const uint32_t f = a.nfirst[c];
        const int s = a.psys[f];
        const SysParams &P = a.sp[s];
        const SysBox &bx = a.box[s];
        const uint32_t lev = a.nlevel[c];
        uint32_t q[3];
        prefix_q(a.key[f], lev, q);
        const double sd = ldexp(bx.L, -(int)lev);
        double rb, hr, delta;
        if (F64) {
            double o[3];
            for (int k = 0; k < 3; ++k) o[k] = __dadd_rn(bx.lo[k], __dmul_rn((double)q[k], sd));
            const double ctr0 = o[0] + 0.5 * sd, ctr1 = o[1] + 0.5 * sd, ctr2 = o[2] + 0.5 * sd;
            const double e0 = a.cx[c] - ctr0, e1 = a.cy[c] - ctr1, e2 = a.cz[c] - ctr2;
            delta = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
            const double bm = __longlong_as_double((long long)a.bmax[c]);
            if (P.mac == 1) rb = 0.5 * bm + sqrt(0.25 * bm * bm + sqrt(3.0 * a.B2[c] / P.a_err));
            else rb = (P.theta > 0.0) ? sd / P.theta + delta : INFINITY;
            hr = P.R2 + P.skin + bm;   // Eq. (15) radius (plus the skin of reused lists)
            const double sacc = fmax(rb, hr);
            a.crit[c] = make_float2((float)(sacc * sacc), P.has_hard ? (float)(hr * hr) : -1.0f);
            a.nD[c] = make_double4_32a(a.cx[c], a.cy[c], a.cz[c], a.M[c]);
            for (int k = 0; k < 3; ++k) a.org[3 * (size_t)c + k] = o[k];
        } else {
            const float sdf = ldexpf((float)bx.L, -(int)lev);
            const float4 A = a.nA[c], B = a.nB[c];
            // cell centre relative to the root corner: (q + 1/2) side, exact in FP32
            const float e0 = (A.x - ((float)q[0] + 0.5f) * sdf) + B.x;
            const float e1 = (A.y - ((float)q[1] + 0.5f) * sdf) + B.y;
            const float e2 = (A.z - ((float)q[2] + 0.5f) * sdf) + B.z;
            const float df = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            const float bm = __uint_as_float(a.bmax32[c]);
            float rbf;
            if (P.mac == 1) rbf = 0.5f * bm + sqrtf(0.25f * bm * bm + sqrtf(3.0f * B.w / (float)P.a_err));
            else rbf = (P.theta > 0.0) ? sdf / (float)P.theta + df : INFINITY;
            const float hrf = P.R2f + P.skinf + bm;
            const float sacc = fmaxf(rbf, hrf);
            a.crit[c] = make_float2(sacc * sacc, P.has_hard ? hrf * hrf : -1.0f);
            // FP64 copies (all lanes busy): moments, b_max, geometry
            const double c0 = bx.lo[0] + ((double)A.x + (double)B.x), c1 = bx.lo[1] + ((double)A.y + (double)B.y),
                         c2 = bx.lo[2] + ((double)A.z + (double)B.z);
            a.M[c] = (double)A.w;
            a.cx[c] = c0;
            a.cy[c] = c1;
            a.cz[c] = c2;
            a.B2[c] = (double)B.w;
            a.bmax[c] = (unsigned long long)__double_as_longlong((double)bm);
            a.nD[c] = make_double4_32a(c0, c1, c2, (double)A.w);
            for (int k = 0; k < 3; ++k) a.org[3 * (size_t)c + k] = __dadd_rn(bx.lo[k], __dmul_rn((double)q[k], sd));
            rb = rbf;
            hr = hrf;
            delta = df;
        }
        const uint32_t k = a.nnch[c];
        a.topo[c] = make_uint4(k ? a.nchild[c] : NONE, k, f, a.ncount[c]);
        a.rb[c] = rb;
        a.hr[c] = hr;
        a.delta[c] = delta;
        a.side[c] = sd;
    }
}

// ---------------------------------------------------------------------------
// Sink groups: first cells (from the root) with count <= n_crit, or leaves.
// Marked at their first particle, compacted in particle order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_group_flag(const uint32_t *__restrict__ lvl,
                                                    const uint32_t *__restrict__ nfirst,
                                                    const uint32_t *__restrict__ ncount,
                                                    const uint32_t *__restrict__ nnch,
                                                    const uint32_t *__restrict__ nparent, int n_crit,
                                                    uint32_t *__restrict__ gflag, const Status *st)
{
    if (st->code) return;
    const uint32_t total = lvl[LEVELS + 1];
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x) {
        const bool stop = ncount[c] <= (uint32_t)n_crit || nnch[c] == 0;
        const uint32_t p = nparent[c];
        const bool parent_goes_on = (p == NONE) || (ncount[p] > (uint32_t)n_crit);
        if (stop && parent_goes_on) gflag[nfirst[c]] = c;
    }
}

__global__ void __launch_bounds__(256) k_group_mark(int64_t N, const uint32_t *__restrict__ gflag,
                                                    uint32_t *__restrict__ gscan, const Status *st)
{
    if (st->code) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        gscan[i] = gflag[i] != NONE ? 1u : 0u;
}

__global__ void __launch_bounds__(256) k_group_compact(int64_t N, const uint32_t *__restrict__ gflag,
                                                       const uint32_t *__restrict__ gscan,
                                                       const uint32_t *__restrict__ ncount,
                                                       const int32_t *__restrict__ psys, uint32_t *gnode,
                                                       uint32_t *gfirst, uint32_t *gcount, uint32_t *gsys,
                                                       const uint64_t *total, int64_t *ngroups, const Status *st)
{
    if (st->code) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ngroups = (int64_t)*total;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = gflag[i];
        if (c != NONE) {
            const uint32_t g = gscan[i];
            gnode[g] = c;
            gfirst[g] = (uint32_t)i;
            gcount[g] = ncount[c];
            gsys[g] = (uint32_t)psys[i];
        }
    }
}

// One warp per group: box of the members (FP64, exact min/max), its centre
// as an FP32 hi/lo pair and its half extents rounded up.
__global__ void __launch_bounds__(256) k_group_box(const int64_t *__restrict__ ngroups,
                                                   const uint32_t *__restrict__ gfirst,
                                                   const uint32_t *__restrict__ gcount, const double *__restrict__ x,
                                                   const double *__restrict__ y, const double *__restrict__ z,
                                                   const int32_t *__restrict__ psys, const SysBox *__restrict__ box,
                                                   double *glo, double *ghi, GroupF *gF, const Status *st)
{
    if (st->code) return;
    const int lane = threadIdx.x & 31;
    const int64_t ng = *ngroups;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // a warp takes B consecutive groups (B = groups per warp, 1 to 32): their boxes one after the other (all
    // lanes), then the FP64 finishing of all B at once, lane k for group g0 + k (a one-lane FP64 instruction costs
    // the FP64 pipe a whole warp's time)
    const int64_t B = max((int64_t)1, min((int64_t)32, ng / nw));
    for (int64_t g0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * B; g0 < ng; g0 += nw * B) {
        const int gn = (int)min(B, ng - g0);
        unsigned long long mine[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
        for (int k = 0; k < gn; ++k) {
            const int64_t g = g0 + k;
            const uint32_t f = gfirst[g], n = gcount[g];
            // exact min/max through the order-preserving integer images (no FP64 pipe work)
            unsigned long long u[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
            for (uint32_t i = f + lane; i < f + n; i += 32) {
                const unsigned long long p0 = ord_dbl(x[i]), p1 = ord_dbl(y[i]), p2 = ord_dbl(z[i]);
                u[0] = min(u[0], p0);
                u[1] = min(u[1], p1);
                u[2] = min(u[2], p2);
                u[3] = max(u[3], p0);
                u[4] = max(u[4], p1);
                u[5] = max(u[5], p2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int j = 0; j < 3; ++j) u[j] = min(u[j], __shfl_xor_sync(0xffffffffu, u[j], o));
#pragma unroll
                for (int j = 3; j < 6; ++j) u[j] = max(u[j], __shfl_xor_sync(0xffffffffu, u[j], o));
            }
            if (lane == k)
#pragma unroll
                for (int j = 0; j < 6; ++j) mine[j] = u[j];
        }
        if (lane < gn) {
            const int64_t g = g0 + lane;
            double v[6];
            for (int j = 0; j < 6; ++j) v[j] = unord_dbl(mine[j]);
            const SysBox b = box[psys[gfirst[g]]];
            float hc[3], lc[3], he[3];
            for (int d = 0; d < 3; ++d) {
                glo[3 * g + d] = v[d];
                ghi[3 * g + d] = v[d + 3];
                const double cc = 0.5 * (v[d] + v[d + 3]) - b.lo[d];   // relative to the root corner
                hc[d] = (float)cc;
                lc[d] = (float)(cc - (double)hc[d]);
                he[d] = __double2float_ru(0.5 * (v[d + 3] - v[d]));
            }
            GroupF G;
            G.c_hi = make_float4(hc[0], hc[1], hc[2], he[0]);
            G.c_lo = make_float4(lc[0], lc[1], lc[2], he[1]);
            G.hz_root = make_float2(he[2], 0.0f);
            gF[g] = G;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid_for(hybrid_ctx *c, int64_t work, int threads, int per_sm = 8)
{
    int64_t g = (work + threads - 1) / threads;
    g = std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)c->nsm * per_sm));
    return (int)g;
}

void launch_box(hybrid_ctx *c)
{
    Status *st = status_dev(c);
    cudaMemsetAsync(c->boxmin.p, 0xff, (size_t)3 * c->S * sizeof(unsigned long long), c->st);
    cudaMemsetAsync(c->boxmax.p, 0x00, (size_t)3 * c->S * sizeof(unsigned long long), c->st);
    k_box<<<std::min(c->nchunks, c->nsm * 16), 256, 0, c->st>>>(
        (const double *)c->x[0].p, (const double *)c->x[1].p, (const double *)c->x[2].p, (const Chunk *)c->chunks_dev.p,
        c->nchunks, (unsigned long long *)c->boxmin.p, (unsigned long long *)c->boxmax.p, st);
    c->launches += 1;
}

void launch_keys_sort(hybrid_ctx *c)
{
    Status *st = status_dev(c);
    const int64_t N = c->N;
    uint64_t *k0 = (uint64_t *)c->keys[0].p, *k1 = (uint64_t *)c->keys[1].p;
    uint32_t *v0 = (uint32_t *)c->vals[0].p, *v1 = (uint32_t *)c->vals[1].p;
    const bool sample = c->ss_ok && !c->sort_fallback;
    const SSys *ss = (const SSys *)c->ss_sys.p;
    uint64_t *spk = (uint64_t *)c->ss_spk.p;
    uint32_t *spv = (uint32_t *)c->ss_spv.p, *cnt = (uint32_t *)c->ss_cnt.p;
    const int64_t *off = (const int64_t *)c->off_dev.p;
    if (sample) {   // splitters from the last build's sorted keys, before the new keys replace them
        k_ss_split<<<std::min(c->S, c->nsm * 2), SSB_THREADS, 0, c->st>>>(k0, off, ss, c->S, spk, spv, cnt);
        c->launches++;
    }
    if (sample) {
        uint32_t *start = (uint32_t *)c->ss_start.p;
        uint32_t *cur = (uint32_t *)c->ss_cur.p, *pb = (uint32_t *)c->ss_pb.p, *flag = (uint32_t *)c->ss_flag.p;
        cudaMemsetAsync(flag, 0, sizeof(uint32_t), c->st);
        k_keys_count<<<grid_for(c, N, 256), 256, 0, c->st>>>(
            N, (const double *)c->x[0].p, (const double *)c->x[1].p, (const double *)c->x[2].p,
            (const int32_t *)c->psys.p, c->S, (const unsigned long long *)c->boxmin.p,
            (const unsigned long long *)c->boxmax.p, (SysBox *)c->box.p, k0, v0, ss, spk, spv, pb, cnt);
        k_ss_scan<<<std::min(c->S, c->nsm * 4), 256, 0, c->st>>>(off, ss, c->S, cnt, start, cur, flag, st, c->op);
        k_ss_scatter<<<grid_for(c, N, 256), 256, 0, c->st>>>(N, k0, pb, start, cur, k1, v1, flag);
        k_ss_sort<<<std::min(c->nbk, c->nsm * 8), SSB_THREADS, (size_t)SS_CAP * 12, c->st>>>(c->nbk, cnt, start, k1,
                                                                                               v1, k0, v0, flag);
        c->launches += 4;
        return;
    }
    k_keys<<<grid_for(c, N, 256), 256, 0, c->st>>>(N, (const double *)c->x[0].p, (const double *)c->x[1].p,
                                                    (const double *)c->x[2].p, (const int32_t *)c->psys.p, c->S,
                                                    (const unsigned long long *)c->boxmin.p,
                                                    (const unsigned long long *)c->boxmax.p, (SysBox *)c->box.p, k0, v0,
                                                    st);
    c->launches++;
    uint32_t *rs = (uint32_t *)c->hist.p;
    uint32_t *counts = rs + RS_HDR, *look = counts + (size_t)2048 * c->S;
    cudaMemsetAsync(rs, 0, ((size_t)RS_HDR + (size_t)2048 * (c->S + c->nchunks)) * sizeof(uint32_t), c->st);
    k_digit_counts<<<std::min(c->nchunks, c->nsm * 4), 256, 0, c->st>>>(k0, (const Chunk *)c->chunks_dev.p, c->nchunks,
                                                                       counts);
    c->launches++;
    const int grid = std::min(c->nchunks, c->nsm * 4);
    const Chunk *chk = (const Chunk *)c->chunks_dev.p;
    for (int pass = 0; pass < 8; ++pass) {
        uint32_t *lk = look + (size_t)pass * 256 * c->nchunks;
        uint32_t *tk = rs + pass;
        switch (c->ipt) {
        case 2: k_onesweep<2><<<grid, 256, 0, c->st>>>(k0, v0, k1, v1, chk, c->nchunks, pass, counts, lk, tk, N, st); break;
        case 4: k_onesweep<4><<<grid, 256, 0, c->st>>>(k0, v0, k1, v1, chk, c->nchunks, pass, counts, lk, tk, N, st); break;
        default: k_onesweep<8><<<grid, 256, 0, c->st>>>(k0, v0, k1, v1, chk, c->nchunks, pass, counts, lk, tk, N, st);
        }
        c->launches++;
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    // after 8 passes the sorted keys/values are back in buffer 0
}

void launch_permute(hybrid_ctx *c)
{
    Status *st = status_dev(c);
    const int64_t N = c->N;
    uint32_t *v0 = (uint32_t *)c->vals[0].p;
    PermArgs a;
    for (int f = 0; f < 7; ++f) {
        a.xin[f] = (const double *)c->x[f].p;
        a.xout[f] = (double *)c->xa[f].p;
    }
    a.id_in = (const int32_t *)c->id.p;
    a.id_out = (int32_t *)c->ida.p;
    a.orig_in = (const int32_t *)c->orig.p;
    a.orig_out = (int32_t *)c->origa.p;
    a.src = v0;
    a.phi = c->p.precision == 1 ? (float4 *)c->phi.p : nullptr;
    a.plo = c->p.precision == 1 ? (float4 *)c->plo.p : nullptr;
    a.pd = c->p.precision == 0 ? (double4_32a *)c->pd.p : nullptr;
    a.disp = c->p.skin > 0.0 ? (float *)c->disp.p : nullptr;
    a.psys = (const int32_t *)c->psys.p;
    a.box = (const SysBox *)c->box.p;
    a.N = N;
    k_permute<<<grid_for(c, N, 256), 256, 0, c->st>>>(a, st);
    c->launches++;
    for (int f = 0; f < 7; ++f) std::swap(c->x[f], c->xa[f]);
    std::swap(c->id, c->ida);
    std::swap(c->orig, c->origa);
    c->swaps ^= 1;
}

bool launch_build_levels(hybrid_ctx *c)
{
    Status *st = status_dev(c);
    const int64_t N = c->N;
    const int gridN = grid_for(c, N, 256, 8);
    int8_t *pc = (int8_t *)c->pc.p;
    uint8_t *pD = (uint8_t *)c->pD.p;
    uint32_t *pn = (uint32_t *)c->pn.p;
    const uint64_t *keys = (const uint64_t *)c->keys[0].p;
    uint64_t *d_tot = (uint64_t *)((char *)c->lvl.p + 256);
    const size_t shm = (size_t)(LD_T + 2 * c->p.n_leaf);
    k_leaf_depth<<<grid_for(c, N, LD_T, 8), LD_T, shm, c->st>>>(N, keys, (const int32_t *)c->psys.p, pc,
                                                                c->p.n_leaf, pD, pn, st);
    scan_u32(c, pn, N, nullptr, N, d_tot);
    unsigned long long *rec = (unsigned long long *)c->rec.p;
    k_records<<<gridN, 256, 0, c->st>>>(N, pc, pD, pn, d_tot, c->capNodes, rec, st, c->op);
    const int ntiles = (int)((c->capNodes + REC_TILE - 1) / REC_TILE);
    uint32_t *rh = (uint32_t *)c->rhist.p;
    k_rec_hist<<<std::min(ntiles, c->nsm * 4), 256, 0, c->st>>>(rec, d_tot, ntiles, rh, st);
    scan_u32(c, rh, (int64_t)NLEV * ntiles, nullptr, (int64_t)NLEV * ntiles, nullptr);
    uint32_t *b2d = (uint32_t *)c->rb2d.p, *d2b = (uint32_t *)c->rd2b.p;
    uint32_t *lvl = (uint32_t *)c->lvl.p;
    k_rec_scatter<<<std::min(ntiles, c->nsm * 4), 256, 0, c->st>>>(rec, d_tot, ntiles, rh, b2d, d2b, lvl, st);
    const int gridT = grid_for(c, c->capNodes, 256, 8);
    k_nodes_a<<<gridT, 256, 0, c->st>>>(d_tot, b2d, d2b, rec, pD, keys, (const int32_t *)c->psys.p,
                                        (const int64_t *)c->off_dev.p, (uint32_t *)c->nfirst.p, (uint32_t *)c->ncount.p,
                                        (uint32_t *)c->nlevel.p, (uint32_t *)c->nchild.p, (uint32_t *)c->nparent.p,
                                        (uint32_t *)c->sysroot.p, st);
    k_nodes_b<<<gridT, 256, 0, c->st>>>(d_tot, lvl, (const uint32_t *)c->nfirst.p, (const uint32_t *)c->ncount.p,
                                        (const uint32_t *)c->nlevel.p, (const uint32_t *)c->nchild.p,
                                        (uint32_t *)c->nnch.p, (uint32_t *)c->nparent.p, st);
    c->launches += 7;
    return true;
}

void launch_moments(hybrid_ctx *c)
{
    Status *st = status_dev(c);
    const int grid = grid_for(c, c->capNodes, 256, 8);
    if (c->p.precision == 0) cudaMemsetAsync(c->nbmax.p, 0, (size_t)c->capNodes * sizeof(unsigned long long), c->st);
    else cudaMemsetAsync(c->nbmax32.p, 0, (size_t)c->capNodes * sizeof(unsigned int), c->st);
    MomArgs a;
    a.lvl = (const uint32_t *)c->lvl.p;
    a.nfirst = (const uint32_t *)c->nfirst.p;
    a.ncount = (const uint32_t *)c->ncount.p;
    a.nnch = (const uint32_t *)c->nnch.p;
    a.nchild = (const uint32_t *)c->nchild.p;
    a.nparent = (const uint32_t *)c->nparent.p;
    a.nlevel = (const uint32_t *)c->nlevel.p;
    a.x = (const double *)c->x[0].p;
    a.y = (const double *)c->x[1].p;
    a.z = (const double *)c->x[2].p;
    a.m = (const double *)c->x[6].p;
    a.key = (const uint64_t *)c->keys[0].p;
    a.psys = (const int32_t *)c->psys.p;
    a.box = (const SysBox *)c->box.p;
    a.M = (double *)c->nM.p;
    a.cx = (double *)c->ncx.p;
    a.cy = (double *)c->ncy.p;
    a.cz = (double *)c->ncz.p;
    a.B2 = (double *)c->nB2.p;
    a.nA = (float4 *)c->nA.p;
    a.nB = (float4 *)c->nB.p;
    a.done = (uint32_t *)c->ndone.p;
    a.bmax64 = (unsigned long long *)c->nbmax.p;
    a.bmax32 = (unsigned int *)c->nbmax32.p;
    a.phi = (const float4 *)c->phi.p;
    a.plo = (const float4 *)c->plo.p;
    unsigned long long *nitems = (unsigned long long *)c->counter.p + 9;
    cudaMemsetAsync(nitems, 0, sizeof(unsigned long long), c->st);
    cudaMemsetAsync(c->ndone.p, 0, (size_t)c->capNodes * sizeof(uint32_t), c->st);
    const int gridw = grid_for(c, c->capNodes * 32, 256, 16);
    uint32_t *bigbase = (uint32_t *)c->nbig.p, *items = (uint32_t *)c->mitems.p;
    if (c->p.precision == 0) {
        k_mom_small<true><<<gridw, 256, 0, c->st>>>(a, nitems, bigbase, items, (uint32_t)c->capItems, st, c->op);
        k_bmax_big<true><<<gridw, 256, 0, c->st>>>(a, nitems, bigbase, items, st);
    } else {
        k_mom_small<false><<<gridw, 256, 0, c->st>>>(a, nitems, bigbase, items, (uint32_t)c->capItems, st, c->op);
        k_bmax_big<false><<<gridw, 256, 0, c->st>>>(a, nitems, bigbase, items, st);
    }
    c->launches += 2;
    FinArgs f;
    f.lvl = a.lvl;
    f.nfirst = a.nfirst;
    f.ncount = a.ncount;
    f.nnch = a.nnch;
    f.nchild = a.nchild;
    f.nlevel = a.nlevel;
    f.key = a.key;
    f.psys = a.psys;
    f.box = a.box;
    f.sp = (const SysParams *)c->sp_dev.p;
    f.M = (double *)c->nM.p;
    f.cx = (double *)c->ncx.p;
    f.cy = (double *)c->ncy.p;
    f.cz = (double *)c->ncz.p;
    f.B2 = (double *)c->nB2.p;
    f.bmax = (unsigned long long *)c->nbmax.p;
    f.bmax32 = (const unsigned int *)c->nbmax32.p;
    f.nA = (const float4 *)c->nA.p;
    f.nB = (const float4 *)c->nB.p;
    f.crit = (float2 *)c->ncrit.p;
    f.topo = (uint4 *)c->ntopo.p;
    f.nD = (double4_32a *)c->nD.p;
    f.rb = (double *)c->nrb.p;
    f.hr = (double *)c->nhr.p;
    f.delta = (double *)c->ndelta.p;
    f.side = (double *)c->nside.p;
    f.org = (double *)c->norg.p;
    if (c->p.precision == 0) k_finalize<true><<<grid, 256, 0, c->st>>>(f, st);
    else k_finalize<false><<<grid, 256, 0, c->st>>>(f, st);
    c->launches += 3;
}

void launch_groups(hybrid_ctx *c)
{
    Status *st = status_dev(c);
    const int64_t N = c->N;
    cudaMemsetAsync(c->gflag.p, 0xff, (size_t)N * sizeof(uint32_t), c->st);
    k_group_flag<<<grid_for(c, c->capNodes, 256), 256, 0, c->st>>>(
        (const uint32_t *)c->lvl.p, (const uint32_t *)c->nfirst.p, (const uint32_t *)c->ncount.p,
        (const uint32_t *)c->nnch.p, (const uint32_t *)c->nparent.p, c->p.n_crit, (uint32_t *)c->gflag.p, st);
    k_group_mark<<<grid_for(c, N, 256), 256, 0, c->st>>>(N, (const uint32_t *)c->gflag.p, (uint32_t *)c->gscan.p, st);
    uint64_t *d_tot = (uint64_t *)((char *)c->lvl.p + 64 * sizeof(uint32_t) + 64 + 8);
    scan_u32(c, (uint32_t *)c->gscan.p, N, nullptr, N, d_tot);
    k_group_compact<<<grid_for(c, N, 256), 256, 0, c->st>>>(
        N, (const uint32_t *)c->gflag.p, (const uint32_t *)c->gscan.p, (const uint32_t *)c->ncount.p,
        (const int32_t *)c->psys.p, (uint32_t *)c->gnode.p, (uint32_t *)c->gfirst.p, (uint32_t *)c->gcount.p,
        (uint32_t *)c->gsys.p, d_tot, (int64_t *)c->ngroups_dev.p, st);
    c->launches += 3;
}

void launch_group_boxes(hybrid_ctx *c)
{
    Status *st = status_dev(c);
    const int64_t N = c->N;
    k_group_box<<<grid_for(c, N * 32 / 16, 256), 256, 0, c->st>>>(
        (const int64_t *)c->ngroups_dev.p, (const uint32_t *)c->gfirst.p, (const uint32_t *)c->gcount.p,
        (const double *)c->x[0].p, (const double *)c->x[1].p, (const double *)c->x[2].p, (const int32_t *)c->psys.p,
        (const SysBox *)c->box.p, (double *)c->glo.p, (double *)c->ghi.p, (GroupF *)c->gF.p, st);
    c->launches += 1;
}

cudaError_t init_tree_kernels()
{
    return cudaFuncSetAttribute(k_ss_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, SS_CAP * 12);
}

void launch_wait_selftest(hybrid_ctx *c, int max_polls)
{
    uint32_t *word = (uint32_t *)((unsigned long long *)c->counter.p + 15);   // a slot nothing else uses
    cudaMemsetAsync(word, 0, sizeof(uint32_t), c->st);
    k_wait_selftest<<<1, 32, 0, c->st>>>(word, max_polls, status_dev(c));
    c->launches++;
}

}  // namespace hy
