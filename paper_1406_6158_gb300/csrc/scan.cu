// scan.cu -- exclusive prefix sums whose length may live on the device.
//
// Two launches: per-segment sums, whose last block to finish (a ticket
// counter, no waiting) also scans the segment sums, and a per-segment block
// scan that adds the segment offset. The length is read
// from device memory when the caller has no host copy (tree levels, group
// counts), so the sequence never waits on the host.
#include "hy_internal.cuh"

namespace hy {

namespace {

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

}  // namespace

// Block-wide exclusive scan of one value per thread; every thread also gets
// the block total.
template <typename T>
__device__ __forceinline__ T block_scan_with_total(T v, T &total)
{
    __shared__ T wsum[SCAN_THREADS / 32];
    __shared__ T tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = (lane < SCAN_THREADS / 32) ? wsum[lane] : T(0);
        T si = warp_incl_scan(s);
        if (lane < SCAN_THREADS / 32) wsum[lane] = si - s;
        if (lane == SCAN_THREADS / 32 - 1) tot = si;
    }
    __syncthreads();
    T r = wsum[w] + inc - v;
    total = tot;
    __syncthreads();
    return r;
}

// Segment sums; the last block to finish scans them (exclusive, in place) and
// writes the grand total. Every block takes a ticket, also when the status
// says to skip the work, so the ticket is back at 0 after every launch.
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const T *data, int64_t n_host, const int64_t *d_n,
                                                               uint64_t *bsum, uint64_t *d_total, unsigned *ticket,
                                                               const Status *st)
{
    const bool skip = st && st->code;
    const int64_t n = skip ? 0 : (d_n ? *d_n : n_host);
    const int64_t nseg = (n + SCAN_SEG - 1) / SCAN_SEG;
    for (int64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const int64_t base = s * SCAN_SEG + (int64_t)threadIdx.x * SCAN_IPT;
        uint64_t acc = 0;
#pragma unroll
        for (int k = 0; k < SCAN_IPT; ++k)
            if (base + k < n) acc += (uint64_t)data[base + k];
        uint64_t tot;
        block_scan_with_total<uint64_t>(acc, tot);
        if (threadIdx.x == 0) bsum[s] = tot;
    }
    __shared__ bool last;
    __threadfence();   // this block's sums are visible before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    uint64_t carry = 0;
    for (int64_t b0 = 0; b0 < nseg; b0 += SCAN_THREADS) {
        const int64_t i = b0 + threadIdx.x;
        const uint64_t v = i < nseg ? __ldcg(bsum + i) : 0ull;
        uint64_t tot;
        const uint64_t ex = block_scan_with_total<uint64_t>(v, tot);
        if (i < nseg) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (d_total && !skip) *d_total = carry;
        *ticket = 0u;
    }
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(T *data, int64_t n_host, const int64_t *d_n,
                                                             const uint64_t *bsum, const Status *st)
{
    if (st && st->code) return;
    const int64_t n = d_n ? *d_n : n_host;
    const int64_t nseg = (n + SCAN_SEG - 1) / SCAN_SEG;
    for (int64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const int64_t base = s * SCAN_SEG + (int64_t)threadIdx.x * SCAN_IPT;
        T v[SCAN_IPT];
        uint64_t acc = 0;
#pragma unroll
        for (int k = 0; k < SCAN_IPT; ++k) {
            v[k] = (base + k < n) ? data[base + k] : T(0);
            acc += (uint64_t)v[k];
        }
        uint64_t tot;
        uint64_t ex = block_scan_with_total<uint64_t>(acc, tot) + bsum[s];
#pragma unroll
        for (int k = 0; k < SCAN_IPT; ++k) {
            if (base + k < n) data[base + k] = (T)ex;
            ex += (uint64_t)v[k];
        }
    }
}

// One block of 1024 threads scans the whole array (short arrays): chunks of
// 1024 x IPT elements, a carry between chunks.
constexpr int SMALL_IPT = 8;
constexpr int64_t SMALL_MAX = 1024 * SMALL_IPT;   // one chunk: a single pass over the array

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_small(T *data, int64_t n_host, const int64_t *d_n, uint64_t *d_total,
                                                     const Status *st)
{
    if (st && st->code) return;
    const int64_t n = d_n ? *d_n : n_host;
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < n; b0 += 1024 * SMALL_IPT) {
        const int64_t base = b0 + (int64_t)threadIdx.x * SMALL_IPT;
        T v[SMALL_IPT];
        uint64_t acc = 0;
#pragma unroll
        for (int k = 0; k < SMALL_IPT; ++k) {
            v[k] = (base + k < n) ? data[base + k] : T(0);
            acc += (uint64_t)v[k];
        }
        const uint64_t inc = warp_incl_scan(acc);
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        if (w == 0) {
            const uint64_t s = wsum[lane];
            wsum[lane] = warp_incl_scan(s) - s;
        }
        __syncthreads();
        const uint64_t c0 = carry;
        uint64_t ex = c0 + wsum[w] + inc - acc;
#pragma unroll
        for (int k = 0; k < SMALL_IPT; ++k) {
            if (base + k < n) data[base + k] = (T)ex;
            ex += (uint64_t)v[k];
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = c0 + wsum[31] + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

template <typename T>
static void scan_impl(hybrid_ctx *c, T *data, int64_t n_host, const int64_t *d_n, int64_t n_max, uint64_t *d_total,
                      bool always)
{
    if (n_max <= SMALL_MAX) {
        k_scan_small<T><<<1, 1024, 0, c->st>>>(data, n_host, d_n, d_total, always ? nullptr : status_dev(c));
        c->launches += 1;
        return;
    }
    const int64_t nseg_max = (n_max + SCAN_SEG - 1) / SCAN_SEG;
    if (nseg_max <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(uint64_t), c->st);
        return;
    }
    ensure(c, c->blocksum, (size_t)nseg_max * sizeof(uint64_t));
    uint64_t *bs = (uint64_t *)c->blocksum.p;
    const int grid = (int)std::min<int64_t>(nseg_max, (int64_t)c->nsm * 8);
    Status *st = always ? nullptr : status_dev(c);
    unsigned *ticket = (unsigned *)((unsigned long long *)c->counter.p + 13);   // 0 between launches
    k_scan_reduce<T><<<grid, SCAN_THREADS, 0, c->st>>>(data, n_host, d_n, bs, d_total, ticket, st);
    k_scan_down<T><<<grid, SCAN_THREADS, 0, c->st>>>(data, n_host, d_n, bs, st);
    c->launches += 2;
}

void scan_u32(hybrid_ctx *c, uint32_t *data, int64_t n_host, const int64_t *d_n, int64_t n_max, uint64_t *d_total,
              bool always)
{
    scan_impl<uint32_t>(c, data, n_host, d_n, n_max, d_total, always);
}

void scan_u64(hybrid_ctx *c, uint64_t *data, int64_t n_host, const int64_t *d_n, int64_t n_max, uint64_t *d_total,
              bool always)
{
    scan_impl<uint64_t>(c, data, n_host, d_n, n_max, d_total, always);
}

}  // namespace hy
