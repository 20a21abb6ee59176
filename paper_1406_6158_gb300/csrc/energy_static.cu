// Allocation-free energy diagnostic: the softened kinetic and potential
// energies of one system by direct FP64 summation (the total-energy check of
// Sec. IV-A), like hybrid_energy, but with no context and no device
// allocation of any kind.
//
// Who needs it: callers that cannot call cudaMalloc/cudaFree (or any library
// call that allocates), namely
//  - code that runs when the device has no free memory left, e.g. a
//    diagnostic taken from an out-of-memory handler, or in a process whose
//    caching allocator already holds the whole device;
//  - latency-sensitive loops that must not pay the implicit device-wide
//    synchronisation cudaFree performs, nor the first-touch cost of a new
//    allocation.
// hybrid_create and hybrid_energy allocate their working buffers, so such
// callers cannot use them.
//
// Scratch is a file-scope __device__ array of fixed size: one (kinetic,
// potential) pair per sink tile plus the two totals. Its address is looked up
// once per device with cudaGetSymbolAddress, with that device current, on the
// first call made there. Every slot a call reads is written earlier in the
// same call (per-tile partials, then the totals), so nothing has to start at
// zero. The scratch is shared by every call on the device: calls that overlap
// in time (two streams, two host threads) race on it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/hybrid.h"

namespace {

constexpr int ES_THREADS = 256;   // sinks per tile = sources per staged tile
constexpr int64_t ES_MAX_TILES = (HYBRID_ENERGY_NOALLOC_MAX_N + ES_THREADS - 1) / ES_THREADS;
constexpr int ES_MAX_DEVICES = 64;

// [2 * tile] kinetic, [2 * tile + 1] potential; the last two slots hold the totals
__device__ __align__(256) double es_scratch[2 * ES_MAX_TILES + 2];

double *g_scratch[ES_MAX_DEVICES];
std::mutex g_mu;

struct alignas(32) Src {
    double x, y, z, m;
};

// One block per tile of ES_THREADS sinks; sources staged through shared
// memory. Writes the tile's kinetic and potential sums (fixed-order block
// reduction) into its own scratch slots.
__global__ void __launch_bounds__(ES_THREADS)
    k_energy_tiles(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                   const double *__restrict__ z, const double *__restrict__ vx, const double *__restrict__ vy,
                   const double *__restrict__ vz, const double *__restrict__ m, double G, double eps2,
                   double *__restrict__ part)
{
    __shared__ Src tile[ES_THREADS];
    __shared__ double red[2][ES_THREADS / 32];
    const int64_t ntiles = (n + ES_THREADS - 1) / ES_THREADS;
    for (int64_t b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const int64_t i = b * ES_THREADS + threadIdx.x;
        const bool ok = i < n;
        const int64_t ii = ok ? i : 0;
        const double xi = x[ii], yi = y[ii], zi = z[ii];
        double W = 0.0;
        for (int64_t j0 = 0; j0 < n; j0 += ES_THREADS) {
            const int64_t j = j0 + threadIdx.x;
            __syncthreads();
            if (j < n) tile[threadIdx.x] = Src{x[j], y[j], z[j], m[j]};
            __syncthreads();
            const int nt = (int)(n - j0 < ES_THREADS ? n - j0 : ES_THREADS);
            for (int k = 0; k < nt; ++k) {
                if (j0 + k == i) continue;
                const Src q = tile[k];
                const double dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
                W += q.m / sqrt(dx * dx + dy * dy + dz * dz + eps2);
            }
        }
        double T = 0.0, P = 0.0;
        if (ok) {
            const double mi = m[i], v0 = vx[i], v1 = vy[i], v2 = vz[i];
            T = 0.5 * mi * (v0 * v0 + v1 * v1 + v2 * v2);
            P = -0.5 * G * mi * W;
        }
        for (int o = 16; o > 0; o >>= 1) {
            T += __shfl_xor_sync(0xffffffffu, T, o);
            P += __shfl_xor_sync(0xffffffffu, P, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = T;
            red[1][threadIdx.x >> 5] = P;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tT = 0.0, tP = 0.0;
            for (int k = 0; k < ES_THREADS / 32; ++k) {
                tT += red[0][k];
                tP += red[1][k];
            }
            part[2 * b] = tT;
            part[2 * b + 1] = tP;
        }
    }
}

// One block: the per-tile sums added in tile order per lane, then a fixed
// tree; writes the totals after the last tile slot.
__global__ void __launch_bounds__(ES_THREADS) k_energy_total(int64_t ntiles, double *part)
{
    __shared__ double red[2][ES_THREADS];
    double T = 0.0, P = 0.0;
    for (int64_t b = threadIdx.x; b < ntiles; b += ES_THREADS) {
        T += part[2 * b];
        P += part[2 * b + 1];
    }
    red[0][threadIdx.x] = T;
    red[1][threadIdx.x] = P;
    __syncthreads();
    for (int s = ES_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * ES_MAX_TILES] = red[0][0];
        part[2 * ES_MAX_TILES + 1] = red[1][0];
    }
}

// Scratch address on the current device, looked up on the first call there.
// The same set-up queries both kernels' attributes, which loads them: under
// lazy module loading a kernel is otherwise loaded (and its code given device
// memory) at its first launch, which an allocation-free caller cannot afford.
cudaError_t scratch_for_current(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= ES_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, es_scratch);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_energy_tiles);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_energy_total);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = (double *)p;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" hybrid_status hybrid_energy_noalloc(int64_t n, const double *x, const double *y, const double *z,
                                               const double *vx, const double *vy, const double *vz,
                                               const double *m, double G, double eps, void *stream,
                                               double *kinetic, double *potential)
{
    if (!kinetic || !potential || n < 0 || !(eps >= 0.0)) return HYBRID_EINVAL;
    if (n > HYBRID_ENERGY_NOALLOC_MAX_N) return HYBRID_ETOOLARGE;
    if (n > 0 && (!x || !y || !z || !vx || !vy || !vz || !m)) return HYBRID_EINVAL;
    double *scratch = nullptr;
    if (scratch_for_current(&scratch) != cudaSuccess) return HYBRID_ECUDA;
    if (n == 0) {
        *kinetic = 0.0;
        *potential = 0.0;
        return HYBRID_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HYBRID_ECUDA;
    const int64_t ntiles = (n + ES_THREADS - 1) / ES_THREADS;
    const int grid = (int)(ntiles < (int64_t)nsm * 8 ? ntiles : (int64_t)nsm * 8);
    k_energy_tiles<<<grid, ES_THREADS, 0, st>>>(n, x, y, z, vx, vy, vz, m, G, eps * eps, scratch);
    k_energy_total<<<1, ES_THREADS, 0, st>>>(ntiles, scratch);
    double v[2];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, scratch + 2 * ES_MAX_TILES, sizeof v, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return HYBRID_ECUDA;
    *kinetic = v[0];
    *potential = v[1];
    return HYBRID_OK;
}
