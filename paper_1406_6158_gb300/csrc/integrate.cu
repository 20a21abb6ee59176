// integrate.cu -- leap-frog kick and drift (Eq. 3-4), the copies between the
// caller's arrays and the context's working state, and the energy diagnostic.
//
// Kicks and drifts run in FP64 with one rounding per product and per sum
// (v <- v + h a; x <- x + dt v), in the order the integrator states them, so
// the FP64 path reproduces a plain CPU evaluation of the same sequence.
#include "hy_internal.cuh"

namespace hy {

namespace {

struct StatePtrs {
    double *x[7];
    int32_t *id, *orig, *psys;
    void *as[3], *ah[3];
    float4 *phi, *plo;      // FP32 hi/lo positions (precision 1)
    float *disp;            // distance bound since the last build (skin > 0), or null
    const SysBox *box;
};

__device__ __forceinline__ void fail(Status *st, int code, int where)
{
    // the first failure wins and keeps its op index: later kernels of the same sequence may fail too (a build
    // after an unsorted one), and the sequence resumes at the first
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

// system of batch position i: binary search over the offsets (S + 1 entries)
__device__ __forceinline__ int sys_of(const int64_t *__restrict__ off, int S, int64_t i)
{
    int lo = 0, hi = S;   // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_copy_in(int64_t N, int S, const int64_t *__restrict__ off,
                                                 const SysIO *__restrict__ io, StatePtrs w, int prec, int with_acc)
{
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < N; gi += (int64_t)gridDim.x * blockDim.x) {
        const int s = sys_of(off, S, gi);
        const SysIO &y = io[s];
        const int64_t li = gi - y.off;
#pragma unroll
        for (int f = 0; f < 7; ++f) w.x[f][gi] = y.x[f][li];
        w.id[gi] = y.id ? y.id[li] : (int32_t)li;
        w.orig[gi] = (int32_t)li;
        w.psys[gi] = s;
        if (with_acc) {
            for (int d = 0; d < 3; ++d) {
                if (prec == 1) {
                    ((float *)w.as[d])[gi] = ((const float *)y.as[d])[li];
                    ((float *)w.ah[d])[gi] = ((const float *)y.ah[d])[li];
                } else {
                    ((double *)w.as[d])[gi] = ((const double *)y.as[d])[li];
                    ((double *)w.ah[d])[gi] = ((const double *)y.ah[d])[li];
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_copy_out(int64_t N, const int32_t *__restrict__ psys,
                                                  const SysIO *__restrict__ io, StatePtrs w, int prec, int state,
                                                  int acc_s, int acc_h, const Status *st)
{
    if (st->code) return;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < N; gi += (int64_t)gridDim.x * blockDim.x) {
        const SysIO &y = io[psys[gi]];
        const int64_t li = gi - y.off;
        if (state) {
#pragma unroll
            for (int f = 0; f < 7; ++f) y.x[f][li] = w.x[f][gi];
            if (y.id) y.id[li] = w.id[gi];
        }
        for (int d = 0; d < 3; ++d) {
            if (prec == 1) {
                if (acc_s) ((float *)y.as[d])[li] = ((const float *)w.as[d])[gi];
                if (acc_h) ((float *)y.ah[d])[li] = ((const float *)w.ah[d])[gi];
            } else {
                if (acc_s) ((double *)y.as[d])[li] = ((const double *)w.as[d])[gi];
                if (acc_h) ((double *)y.ah[d])[li] = ((const double *)w.ah[d])[gi];
            }
        }
    }
}

struct KickSpec {
    int n;            // number of kicks, applied in order
    int which[4];     // 0 soft, 1 hard
    int mode[4];      // 0: h = val; 1: h = dt_soft / 2; 2: h = (dt_soft / n_hard) / 2
    double val[4];
    int dmode;        // -1: no drift; 0: dt = dval; 2: dt = dt_soft / n_hard
    double dval;
    int resplit;      // after the drift: new FP32 hi/lo positions and the distance bound (reused lists)
    int where;        // op index, recorded when a particle has moved more than skin / 2
};

// Exact FP32 -> FP64 conversion of a normal number with integer operations
// (sign, exponent rebiased by 1023 - 127, mantissa moved up 29 bits); zero keeps
// its sign, and subnormals, infinities and NaNs take the ordinary conversion.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    if (e == 0u || e == 0xffu) return (b & 0x7fffffffu) == 0u ? __longlong_as_double((long long)sign) : (double)f;
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double widen(double f) { return f; }

// The step sizes of each kind are per-system constants (SysParams), so a
// particle's update is the three products and sums per vector and nothing else.
template <typename A>
__global__ void __launch_bounds__(256) k_kick_drift(int64_t N, StatePtrs w, const SysParams *__restrict__ sp,
                                                    KickSpec ks, Status *st)
{
    if (st->code) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const SysParams &P = sp[w.psys[i]];
        double v0 = w.x[3][i], v1 = w.x[4][i], v2 = w.x[5][i];
        for (int k = 0; k < ks.n; ++k) {
            const double h = ks.mode[k] == 1 ? P.h_soft : ks.mode[k] == 2 ? P.h_hard : ks.val[k];
            void *const *acc = ks.which[k] ? w.ah : w.as;
            const double a0 = widen(((const A *)acc[0])[i]);
            const double a1 = widen(((const A *)acc[1])[i]);
            const double a2 = widen(((const A *)acc[2])[i]);
            v0 = __dadd_rn(v0, __dmul_rn(h, a0));
            v1 = __dadd_rn(v1, __dmul_rn(h, a1));
            v2 = __dadd_rn(v2, __dmul_rn(h, a2));
        }
        w.x[3][i] = v0;
        w.x[4][i] = v1;
        w.x[5][i] = v2;
        if (ks.dmode >= 0) {
            const double dt = ks.dmode == 0 ? ks.dval : P.dt_hard;
            const double x0 = __dadd_rn(w.x[0][i], __dmul_rn(dt, v0));
            const double x1 = __dadd_rn(w.x[1][i], __dmul_rn(dt, v1));
            const double x2 = __dadd_rn(w.x[2][i], __dmul_rn(dt, v2));
            w.x[0][i] = x0;
            w.x[1][i] = x1;
            w.x[2][i] = x2;
            if (ks.resplit) {
                // the pair kernels' copy of the moved positions, and the distance of this drift (from the old
                // and new hi/lo copies: hi differences are exact) added to the bound since the last build
                const SysBox &b = w.box[w.psys[i]];
                float h0, h1, h2, l0, l1, l2;
                grid_split(x0, b.lo[0], b, h0, l0);
                grid_split(x1, b.lo[1], b, h1, l1);
                grid_split(x2, b.lo[2], b, h2, l2);
                const float4 oh = w.phi[i], ol = w.plo[i];
                const float d0 = (h0 - oh.x) + (l0 - ol.x), d1 = (h1 - oh.y) + (l1 - ol.y), d2 = (h2 - oh.z) + (l2 - ol.z);
                w.phi[i] = make_float4(h0, h1, h2, oh.w);
                w.plo[i] = make_float4(l0, l1, l2, 0.0f);
                // rounded up by a few units in the last place: a bound, not an estimate
                const float moved = w.disp[i] + sqrtf(d0 * d0 + d1 * d1 + d2 * d2) * 1.000001f + 1e-30f;
                w.disp[i] = moved;
                if (moved > P.half_skinf) fail(st, ST_SKIN, ks.where);
            }
        }
    }
}

// caller-array kick and drift (hybrid_kick / hybrid_drift)
template <typename A>
__global__ void __launch_bounds__(256) k_kick_ext(int64_t n, double *vx, double *vy, double *vz, const A *ax,
                                                  const A *ay, const A *az, double h)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        vx[i] = __dadd_rn(vx[i], __dmul_rn(h, widen(ax[i])));
        vy[i] = __dadd_rn(vy[i], __dmul_rn(h, widen(ay[i])));
        vz[i] = __dadd_rn(vz[i], __dmul_rn(h, widen(az[i])));
    }
}

__global__ void __launch_bounds__(256) k_drift_ext(int64_t n, double *x, double *y, double *z, const double *vx,
                                                   const double *vy, const double *vz, double dt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = __dadd_rn(x[i], __dmul_rn(dt, vx[i]));
        y[i] = __dadd_rn(y[i], __dmul_rn(dt, vy[i]));
        z[i] = __dadd_rn(z[i], __dmul_rn(dt, vz[i]));
    }
}

// Softened energies by direct FP64 summation: one thread per sink, sources of
// the same system staged through shared memory; per-system sums by atomics.
constexpr int EN_THREADS = 256;
__global__ void __launch_bounds__(EN_THREADS) k_energy(const Chunk *__restrict__ chunks, int nchunks, int SUB,
                                                       const int64_t *__restrict__ off, StatePtrs w,
                                                       const SysParams *__restrict__ sp, double *out)
{
    __shared__ double4_32a tile[EN_THREADS];
    __shared__ double red[2][EN_THREADS / 32];
    // SUB = sink tiles of EN_THREADS per radix chunk
    for (int b = blockIdx.x; b < nchunks * SUB; b += gridDim.x) {
        const Chunk ch = chunks[b / SUB];
        const int t0 = (b % SUB) * EN_THREADS;
        if (t0 >= ch.len) continue;
        const SysParams P = sp[ch.sys];
        const int64_t s0 = off[ch.sys], s1 = off[ch.sys + 1];
        {
            const int t = t0 + threadIdx.x;
            const bool ok = t < ch.len;
            const int64_t i = ch.start + (ok ? t : 0);
            const double xi = w.x[0][i], yi = w.x[1][i], zi = w.x[2][i], mi = w.x[6][i];
            double W = 0.0;
            for (int64_t j0 = s0; j0 < s1; j0 += EN_THREADS) {
                const int64_t j = j0 + threadIdx.x;
                __syncthreads();
                if (j < s1) tile[threadIdx.x] = make_double4_32a(w.x[0][j], w.x[1][j], w.x[2][j], w.x[6][j]);
                __syncthreads();
                const int nt = (int)min((int64_t)EN_THREADS, s1 - j0);
                for (int k = 0; k < nt; ++k) {
                    if (j0 + k == i) continue;
                    const double4_32a q = tile[k];
                    const double dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
                    W += q.w / sqrt(dx * dx + dy * dy + dz * dz + P.eps2);
                }
            }
            double T = 0.0, Wi = 0.0;
            if (ok) {
                const double v0 = w.x[3][i], v1 = w.x[4][i], v2 = w.x[5][i];
                T = 0.5 * mi * (v0 * v0 + v1 * v1 + v2 * v2);
                Wi = -0.5 * P.G * mi * W;
            }
            for (int o = 16; o > 0; o >>= 1) {
                T += __shfl_xor_sync(0xffffffffu, T, o);
                Wi += __shfl_xor_sync(0xffffffffu, Wi, o);
            }
            if ((threadIdx.x & 31) == 0) {
                red[0][threadIdx.x >> 5] = T;
                red[1][threadIdx.x >> 5] = Wi;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double tT = 0.0, tW = 0.0;
                for (int k = 0; k < EN_THREADS / 32; ++k) {
                    tT += red[0][k];
                    tW += red[1][k];
                }
                atomicAdd(&out[2 * ch.sys], tT);
                atomicAdd(&out[2 * ch.sys + 1], tW);
            }
            __syncthreads();
        }
    }
}

StatePtrs state_ptrs(hybrid_ctx *c)
{
    StatePtrs w;
    for (int f = 0; f < 7; ++f) w.x[f] = (double *)c->x[f].p;
    w.id = (int32_t *)c->id.p;
    w.orig = (int32_t *)c->orig.p;
    w.psys = (int32_t *)c->psys.p;
    for (int d = 0; d < 3; ++d) {
        w.as[d] = c->acc_s[d].p;
        w.ah[d] = c->acc_h[d].p;
    }
    w.phi = (float4 *)c->phi.p;
    w.plo = (float4 *)c->plo.p;
    w.disp = (float *)c->disp.p;
    w.box = (const SysBox *)c->box.p;
    return w;
}

}  // namespace

static int grid_n(hybrid_ctx *c, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)c->nsm * 8));
}

void launch_copy_in(hybrid_ctx *c, const SysIO *d_io, bool with_acc)
{
    k_copy_in<<<grid_n(c, c->N), 256, 0, c->st>>>(c->N, c->S, (const int64_t *)c->off_dev.p, d_io, state_ptrs(c),
                                                   c->p.precision, with_acc ? 1 : 0);
    c->launches++;
}

void launch_copy_out(hybrid_ctx *c, const SysIO *d_io, bool state, bool acc_s, bool acc_h)
{
    k_copy_out<<<grid_n(c, c->N), 256, 0, c->st>>>(c->N, (const int32_t *)c->psys.p, d_io, state_ptrs(c),
                                                    c->p.precision, state, acc_s, acc_h, status_dev(c));
    c->launches++;
}

void launch_kick_seq(hybrid_ctx *c, int n, const int *which, const int *mode, const double *val, int dmode,
                     double dval, bool resplit)
{
    KickSpec ks;
    ks.resplit = resplit && dmode >= 0 && c->p.precision == 1 && c->p.skin > 0.0;
    ks.where = c->op;
    ks.n = n;
    for (int k = 0; k < 4; ++k) {
        ks.which[k] = k < n ? which[k] : 0;
        ks.mode[k] = k < n ? mode[k] : 0;
        ks.val[k] = k < n ? val[k] : 0.0;
    }
    ks.dmode = dmode;
    ks.dval = dval;
    const int64_t N = c->N;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)c->nsm * 8));
    cudaEvent_t e0 = nullptr;
    prof_begin(c, PROF_INTEG, &e0);
    if (c->p.precision == 1)
        k_kick_drift<float><<<grid, 256, 0, c->st>>>(N, state_ptrs(c), (const SysParams *)c->sp_dev.p, ks,
                                                      status_dev(c));
    else
        k_kick_drift<double><<<grid, 256, 0, c->st>>>(N, state_ptrs(c), (const SysParams *)c->sp_dev.p, ks,
                                                       status_dev(c));
    prof_end(c, PROF_INTEG, e0);
    c->launches++;
}

void launch_kick_ext(hybrid_ctx *c, const hybrid_system *s, int which, double h)
{
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((s->n + 255) / 256, (int64_t)c->nsm * 8));
    void *ax = which ? s->ax_h : s->ax_s, *ay = which ? s->ay_h : s->ay_s, *az = which ? s->az_h : s->az_s;
    if (c->p.precision == 1)
        k_kick_ext<float><<<grid, 256, 0, c->st>>>(s->n, s->vx, s->vy, s->vz, (const float *)ax, (const float *)ay,
                                                    (const float *)az, h);
    else
        k_kick_ext<double><<<grid, 256, 0, c->st>>>(s->n, s->vx, s->vy, s->vz, (const double *)ax,
                                                     (const double *)ay, (const double *)az, h);
    c->launches++;
}

void launch_drift_ext(hybrid_ctx *c, const hybrid_system *s, double dt)
{
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((s->n + 255) / 256, (int64_t)c->nsm * 8));
    k_drift_ext<<<grid, 256, 0, c->st>>>(s->n, s->x, s->y, s->z, s->vx, s->vy, s->vz, dt);
    c->launches++;
}

void launch_energy(hybrid_ctx *c, double *d_out)
{
    cudaMemsetAsync(d_out, 0, (size_t)2 * c->S * sizeof(double), c->st);
    const int sub = c->tile / EN_THREADS;
    k_energy<<<std::min(c->nchunks * sub, c->nsm * 8), EN_THREADS, 0, c->st>>>(
        (const Chunk *)c->chunks_dev.p, c->nchunks, sub, (const int64_t *)c->off_dev.p, state_ptrs(c),
        (const SysParams *)c->sp_dev.p, d_out);
    c->launches++;
}

}  // namespace hy
