// serve.cu -- continuous batching of independent simulations on one context.
//
// The method advances one system (or a fixed batch) per call; a server takes
// requests as they arrive and keeps every admitted one resident on the device
// between steps. Each hybrid_server_step
//   1. admits queued requests in arrival order while the device bytes charged
//      for them (HYBRID_SERVER_BYTES_PER_PARTICLE per particle: the request's
//      own arrays and its share of the context's working buffers) fit the
//      budget; a request's arrays are one stream-ordered allocation;
//   2. computes the first forces of the newly admitted requests (one batched
//      call with no step, so later steps start from valid forces, as a lone
//      run does);
//   3. advances every admitted request by one soft step (Sec. II-C) in one
//      batched call: every kernel launch covers all of them;
//   4. retires the requests whose steps are done: their state goes back to
//      the host copy the server keeps and their device arrays are freed.
// Requests are independent, so a request's result does not depend on the mix
// it ran in (bitwise in the FP64 form; to FP32 rounding order otherwise).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "../../include/hybrid.h"

namespace {

struct Request {
    int64_t tag = 0, n = 0;
    int32_t steps_left = 0;
    hybrid_params p;
    std::vector<double> h;   // x, y, z, vx, vy, vz, m back to back (n each): input, then result in key order
    std::vector<int32_t> hid;   // result: input index of each particle of h
    void *dev = nullptr;     // one block: 7 FP64 arrays, 6 acceleration arrays, id
    hybrid_system sys;
    double charge = 0.0;
};

}  // namespace

struct hybrid_server {
    hybrid_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    hybrid_params p;
    double budget = 0.0, used = 0.0;
    size_t acc_bytes = 4;
    std::deque<Request *> queued;
    std::vector<Request *> active;
    std::deque<Request *> finished;
    std::string err;
};

namespace {

void srv_err(hybrid_server *s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s->err = buf;
}

size_t dev_bytes(const hybrid_server *s, int64_t n)
{
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return 7 * up((size_t)n * 8) + 6 * up((size_t)n * s->acc_bytes) + up((size_t)n * 4);
}

void release(hybrid_server *s, Request *r)
{
    if (r->dev) cudaFreeAsync(r->dev, s->st);
    r->dev = nullptr;
    s->used -= r->charge;
    r->charge = 0.0;
}

// one batched call over the given requests; forces_valid is carried back
hybrid_status run_batch(hybrid_server *s, const std::vector<Request *> &rs, int steps)
{
    std::vector<hybrid_system> arr(rs.size());
    for (size_t k = 0; k < rs.size(); ++k) arr[k] = rs[k]->sys;
    hybrid_status r = hybrid_step_batched(s->ctx, arr.data(), (int)arr.size(), steps);
    for (size_t k = 0; k < rs.size(); ++k) rs[k]->sys.forces_valid = arr[k].forces_valid;
    if (r != HYBRID_OK) srv_err(s, "batched step: %s", hybrid_last_error(s->ctx));
    return r;
}

}  // namespace

extern "C" {

hybrid_status hybrid_server_create(hybrid_server **out, const hybrid_params *p, double budget_bytes, void *stream)
{
    if (!out || !p || !(budget_bytes > 0.0)) return HYBRID_EINVAL;
    *out = nullptr;
    hybrid_server *s = new hybrid_server();
    s->p = *p;
    s->st = (cudaStream_t)stream;
    s->budget = budget_bytes;
    s->acc_bytes = p->precision == 1 ? 4 : 8;
    hybrid_status r = hybrid_create(&s->ctx, p, stream);
    if (r != HYBRID_OK) {
        delete s;
        return r;
    }
    *out = s;
    return HYBRID_OK;
}

hybrid_status hybrid_server_destroy(hybrid_server *s)
{
    if (!s) return HYBRID_OK;
    cudaStreamSynchronize(s->st);
    for (Request *r : s->active) release(s, r), delete r;
    for (Request *r : s->queued) delete r;
    for (Request *r : s->finished) delete r;
    cudaStreamSynchronize(s->st);
    hybrid_destroy(s->ctx);
    delete s;
    return HYBRID_OK;
}

hybrid_status hybrid_server_submit(hybrid_server *s, int64_t tag, int64_t n, const double *x, const double *y,
                                   const double *z, const double *vx, const double *vy, const double *vz,
                                   const double *m, const hybrid_params *params, int32_t n_steps)
{
    if (!s || tag < 0 || n < 1 || n_steps < 1 || !x || !y || !z || !vx || !vy || !vz || !m) return HYBRID_EINVAL;
    if ((double)n * HYBRID_SERVER_BYTES_PER_PARTICLE > s->budget) {
        srv_err(s, "request %lld: %lld particles exceed the budget", (long long)tag, (long long)n);
        return HYBRID_ETOOLARGE;
    }
    Request *r = new Request();
    r->tag = tag;
    r->n = n;
    r->steps_left = n_steps;
    r->p = s->p;
    if (params) {   // per-request values of the fields a system may override
        r->p.G = params->G;
        r->p.eps = params->eps;
        r->p.theta = params->theta;
        r->p.R1 = params->R1;
        r->p.R2 = params->R2;
        r->p.dt_soft = params->dt_soft;
        r->p.a_err = params->a_err;
        r->p.mac = params->mac;
    }
    r->h.resize((size_t)7 * n);
    const double *src[7] = {x, y, z, vx, vy, vz, m};
    for (int f = 0; f < 7; ++f) memcpy(r->h.data() + (size_t)f * n, src[f], (size_t)n * sizeof(double));
    s->queued.push_back(r);
    return HYBRID_OK;
}

hybrid_status hybrid_server_step(hybrid_server *s, int32_t *n_active, int32_t *n_queued, int32_t *n_finished)
{
    if (!s) return HYBRID_EINVAL;
    // 1. admission, in arrival order, by charged bytes
    std::vector<Request *> fresh;
    while (!s->queued.empty()) {
        Request *r = s->queued.front();
        const double charge = (double)r->n * HYBRID_SERVER_BYTES_PER_PARTICLE;
        if (s->used + charge > s->budget) break;
        const size_t bytes = dev_bytes(s, r->n);
        if (cudaMallocAsync(&r->dev, bytes, s->st) != cudaSuccess) {
            cudaGetLastError();
            r->dev = nullptr;
            if (s->active.empty() && fresh.empty()) {
                srv_err(s, "device allocation of %zu bytes failed", bytes);
                return HYBRID_ENOMEM;
            }
            break;   // try again once others have left
        }
        char *b = (char *)r->dev;
        auto take = [&](size_t sz) {
            void *q = b;
            b += (sz + 255) / 256 * 256;
            return q;
        };
        double *st7[7];
        for (int f = 0; f < 7; ++f) {
            st7[f] = (double *)take((size_t)r->n * 8);
            cudaMemcpyAsync(st7[f], r->h.data() + (size_t)f * r->n, (size_t)r->n * 8, cudaMemcpyHostToDevice, s->st);
        }
        void *acc[6];
        for (int f = 0; f < 6; ++f) acc[f] = take((size_t)r->n * s->acc_bytes);
        int32_t *id = (int32_t *)take((size_t)r->n * 4);
        hybrid_system &y = r->sys;
        memset(&y, 0, sizeof y);
        y.n = r->n;
        y.x = st7[0];
        y.y = st7[1];
        y.z = st7[2];
        y.vx = st7[3];
        y.vy = st7[4];
        y.vz = st7[5];
        y.m = st7[6];
        y.id = id;
        y.ax_s = acc[0];
        y.ay_s = acc[1];
        y.az_s = acc[2];
        y.ax_h = acc[3];
        y.ay_h = acc[4];
        y.az_h = acc[5];
        y.params = &r->p;
        y.forces_valid = 0;
        r->charge = charge;
        s->used += charge;
        fresh.push_back(r);
        s->queued.pop_front();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        srv_err(s, "admission copies: %s", cudaGetErrorString(e));
        return HYBRID_ECUDA;
    }
    hybrid_status r = HYBRID_OK;
    // 2. first forces of the newly admitted requests
    if (!fresh.empty()) {
        for (Request *q : fresh) {   // labels 0..n-1 in input order (the state is kept in key order)
            std::vector<int32_t> ids((size_t)q->n);
            for (int64_t i = 0; i < q->n; ++i) ids[(size_t)i] = (int32_t)i;
            cudaMemcpyAsync(q->sys.id, ids.data(), (size_t)q->n * 4, cudaMemcpyHostToDevice, s->st);
            cudaStreamSynchronize(s->st);
        }
        r = run_batch(s, fresh, 0);
        s->active.insert(s->active.end(), fresh.begin(), fresh.end());
        if (r != HYBRID_OK) return r;
    }
    // 3. one soft step of every admitted request
    if (!s->active.empty()) {
        if ((r = run_batch(s, s->active, 1)) != HYBRID_OK) return r;
        // 4. retire the finished ones
        std::vector<Request *> keep;
        for (Request *q : s->active) {
            if (--q->steps_left > 0) {
                keep.push_back(q);
                continue;
            }
            const double *dst[7] = {q->sys.x, q->sys.y, q->sys.z, q->sys.vx, q->sys.vy, q->sys.vz, q->sys.m};
            for (int f = 0; f < 7; ++f)
                cudaMemcpyAsync(q->h.data() + (size_t)f * q->n, dst[f], (size_t)q->n * 8, cudaMemcpyDeviceToHost,
                                s->st);
            q->hid.resize((size_t)q->n);
            cudaMemcpyAsync(q->hid.data(), q->sys.id, (size_t)q->n * 4, cudaMemcpyDeviceToHost, s->st);
            release(s, q);
            s->finished.push_back(q);
        }
        s->active.swap(keep);
        if ((e = cudaStreamSynchronize(s->st)) != cudaSuccess) {
            srv_err(s, "retirement copies: %s", cudaGetErrorString(e));
            return HYBRID_ECUDA;
        }
    }
    if (n_active) *n_active = (int32_t)s->active.size();
    if (n_queued) *n_queued = (int32_t)s->queued.size();
    if (n_finished) *n_finished = (int32_t)s->finished.size();
    return HYBRID_OK;
}

hybrid_status hybrid_server_next(hybrid_server *s, int64_t *tag, int64_t *n, double *x, double *y, double *z,
                                 double *vx, double *vy, double *vz, double *m)
{
    if (!s || !tag || !n) return HYBRID_EINVAL;
    if (s->finished.empty()) {
        *tag = -1;
        *n = 0;
        return HYBRID_OK;
    }
    Request *r = s->finished.front();
    *tag = r->tag;
    *n = r->n;
    double *dst[7] = {x, y, z, vx, vy, vz, m};
    bool all = true, none = true;
    for (int f = 0; f < 7; ++f) {
        all = all && dst[f];
        none = none && !dst[f];
    }
    if (none) return HYBRID_OK;   // a peek
    if (!all) return HYBRID_EINVAL;
    for (int f = 0; f < 7; ++f) {   // back to the request's input order
        const double *src = r->h.data() + (size_t)f * r->n;
        for (int64_t k = 0; k < r->n; ++k) dst[f][r->hid[(size_t)k]] = src[k];
    }
    s->finished.pop_front();
    delete r;
    return HYBRID_OK;
}

double hybrid_server_used_bytes(hybrid_server *s) { return s ? s->used : 0.0; }

const char *hybrid_server_last_error(hybrid_server *s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
