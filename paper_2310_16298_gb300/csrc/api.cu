// Host runtime behind include/stencil.h: plans, the time loop, asynchronous
// submission, batches and error norms.  Every step of a sweep runs in the
// library's own CUDA kernels; there is no host fallback.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/stencil.h"
#include "common.cuh"
#include "kernels.h"
#include "mx.h"
#include "plan.h"
#include "runtime.h"

using namespace stx;

namespace stx {

thread_local std::string g_err;

stencil_status fail(stencil_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

stencil_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return STENCIL_ECUDA;
}

const std::string& last_error_string() { return g_err; }

GatherProblem gather_problem(const stencil_plan_s* p) {
    GatherProblem g;
    g.ndim = p->ndim;
    for (int d = 0; d < 3; ++d) g.n[d] = p->n[d];
    g.r = p->r;
    g.star = p->star;
    g.f64 = p->f64;
    g.bc = p->bc;
    g.cg = p->cg.data();
    g.err = p->err_dev;
    g.ldx = p->ldx;
    return g;
}

// One sweep of depth `tb` from src to dst.
cudaError_t run_sweep(const stencil_plan_s* p, const void* src, void* dst, int tb, cudaStream_t s) {
    if (p->impl == STENCIL_IMPL_MATRIXIZED) return mx_sweep(*p->mx, src, dst, tb, s);
    GatherProblem g = gather_problem(p);
    return gather_sweep(g, src, dst, tb, s);
}

// Time loop (Sec. 2.2: two grid copies used alternately).  The copies are the
// caller's output and the plan's scratch grid, ordered so that the last
// sweep writes d_out and no sweep reads the buffer it writes.
// Strided copy between the caller's layout (row stride pitch) and the padded
// layout of a repacking plan (row stride ldx).
cudaError_t repack_copy(const stencil_plan_s* p, void* dst, int64_t dld, const void* src, int64_t sld, cudaStream_t s) {
    const size_t es = p->f64 ? 8 : 4;
    const size_t rows = (size_t)(p->points / p->n[p->ndim - 1]);
    return cudaMemcpy2DAsync(dst, (size_t)dld * es, src, (size_t)sld * es, (size_t)p->n[p->ndim - 1] * es, rows,
                             cudaMemcpyDeviceToDevice, s);
}

stencil_status time_loop(const stencil_plan_s* p, const void* d_in, void* d_out, int64_t steps,
                         cudaStream_t s, void* scratch) {
    if (steps > 0 && p->repack) {
        // the field goes into the plan's padded grids, is advanced there and comes back
        void* g[2] = {p->pad, p->scratch};
        cudaError_t e = repack_copy(p, g[0], p->ldx, d_in, p->pitch, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync");
        const int tb = p->tb;
        const int64_t nsweep = (steps + tb - 1) / tb;
        for (int64_t k = 0; k < nsweep; ++k) {
            const int depth = (int)((k == nsweep - 1) ? (steps - (nsweep - 1) * tb) : tb);
            e = run_sweep(p, g[k & 1], g[(k + 1) & 1], depth, s);
            if (e != cudaSuccess) return cuda_fail(e, "stencil sweep launch");
        }
        e = repack_copy(p, d_out, p->pitch, g[nsweep & 1], p->ldx, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync");
        return STENCIL_OK;
    }
    if (steps == 0) {
        if (d_in != d_out) {
            cudaError_t e = cudaMemcpyAsync(d_out, d_in, p->grid_bytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        }
        return STENCIL_OK;
    }
    const int tb = p->tb;
    const int64_t nsweep = (steps + tb - 1) / tb;
    const void* src = d_in;
    if (d_in == d_out && (nsweep & 1)) {
        cudaError_t e = cudaMemcpyAsync(scratch, d_in, p->grid_bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        src = scratch;
    }
    for (int64_t k = 0; k < nsweep; ++k) {
        const int64_t left = nsweep - 1 - k;  // sweeps after this one
        void* dst = (left & 1) ? scratch : d_out;
        const int depth = (int)((k == nsweep - 1) ? (steps - (nsweep - 1) * tb) : tb);
        cudaError_t e = run_sweep(p, src, dst, depth, s);
        if (e != cudaSuccess) return cuda_fail(e, "stencil sweep launch");
        src = dst;
    }
    return STENCIL_OK;
}

unsigned int plan_error_bits(const stencil_plan_s* p) {
    unsigned int w = *(volatile const unsigned int*)&p->host_error;
    if (p->mx) w |= mx_device_error(*p->mx);
    if (p->err_host) w |= *(volatile const unsigned int*)p->err_host;
    return w;
}

stencil_status plan_error_status(const stencil_plan_s* p, const char* where) {
    const unsigned int w = plan_error_bits(p);
    if (!w) return STENCIL_OK;
    char buf[64];
    snprintf(buf, sizeof(buf), "0x%x", w);
    return fail(STENCIL_ECUDA, std::string(where) + ": a kernel of this plan gave up a bounded wait (error bits " +
                                   buf + "); the plan's results since then are not valid: destroy the plan");
}

}  // namespace stx

namespace {

// ----------------------------------------------------------------- live plans
// Tickets name their plan by id, so a poll after the plan was destroyed finds
// no plan instead of a dangling pointer.
std::mutex g_plans_mu;
std::unordered_map<uint64_t, stencil_plan_s*> g_plans;
uint64_t g_next_plan_id = 1;

void plan_register(stencil_plan_s* p) {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    p->id = g_next_plan_id++;
    g_plans[p->id] = p;
}

void plan_unregister(stencil_plan_s* p) {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    g_plans.erase(p->id);
}

// Error status of the plan with this id once its work has completed (OK when
// the plan no longer exists).
stencil_status plan_error_status_by_id(uint64_t id, const char* where) {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    auto it = g_plans.find(id);
    if (it == g_plans.end()) return STENCIL_OK;
    return plan_error_status(it->second, where);
}

// ----------------------------------------------------------------- tickets
struct Ticket {
    cudaEvent_t ev;
    uint64_t plan_id;
};
std::mutex g_tk_mu;
std::unordered_map<uint64_t, Ticket> g_tickets;
std::vector<cudaEvent_t> g_event_pool;
uint64_t g_next_ticket = 1;

stencil_status ticket_status(uint64_t ticket, Ticket* t) {
    std::lock_guard<std::mutex> lk(g_tk_mu);
    auto it = g_tickets.find(ticket);
    if (it == g_tickets.end()) return fail(STENCIL_EINVAL, "unknown or already released ticket");
    *t = it->second;
    return STENCIL_OK;
}

void ticket_release(uint64_t ticket) {
    std::lock_guard<std::mutex> lk(g_tk_mu);
    auto it = g_tickets.find(ticket);
    if (it != g_tickets.end()) {
        g_event_pool.push_back(it->second.ev);
        g_tickets.erase(it);
    }
}

// Status of a ticket whose event has completed with `e`.
stencil_status ticket_done(uint64_t ticket, const Ticket& t, cudaError_t e) {
    ticket_release(ticket);
    if (e != cudaSuccess) return cuda_fail(e, "submitted work");
    return plan_error_status_by_id(t.plan_id, "submitted work");
}

}  // namespace

// =================================================================== plans
namespace {

// Free everything a plan (complete or half-built) owns.
void plan_free(stencil_plan_s* p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->scratch) cudaFree(p->scratch);
    if (p->staging) cudaFree(p->staging);
    if (p->pad) cudaFree(p->pad);
    if (p->err_host) cudaFreeHost(p->err_host);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (p->mx) {
        mx_plan_free(p->mx);
        delete p->mx;
    }
    delete p;
}

struct PlanFree {
    void operator()(stencil_plan_s* p) const { plan_free(p); }
};

// ----------------------------------------------------------------- cover choice
// The covers of a 3D star (all lines on the tensor cores, or the contiguous-
// axis line there and the off-axis weights on the CUDA cores) trade MMA work
// against epilogue work differently for each order, precision and grid size
// (Sec. 5.2 measured the same trade on the paper's machine).  The plan times
// one sweep of each on its own grids and keeps the faster; the result is
// cached per order, precision, boundary and grid size class.
std::mutex g_cover_mu;
std::map<std::tuple<int, int, int, int>, int> g_cover_cache;

// Mean time of three sweeps (after one untimed) of a matrixized plan, in ms;
// negative when a launch failed.
float time_mx_sweeps(const MxPlan& m, const void* src, void* dst, cudaStream_t s) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        cudaGetLastError();
        return -1.f;
    }
    float ms = -1.f;
    bool ok = mx_sweep(m, src, dst, 1, s) == cudaSuccess && cudaEventRecord(a, s) == cudaSuccess;
    for (int k = 0; k < 3 && ok; ++k) ok = mx_sweep(m, src, dst, 1, s) == cudaSuccess;
    if (ok && cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, a, b) == cudaSuccess && mx_device_error(m) == 0)
        ms /= 3.f;
    else
        ms = -1.f;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGetLastError();
    return ms;
}

int pick_star_cover(const MxRequest& base, size_t grid_bytes, void* scratch, cudaStream_t s) {
    int64_t pts = base.n[0] * base.n[1] * base.n[2];
    int lg = 0;
    while ((int64_t)1 << (lg + 1) <= pts) ++lg;
    const auto key = std::make_tuple(base.r, base.prec, base.bc, lg);
    {
        std::lock_guard<std::mutex> lk(g_cover_mu);
        auto it = g_cover_cache.find(key);
        if (it != g_cover_cache.end()) return it->second;
    }
    int best = STENCIL_COVER_HYBRID;
    void* tmp = nullptr;
    if (cudaMalloc(&tmp, grid_bytes) != cudaSuccess) {
        cudaGetLastError();
        return best;   // no room to time: the default, not cached
    }
    float best_t = 0.f;
    for (int cover : {STENCIL_COVER_PARALLEL, STENCIL_COVER_HYBRID}) {
        MxRequest q = base;
        q.cover = cover;
        std::string why;
        if (!mx_supported(q, &why)) continue;
        MxPlan m;
        if (mx_plan_build(q, &m, &why) != STENCIL_OK) continue;
        const float t = time_mx_sweeps(m, scratch, tmp, s);
        mx_plan_free(&m);
        if (t > 0.f && (best_t == 0.f || t < best_t)) {
            best_t = t;
            best = cover;
        }
    }
    cudaFree(tmp);
    if (best_t > 0.f) {
        std::lock_guard<std::mutex> lk(g_cover_mu);
        g_cover_cache[key] = best;
    }
    return best;
}

}  // namespace

extern "C" stencil_status stencil_plan_create(stencil_plan_t* out, int ndim, const int64_t* shape,
                                              int radius, stencil_kind kind, const double* coeffs,
                                              stencil_dtype dtype, const stencil_options* opt) {
    if (!out) return fail(STENCIL_EINVAL, "out is NULL");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(STENCIL_EINVAL, "ndim must be 2 or 3");
    if (radius < 1 || radius > kMaxRadius) return fail(STENCIL_EINVAL, "radius must be in 1..4");
    if (!shape || !coeffs) return fail(STENCIL_EINVAL, "shape or coeffs is NULL");
    if (kind != STENCIL_STAR && kind != STENCIL_BOX) return fail(STENCIL_EINVAL, "kind must be STAR or BOX");
    if (dtype != STENCIL_F32 && dtype != STENCIL_F64) return fail(STENCIL_EINVAL, "dtype must be F32 or F64");
    stencil_options o{};
    if (opt) o = *opt;
    if (o.bc != STENCIL_BC_DIRICHLET_ZERO && o.bc != STENCIL_BC_PERIODIC)
        return fail(STENCIL_EINVAL, "bc must be DIRICHLET_ZERO or PERIODIC");
    if (o.impl < STENCIL_IMPL_AUTO || o.impl > STENCIL_IMPL_MATRIXIZED)
        return fail(STENCIL_EINVAL, "impl out of range");
    if (o.tb < 0 || o.tb > 16) return fail(STENCIL_EINVAL, "tb must be in 0..16");
    if (o.cover < STENCIL_COVER_AUTO || o.cover > STENCIL_COVER_HYBRID)
        return fail(STENCIL_EINVAL, "cover out of range");
    const int64_t es = (dtype == STENCIL_F64) ? 8 : 4;
    if (o.pitch < 0) return fail(STENCIL_EINVAL, "pitch must be >= 0");
    if (o.unit_planes < 0 || o.unit_planes > 1024) return fail(STENCIL_EINVAL, "unit_planes must be in 0..1024");
    if (o.pitch > 0 && (o.pitch < shape[ndim - 1] || (o.pitch * es) % 16 != 0))
        return fail(STENCIL_EINVAL, "pitch must be at least the contiguous extent and give 16-byte rows");
    const int W = 2 * radius + 1;
    int64_t nco = 1, points = 1;
    for (int d = 0; d < ndim; ++d) {
        if (shape[d] < W) return fail(STENCIL_EINVAL, "every extent must be at least 2*radius+1");
        if (shape[d] > (int64_t)1 << 31) return fail(STENCIL_EINVAL, "extent too large");
        nco *= W;
        points *= shape[d];
    }
    for (int64_t i = 0; i < nco; ++i)
        if (!std::isfinite(coeffs[i])) return fail(STENCIL_EINVAL, "coefficients must be finite");
    if (kind == STENCIL_STAR) {
        for (int64_t t = 0; t < nco; ++t) {
            int64_t rem = t;
            int off = 0;
            for (int d = ndim - 1; d >= 0; --d) {
                off += (rem % W) != radius;
                rem /= W;
            }
            if (off > 1 && coeffs[t] != 0.0)
                return fail(STENCIL_EINVAL, "a STAR stencil must have zero off-axis coefficients");
        }
    }
    const bool f64 = (dtype == STENCIL_F64);
    const int prec = o.prec;
    if (prec < STENCIL_PREC_NATIVE || prec > STENCIL_PREC_BF16_W2) return fail(STENCIL_EINVAL, "prec out of range");
    if (f64 && prec != STENCIL_PREC_NATIVE) return fail(STENCIL_EINVAL, "TF32/BF16 precisions need F32 storage");
    if (o.impl == STENCIL_IMPL_GATHER && prec != STENCIL_PREC_NATIVE)
        return fail(STENCIL_EINVAL, "the gather kernel computes in the storage type (prec NATIVE)");

    std::unique_ptr<stencil_plan_s, PlanFree> p(new stencil_plan_s);
    p->ndim = ndim;
    for (int d = 0; d < ndim; ++d) p->n[d] = shape[d];
    p->r = radius;
    p->star = (kind == STENCIL_STAR);
    p->f64 = f64;
    p->bc = o.bc;
    p->cg.assign(coeffs, coeffs + nco);
    p->points = points;
    const int64_t nlast = shape[ndim - 1];
    p->pitch = o.pitch > 0 ? o.pitch : nlast;
    p->grid_bytes = (size_t)(points / nlast) * (size_t)p->pitch * (size_t)es;
    p->ldx = p->pitch;

    // Implementation choice.  For the outer-product kernels, NATIVE means the
    // FP32-accuracy split (TF32X3); FP64 runs on the CUDA-core kernel.
    std::string why;
    MxRequest req;
    req.ndim = ndim;
    for (int d = 0; d < 3; ++d) req.n[d] = p->n[d];
    req.r = radius;
    req.star = p->star;
    req.f64 = f64;
    req.bc = o.bc;
    req.cg = p->cg.data();
    req.prec = (prec == STENCIL_PREC_NATIVE) ? STENCIL_PREC_TF32X3 : prec;
    req.tb = o.tb;
    req.unit_planes = o.unit_planes;
    // The tensor-core kernels stage rows with TMA, which needs 16-byte rows:
    // packed grids whose rows are not run on padded copies the plan owns.
    const bool aligned_rows = (p->pitch * es) % 16 == 0;
    req.ldx = aligned_rows ? p->pitch : (p->pitch + (16 / es) - 1) / (16 / es) * (16 / es);
    req.cover = o.cover;
    const bool mx_ok = (o.impl != STENCIL_IMPL_GATHER) && mx_supported(req, &why);
    const bool want_mx = (o.impl == STENCIL_IMPL_MATRIXIZED) || (prec != STENCIL_PREC_NATIVE);
    if (want_mx && !mx_ok) return fail(STENCIL_EUNSUPPORTED, "matrixized kernel not available: " + why);
    if (mx_ok) {
        p->impl = STENCIL_IMPL_MATRIXIZED;
        p->prec = req.prec;
        p->ldx = req.ldx;
        p->repack = !aligned_rows;
    } else {
        p->impl = STENCIL_IMPL_GATHER;
        p->prec = STENCIL_PREC_NATIVE;
    }

    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    // scratch: the second grid of the ping-pong (padded like the kernels' grids
    // when the plan repacks, and then with a first padded grid beside it)
    p->pad_bytes = (size_t)(points / nlast) * (size_t)p->ldx * (size_t)es;
    e = cudaMalloc(&p->scratch, p->repack ? p->pad_bytes : p->grid_bytes);
    if (e == cudaSuccess && p->repack) e = cudaMalloc(&p->pad, p->pad_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(STENCIL_ENOMEM, std::string("scratch grid: ") + cudaGetErrorString(e));
    }
    e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        p->stream = nullptr;
        return cuda_fail(e, "cudaStreamCreate");
    }

    // Temporal blocking depth.
    if (p->impl == STENCIL_IMPL_GATHER) {
        e = cudaHostAlloc((void**)&p->err_host, sizeof(unsigned int), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&p->err_dev, p->err_host, 0);
        if (e != cudaSuccess) return cuda_fail(e, "error word");
        *p->err_host = 0;
        p->tb = o.tb > 0 ? o.tb : 1;
        GatherProblem g = gather_problem(p.get());
        int max_smem = 0;
        e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        if (gather_smem_bytes(g, p->tb) > (size_t)max_smem)
            return fail(STENCIL_EUNSUPPORTED, "temporal block depth too large for shared memory");
    } else {
        if (ndim == 3 && p->star && o.cover == STENCIL_COVER_AUTO)
            req.cover = pick_star_cover(req, p->repack ? p->pad_bytes : p->grid_bytes, p->scratch, p->stream);
        p->mx = new MxPlan();
        stencil_status st = mx_plan_build(req, p->mx, &why);
        if (st != STENCIL_OK) {
            delete p->mx;
            p->mx = nullptr;
            return fail(st, "matrixized plan: " + why);
        }
        p->tb = p->mx->tb;
    }
    plan_register(p.get());
    *out = p.release();
    return STENCIL_OK;
}

extern "C" stencil_status stencil_plan_destroy(stencil_plan_t p) {
    if (!p) return STENCIL_OK;
    plan_unregister(p);
    plan_free(p);
    return STENCIL_OK;
}

extern "C" stencil_status stencil_plan_info(stencil_plan_t p, stencil_plan_info_t* info) {
    if (!p || !info) return fail(STENCIL_EINVAL, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->impl = p->impl;
    info->prec = p->prec;
    info->tb = p->tb;
    info->scratch_bytes = (int64_t)(p->repack ? 2 * p->pad_bytes : p->grid_bytes) +
                          (p->mx ? (int64_t)p->mx->operand_bytes : 0);
    if (p->mx) {
        info->n_lines = p->mx->n_lines;
        info->n_scalar = p->mx->n_scalar;
        info->tile_n = p->mx->nb;
        info->cover = p->mx->cover;
    }
    info->kernels_per_sweep = p->mx && p->mx->n_edge_terms > 0 ? 2 : 1;
    info->device_error = (int32_t)plan_error_bits(p);
    return STENCIL_OK;
}

extern "C" stencil_status stencil_plan_raise_error(stencil_plan_t p, uint32_t bits) {
    if (!p) return fail(STENCIL_EINVAL, "NULL plan");
    if (!bits) return fail(STENCIL_EINVAL, "bits must be nonzero");
    __atomic_fetch_or(&p->host_error, bits, __ATOMIC_SEQ_CST);
    return STENCIL_OK;
}

// =================================================================== sweeps
extern "C" stencil_status stencil_apply(stencil_plan_t p, const void* d_in, void* d_out, int64_t steps,
                                        stencil_stream_t stream) {
    if (!p || !d_in || !d_out) return fail(STENCIL_EINVAL, "NULL argument");
    if (steps < 0) return fail(STENCIL_EINVAL, "steps must be >= 0");
    stencil_status st = plan_error_status(p, "stencil_apply");
    if (st != STENCIL_OK) return st;
    return time_loop(p, d_in, d_out, steps, (cudaStream_t)stream, p->scratch);
}

// The field goes to the plan's staging grid, is advanced there in place (the
// time loop ping-pongs through the plan's scratch grid) and comes back: one
// device grid beyond the plan's own, allocated by the first call.
extern "C" stencil_status stencil_apply_host(stencil_plan_t p, const void* h_in, void* h_out, int64_t steps) {
    if (!p || !h_in || !h_out) return fail(STENCIL_EINVAL, "NULL argument");
    if (steps < 0) return fail(STENCIL_EINVAL, "steps must be >= 0");
    stencil_status st = plan_error_status(p, "stencil_apply_host");
    if (st != STENCIL_OK) return st;
    cudaError_t e;
    if (!p->staging) {
        e = cudaMalloc(&p->staging, p->grid_bytes);
        if (e != cudaSuccess) {
            p->staging = nullptr;
            cudaGetLastError();
            return fail(STENCIL_ENOMEM, std::string("staging grid: ") + cudaGetErrorString(e));
        }
    }
    e = cudaMemcpyAsync(p->staging, h_in, p->grid_bytes, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "H2D copy");
    if (st == STENCIL_OK) st = time_loop(p, p->staging, p->staging, steps, p->stream, p->scratch);
    if (st == STENCIL_OK) {
        e = cudaMemcpyAsync(h_out, p->staging, p->grid_bytes, cudaMemcpyDeviceToHost, p->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "D2H copy");
    }
    e = cudaStreamSynchronize(p->stream);
    if (st == STENCIL_OK && e != cudaSuccess) st = cuda_fail(e, "stencil_apply_host");
    if (st == STENCIL_OK) st = plan_error_status(p, "stencil_apply_host");
    return st;
}

// =================================================================== no-allocation apply
//
// A second way to run stencil_apply for callers that must not allocate device
// memory while they step a field: for example code running inside another
// runtime's stream-ordered work, a process whose device memory is budgeted
// once at start-up, or a real-time loop where cudaMalloc's implicit
// synchronisation is not acceptable.  The ping-pong copy lives in this
// file-scope device array instead of the plan's scratch grid.  Every GPU that
// loads the library holds the array until the process exits.

static constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB: 4 Mi FP32 or 2 Mi FP64 points
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
stencil_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(STENCIL_EUNSUPPORTED, "device ordinal beyond the no-allocation table");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return STENCIL_OK;
}

}  // namespace

extern "C" stencil_status stencil_apply_noalloc(stencil_plan_t p, const void* d_in, void* d_out, int64_t steps,
                                                stencil_stream_t stream) {
    if (!p || !d_in || !d_out) return fail(STENCIL_EINVAL, "NULL argument");
    if (steps < 0) return fail(STENCIL_EINVAL, "steps must be >= 0");
    if (p->repack)
        return fail(STENCIL_EINVAL, "stencil_apply_noalloc: rows that are not 16-byte multiples run on the plan's "
                                    "padded grids; use stencil_apply or pass a pitch");
    if (p->grid_bytes > kNoAllocScratchBytes)
        return fail(STENCIL_EINVAL, "grid of " + std::to_string(p->grid_bytes) +
                                        " bytes exceeds the 16 MiB static scratch of stencil_apply_noalloc");
    stencil_status st = plan_error_status(p, "stencil_apply_noalloc");
    if (st != STENCIL_OK) return st;
    void* scratch = nullptr;
    st = noalloc_scratch(&scratch);
    if (st != STENCIL_OK) return st;
    return time_loop(p, d_in, d_out, steps, (cudaStream_t)stream, scratch);
}

// =================================================================== async
extern "C" stencil_status stencil_submit(stencil_plan_t p, const void* d_in, void* d_out, int64_t steps,
                                         uint64_t* ticket) {
    if (!p || !d_in || !d_out || !ticket) return fail(STENCIL_EINVAL, "NULL argument");
    if (steps < 0) return fail(STENCIL_EINVAL, "steps must be >= 0");
    stencil_status st = plan_error_status(p, "stencil_submit");
    if (st != STENCIL_OK) return st;
    st = time_loop(p, d_in, d_out, steps, p->stream, p->scratch);
    if (st != STENCIL_OK) return st;
    cudaEvent_t ev = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_tk_mu);
        if (!g_event_pool.empty()) {
            ev = g_event_pool.back();
            g_event_pool.pop_back();
        }
    }
    cudaError_t e = cudaSuccess;
    if (!ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    e = cudaEventRecord(ev, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    std::lock_guard<std::mutex> lk(g_tk_mu);
    *ticket = g_next_ticket++;
    g_tickets[*ticket] = Ticket{ev, p->id};
    return STENCIL_OK;
}

extern "C" stencil_status stencil_poll(uint64_t ticket) {
    Ticket t;
    stencil_status st = ticket_status(ticket, &t);
    if (st != STENCIL_OK) return st;
    cudaError_t e = cudaEventQuery(t.ev);
    if (e == cudaErrorNotReady) return fail(STENCIL_ENOTREADY, "work not finished");
    return ticket_done(ticket, t, e);
}

extern "C" stencil_status stencil_wait(uint64_t ticket, int64_t timeout_ms) {
    Ticket t;
    stencil_status st = ticket_status(ticket, &t);
    if (st != STENCIL_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(t.ev);
        if (e != cudaErrorNotReady) return ticket_done(ticket, t, e);
        if (timeout_ms >= 0) {
            const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
                                 std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_ms) return fail(STENCIL_ETIMEDOUT, "wait timed out; work still queued");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

extern "C" const char* stencil_last_error(void) { return g_err.c_str(); }

// =================================================================== norms
extern "C" stencil_status stencil_error_norms(const void* d_got, stencil_dtype got_dtype, const double* d_ref,
                                              int64_t count, double* out, stencil_stream_t stream) {
    if (!d_got || !d_ref || !out) return fail(STENCIL_EINVAL, "NULL argument");
    if (count < 0) return fail(STENCIL_EINVAL, "count must be >= 0");
    if (got_dtype != STENCIL_F32 && got_dtype != STENCIL_F64) return fail(STENCIL_EINVAL, "bad dtype");
    double* scratch = nullptr;
    const size_t pb = norms_partials_bytes();
    cudaError_t e = cudaMalloc(&scratch, pb + 4 * sizeof(double));
    if (e != cudaSuccess) return fail(STENCIL_ENOMEM, "norm scratch");
    cudaStream_t s = (cudaStream_t)stream;
    e = error_norms(d_got, got_dtype == STENCIL_F64, d_ref, count, scratch,
                    scratch + pb / sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch + pb / sizeof(double), 4 * sizeof(double),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(e, "error norms");
    return STENCIL_OK;
}

// =================================================================== synthetic fields
extern "C" stencil_status stencil_fill_uniform(void* d_out, stencil_dtype dtype, int64_t count, uint64_t seed,
                                               int64_t offset, double lo, double hi, stencil_stream_t stream) {
    if (!d_out && count > 0) return fail(STENCIL_EINVAL, "NULL argument");
    if (count < 0 || offset < 0) return fail(STENCIL_EINVAL, "count and offset must be >= 0");
    if (dtype != STENCIL_F32 && dtype != STENCIL_F64) return fail(STENCIL_EINVAL, "bad dtype");
    cudaError_t e = fill_uniform(d_out, dtype == STENCIL_F64, count, seed, offset, lo, hi, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fill launch");
    return STENCIL_OK;
}

// =================================================================== host algebra
extern "C" stencil_status stencil_band_operand(int radius, const double* line, int n, int pad, double* band) {
    if (!line || !band) return fail(STENCIL_EINVAL, "NULL argument");
    if (radius < 1 || radius > kMaxRadius || n < 1 || pad < radius)
        return fail(STENCIL_EINVAL, "need 1 <= radius <= 4, n >= 1, pad >= radius");
    band_operand(radius, line, n, pad, band);
    return STENCIL_OK;
}

extern "C" stencil_status stencil_line_cover(int ndim, int radius, stencil_kind kind, int option, int n,
                                             int32_t* n_lines, int64_t* outer_products) {
    if (!n_lines || !outer_products) return fail(STENCIL_EINVAL, "NULL argument");
    if (ndim != 2 && ndim != 3) return fail(STENCIL_EINVAL, "ndim must be 2 or 3");
    if (radius < 1 || radius > kMaxRadius || n < 1) return fail(STENCIL_EINVAL, "bad radius or n");
    const int W = 2 * radius + 1;
    int64_t nco = 1;
    for (int d = 0; d < ndim; ++d) nco *= W;
    // Unit weights on the stencil's support: every point of a box, the axes of a star.
    std::vector<double> cg((size_t)nco, 0.0);
    for (int64_t t = 0; t < nco; ++t) {
        int64_t rem = t;
        int off = 0;
        for (int d = ndim - 1; d >= 0; --d) {
            off += (rem % W) != radius;
            rem /= W;
        }
        cg[(size_t)t] = (kind == STENCIL_BOX || off <= 1) ? 1.0 : 0.0;
    }
    // Parallel lines run along the axis the paper's tables use: i in 2D
    // (CLS(*,j)), j in 3D (CLS(i,*,k)).
    const int axis_par = (ndim == 2) ? 0 : 1;
    std::vector<CoefLine> lines;
    std::string why;
    if (!cover_lines(ndim, radius, kind == STENCIL_STAR, cg.data(), option, axis_par, &lines, &why))
        return fail(STENCIL_EINVAL, why);
    int64_t ops = 0;
    for (const auto& l : lines) ops += line_outer_products(l, n);
    *n_lines = (int32_t)lines.size();
    *outer_products = ops;
    return STENCIL_OK;
}

// Minimal axis-parallel line cover of a 2D weight pattern (Sec. 3.5): the
// rows and the columns of the weight matrix are the two vertex sets of a
// bipartite graph and every weight is an edge, so a minimal set of lines is a
// minimum vertex cover.  A maximum matching is grown by augmenting paths; by
// Konig's theorem the rows that the alternating paths from the unmatched rows
// do not reach, together with the columns they do reach, form a vertex cover
// with as many vertices as the matching has edges, hence a minimum one.
namespace {
constexpr int kMaxCoverSide = 64;

bool augment(int u, int n, const uint8_t* mask, std::vector<int>& row_of_col, std::vector<int>& col_of_row,
             std::vector<char>& seen) {
    for (int v = 0; v < n; ++v) {
        if (!mask[(size_t)u * n + v] || seen[v]) continue;
        seen[v] = 1;
        if (row_of_col[v] < 0 || augment(row_of_col[v], n, mask, row_of_col, col_of_row, seen)) {
            row_of_col[v] = u;
            col_of_row[u] = v;
            return true;
        }
    }
    return false;
}
}  // namespace

extern "C" stencil_status stencil_min_line_cover(int n, const uint8_t* mask, int32_t* rows, int32_t* cols,
                                                 int32_t* n_lines) {
    if (!mask || !rows || !cols || !n_lines) return fail(STENCIL_EINVAL, "NULL argument");
    if (n < 1 || n > kMaxCoverSide) return fail(STENCIL_EINVAL, "n must be in 1..64");
    std::vector<int> row_of_col(n, -1), col_of_row(n, -1);
    std::vector<char> seen(n);
    for (int u = 0; u < n; ++u) {
        std::fill(seen.begin(), seen.end(), 0);
        augment(u, n, mask, row_of_col, col_of_row, seen);
    }
    // Alternating paths from the unmatched rows: row -> column along any
    // weight, column -> row along its matching edge.
    std::vector<char> zr(n, 0), zc(n, 0);
    std::vector<int> todo;
    for (int u = 0; u < n; ++u)
        if (col_of_row[u] < 0) {
            zr[u] = 1;
            todo.push_back(u);
        }
    while (!todo.empty()) {
        const int u = todo.back();
        todo.pop_back();
        for (int v = 0; v < n; ++v) {
            if (!mask[(size_t)u * n + v] || zc[v]) continue;
            zc[v] = 1;
            const int w = row_of_col[v];
            if (w >= 0 && !zr[w]) {
                zr[w] = 1;
                todo.push_back(w);
            }
        }
    }
    int32_t count = 0;
    for (int i = 0; i < n; ++i) {
        rows[i] = zr[i] ? 0 : 1;
        cols[i] = zc[i] ? 1 : 0;
        count += rows[i] + cols[i];
    }
    *n_lines = count;
    return STENCIL_OK;
}

extern "C" const char* stencil_version(void) { return "stencil-gb300 0.1 (sm_103a)"; }
