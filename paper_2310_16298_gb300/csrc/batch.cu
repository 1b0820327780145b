// Batches of independent problems: one schedule of persistent launches that
// advances every problem by its own number of time steps, with the
// temporal-blocking depth chosen by timing candidates on the batch itself,
// and the whole launch sequence captured once in a CUDA graph.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "runtime.h"

using namespace stx;

struct stencil_batch_s {
    int n = 0;
    bool packed = false;  // one persistent kernel per launch (else per-problem sweeps)
    int tb = 1;
    int shape = 0;        // batch tile shape of the packed launches
    int launches = 0;
    int64_t tiles = 0;
    int64_t updates = 0;
    void* d_tables = nullptr;  // BatchProblem tables of every launch + coefficient rows
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const stencil_plan_s*> plans;  // error bits are checked at every launch
};

namespace {

struct Launch {
    size_t table_off;  // byte offset of its BatchProblem array in d_tables
    int nprob;
    int tiles;
    int max_depth;
};

struct Schedule {
    std::vector<BatchProblem> probs;  // all launches, concatenated
    std::vector<Launch> launches;
    std::vector<std::tuple<const void*, void*, size_t>> copies;  // done before the first launch
    int64_t tiles = 0;
};

// Per-problem ping-pong: sweep k of problem i goes from src to dst so that
// the last sweep writes d_out[i] and no sweep reads what it writes.
void build_schedule(int n, const stencil_plan_t* plans, const void* const* d_in, void* const* d_out,
                    const int64_t* steps, int tb, int shape, Schedule* S) {
    int ty = 0, tx = 0;
    gather_batch_tile_shape(shape, &ty, &tx);
    int64_t max_sweeps = 0;
    std::vector<int64_t> sweeps(n);
    std::vector<const void*> cur(n);
    for (int i = 0; i < n; ++i) {
        sweeps[i] = (steps[i] + tb - 1) / tb;
        max_sweeps = std::max(max_sweeps, sweeps[i]);
        cur[i] = d_in[i];
        if (steps[i] == 0) {
            if (d_in[i] != d_out[i]) S->copies.emplace_back(d_in[i], d_out[i], plans[i]->grid_bytes);
        } else if (d_in[i] == d_out[i] && (sweeps[i] & 1)) {
            S->copies.emplace_back(d_in[i], plans[i]->scratch, plans[i]->grid_bytes);
            cur[i] = plans[i]->scratch;
        }
    }
    for (int64_t k = 0; k < max_sweeps; ++k) {
        Launch L;
        L.table_off = S->probs.size() * sizeof(BatchProblem);
        L.nprob = 0;
        L.tiles = 0;
        L.max_depth = 1;
        for (int i = 0; i < n; ++i) {
            if (sweeps[i] <= k) continue;
            const stencil_plan_s* p = plans[i];
            const int64_t left = sweeps[i] - 1 - k;
            void* dst = (left & 1) ? p->scratch : d_out[i];
            BatchProblem b;
            memset(&b, 0, sizeof(b));
            b.src = cur[i];
            b.dst = dst;
            b.ny = (int)p->n[0];
            b.nx = (int)p->n[1];
            b.depth = (int)((k == sweeps[i] - 1) ? (steps[i] - (sweeps[i] - 1) * tb) : tb);
            b.bc = p->bc;
            b.tiles_x = (int)((p->n[1] + tx - 1) / tx);
            b.tile0 = L.tiles;
            b.coef_index = i;
            L.tiles += b.tiles_x * (int)((p->n[0] + ty - 1) / ty);
            L.max_depth = std::max(L.max_depth, b.depth);
            S->probs.push_back(b);
            ++L.nprob;
            cur[i] = dst;
        }
        S->tiles += L.tiles;
        S->launches.push_back(L);
    }
}

// Upload tables + coefficient rows (in the storage type) to one allocation.
stencil_status upload_tables(int n, const stencil_plan_t* plans, const Schedule& S, bool f64, void** out,
                             size_t* coef_off) {
    const int nc = (int)plans[0]->cg.size();
    const size_t tbytes = S.probs.size() * sizeof(BatchProblem);
    *coef_off = (tbytes + 255) / 256 * 256;
    const size_t es = f64 ? 8 : 4;
    const size_t total = *coef_off + (size_t)n * nc * es;
    std::vector<unsigned char> host(total, 0);
    if (tbytes) memcpy(host.data(), S.probs.data(), tbytes);
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < nc; ++c) {
            unsigned char* dst = host.data() + *coef_off + ((size_t)i * nc + c) * es;
            if (f64) {
                const double v = plans[i]->cg[c];
                memcpy(dst, &v, 8);
            } else {
                const float v = (float)plans[i]->cg[c];
                memcpy(dst, &v, 4);
            }
        }
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, total);
    if (e != cudaSuccess) return fail(STENCIL_ENOMEM, "batch tables");
    e = cudaMemcpy(d, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "batch table upload");
    }
    *out = d;
    return STENCIL_OK;
}

cudaError_t enqueue(const stencil_plan_s* p0, const Schedule& S, void* d_tables, size_t coef_off, int shape,
                    cudaStream_t s) {
    for (const auto& c : S.copies) {
        cudaError_t e = cudaMemcpyAsync(std::get<1>(c), std::get<0>(c), std::get<2>(c), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    for (const Launch& L : S.launches) {
        cudaError_t e = gather_batch_sweep(p0->f64, p0->star, p0->r,
                                           (const BatchProblem*)((char*)d_tables + L.table_off), L.nprob, L.tiles,
                                           (const char*)d_tables + coef_off, L.max_depth, shape, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Autotuner cache: (order, star, f64, log2 of the batch's points, fixed
// depth or 0, fixed shape or -1) -> (tile shape, depth).
std::mutex g_tune_mu;
std::map<std::tuple<int, bool, bool, int, int, int>, std::pair<int, int>> g_tune;

// Time one launch of the batch's first sweep for each candidate (tile shape,
// depth) pair -- the depth held when tb_fixed > 0, the shape when
// shape_fixed >= 0 -- (the outputs go to the plans' scratch grids, the inputs
// are only read) and keep the pair with the lowest time per time step.
std::pair<int, int> autotune(int n, const stencil_plan_t* plans, const void* const* d_in, const int64_t* steps,
                             int tb_fixed, int shape_fixed) {
    const stencil_plan_s* p0 = plans[0];
    int64_t pts = 0;
    for (int i = 0; i < n; ++i) pts += plans[i]->points;
    const auto key = std::make_tuple(p0->r, p0->star, p0->f64, (int)std::log2((double)std::max<int64_t>(pts, 1)),
                                     tb_fixed, shape_fixed);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    std::vector<void*> scratch_out(n);
    std::vector<int64_t> one(n);
    for (int i = 0; i < n; ++i) scratch_out[i] = plans[i]->scratch;
    std::pair<int, int> best{shape_fixed >= 0 ? shape_fixed : 0, tb_fixed > 0 ? tb_fixed : 1};
    double best_t = 1e30;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return best;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int s_lo = shape_fixed >= 0 ? shape_fixed : 0;
    const int s_hi = shape_fixed >= 0 ? shape_fixed : gather_batch_shapes() - 1;
    const int t_lo = tb_fixed > 0 ? tb_fixed : 1, t_hi = tb_fixed > 0 ? tb_fixed : 4;
    for (int shape = s_lo; shape <= s_hi; ++shape)
        for (int tb = t_lo; tb <= t_hi; ++tb) {
            if (gather_batch_smem_bytes(p0->f64, p0->r, tb, shape) > (size_t)max_smem) break;
            for (int i = 0; i < n; ++i) one[i] = std::min<int64_t>(steps[i], tb) > 0 ? tb : 0;
            Schedule S;
            build_schedule(n, plans, d_in, scratch_out.data(), one.data(), tb, shape, &S);
            S.copies.clear();
            void* d = nullptr;
            size_t coef_off = 0;
            if (upload_tables(n, plans, S, p0->f64, &d, &coef_off) != STENCIL_OK) break;
            float ms = 0.0f;
            bool ok = enqueue(p0, S, d, coef_off, shape, s) == cudaSuccess;  // warm-up
            ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
            for (int rep = 0; rep < 2 && ok; ++rep) ok = enqueue(p0, S, d, coef_off, shape, s) == cudaSuccess;
            ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            cudaFree(d);
            if (!ok) break;
            const double per_step = ms / (2.0 * tb);
            if (per_step < best_t) {
                best_t = per_step;
                best = {shape, tb};
            }
        }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    return best;
}

void batch_free(stencil_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_tables) cudaFree(b->d_tables);
    delete b;
}

}  // namespace

extern "C" stencil_status stencil_batch_create_ex(stencil_batch_t* out, int n, const stencil_plan_t* plans,
                                                  const void* const* d_in, void* const* d_out,
                                                  const int64_t* steps, int32_t tb, int32_t tile_shape) {
    if (!out) return fail(STENCIL_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1) return fail(STENCIL_EINVAL, "n must be >= 1");
    if (!plans || !d_in || !d_out || !steps) return fail(STENCIL_EINVAL, "NULL argument");
    if (tb < 0 || tb > 8) return fail(STENCIL_EINVAL, "tb must be in 0..8");
    if (tile_shape < -1 || tile_shape >= gather_batch_shapes())
        return fail(STENCIL_EINVAL, "tile_shape must be -1 or in 0.." + std::to_string(gather_batch_shapes() - 1));
    for (int i = 0; i < n; ++i)
        if (!plans[i] || !d_in[i] || !d_out[i] || steps[i] < 0)
            return fail(STENCIL_EINVAL, "invalid entry " + std::to_string(i));
    const stencil_plan_s* p0 = plans[0];
    // packed launches take 2D plans of one order, kind and dtype with packed rows
    bool packed = (p0->ndim == 2) && p0->r <= 3;
    for (int i = 0; i < n && packed; ++i) {
        const stencil_plan_s* p = plans[i];
        packed = p->ndim == 2 && p->r == p0->r && p->star == p0->star && p->f64 == p0->f64 && p->pitch == p->n[1];
    }
    std::unique_ptr<stencil_batch_s, void (*)(stencil_batch_s*)> b(new stencil_batch_s, batch_free);
    b->n = n;
    b->packed = packed;
    b->plans.assign(plans, plans + n);
    for (int i = 0; i < n; ++i) b->updates += plans[i]->points * steps[i];
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    Schedule S;
    size_t coef_off = 0;
    if (packed) {
        if (tile_shape >= 0 && tb > 0) {
            b->shape = tile_shape;
            b->tb = tb;
        } else {
            const std::pair<int, int> t = autotune(n, plans, d_in, steps, tb, tile_shape);
            b->shape = t.first;
            b->tb = t.second;
        }
        int dev = 0, max_smem = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (gather_batch_smem_bytes(p0->f64, p0->r, b->tb, b->shape) > (size_t)max_smem)
            return fail(STENCIL_EUNSUPPORTED, "temporal block depth too large for shared memory");
        build_schedule(n, plans, d_in, d_out, steps, b->tb, b->shape, &S);
        stencil_status st = upload_tables(n, plans, S, p0->f64, &b->d_tables, &coef_off);
        if (st != STENCIL_OK) return st;
        // set the kernel's attributes outside the capture (a launch of no tiles)
        e = gather_batch_sweep(p0->f64, p0->star, p0->r, (const BatchProblem*)b->d_tables, 0, 0, b->d_tables,
                               b->tb, b->shape, b->cap);
        if (e != cudaSuccess) return cuda_fail(e, "batched kernel set-up");
        b->launches = (int)S.launches.size();
        b->tiles = S.tiles;
    }
    // Capture the whole schedule once; stencil_batch_launch replays it.
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    stencil_status st = STENCIL_OK;
    if (packed) {
        e = enqueue(p0, S, b->d_tables, coef_off, b->shape, b->cap);
        if (e != cudaSuccess) st = cuda_fail(e, "batched sweep launch");
    } else {
        for (int i = 0; i < n && st == STENCIL_OK; ++i)
            st = time_loop(plans[i], d_in[i], d_out[i], steps[i], b->cap, plans[i]->scratch);
        b->launches = -1;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap, &graph);
    if (st != STENCIL_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b->graph = graph;
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    *out = b.release();
    return STENCIL_OK;
}

extern "C" stencil_status stencil_batch_create(stencil_batch_t* out, int n, const stencil_plan_t* plans,
                                               const void* const* d_in, void* const* d_out, const int64_t* steps,
                                               int32_t tb) {
    return stencil_batch_create_ex(out, n, plans, d_in, d_out, steps, tb, -1);
}

extern "C" stencil_status stencil_batch_launch(stencil_batch_t b, stencil_stream_t stream) {
    if (!b) return fail(STENCIL_EINVAL, "NULL batch");
    for (const stencil_plan_s* p : b->plans) {
        stencil_status st = plan_error_status(p, "stencil_batch_launch");
        if (st != STENCIL_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return STENCIL_OK;
}

extern "C" stencil_status stencil_batch_info(stencil_batch_t b, stencil_batch_info_t* info) {
    if (!b || !info) return fail(STENCIL_EINVAL, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->packed = b->packed ? 1 : 0;
    info->tb = b->tb;
    info->launches = b->launches;
    info->tile_shape = b->packed ? b->shape : -1;
    info->tiles = b->tiles;
    info->updates = b->updates;
    return STENCIL_OK;
}

extern "C" stencil_status stencil_batch_destroy(stencil_batch_t b) {
    if (!b) return STENCIL_OK;
    if (b->cap) cudaStreamSynchronize(b->cap);
    batch_free(b);
    return STENCIL_OK;
}

extern "C" stencil_status stencil_batch_run(int n, const stencil_plan_t* plans, const void* const* d_in,
                                            void* const* d_out, const int64_t* steps, stencil_stream_t stream) {
    if (n < 0) return fail(STENCIL_EINVAL, "n must be >= 0");
    if (n == 0) return STENCIL_OK;
    stencil_batch_t b = nullptr;
    stencil_status st = stencil_batch_create(&b, n, plans, d_in, d_out, steps, 0);
    if (st != STENCIL_OK) return st;
    st = stencil_batch_launch(b, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    stencil_batch_destroy(b);
    if (st == STENCIL_OK && e != cudaSuccess) st = cuda_fail(e, "batch run");
    for (int i = 0; i < n && st == STENCIL_OK; ++i) st = plan_error_status(plans[i], "stencil_batch_run");
    return st;
}
