// Batch driver: many independent solves (different trees, operator sets, right-hand sides) in
// one stream-ordered call that can be captured as a single CUDA graph. The paper solves one
// problem at a time; this is the serving-side counterpart.
//
// Schedule: the items are sorted by an estimate of their work and dealt to the side stream
// with the least work so far (longest processing time first). Every side stream is forked
// from the caller's stream by an event and joined back by another, so the whole batch is
// ordered after the caller's earlier work and before its later work, and a stream capture of
// the call records the concurrency as parallel branches of one graph.
#include <algorithm>
#include <numeric>
#include <vector>

#include "ops.cuh"
#include "vfmm_internal.cuh"

using namespace vfmm;

struct vfmm_batch {
    int n_streams = 0;  // created side streams
    int active = 0;     // side streams used by the next call (vfmm_batch_tune sets it)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};

namespace {

void destroy_batch(vfmm_batch* b) {
    for (cudaStream_t s : b->side)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// Work estimate of one item: near-field table applies plus the far-field translations.
double item_cost(const vfmm_batch_item& it) {
    const DeviceTree& T = it.tree->t;
    const double kk = (double)it.ops->k * it.ops->k, P = (double)it.ops->p + 1;
    return (double)it.nrhs * (6.0 * kk * kk * (double)T.llen[VFMM_LIST_U] + 8.0 * P * P * (double)T.llen[VFMM_LIST_V] +
                              16.0 * P * P * (double)T.n_boxes + 12.0 * kk * P * (double)T.n_leaves);
}

// assignment[i] = side stream of item i (LPT); order = items by descending cost.
void schedule(int n, const vfmm_batch_item* items, int S, std::vector<int>& order, std::vector<int>& assignment) {
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) cost[i] = item_cost(items[i]);
    order.resize(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(S, 0.0);
    assignment.assign(n, 0);
    for (int i : order) {
        int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        assignment[i] = s;
        load[s] += cost[i];
    }
}

int run_batch(vfmm_batch* b, int n, const vfmm_batch_item* items, int S, cudaStream_t st) {
    std::vector<int> order, assignment;
    schedule(n, items, S, order, assignment);
    VFMM_CUDA(cudaEventRecord(b->fork, st));
    for (int s = 0; s < S; ++s) VFMM_CUDA(cudaStreamWaitEvent(b->side[s], b->fork, 0));
    int rc = VFMM_OK;
    for (int i : order) {
        const vfmm_batch_item& it = items[i];
        // each item on its own side stream only: the batch's streams already run items side by side
        rc = volume_potential(it.tree, it.ops, it.f, it.nrhs, it.u, it.ux, it.uy, it.workspace, it.workspace_bytes,
                              b->side[assignment[i]], false);
        if (rc != VFMM_OK) break;
    }
    // join every side stream even after an error, so that a capture in progress stays well formed
    for (int s = 0; s < S; ++s) {
        cudaError_t e1 = cudaEventRecord(b->join[s], b->side[s]);
        cudaError_t e2 = cudaStreamWaitEvent(st, b->join[s], 0);
        if (rc == VFMM_OK && e1 != cudaSuccess) rc = cuda_fail(e1, "cudaEventRecord");
        if (rc == VFMM_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamWaitEvent");
    }
    return rc;
}

int check_items(int n, const vfmm_batch_item* items) {
    if (n < 0 || (n > 0 && !items)) return fail(VFMM_ERR_INVALID_ARG, "bad item list");
    for (int i = 0; i < n; ++i)
        if (!items[i].tree || !items[i].ops) return fail(VFMM_ERR_INVALID_ARG, "item without tree or ops");
    return VFMM_OK;
}

int capture(vfmm_batch* b, int n, const vfmm_batch_item* items, int S, cudaStream_t st, vfmm_graph** out) {
    vfmm_graph* g = new vfmm_graph();
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    int rc = run_batch(b, n, items, S, st);
    e = cudaStreamEndCapture(st, &g->graph);
    if (rc != VFMM_OK || e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc != VFMM_OK ? rc : cuda_fail(e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = g;
    return VFMM_OK;
}

}  // namespace

extern "C" int vfmm_batch_create(int32_t n_streams, vfmm_batch** out) {
    if (!out) return fail(VFMM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (n_streams < 1 || n_streams > VFMM_BATCH_MAX_STREAMS)
        return fail(VFMM_ERR_INVALID_ARG, "n_streams must be in [1, VFMM_BATCH_MAX_STREAMS]");
    vfmm_batch* b = new vfmm_batch();
    b->n_streams = b->active = n_streams;
    b->side.assign(n_streams, nullptr);
    b->join.assign(n_streams, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int s = 0; s < n_streams && e == cudaSuccess; ++s) {
        e = cudaStreamCreateWithFlags(&b->side[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy_batch(b);
        return cuda_fail(e, "creating batch streams");
    }
    *out = b;
    return VFMM_OK;
}

extern "C" int vfmm_batch_destroy(vfmm_batch* b) {
    if (b) destroy_batch(b);
    return VFMM_OK;
}

extern "C" int vfmm_batch_potential(vfmm_batch* b, int32_t n, const vfmm_batch_item* items, void* stream) {
    if (!b) return fail(VFMM_ERR_INVALID_ARG, "null batch");
    VFMM_CHECK(check_items(n, items));
    return run_batch(b, n, items, b->active, (cudaStream_t)stream);
}

extern "C" int vfmm_batch_graph_create(vfmm_batch* b, int32_t n, const vfmm_batch_item* items, void* stream,
                                       vfmm_graph** out) {
    if (!b || !out) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (st == nullptr) return fail(VFMM_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    VFMM_CHECK(check_items(n, items));
    // one ordinary run first: schedules and one-time kernel attributes are set outside the capture
    VFMM_CHECK(run_batch(b, n, items, b->active, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    return capture(b, n, items, b->active, st, out);
}

extern "C" int vfmm_batch_tune(vfmm_batch* b, int32_t n, const vfmm_batch_item* items, void* stream,
                               int32_t* best_streams, float* best_ms) {
    if (!b || !best_streams || !best_ms) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (st == nullptr) return fail(VFMM_ERR_INVALID_ARG, "tuning needs a non-default stream");
    VFMM_CHECK(check_items(n, items));
    VFMM_CHECK(run_batch(b, n, items, b->n_streams, st));
    VFMM_CUDA(cudaStreamSynchronize(st));
    cudaEvent_t e0, e1;
    VFMM_CUDA(cudaEventCreate(&e0));
    VFMM_CUDA(cudaEventCreate(&e1));
    int best = b->active;
    float best_t = -1.0f;
    int rc = VFMM_OK;
    for (int S = 1; S <= b->n_streams && rc == VFMM_OK; S *= 2) {
        vfmm_graph* g = nullptr;
        rc = capture(b, n, items, S, st, &g);
        if (rc != VFMM_OK) break;
        float total = 0.0f;
        for (int rep = 0; rep < 4 && rc == VFMM_OK; ++rep) {
            cudaError_t e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) rc = cuda_fail(e, "timing a batch graph");
            if (rep > 0) total += ms;  // the first replay warms up
        }
        cudaGraphExecDestroy(g->exec);
        cudaGraphDestroy(g->graph);
        delete g;
        if (rc == VFMM_OK && (best_t < 0.0f || total / 3.0f < best_t)) {
            best_t = total / 3.0f;
            best = S;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != VFMM_OK) return rc;
    b->active = best;
    *best_streams = best;
    *best_ms = best_t;
    return VFMM_OK;
}

extern "C" int vfmm_batch_streams(const vfmm_batch* b, int32_t* active) {
    if (!b || !active) return fail(VFMM_ERR_INVALID_ARG, "null argument");
    *active = b->active;
    return VFMM_OK;
}
