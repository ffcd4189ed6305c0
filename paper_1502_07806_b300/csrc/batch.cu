// Batched PFSM solves of many independent problems of uneven order (k-points / spin channels of
// one SCF step), replayed as one captured CUDA graph.
//
// Every problem keeps its own workspace (a pfsm handle). The problems are spread over a set of
// internal streams, longest first (estimated cost N^3) onto the least-loaded stream, so small
// problems run concurrently with the large ones and fill the SMs the large ones leave idle. The
// first call with a given set of buffers captures the whole fork/join -- the caller's stream
// forks to the internal streams, each enqueues its problems' solves, the caller's stream joins
// them -- into a CUDA graph; later calls with the same buffers replay it with a single graph
// launch, which removes the host launch overhead of the per-problem kernel sequences.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "pfsm_internal.cuh"

using namespace pfsm;

struct pfsm_batch_s {
    int32_t count = 0;
    std::vector<pfsm_handle_t> h;
    std::vector<int32_t> stream_of;          // problem -> internal stream
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;              // private stream the graph is captured on and runs on
    cudaEvent_t enter = nullptr, leave = nullptr;
    // graph cache for the last set of buffers
    std::vector<const void *> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last_stream = nullptr;
};

namespace {

int bfail(int code, const char *msg)
{
    pfsm::set_last_error(msg);
    return code;
}

void release(pfsm_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->enter) cudaEventDestroy(b->enter);
    if (b->leave) cudaEventDestroy(b->leave);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (pfsm_handle_t h : b->h) pfsm_destroy(h);
    delete b;
}

}  // namespace

extern "C" {

int pfsm_batch_init(int32_t count, const int64_t *N, const int32_t *nblocks, const pfsm_params_t *p,
                    pfsm_batch_t *out)
{
    if (!out || !N || !nblocks || count < 1 || count > 4096)
        return bfail(PFSM_ERR_INVALID_ARG, "pfsm_batch_init: bad count or null argument");
    *out = nullptr;
    pfsm_params_t prm;
    pfsm_default_params(&prm);
    if (p) prm = *p;
    prm.slice_sizes = nullptr;              // per-problem slice sizes are not supported here
    pfsm_batch_s *b = new pfsm_batch_s();
    b->count = count;
    b->h.assign(count, nullptr);
    for (int32_t i = 0; i < count; i++) {
        int rc = pfsm_init(N[i], nblocks[i], &prm, &b->h[i]);
        if (rc != PFSM_OK) {
            std::string msg = std::string("pfsm_batch_init: problem ") + std::to_string(i) + ": " + pfsm_last_error();
            release(b);
            return bfail(rc, msg.c_str());
        }
    }
    // longest-processing-time-first assignment to the least-loaded stream
    const int ns = count < 16 ? count : 16;
    b->streams.assign(ns, nullptr);
    b->join.assign(ns, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->enter, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->leave, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int s = 0; s < ns && e == cudaSuccess; s++) {
        e = cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        release(b);
        return bfail(PFSM_ERR_CUDA, cudaGetErrorString(e));
    }
    std::vector<int32_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return N[a] > N[c]; });
    std::vector<double> load(ns, 0.0);
    b->stream_of.assign(count, 0);
    for (int32_t i : order) {
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->stream_of[i] = s;
        load[s] += (double)N[i] * N[i] * N[i];
    }
    *out = b;
    return PFSM_OK;
}

int pfsm_solve_batched(pfsm_batch_t b, const double *const *A, const double *const *prev,
                       double *const *eigvals_out, double *const *V_out, void *stream)
{
    if (!b || !A || !prev || !eigvals_out || !V_out)
        return bfail(PFSM_ERR_INVALID_ARG, "pfsm_solve_batched: null argument");
    const int32_t n = b->count;
    std::vector<const void *> key;
    key.reserve(4 * (size_t)n);
    for (int32_t i = 0; i < n; i++) {
        if (!A[i] || !prev[i] || !eigvals_out[i] || !V_out[i])
            return bfail(PFSM_ERR_INVALID_ARG, "pfsm_solve_batched: null buffer");
        key.push_back(A[i]);
        key.push_back(prev[i]);
        key.push_back(eigvals_out[i]);
        key.push_back(V_out[i]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->exec || key != b->key) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        cudaStream_t cs = b->cap;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bfail(PFSM_ERR_CUDA, cudaGetErrorString(e));
        int rc = PFSM_OK;
        e = cudaEventRecord(b->fork, cs);
        for (size_t s = 0; s < b->streams.size() && e == cudaSuccess; s++)
            e = cudaStreamWaitEvent(b->streams[s], b->fork, 0);
        for (int32_t i = 0; i < n && e == cudaSuccess && rc == PFSM_OK; i++)
            rc = pfsm_solve(b->h[i], A[i], prev[i], eigvals_out[i], V_out[i], b->streams[b->stream_of[i]]);
        for (size_t s = 0; s < b->streams.size() && e == cudaSuccess; s++) {
            e = cudaEventRecord(b->join[s], b->streams[s]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b->join[s], 0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (rc != PFSM_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;                      // pfsm_solve already recorded the message
        }
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(PFSM_ERR_CUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return bfail(PFSM_ERR_CUDA, cudaGetErrorString(e));
        }
        b->graph = g;
        b->key = key;
    }
    // order the graph after the caller's prior work and the caller's later work after the graph
    cudaError_t e = cudaEventRecord(b->enter, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->enter, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->cap);
    if (e == cudaSuccess) e = cudaEventRecord(b->leave, b->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->leave, 0);
    if (e != cudaSuccess) return bfail(PFSM_ERR_CUDA, cudaGetErrorString(e));
    b->last_stream = st;
    return PFSM_OK;
}

int pfsm_batch_get_status(pfsm_batch_t b, int32_t *statuses)
{
    if (!b || !statuses) return bfail(PFSM_ERR_INVALID_ARG, "pfsm_batch_get_status: null argument");
    cudaError_t e = cudaStreamSynchronize(b->last_stream);
    if (e != cudaSuccess) return bfail(PFSM_ERR_CUDA, cudaGetErrorString(e));
    for (int32_t i = 0; i < b->count; i++) {
        e = cudaMemcpy(&statuses[i], b->h[i]->ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bfail(PFSM_ERR_CUDA, cudaGetErrorString(e));
    }
    return PFSM_OK;
}

int pfsm_batch_destroy(pfsm_batch_t b)
{
    if (!b) return PFSM_OK;
    cudaDeviceSynchronize();
    release(b);
    return PFSM_OK;
}

}  // extern "C"
