// lscan_graph.cu -- a scan captured once into a CUDA graph and replayed.
//
// The graph owns a private scratch set (control block + status words).  The
// kernel re-arms that scratch itself at the end of every launch (ticket back
// to 0, epoch + 1), so each replay is exactly one kernel node with no memset
// node, and the baked kernel parameters stay valid.  Replays of one graph
// must be ordered (one stream, or synchronised), since they share scratch.
#include <cuda_runtime.h>

#include <set>

#include "../../include/lscan.h"
#include "kernel_table.h"
#include "lscan_internal.h"
#include "scan_common.h"

struct lscan_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t *ctl = nullptr;
    uint64_t *status = nullptr;
    size_t status_words = 0;
    uint64_t replays = 0;
    int device = 0;
};

namespace lscan {
namespace {
std::set<lscan_graph *> g_graphs;

void destroy_graph(lscan_graph *g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->status) cudaFree(g->status);
    if (g->ctl) cudaFree(g->ctl);
    cudaSetDevice(cur);
    delete g;
}

lscan_status create_graph(const LaunchSpec &ls, lscan_graph **out) {
    if (out == nullptr) return LSCAN_ERR_INVALID;
    *out = nullptr;
    if (ls.n == 0) return LSCAN_ERR_INVALID;  // nothing to capture
    lscan_graph *g = new lscan_graph();
    cudaGetDevice(&g->device);
    const size_t words = ls.status_words > 0 ? ls.status_words : 1;
    g->status_words = words;
    cudaStream_t cs = nullptr;
    lscan_status st = LSCAN_OK;
    if (cudaMalloc(&g->ctl, CTL_WORDS * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&g->status, words * sizeof(uint64_t)) != cudaSuccess) {
        destroy_graph(g);
        return LSCAN_ERR_NOMEM;
    }
    if (cudaMemset(g->ctl, 0, CTL_WORDS * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(g->status, 0, words * sizeof(uint64_t)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        destroy_graph(g);
        return LSCAN_ERR_CUDA;
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        destroy_graph(g);
        return LSCAN_ERR_CUDA;
    }
    DevBuffers b{g->ctl, g->status};
    st = launch_scan(ls, b, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (st != LSCAN_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        destroy_graph(g);
        return st != LSCAN_OK ? st : LSCAN_ERR_CUDA;
    }
    g->graph = graph;
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        destroy_graph(g);
        return LSCAN_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(api_mutex());
        g_graphs.insert(g);
    }
    *out = g;
    return LSCAN_OK;
}
}  // namespace

void shutdown_graphs_locked() {
    for (lscan_graph *g : g_graphs) destroy_graph(g);
    g_graphs.clear();
}

}  // namespace lscan

using namespace lscan;

extern "C" {

lscan_status lscan_graph_create_scan(lscan_op op, lscan_dtype dtype, int inclusive,
                                     const void *x, void *y, int64_t n,
                                     const lscan_options *opts, lscan_graph **out) {
    LaunchSpec ls;
    lscan_status st =
        plan_scan(op, dtype, inclusive, x, y, n, opts, MODE_SINGLE, nullptr, 0, &ls);
    if (st != LSCAN_OK) return st;
    return create_graph(ls, out);
}

lscan_status lscan_graph_create_batched(lscan_op op, lscan_dtype dtype, int inclusive,
                                        const void *x, void *y,
                                        const int64_t *d_offsets, int64_t n_seg,
                                        int64_t n_total, const lscan_options *opts,
                                        lscan_graph **out) {
    if (n_seg <= 0 || n_total < 0 || d_offsets == nullptr) return LSCAN_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(d_offsets) % 8 != 0) return LSCAN_ERR_INVALID;
    LaunchSpec ls;
    lscan_status st = plan_scan(op, dtype, inclusive, x, y, n_total, opts,
                                MODE_SEGMENTED, d_offsets, n_seg, &ls);
    if (st != LSCAN_OK) return st;
    return create_graph(ls, out);
}

lscan_status lscan_graph_launch(lscan_graph *g, void *stream) {
    if (g == nullptr || g->exec == nullptr) return LSCAN_ERR_INVALID;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (++g->replays >= (1ull << 30) - 1) {
        // keep the 30-bit epoch tag from wrapping (see lscan_api.cu)
        const size_t words = g->status_words;
        if (cudaMemsetAsync(g->ctl, 0, CTL_WORDS * sizeof(uint32_t), cs) != cudaSuccess ||
            cudaMemsetAsync(g->status, 0, words * sizeof(uint64_t), cs) != cudaSuccess)
            return LSCAN_ERR_CUDA;
        g->replays = 0;
    }
    if (cudaGraphLaunch(g->exec, cs) != cudaSuccess) return LSCAN_ERR_CUDA;
    note_launch();
    return LSCAN_OK;
}

lscan_status lscan_graph_status(lscan_graph *g) {
    if (g == nullptr) return LSCAN_ERR_INVALID;
    if (cudaDeviceSynchronize() != cudaSuccess) return LSCAN_ERR_CUDA;
    uint32_t err = 0;
    if (cudaMemcpy(&err, g->ctl + CTL_ERROR, sizeof(err), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return LSCAN_ERR_CUDA;
    if (err == 0) return LSCAN_OK;
    cudaMemset(g->ctl + CTL_ERROR, 0, sizeof(uint32_t));
    if (err & (DEV_ERR_CARRY_WAIT | DEV_ERR_BARRIER_WAIT)) return LSCAN_ERR_TIMEOUT;
    return LSCAN_ERR_DEVICE;
}

void lscan_graph_destroy(lscan_graph *g) {
    if (g == nullptr) return;
    {
        std::lock_guard<std::mutex> lk(api_mutex());
        g_graphs.erase(g);
    }
    destroy_graph(g);
}

}  // extern "C"
