// Host-side launches of the sampler (csrc/sample.cu): plain stream launches and
// kernel nodes of the replayed CUDA graph.
#include <algorithm>

#include "agis_internal.h"

namespace agis {

// The persisting-L2 access window of sampler launches on g: its hub bitmaps, laid out
// in decreasing degree order, up to g->l2_window_bytes (within the device's window
// and set-aside limits).  Probes of the hottest hubs' bitmaps are the sampler's most
// frequent random sectors; marked persisting they stay in L2 instead of competing
// with the streamed rows.  The context's set-aside is raised to the window's size at
// the first such launch and restored when the context is released.  Returns false
// (no window) when off, without hubs, or when the device has no set-aside.
static bool l2_window(agis_graph *g, cudaAccessPolicyWindow *w)
{
    if (g->l2_window_bytes == 0 || !g->hub_bits || g->n_hubs <= 0) return false;
    agis_ctx *c = g->ctx;
    int max_set = 0, max_win = 0;
    if (cudaDeviceGetAttribute(&max_set, cudaDevAttrMaxPersistingL2CacheSize, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, c->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (max_set <= 0 || max_win <= 0) return false;
    size_t want = (size_t)g->l2_window_bytes;
    want = std::min(want, (size_t)g->n_hubs * (size_t)g->hub_words * sizeof(uint32_t));
    want = std::min(want, (size_t)max_win);
    want = std::min(want, (size_t)max_set);
    if (want == 0) return false;
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cur < want) {
        if (!c->l2_limit_set) {
            c->l2_limit_before = cur;
            c->l2_limit_set = true;
        }
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    w->base_ptr = (void *)g->hub_bits;
    w->num_bytes = want;
    w->hitRatio = 1.0f;
    w->hitProp = cudaAccessPropertyPersisting;
    w->missProp = cudaAccessPropertyStreaming;
    return true;
}

// The device's greatest (most urgent) stream priority.
static int urgent_priority()
{
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
    return greatest;
}

// Enqueue one sampler launch over lb's staged queries and items (already on the
// device; lb.d_counter[0] = the first item, lb.d_counter[1] = the end of the items).
// With implicit_count > 0 the items are implicit runs of implicit_span tiles of query
// 0 (see the kernel).  An urgent launch gets its CTAs placed before those of a
// scatter launch enqueued beside it.
int launch_sampler(agis_graph *g, LaunchBuffers &lb, int grid, const DumpView *dump,
                   cudaStream_t stream, uint64_t implicit_first, uint64_t implicit_count,
                   uint32_t implicit_span, uint64_t *tile_out, bool anchor, bool urgent)
{
    GraphView gv{g->off, g->cols, g->nv, g->nnz, g->hub_id, g->hub_bits, g->hub_words, g->rp_base};
    DumpView dv = dump ? *dump : DumpView{nullptr, nullptr, nullptr, nullptr, 0};
    const DevQuery *q = lb.d_queries;
    const WorkItem *items = implicit_count ? nullptr : lb.d_items;
    const uint32_t *nptr = lb.d_counter + 1;
    uint32_t *ctr = lb.d_counter;
    uint64_t *out = tile_out ? tile_out : lb.d_out;
    char *scr = (char *)lb.d_scratch;
    uint32_t cap = lb.scratch_cap;
    void *args[] = {&gv, &q, &items, &nptr, &ctr, &out, &dv, &implicit_first, &implicit_count, &implicit_span,
                    &scr, &cap};
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    unsigned na = 0;
    if (urgent) {
        attr[na].id = cudaLaunchAttributePriority;
        attr[na++].val.priority = urgent_priority();
    }
    cudaAccessPolicyWindow w;
    if (l2_window(g, &w)) {
        attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[na++].val.accessPolicyWindow = w;
    }
    cfg.attrs = na ? attr : nullptr;
    cfg.numAttrs = na;
    return cuda_status(cudaLaunchKernelExC(&cfg, sampler_function(dump != nullptr, anchor), args));
}

// Adds the sampler as a kernel node of a CUDA graph (explicit items, no dump).  The
// argument values are copied into the node when it is added.
int add_sampler_node(agis_graph *g, LaunchBuffers &lb, int grid, cudaGraph_t graph,
                     const cudaGraphNode_t *deps, size_t ndeps, cudaGraphNode_t *node, bool anchor, bool urgent)
{
    GraphView gv{g->off, g->cols, g->nv, g->nnz, g->hub_id, g->hub_bits, g->hub_words, g->rp_base};
    DumpView none{nullptr, nullptr, nullptr, nullptr, 0};
    const DevQuery *q = lb.d_queries;
    const WorkItem *it = lb.d_items;
    const uint32_t *nptr = lb.d_counter + 1;
    uint32_t *ctr = lb.d_counter;
    uint64_t *out = lb.d_out;
    uint64_t z0 = 0, z1 = 0;
    uint32_t span1 = 1;
    char *scr = (char *)lb.d_scratch;
    uint32_t cap = lb.scratch_cap;
    void *args[] = {&gv, &q, &it, &nptr, &ctr, &out, &none, &z0, &z1, &span1, &scr, &cap};
    cudaKernelNodeParams p = {};
    p.func = const_cast<void *>(sampler_function(false, anchor));
    p.gridDim = dim3(grid);
    p.blockDim = dim3(kBlock);
    p.sharedMemBytes = 0;
    p.kernelParams = args;
    int rc = cuda_status(cudaGraphAddKernelNode(node, graph, deps, ndeps, &p));
    if (rc != AGIS_OK) return rc;
    cudaKernelNodeAttrValue w = {};
    if (l2_window(g, &w.accessPolicyWindow) &&
        (rc = cuda_status(cudaGraphKernelNodeSetAttribute(*node, cudaLaunchAttributeAccessPolicyWindow, &w))) != AGIS_OK)
        return rc;
    if (!urgent) return rc;
    cudaKernelNodeAttrValue v = {};
    v.priority = urgent_priority();
    return cuda_status(cudaGraphKernelNodeSetAttribute(*node, cudaLaunchAttributePriority, &v));
}

// The scatter kernel's arguments: the tail items are the first lb.d_counter[3] staged
// items, lb.d_counter[2] its trial counter; its warps' candidate lists follow those
// of the first `scratch_skip` CTAs (a sampler launch running beside it uses those).
struct ScatterArgs {
    GraphView gv;
    const DevQuery *q;
    const WorkItem *items;
    const uint32_t *nptr;
    uint32_t *ctr;
    ScatterView sv;
    char *scr;
    uint32_t cap;
    uint64_t *out;
    void *args[8];
    void *rargs[4];

    ScatterArgs(agis_graph *g, LaunchBuffers &lb, int scratch_skip)
    {
        gv = GraphView{g->off, g->cols, g->nv, g->nnz, g->hub_id, g->hub_bits, g->hub_words, g->rp_base};
        q = lb.d_queries;
        items = lb.d_items;
        nptr = lb.d_counter + 3;
        ctr = lb.d_counter + 2;
        sv = ScatterView{lb.d_sx, lb.d_shit, lb.d_ssec};
        scr = (char *)lb.d_scratch + scratch_stride(lb.scratch_cap) * (size_t)scratch_skip * kWarps;
        cap = lb.scratch_cap;
        out = lb.d_out;
        void *a[] = {&gv, &q, &items, &nptr, &ctr, &sv, &scr, &cap};
        void *r[] = {&items, &nptr, &sv, &out};
        std::copy(a, a + 8, args);
        std::copy(r, r + 4, rargs);
    }
};

// The scatter kernel on `grid` CTAs, then one tile-reduction CTA per tail item
// (`rgrid` CTAs, those past the items return at once), writing lb.d_out.
int launch_scatter(agis_graph *g, LaunchBuffers &lb, int grid, int scratch_skip, size_t rgrid, cudaStream_t stream,
                   bool anchor)
{
    ScatterArgs a(g, lb, scratch_skip);
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    if (l2_window(g, &attr[0].val.accessPolicyWindow)) {
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelExC(&cfg, scatter_function(anchor), a.args);
    if (e != cudaSuccess) return AGIS_ERR_CUDA;
    count_launch();
    return cuda_status(cudaLaunchKernel(tile_reduce_function(), dim3((unsigned)std::max<size_t>(rgrid, 1)),
                                        dim3(kBlock), a.rargs, 0, stream));
}

// The same two kernels as nodes of a CUDA graph (after deps).
int add_scatter_nodes(agis_graph *g, LaunchBuffers &lb, int grid, int scratch_skip, size_t rgrid, cudaGraph_t graph,
                      const cudaGraphNode_t *deps, size_t ndeps, cudaGraphNode_t *kernel, cudaGraphNode_t *reduce,
                      bool anchor)
{
    ScatterArgs a(g, lb, scratch_skip);
    cudaKernelNodeParams p = {};
    p.func = const_cast<void *>(scatter_function(anchor));
    p.gridDim = dim3(grid);
    p.blockDim = dim3(kBlock);
    p.kernelParams = a.args;
    cudaError_t e = cudaGraphAddKernelNode(kernel, graph, deps, ndeps, &p);
    if (e != cudaSuccess) return AGIS_ERR_CUDA;
    cudaKernelNodeAttrValue v = {};
    if (l2_window(g, &v.accessPolicyWindow) &&
        cudaGraphKernelNodeSetAttribute(*kernel, cudaLaunchAttributeAccessPolicyWindow, &v) != cudaSuccess)
        return AGIS_ERR_CUDA;
    cudaKernelNodeParams r = {};
    r.func = const_cast<void *>(tile_reduce_function());
    r.gridDim = dim3((unsigned)std::max<size_t>(rgrid, 1));
    r.blockDim = dim3(kBlock);
    r.kernelParams = a.rargs;
    return cuda_status(cudaGraphAddKernelNode(reduce, graph, kernel, 1, &r));
}

}  // namespace agis
