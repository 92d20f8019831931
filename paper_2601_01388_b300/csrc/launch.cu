// Host-side launches of the sampler (csrc/sample.cu): plain stream launches and
// kernel nodes of the replayed CUDA graph.
#include <algorithm>

#include "agis_internal.h"

namespace agis {

// Enqueue one sampler launch over lb's staged queries and items (already on the
// device; lb.d_counter[0] zeroed and lb.d_counter[1] = number of items).  With
// implicit_count > 0 the items are implicit runs of implicit_span tiles of query 0
// (see the kernel).
int launch_sampler(agis_graph *g, LaunchBuffers &lb, int grid, const DumpView *dump,
                   cudaStream_t stream, uint64_t implicit_first, uint64_t implicit_count,
                   uint32_t implicit_span, uint64_t *tile_out, bool anchor)
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
    return cuda_status(cudaLaunchKernel(sampler_function(dump != nullptr, anchor), dim3(grid), dim3(kBlock),
                                        args, 0, stream));
}

// Adds the sampler as a kernel node of a CUDA graph (explicit items, no dump).  The
// argument values are copied into the node when it is added.
int add_sampler_node(agis_graph *g, LaunchBuffers &lb, int grid, cudaGraph_t graph,
                     const cudaGraphNode_t *deps, size_t ndeps, cudaGraphNode_t *node, bool anchor)
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
    return cuda_status(cudaGraphAddKernelNode(node, graph, deps, ndeps, &p));
}

static void scatter_args(agis_graph *g, LaunchBuffers &lb, GraphView &gv, ScatterView &sv)
{
    gv = GraphView{g->off, g->cols, g->nv, g->nnz, g->hub_id, g->hub_bits, g->hub_words, g->rp_base};
    sv = ScatterView{lb.d_sx, lb.d_shit, lb.d_ssec};
}

// A scatter epoch: the scatter kernel on `grid` CTAs over the n staged single-tile
// items (lb.d_counter[0] zeroed, lb.d_counter[1] = n), then one tile-reduction CTA
// per item, writing lb.d_out.
int launch_scatter(agis_graph *g, LaunchBuffers &lb, int grid, size_t n, cudaStream_t stream, bool anchor)
{
    GraphView gv;
    ScatterView sv;
    scatter_args(g, lb, gv, sv);
    const DevQuery *q = lb.d_queries;
    const WorkItem *items = lb.d_items;
    const uint32_t *nptr = lb.d_counter + 1;
    uint32_t *ctr = lb.d_counter;
    char *scr = (char *)lb.d_scratch;
    uint32_t cap = lb.scratch_cap;
    uint64_t *out = lb.d_out;
    void *args[] = {&gv, &q, &items, &nptr, &ctr, &sv, &scr, &cap};
    count_launch();
    cudaError_t e = cudaLaunchKernel(scatter_function(anchor), dim3(grid), dim3(kBlock), args, 0, stream);
    if (e != cudaSuccess) return AGIS_ERR_CUDA;
    void *rargs[] = {&items, &nptr, &sv, &out};
    count_launch();
    return cuda_status(cudaLaunchKernel(tile_reduce_function(), dim3((unsigned)std::max<size_t>(n, 1)), dim3(kBlock),
                                        rargs, 0, stream));
}

// The same two kernels as nodes of a CUDA graph (after deps); the reduction's grid
// is patched per epoch by set_reduce_node_items.
int add_scatter_nodes(agis_graph *g, LaunchBuffers &lb, int grid, size_t n, cudaGraph_t graph,
                      const cudaGraphNode_t *deps, size_t ndeps, cudaGraphNode_t *kernel, cudaGraphNode_t *reduce,
                      bool anchor)
{
    GraphView gv;
    ScatterView sv;
    scatter_args(g, lb, gv, sv);
    const DevQuery *q = lb.d_queries;
    const WorkItem *items = lb.d_items;
    const uint32_t *nptr = lb.d_counter + 1;
    uint32_t *ctr = lb.d_counter;
    char *scr = (char *)lb.d_scratch;
    uint32_t cap = lb.scratch_cap;
    uint64_t *out = lb.d_out;
    void *args[] = {&gv, &q, &items, &nptr, &ctr, &sv, &scr, &cap};
    cudaKernelNodeParams p = {};
    p.func = const_cast<void *>(scatter_function(anchor));
    p.gridDim = dim3(grid);
    p.blockDim = dim3(kBlock);
    p.kernelParams = args;
    cudaError_t e = cudaGraphAddKernelNode(kernel, graph, deps, ndeps, &p);
    if (e != cudaSuccess) return AGIS_ERR_CUDA;
    void *rargs[] = {&items, &nptr, &sv, &out};
    cudaKernelNodeParams r = {};
    r.func = const_cast<void *>(tile_reduce_function());
    r.gridDim = dim3((unsigned)std::max<size_t>(n, 1));
    r.blockDim = dim3(kBlock);
    r.kernelParams = rargs;
    return cuda_status(cudaGraphAddKernelNode(reduce, graph, kernel, 1, &r));
}

int set_reduce_node_items(LaunchBuffers &lb, cudaGraphExec_t exec, cudaGraphNode_t node, size_t n)
{
    const WorkItem *items = lb.d_items;
    const uint32_t *nptr = lb.d_counter + 1;
    ScatterView sv{lb.d_sx, lb.d_shit, lb.d_ssec};
    uint64_t *out = lb.d_out;
    void *rargs[] = {&items, &nptr, &sv, &out};
    cudaKernelNodeParams r = {};
    r.func = const_cast<void *>(tile_reduce_function());
    r.gridDim = dim3((unsigned)std::max<size_t>(n, 1));
    r.blockDim = dim3(kBlock);
    r.kernelParams = rargs;
    return cuda_status(cudaGraphExecKernelNodeSetParams(exec, node, &r));
}

}  // namespace agis
