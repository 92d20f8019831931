// Host-side launches of the sampler (csrc/sample.cu): plain stream launches and
// kernel nodes of the replayed CUDA graph.
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

}  // namespace agis
