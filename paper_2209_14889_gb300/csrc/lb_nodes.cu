// lb_nodes.cu -- the node kernel: one CTA per block of ring nodes (lb_node.cuh).
#include <cuda_runtime.h>

#include "lb_node.cuh"

namespace vlb {

namespace {

using namespace node;

__global__ void __launch_bounds__(NODE_THREADS) k_nodes(const NodeArgs a)
{
    __shared__ NodeSmem S;
    node_block(a, blockIdx.x, S);
}

}  // namespace

cudaError_t launch_nodes(const NodeArgs& a, cudaStream_t s, bool pdl)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.n_ctas);
    cfg.blockDim = dim3(NODE_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_nodes, a);
}

}  // namespace vlb
