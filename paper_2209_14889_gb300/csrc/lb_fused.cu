// lb_fused.cu -- the tile kernels: one CTA per 32 x 16 tile of the fused step (lb_tile.cuh), one
// cell per thread (tile_step) or two neighbouring cells per thread on paired FP32 instructions
// (tile_step2).
#include <cuda_runtime.h>

#include "lb_tile.cuh"

namespace vlb {

namespace {

using namespace tile;

template <int MODE, int PREC>
__global__ void __launch_bounds__(NT, 3) k_fused(const FusedArgs a)
{
    extern __shared__ __align__(16) float sm[];
    tile_step<MODE, PREC, TILE_X, TILE_Y>(a, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, sm);
}

template <int MODE, int PREC>
__global__ void __launch_bounds__(NT, 2) k_fused_pair(const FusedArgs a)
{
    extern __shared__ __align__(16) float sm[];
    tile_step2<MODE, PREC, TILE_X, TILE_Y>(a, blockIdx.x, blockIdx.y, blockIdx.y * gridDim.x + blockIdx.x, sm);
}

}  // namespace

int fused_ctas(int nx, int ny) { return ((nx + TILE_X - 1) / TILE_X) * ((ny + TILE_Y - 1) / TILE_Y); }

template <int MODE, int PREC, bool PAIR>
static cudaError_t launch_one(const FusedArgs& a, dim3 grid, cudaStream_t s, bool pdl)
{
    static bool attr_done = false;
    auto kern = PAIR ? k_fused_pair<MODE, PREC> : k_fused<MODE, PREC>;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)TileGeo<TILE_X, TILE_Y>::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = TileGeo<TILE_X, TILE_Y>::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <bool PAIR>
static cudaError_t launch_form(const FusedArgs& a, int mode, dim3 grid, cudaStream_t s, bool pdl)
{
    if (a.prec == PREC_FP32)
        return mode == MODE_STEP ? launch_one<MODE_STEP, PREC_FP32, PAIR>(a, grid, s, pdl)
                                 : launch_one<MODE_MOMENTS, PREC_FP32, PAIR>(a, grid, s, false);
    return mode == MODE_STEP ? launch_one<MODE_STEP, PREC_LP, PAIR>(a, grid, s, pdl)
                             : launch_one<MODE_MOMENTS, PREC_LP, PAIR>(a, grid, s, false);
}

cudaError_t launch_fused(const FusedArgs& a, int mode, cudaStream_t s, int* grid_ctas, bool pdl, bool pair)
{
    dim3 grid((a.nx + TILE_X - 1) / TILE_X, (a.ny + TILE_Y - 1) / TILE_Y);
    if (grid_ctas) *grid_ctas = grid.x * grid.y;
    return pair ? launch_form<true>(a, mode, grid, s, pdl) : launch_form<false>(a, mode, grid, s, pdl);
}

}  // namespace vlb
