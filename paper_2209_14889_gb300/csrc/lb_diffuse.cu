// lb_diffuse.cu -- the stress-diffusion sub-step kernel (lb_diffuse.cuh) and its launcher.
#include <cuda_runtime.h>

#include "lb_diffuse.cuh"

namespace vlb {

using namespace dif;

int diffuse_smem_floats() { return SMEM; }
int diffuse_tiles_x(int nx) { return (nx + DX - 1) / DX; }
int diffuse_tiles_y(int ny) { return (ny + DY - 1) / DY; }

namespace {

__global__ void __launch_bounds__(DNT) k_diffuse(const float* src, float* dst, long long NP, int nx, int ny, float D)
{
    extern __shared__ __align__(16) float sm[];
    diffuse_tile(src, dst, NP, nx, ny, D, blockIdx.x, blockIdx.y, sm);
}

__global__ void k_copy3(const float* src, float* dst, long long NP)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NP) {
        dst[i] = src[i];
        dst[NP + i] = src[NP + i];
        dst[2 * NP + i] = src[2 * NP + i];
    }
}

}  // namespace

cudaError_t launch_diffusion(float* sig_new, float* sig_tmp, long long NP, int nx, int ny, float D, int substeps,
                             cudaStream_t s)
{
    const dim3 grid(diffuse_tiles_x(nx), diffuse_tiles_y(ny));
    const size_t smem = sizeof(float) * diffuse_smem_floats();
    for (int k = 0; k < substeps; ++k) {
        const bool even = (k & 1) == 0;
        k_diffuse<<<grid, DNT, smem, s>>>(even ? sig_new : sig_tmp, even ? sig_tmp : sig_new, NP, nx, ny, D);
    }
    if (substeps & 1) k_copy3<<<(unsigned)((NP + 255) / 256), 256, 0, s>>>(sig_tmp, sig_new, NP);
    return cudaGetLastError();
}

}  // namespace vlb
