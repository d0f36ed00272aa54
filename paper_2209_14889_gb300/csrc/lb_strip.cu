// lb_strip.cu -- launch of the warp-strip lattice kernel (device code in lb_strip.cuh): one CTA
// of four warps per four strips of a rows chunk, three CTAs per SM.
#include <cuda_runtime.h>

#include <cmath>

#include "lb_strip.cuh"

namespace vlb {

namespace {

template <int PREC, bool SCALAR>
__global__ void __launch_bounds__(SNT, 3) k_strip(const FusedArgs a, const int H)
{
    extern __shared__ __align__(16) float smem[];
    strip_body<PREC, SCALAR>(a, a.t, H, blockIdx.x, blockIdx.y, (long long)blockIdx.y * gridDim.x + blockIdx.x, smem);
}

template <int PREC, bool SCALAR>
cudaError_t launch_strip_t(const FusedArgs& a, int H, dim3 grid, cudaStream_t s, bool pdl)
{
    static unsigned long long attr_done = 0;     // per device
    auto kern = k_strip<PREC, SCALAR>;
    if (!done_on_device(attr_done)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STRIP_SMEM);
        if (e != cudaSuccess) {
            attr_done = 0;
            return e;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(SNT);
    cfg.dynamicSmemBytes = STRIP_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a, H);
}

}  // namespace

bool strip_eligible(int nx, int ny, int walls)
{
    // 32 distinct columns per warp, a spreading window (the sub-chunk's rows and the kernel's
    // support) that does not wrap onto itself, even nx (the 2-byte form copies column pairs), and
    // 32-bit flat indices over the 14 planes
    return !walls && nx >= 64 && (nx & 1) == 0 && ny >= 32 && (long long)nx * ny * N_PLANES < (1LL << 31);
}

// Rows per warp chunk: 64 (the chunk ends recompute (64 + 6) / 64 of the stage rows), fewer when
// the lattice would otherwise not give every SM its three CTAs.
int strip_chunk(int nx, int ny, int n_sm)
{
    const int strips = (nx + SOWN - 1) / SOWN;
    const long long cx = (strips + SWARPS - 1) / SWARPS;
    int H = 64;
    while (H > 16 && cx * ((ny + H - 1) / H) < 3LL * n_sm) H /= 2;
    return H;
}

// The strip kernel is latency-bound per warp (each row runs its stages as one dependent chain),
// so it needs many resident warps and many waves of CTAs to keep the SMs issuing.  Measured on
// GB300 (per time step, 16 rings at 4096^2, one ring below): 4096^2 899 us against 1098 us for the
// tile kernel (precision form 964 / 1136, scalar model 665 / 848), 2048^2 308 / 272 us, 1024^2
// 150 / 75 us.  It is preferred where its grid of 64-row chunks fills at least four waves of
// three CTAs per SM.
bool strip_preferred(int nx, int ny, int n_sm)
{
    const int strips = (nx + SOWN - 1) / SOWN;
    const long long ctas = (long long)((strips + SWARPS - 1) / SWARPS) * ((ny + 63) / 64);
    return ctas >= 4LL * 3 * n_sm;
}

int strip_ctas(int nx, int ny, int H)
{
    const int strips = (nx + SOWN - 1) / SOWN;
    return ((strips + SWARPS - 1) / SWARPS) * ((ny + H - 1) / H);
}

cudaError_t launch_strip(const FusedArgs& a, int H, cudaStream_t s, bool pdl)
{
    const int strips = (a.nx + SOWN - 1) / SOWN;
    dim3 grid((strips + SWARPS - 1) / SWARPS, (a.ny + H - 1) / H);
    if (a.scalar) return launch_strip_t<0, true>(a, H, grid, s, pdl);
    return a.prec == 0 ? launch_strip_t<0, false>(a, H, grid, s, pdl) : launch_strip_t<1, false>(a, H, grid, s, pdl);
}

}  // namespace vlb
