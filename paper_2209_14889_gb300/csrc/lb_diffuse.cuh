// lb_diffuse.cuh -- explicit stress-diffusion sub-steps for D_p beyond the Heun bound (device
// code shared by the diffusion kernel and the batched persistent kernel).
//
// Heun with the 5-point Laplacian is stable for 8 D_p <= 2.  For larger D_p the step takes the
// polymer-stress update of Eq. StiffCons without its diffusion term and then applies s Heun
// sub-steps of d sigma / dt = (D_p / s) lap sigma (periodic), each
//   sigma* = sigma + (D_p/s) lap sigma,  sigma' = sigma + (D_p/s) (lap sigma + lap sigma*) / 2.
// A sub-step reads the three sigma planes of one buffer and writes those of another; the tile
// stages sigma with a 2-cell halo and forms the predictor on a 1-cell halo.
#pragma once
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace vlb {
namespace dif {

constexpr int DX = 32, DY = 16, DNT = 256;
constexpr int D2W = DX + 4, D2H = DY + 4, D2 = D2W * D2H;
constexpr int D1W = DX + 2, D1H = DY + 2, D1 = D1W * D1H;

__device__ __forceinline__ int wrapd(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// One DX x DY tile of a diffusion sub-step; sm: SMEM floats.
__device__ __forceinline__ void diffuse_tile(const float* src, float* dst, long long NP, int nx, int ny,
                             float D, int bx, int by, float* sm)
{
    float* sA = sm;               // sigma on the halo-2 region [3][D2]
    float* sB = sm + 3 * D2;      // predictor on the halo-1 region [3][D1]
    const int x0 = bx * DX, y0 = by * DY;
    // a staged index lies within one period of the lattice when the lattice is at least a tile and
    // its halo wide: one conditional add or subtract wraps it; smaller lattices take the modulo
    const bool near = nx >= D2W && ny >= D2H;
    for (int i = threadIdx.x; i < D2; i += blockDim.x) {
        const int ly = i / D2W, lx = i - ly * D2W;
        int x = x0 - 2 + lx, y = y0 - 2 + ly;
        if (near) {
            x += x < 0 ? nx : (x >= nx ? -nx : 0);
            y += y < 0 ? ny : (y >= ny ? -ny : 0);
        } else {
            x = wrapd(x, nx);
            y = wrapd(y, ny);
        }
        const float* p = src + (long long)y * nx + x;
        for (int c = 0; c < 3; ++c) sA[c * D2 + i] = __ldcg(p + c * NP);   // written by the previous sub-step
    }
    __syncthreads();
    for (int i = threadIdx.x; i < D1; i += blockDim.x) {
        const int ly = i / D1W, lx = i - ly * D1W;
        const int j = (ly + 1) * D2W + lx + 1;
        for (int c = 0; c < 3; ++c) {
            const float* a = sA + c * D2;
            sB[c * D1 + i] = a[j] + D * (a[j + 1] + a[j - 1] + a[j + D2W] + a[j - D2W] - 4.f * a[j]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < DX * DY; i += blockDim.x) {
        const int ly = i / DX, lx = i - ly * DX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const int j = (ly + 2) * D2W + lx + 2, k = (ly + 1) * D1W + lx + 1;
        float* q = dst + (long long)gy * nx + gx;
        for (int c = 0; c < 3; ++c) {
            const float* a = sA + c * D2;
            const float* b = sB + c * D1;
            const float l0 = a[j + 1] + a[j - 1] + a[j + D2W] + a[j - D2W] - 4.f * a[j];
            const float l1 = b[k + 1] + b[k - 1] + b[k + D1W] + b[k - D1W] - 4.f * b[k];
            q[c * NP] = a[j] + 0.5f * D * (l0 + l1);
        }
    }
    __syncthreads();
}

constexpr int SMEM = 3 * D2 + 3 * D1;

}  // namespace dif
}  // namespace vlb
