// lb_unet.cu -- the network of the learned stepper: a 4-level convolutional U-Net on NHWC BF16
// activations with FP32 accumulation, forward and backward, trained on the GPU.
//
// Convolutions (3x3, stride 1, zero padding) are implicit GEMMs on the tensor cores:
//   forward      y[p, o]  = b[o] + sum_{t, c} x[p + off_t, c] w[t, o, c]      (M = pixels, N = Co,
//                                                                           K = 9 Ci)
//   data grad    gx[q, c] = sum_{t', o} gz[q + off_t', o] w'[t', c, o],  w'[t'] = w[8 - t']^T
//                (the forward kernel on the flipped, transposed weights)
//   weight grad  gw[t, o, c] = sum_p gz[p, o] x[p + off_t, c]                (M = Co, N = Ci,
//                                                                           K = pixels)
// with off_t = (t / 3 - 1, t % 3 - 1).  Tiles are staged in shared memory (rows padded to 48 or
// 144 bytes, so the 8 rows of each ldmatrix fall in distinct banks) and multiplied with
// mma.sync m16n8k16 BF16 -> FP32; by default the forward and the data gradient run instead on
// tcgen05 (k_conv3x3_tc: pixels as M, output channels as N, accumulators in tensor memory).
// Weight gradients are reduced over pixel tiles in a fixed
// order (per-CTA partials, then a sum over CTAs), so training is bitwise reproducible.
// Joins: 2x2 average pooling, nearest 2x upsampling written into a channel slice of the
// concatenation buffer (the skip is written there by its producing convolution), LeakyReLU
// (slope 0.1) fused into the convolution epilogue.  Optimiser: Adam on FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace vlb {
namespace net {

using bf16 = __nv_bfloat16;
constexpr float SLOPE = 0.1f;

// ------------------------------------------------------------------ tensor-core primitives

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
// D += A (16x16, row) * B (16x8, col); BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------------ convolution forward

constexpr int CT_H = 8, CT_W = 16;              // output tile: 8 rows x 16 pixels (4 warps x 2 rows)
constexpr int CT_IH = CT_H + 2, CT_IW = CT_W + 2;
constexpr int CT_CO = 64;                       // output channels per CTA
constexpr int PS = 24;                          // shared row of 16 channels + 8 pad (48 bytes)

struct ConvArgs {
    const bf16* x;          // input, pixel stride ldx, channels at xoff .. xoff + Ci
    long long ldx;
    int xoff;
    const bf16* w;          // [9][Co][Ci]
    const float* bias;      // [Co] or nullptr
    bf16* y;                // BF16 output (pixel stride ldy, channel offset yoff), or
    float* yf;              // FP32 output
    long long ldy;
    int yoff;
    int B, H, W, Ci, Co;
    int act;                // 1: LeakyReLU
};

__global__ void __launch_bounds__(128) k_conv3x3(const ConvArgs a)
{
    __shared__ __align__(16) bf16 sx[CT_IH * CT_IW * PS];
    __shared__ __align__(16) bf16 sw[9 * CT_CO * PS];
    const int n_cot = (a.Co + CT_CO - 1) / CT_CO;
    const int b = blockIdx.z / n_cot, co0 = (blockIdx.z % n_cot) * CT_CO;
    const int tx0 = blockIdx.x * CT_W, ty0 = blockIdx.y * CT_H;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);

    for (int c0 = 0; c0 < a.Ci; c0 += 16) {
        for (int q = tid; q < CT_IH * CT_IW * 2; q += 128) {
            const int p = q >> 1, h = q & 1;
            const int py = p / CT_IW, px = p - py * CT_IW;
            const int gy = ty0 - 1 + py, gx = tx0 - 1 + px;
            uint4 v = zero;
            if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
                v = *reinterpret_cast<const uint4*>(a.x + ((long long)(b * a.H + gy) * a.W + gx) * a.ldx + a.xoff + c0 +
                                                    h * 8);
            *reinterpret_cast<uint4*>(sx + p * PS + h * 8) = v;
        }
        for (int q = tid; q < 9 * CT_CO * 2; q += 128) {
            const int t = q / (CT_CO * 2), r = q - t * (CT_CO * 2);
            const int co = r >> 1, h = r & 1;
            uint4 v = zero;
            if (co0 + co < a.Co)
                v = *reinterpret_cast<const uint4*>(a.w + ((long long)t * a.Co + co0 + co) * a.Ci + c0 + h * 8);
            *reinterpret_cast<uint4*>(sw + (t * CT_CO + co) * PS + h * 8) = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            const int dy = t / 3 - 1, dx = t % 3 - 1;
            unsigned A[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int orow = warp * 2 + mi;
                const int pix = (lane & 7) + ((lane >> 3) & 1) * 8;
                const int sp = (orow + 1 + dy) * CT_IW + (pix + 1 + dx);
                ldsm_x4(A[mi], sx + sp * PS + (lane >> 4) * 8);
            }
#pragma unroll
            for (int nj = 0; nj < 8; nj += 2) {
                unsigned Bf[4];
                const int n = nj * 8 + (lane & 7) + (lane >> 4) * 8;
                ldsm_x4(Bf, sw + (t * CT_CO + n) * PS + ((lane >> 3) & 1) * 8);
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    mma_bf16(acc[mi][nj], A[mi], Bf[0], Bf[1]);
                    mma_bf16(acc[mi][nj + 1], A[mi], Bf[2], Bf[3]);
                }
            }
        }
        __syncthreads();
    }

    // epilogue: bias, activation, store (thread holds rows g, g+8 and channel pairs 2t, 2t+1)
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int gy = ty0 + warp * 2 + mi;
        if (gy >= a.H) continue;
#pragma unroll
        for (int nj = 0; nj < 8; ++nj) {
            const int co = co0 + nj * 8 + 2 * tq;
            if (co >= a.Co) continue;
            const float b0 = a.bias ? a.bias[co] : 0.f, b1 = a.bias ? a.bias[co + 1] : 0.f;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int gx = tx0 + g + 8 * hh;
                if (gx >= a.W) continue;
                float v0 = acc[mi][nj][2 * hh] + b0, v1 = acc[mi][nj][2 * hh + 1] + b1;
                if (a.act) {
                    v0 = v0 > 0.f ? v0 : SLOPE * v0;
                    v1 = v1 > 0.f ? v1 : SLOPE * v1;
                }
                const long long o = ((long long)(b * a.H + gy) * a.W + gx) * a.ldy + a.yoff + co;
                if (a.yf) {
                    a.yf[o] = v0;
                    a.yf[o + 1] = v1;
                } else {
                    *reinterpret_cast<__nv_bfloat162*>(a.y + o) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ tcgen05 descriptors

// shared-memory matrix descriptor: start address, leading (K-direction core-matrix) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // version 1, no swizzle
}

// ------------------------------------------------------------------ convolution forward, tcgen05
//
// The convolution on the 5th-generation tensor cores, with the output pixels as the MMA's M
// dimension and the output channels as N, so that layers with 32 or 64 output channels fill the
// tensor core.  A CTA computes 4 output rows x 30 pixels.  Its input tile is staged as 6 rows of 32
// pixels (x0 - 1 .. x0 + 30), so a tap (dy, dx) reads the 128 consecutive staged pixels that
// start at (1 + dy) 32 + (1 + dx): position m = 32 r + c of that window is output pixel (r, c)
// for c < 30 (c = 30, 31 fall beyond the tile and are not stored).  One chunk of 16 input
// channels is then 9 MMAs, M = 128, N = Co (up to 128, a multiple of 16), K = 16, into one
// accumulator of N columns in tensor memory; the next chunk's input and weights are copied
// asynchronously (cp.async) into the other of two buffers while the MMAs of this one run.
// Operands in the canonical K-major layout without swizzle: input [2 k-halves][200 pixels][8],
// weights [9 taps][2 k-halves][N channels][8]; 8-row groups 128 bytes apart.

constexpr int T2_GW = 32, T2_OW = T2_GW - 2, T2_OH = 4, T2_IH = T2_OH + 2;
constexpr int T2_NPIX = T2_IH * T2_GW + 8;                          // + zero slack for the last tap
constexpr int T2_SX = 2 * T2_NPIX * 8;                              // BF16 per input buffer
constexpr int T2_COMAX = 128;

__host__ __device__ constexpr int t2_smem_bytes(int cop)
{
    return (2 * T2_SX + 2 * 9 * 2 * cop * 8) * 2 + 64 + 1024;
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(sdst)), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// bounded wait for the phase of parity `parity` of an mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* mb, unsigned parity)
{
    unsigned done = 0;
    for (long it = 0; it < (1L << 26) && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(mb)), "r"(parity));
    }
    return done != 0;
}

__global__ void __launch_bounds__(128) k_conv3x3_tc(const ConvArgs a, int cop, int* err)
{
    extern __shared__ __align__(128) unsigned char t2_smem[];
    const int swn = 9 * 2 * cop * 8;
    bf16* const sx0 = reinterpret_cast<bf16*>(t2_smem);
    bf16* const sw0 = sx0 + 2 * T2_SX;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(t2_smem + (size_t)(2 * T2_SX + 2 * swn) * 2);
    unsigned* tslot = reinterpret_cast<unsigned*>(mbar + 2);

    const int n_cot = (a.Co + cop - 1) / cop;
    const int b = blockIdx.z / n_cot, co0 = (blockIdx.z % n_cot) * cop;
    const int tx0 = blockIdx.x * T2_OW, ty0 = blockIdx.y * T2_OH;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned ncol = cop <= 32 ? 32u : (cop <= 64 ? 64u : 128u);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;

    // asynchronous copies of chunk k (16 input channels) into buffer k & 1; out-of-range pixels
    // and channels are zero-filled
    auto stage = [&](int k) {
        const int c0 = k * 16;
        bf16* sx = sx0 + (k & 1) * T2_SX;
        bf16* sw = sw0 + (k & 1) * swn;
        for (int q = tid; q < T2_NPIX * 2; q += 128) {
            const int p = q >> 1, h = q & 1;
            const int py = p / T2_GW, px = p - py * T2_GW;
            const int gy = ty0 - 1 + py, gx = tx0 - 1 + px;
            const bool in = p < T2_IH * T2_GW && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
            const bf16* src = in ? a.x + ((long long)(b * a.H + gy) * a.W + gx) * a.ldx + a.xoff + c0 + h * 8 : a.x;
            cp_async16(sx + (h * T2_NPIX + p) * 8, src, in ? 16 : 0);
        }
        for (int q = tid; q < 9 * 2 * cop; q += 128) {
            const int t = q / (2 * cop), r = q - t * (2 * cop);
            const int h = r / cop, co = r - h * cop;
            const bool in = co0 + co < a.Co;
            const bf16* src = in ? a.w + ((long long)t * a.Co + co0 + co) * a.Ci + c0 + h * 8 : a.w;
            cp_async16(sw + ((t * 2 + h) * cop + co) * 8, src, in ? 16 : 0);
        }
        cp_async_commit();
    };

    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(cop >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const int nchunk = a.Ci / 16;
    bool ok = true;
    stage(0);
    for (int k = 0; k < nchunk; ++k) {
        if (k + 1 < nchunk) {
            // the other buffer was last read by the MMAs of chunk k - 1 (one decision for all threads)
            if (k >= 1 && !__syncthreads_and(mbar_wait(mbar + ((k - 1) & 1), (unsigned)(((k - 1) >> 1) & 1)))) {
                ok = false;
                break;
            }
            stage(k + 1);
            cp_async_wait<1>();     // chunk k has landed; chunk k + 1 may still be in flight
        } else {
            cp_async_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sxa = smem_u32(sx0 + (k & 1) * T2_SX), swa = smem_u32(sw0 + (k & 1) * swn);
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3 - 1, dx = t % 3 - 1;
                const int p0 = (1 + dy) * T2_GW + (1 + dx);
                const uint64_t ad = tc_desc(sxa + (unsigned)(p0 * 16), T2_NPIX * 16, 128);
                const uint64_t bd = tc_desc(swa + (unsigned)(t * 2 * cop * 16), (unsigned)(cop * 16), 128);
                const int acc = (k > 0 || t > 0) ? 1 : 0;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(mbar + (k & 1))));
        }
    }
    cp_async_wait<0>();     // no copy in flight past this point, whatever happened above
    if (ok) ok = mbar_wait(mbar + ((nchunk - 1) & 1), (unsigned)(((nchunk - 1) >> 1) & 1));
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (ok) {
        // epilogue: warp w holds output row w, lane c its column; columns of the accumulator are
        // the output channels co0 ..
        const int gy = ty0 + warp, gx = tx0 + lane;
        const bool valid = lane < T2_OW && gy < a.H && gx < a.W;
        const long long o0 = ((long long)(b * a.H + gy) * a.W + gx) * a.ldy + a.yoff + co0;
        for (int j = 0; j < cop; j += 16) {
            unsigned v[16];
            const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)j;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!valid) continue;
            float f[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int co = co0 + j + e;
                float val = __uint_as_float(v[e]) + ((a.bias && co < a.Co) ? a.bias[co] : 0.f);
                if (a.act) val = val > 0.f ? val : SLOPE * val;
                f[e] = val;
            }
            if (a.yf) {
                for (int e = 0; e < 16; ++e)
                    if (co0 + j + e < a.Co) a.yf[o0 + j + e] = f[e];
            } else if (co0 + j + 16 <= a.Co && ((o0 + j) & 7) == 0) {
                uint4 w0, w1;
                unsigned* u0 = &w0.x;
                unsigned* u1 = &w1.x;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const __nv_bfloat162 p = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
                    const __nv_bfloat162 q = __floats2bfloat162_rn(f[8 + 2 * e], f[8 + 2 * e + 1]);
                    u0[e] = *reinterpret_cast<const unsigned*>(&p);
                    u1[e] = *reinterpret_cast<const unsigned*>(&q);
                }
                *reinterpret_cast<uint4*>(a.y + o0 + j) = w0;
                *reinterpret_cast<uint4*>(a.y + o0 + j + 8) = w1;
            } else {
                for (int e = 0; e < 16; ++e)
                    if (co0 + j + e < a.Co) a.y[o0 + j + e] = __float2bfloat16_rn(f[e]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol));
    }
}

// ------------------------------------------------------------------ weight gradient

constexpr int WG_CO = 64, WG_CI = 16;           // output block of gw per CTA: [9][64][16]
constexpr int DZS = WG_CO + 8;                  // shared row of 64 channels + 8 pad (144 bytes)

struct WgradArgs {
    const bf16* x;          // layer input (pixel stride ldx, offset xoff)
    long long ldx;
    int xoff;
    const bf16* gz;         // gradient at the layer's pre-activation output [P][Co] (stride ldz)
    long long ldz;
    float* part;            // [S][9][Co][Ci] partial sums
    int B, H, W, Ci, Co, S;
};

__global__ void __launch_bounds__(128) k_conv_wgrad(const WgradArgs a)
{
    __shared__ __align__(16) bf16 sdz[CT_H * CT_W * DZS];
    __shared__ __align__(16) bf16 sx[CT_IH * CT_IW * PS];
    const int co0 = blockIdx.x * WG_CO, ci0 = blockIdx.y * WG_CI, s = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (a.W + CT_W - 1) / CT_W, tiles_y = (a.H + CT_H - 1) / CT_H;
    const int n_tiles = a.B * tiles_x * tiles_y;
    float acc[9][2][4];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[t][j][k] = 0.f;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);

    for (int tile = s; tile < n_tiles; tile += a.S) {
        const int b = tile / (tiles_x * tiles_y), r = tile - b * (tiles_x * tiles_y);
        const int ty0 = (r / tiles_x) * CT_H, tx0 = (r % tiles_x) * CT_W;
        // gz tile: 128 pixels x 64 channels (8 chunks of 8)
        for (int q = tid; q < CT_H * CT_W * 8; q += 128) {
            const int p = q >> 3, h = q & 7;
            const int gy = ty0 + p / CT_W, gx = tx0 + p % CT_W;
            uint4 v = zero;
            if (gy < a.H && gx < a.W && co0 + h * 8 < a.Co)
                v = *reinterpret_cast<const uint4*>(a.gz + ((long long)(b * a.H + gy) * a.W + gx) * a.ldz + co0 + h * 8);
            *reinterpret_cast<uint4*>(sdz + p * DZS + h * 8) = v;
        }
        for (int q = tid; q < CT_IH * CT_IW * 2; q += 128) {
            const int p = q >> 1, h = q & 1;
            const int py = p / CT_IW, px = p - py * CT_IW;
            const int gy = ty0 - 1 + py, gx = tx0 - 1 + px;
            uint4 v = zero;
            if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
                v = *reinterpret_cast<const uint4*>(a.x + ((long long)(b * a.H + gy) * a.W + gx) * a.ldx + a.xoff + ci0 +
                                                    h * 8);
            *reinterpret_cast<uint4*>(sx + p * PS + h * 8) = v;
        }
        __syncthreads();
        const int j = lane >> 3, rr = lane & 7;
#pragma unroll 1
        for (int ks = 0; ks < CT_H; ++ks) {             // 16 pixels (one tile row) per k-step
            unsigned A[4];                               // (co, p): rows p of sdz, transposed
            ldsm_x4_t(A, sdz + (ks * CT_W + rr + (j >> 1) * 8) * DZS + warp * 16 + (j & 1) * 8);
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3 - 1, dx = t % 3 - 1;
                unsigned Bf[4];                          // (p, ci): rows p of the shifted input
                const int k = rr + (j & 1) * 8;
                ldsm_x4_t(Bf, sx + ((ks + 1 + dy) * CT_IW + (k + 1 + dx)) * PS + (j >> 1) * 8);
                mma_bf16(acc[t][0], A, Bf[0], Bf[1]);
                mma_bf16(acc[t][1], A, Bf[2], Bf[3]);
            }
        }
        __syncthreads();
    }
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int jn = 0; jn < 2; ++jn)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int co = co0 + warp * 16 + g + 8 * hh;
                const int ci = ci0 + jn * 8 + 2 * tq;
                if (co < a.Co) {
                    float* o = a.part + (((long long)s * 9 + t) * a.Co + co) * a.Ci + ci;
                    o[0] = acc[t][jn][2 * hh];
                    o[1] = acc[t][jn][2 * hh + 1];
                }
            }
}

// sum of S partial arrays of n floats, in order: out[i] = sum_s part[s][i]
__global__ void k_sum_parts(const float* part, int S, long long n, float* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = 0.f;
    for (int s = 0; s < S; ++s) v += part[(long long)s * n + i];
    out[i] = v;
}

// bias gradient partials: part[s][o] = sum over pixels p = s, s + S, ... of gz[p][o]
__global__ void k_bias_parts(const bf16* gz, long long ldz, long long P, int Co, int S, float* part)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
    if (o >= Co) return;
    float v = 0.f;
    for (long long p = s; p < P; p += S) v += __bfloat162float(gz[p * ldz + o]);
    part[(long long)s * Co + o] = v;
}

// w'[t'][c][o] = w[8 - t'][o][c]
__global__ void k_flip_transpose(const bf16* w, int Co, int Ci, bf16* wt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = 9LL * Co * Ci;
    if (i >= n) return;
    const int t = (int)(i / ((long long)Co * Ci));
    const long long r = i - (long long)t * Co * Ci;
    const int o = (int)(r / Ci), c = (int)(r - (long long)o * Ci);
    wt[((long long)(8 - t) * Ci + c) * Co + o] = w[i];
}

// ------------------------------------------------------------------ joins and pointwise

// gz = gy * LeakyReLU'(from the sign of the activation output y); gy BF16 or FP32
__global__ void k_leaky_bwd(const bf16* y, long long ldy, int yoff, const bf16* gy, const float* gyf, long long ldg,
                            int goff, long long P, int C, bf16* gz)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * C) return;
    const long long p = i / C;
    const int c = (int)(i - p * C);
    const float g = gyf ? gyf[p * ldg + goff + c] : __bfloat162float(gy[p * ldg + goff + c]);
    const float v = __bfloat162float(y[p * ldy + yoff + c]);
    gz[i] = __float2bfloat16_rn(v > 0.f ? g : SLOPE * g);
}

// FP32 -> BF16 (dense)
__global__ void k_to_bf16(const float* x, long long n, bf16* y)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// y[b, i, j, c] = mean of x[b, 2i + {0,1}, 2j + {0,1}, c]  (x: stride ldx, offset xoff)
__global__ void k_pool2(const bf16* x, long long ldx, int xoff, int B, int H, int W, int C, bf16* y)
{
    const long long n = (long long)B * (H / 2) * (W / 2) * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int j = (int)(r % (W / 2));
    r /= (W / 2);
    const int ii = (int)(r % (H / 2));
    const int b = (int)(r / (H / 2));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
            s += __bfloat162float(x[((long long)(b * H + 2 * ii + dy) * W + 2 * j + dx) * ldx + xoff + c]);
    y[i] = __float2bfloat16_rn(0.25f * s);
}

// g[b, y, x, c] = gp[b, y/2, x/2, c] / 4 + gs[b, y, x, c] (gs: stride lds, offset soff)
__global__ void k_pool2_bwd_add(const bf16* gp, const bf16* gs, long long lds, int soff, int B, int H, int W, int C,
                                bf16* g)
{
    const long long n = (long long)B * H * W * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int x = (int)(p % W);
    const long long r = p / W;
    const int y = (int)(r % H), b = (int)(r / H);
    const float v = 0.25f * __bfloat162float(gp[((long long)(b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]) +
                    __bfloat162float(gs[p * lds + soff + c]);
    g[i] = __float2bfloat16_rn(v);
}

// y[b, y, x, yoff + c] = x[b, y/2, x/2, c]   (y at full resolution H x W, stride ldy)
__global__ void k_up2(const bf16* x, int B, int H, int W, int C, bf16* y, long long ldy, int yoff)
{
    const long long n = (long long)B * H * W * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int xx = (int)(p % W);
    const long long r = p / W;
    const int yy = (int)(r % H), b = (int)(r / H);
    y[p * ldy + yoff + c] = x[((long long)(b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c];
}

// g[b, i, j, c] = sum of gy[b, 2i + {0,1}, 2j + {0,1}, goff + c]  (gy at H x W, stride ldg)
__global__ void k_up2_bwd(const bf16* gy, long long ldg, int goff, int B, int H, int W, int C, bf16* g)
{
    const long long n = (long long)B * (H / 2) * (W / 2) * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    long long r = i / C;
    const int j = (int)(r % (W / 2));
    r /= (W / 2);
    const int ii = (int)(r % (H / 2));
    const int b = (int)(r / (H / 2));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
            s += __bfloat162float(gy[((long long)(b * H + 2 * ii + dy) * W + 2 * j + dx) * ldg + goff + c]);
    g[i] = __float2bfloat16_rn(s);
}

// masked mean squared error: per-block partial sums of (pred - target)^2 and the gradient
// 2 (pred - target) mask / n
__global__ void k_mse(const float* pred, const float* target, const float* mask, long long P, float inv_n,
                      float* grad, double* part)
{
    __shared__ double red[256];
    double acc = 0.0;
    const long long n = P * 16;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = (pred[i] - target[i]) * mask[i & 15];
        acc += (double)d * d;
        grad[i] = 2.f * d * inv_n;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam on FP32 master weights; writes the BF16 copy of the weights (not of the biases)
__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, bf16* pb)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
}

}  // namespace net
}  // namespace vlb

// ==================================================================== host side

using vlb::net::bf16;

namespace {

struct NetLayer {
    const char* name;
    int ci, co;
    bool act;
    long long w_off, b_off;      // offsets of w [9][co][ci] and b [co] in the flat parameter array
};

// (name, Ci, Co, activation) in execution order; the same table as the FP64 oracle
const struct {
    const char* name;
    int ci, co;
    bool act;
} NET_LAYERS[] = {
    {"e0a", 16, 32, true},       {"e0b", 32, 32, true},  {"e1a", 32, 64, true},  {"e1b", 64, 64, true},
    {"e2a", 64, 96, true},       {"e2b", 96, 96, true},  {"bta", 96, 128, true}, {"btb", 128, 128, true},
    {"d2a", 128 + 96, 96, true}, {"d2b", 96, 96, true},  {"d1a", 96 + 64, 64, true}, {"d1b", 64, 64, true},
    {"d0a", 64 + 32, 32, true},  {"d0b", 32, 32, true},  {"head", 32, 16, false},
};
constexpr int N_LAYERS = 15;
enum { E0A, E0B, E1A, E1B, E2A, E2B, BTA, BTB, D2A, D2B, D1A, D1B, D0A, D0B, HEAD };

int blocks(long long n, int t = 256) { return (int)((n + t - 1) / t); }

}  // namespace

struct lb_net {
    int B = 0, H = 0, W = 0;
    cudaStream_t stream = nullptr;
    NetLayer L[N_LAYERS];
    long long n_params = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16* wb = nullptr;          // BF16 copy of the parameters (weights used)
    bf16* wt = nullptr;          // flipped, transposed BF16 weights for the data gradients
    // activations (BF16 NHWC)
    bf16 *x_in = nullptr, *t0 = nullptr, *cat0 = nullptr, *p1 = nullptr, *t1 = nullptr, *cat1 = nullptr;
    bf16 *p2 = nullptr, *t2 = nullptr, *cat2 = nullptr, *p3 = nullptr, *t3 = nullptr, *bt = nullptr;
    bf16 *u2 = nullptr, *d2 = nullptr, *u1 = nullptr, *d1 = nullptr, *u0 = nullptr, *d0 = nullptr;
    float* y = nullptr;          // head output FP32 [P0][16]
    float* gy = nullptr;         // loss gradient FP32 [P0][16]
    bf16* gs[6] = {};            // gradient scratch, P0 x 96 each
    float* part = nullptr;       // weight-gradient partials
    long long part_n = 0;
    double* lpart = nullptr;     // loss partials
    int adam_t = 0;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

using namespace vlb::net;

int nfail(lb_net* n, int code, const std::string& msg)
{
    if (n) n->err = msg;
    return code;
}

#define NCK(n, call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (n) n->err = std::string(#call) + ": " + cudaGetErrorString(e_);        \
            return e_ == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA;             \
        }                                                                              \
    } while (0)

template <class T>
cudaError_t nalloc(lb_net* n, T** ptr, long long count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (size_t)count);
    if (e == cudaSuccess) {
        n->allocs.push_back(q);
        *ptr = static_cast<T*>(q);
    }
    return e;
}

int S_parts(int B, int H, int W)
{
    const int tiles = B * ((W + CT_W - 1) / CT_W) * ((H + CT_H - 1) / CT_H);
    return tiles < 64 ? tiles : 64;
}

// convolution kernel: 0 mma.sync, 1 tcgen05 (TMEM accumulators, the default)
int g_conv_kernel = 1;
int* g_conv_err = nullptr;      // device flag: a tcgen05 convolution's bounded wait gave up

cudaError_t conv_fwd(cudaStream_t s, const bf16* x, long long ldx, int xoff, const bf16* w, const float* bias, bf16* y,
                     float* yf, long long ldy, int yoff, int B, int H, int W, int Ci, int Co, int act)
{
    ConvArgs a;
    a.x = x; a.ldx = ldx; a.xoff = xoff; a.w = w; a.bias = bias; a.y = y; a.yf = yf; a.ldy = ldy; a.yoff = yoff;
    a.B = B; a.H = H; a.W = W; a.Ci = Ci; a.Co = Co; a.act = act;
    if (g_conv_kernel == 1) {
        static unsigned long long attr = 0;      // per device
        if (!vlb::done_on_device(attr)) {
            cudaError_t e =
                cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, t2_smem_bytes(T2_COMAX));
            if (e != cudaSuccess) {
                attr = 0;
                return e;
            }
        }
        if (!g_conv_err) {
            cudaError_t e = cudaMalloc(&g_conv_err, sizeof(int));
            if (e == cudaSuccess) e = cudaMemset(g_conv_err, 0, sizeof(int));
            if (e != cudaSuccess) return e;
        }
        if (Ci % 16 != 0) return cudaErrorInvalidValue;
        int cop = (Co + 15) / 16 * 16;
        if (cop > T2_COMAX) cop = T2_COMAX;
        dim3 grid((W + T2_OW - 1) / T2_OW, (H + T2_OH - 1) / T2_OH, B * ((Co + cop - 1) / cop));
        k_conv3x3_tc<<<grid, 128, t2_smem_bytes(cop), s>>>(a, cop, g_conv_err);
        return cudaGetLastError();
    }
    dim3 grid((W + CT_W - 1) / CT_W, (H + CT_H - 1) / CT_H, B * ((Co + CT_CO - 1) / CT_CO));
    k_conv3x3<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// weight and bias gradients of one layer from its input x and pre-activation gradient gz
cudaError_t conv_wgrad(cudaStream_t s, const bf16* x, long long ldx, int xoff, const bf16* gz, int B, int H, int W,
                       int Ci, int Co, float* part, float* gw, float* gb)
{
    const int S = S_parts(B, H, W);
    WgradArgs a;
    a.x = x; a.ldx = ldx; a.xoff = xoff; a.gz = gz; a.ldz = Co; a.part = part;
    a.B = B; a.H = H; a.W = W; a.Ci = Ci; a.Co = Co; a.S = S;
    dim3 grid((Co + WG_CO - 1) / WG_CO, Ci / WG_CI, S);
    k_conv_wgrad<<<grid, 128, 0, s>>>(a);
    const long long nw = 9LL * Co * Ci;
    k_sum_parts<<<blocks(nw), 256, 0, s>>>(part, S, nw, gw);
    const long long P = (long long)B * H * W;
    k_bias_parts<<<dim3((Co + 127) / 128, S), 128, 0, s>>>(gz, Co, P, Co, S, part);
    k_sum_parts<<<blocks(Co), 256, 0, s>>>(part, S, Co, gb);
    return cudaGetLastError();
}

cudaError_t refresh_weights(lb_net* n)
{
    for (int l = 0; l < N_LAYERS; ++l) {
        const NetLayer& Ly = n->L[l];
        const long long nw = 9LL * Ly.co * Ly.ci;
        k_flip_transpose<<<blocks(nw), 256, 0, n->stream>>>(n->wb + Ly.w_off, Ly.co, Ly.ci, n->wt + Ly.w_off);
    }
    return cudaGetLastError();
}

// forward of layer l: input (x, ldx, xoff) at resolution H x W -> output (y | yf, ldy, yoff)
cudaError_t layer_fwd(lb_net* n, int l, const bf16* x, long long ldx, int xoff, bf16* y, float* yf, long long ldy,
                      int yoff, int H, int W)
{
    const NetLayer& Ly = n->L[l];
    return conv_fwd(n->stream, x, ldx, xoff, n->wb + Ly.w_off, n->p + Ly.b_off, y, yf, ldy, yoff, n->B, H, W, Ly.ci,
                    Ly.co, Ly.act ? 1 : 0);
}

// backward of layer l given the gradient at its (activated) output g_out (BF16, stride ldg,
// offset goff) and its output y (stride ldy, offset yoff): weight/bias gradients, and the
// gradient at its input into gx (dense [P][ci]) when gx is not null.  gz: scratch [P][co].
cudaError_t layer_bwd(lb_net* n, int l, const bf16* x, long long ldx, int xoff, const bf16* y, long long ldy, int yoff,
                      const bf16* g_out, long long ldg, int goff, bf16* gz, bf16* gx, int H, int W)
{
    const NetLayer& Ly = n->L[l];
    const long long P = (long long)n->B * H * W;
    const bf16* gzz = g_out;
    if (Ly.act) {
        k_leaky_bwd<<<blocks(P * Ly.co), 256, 0, n->stream>>>(y, ldy, yoff, g_out, nullptr, ldg, goff, P, Ly.co, gz);
        gzz = gz;
    }
    cudaError_t e = conv_wgrad(n->stream, x, ldx, xoff, gzz, n->B, H, W, Ly.ci, Ly.co, n->part, n->g + Ly.w_off,
                               n->g + Ly.b_off);
    if (e != cudaSuccess) return e;
    if (gx)
        e = conv_fwd(n->stream, gzz, Ly.co, 0, n->wt + Ly.w_off, nullptr, gx, nullptr, Ly.ci, 0, n->B, H, W, Ly.co,
                     Ly.ci, 0);
    return e;
}

int net_forward(lb_net* n)
{
    const int H = n->H, W = n->W, B = n->B;
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
    cudaStream_t s = n->stream;
    NCK(n, layer_fwd(n, E0A, n->x_in, 16, 0, n->t0, nullptr, 32, 0, H, W));
    NCK(n, layer_fwd(n, E0B, n->t0, 32, 0, n->cat0, nullptr, 96, 64, H, W));
    k_pool2<<<blocks((long long)B * H1 * W1 * 32), 256, 0, s>>>(n->cat0, 96, 64, B, H, W, 32, n->p1);
    NCK(n, layer_fwd(n, E1A, n->p1, 32, 0, n->t1, nullptr, 64, 0, H1, W1));
    NCK(n, layer_fwd(n, E1B, n->t1, 64, 0, n->cat1, nullptr, 160, 96, H1, W1));
    k_pool2<<<blocks((long long)B * H2 * W2 * 64), 256, 0, s>>>(n->cat1, 160, 96, B, H1, W1, 64, n->p2);
    NCK(n, layer_fwd(n, E2A, n->p2, 64, 0, n->t2, nullptr, 96, 0, H2, W2));
    NCK(n, layer_fwd(n, E2B, n->t2, 96, 0, n->cat2, nullptr, 224, 128, H2, W2));
    k_pool2<<<blocks((long long)B * H3 * W3 * 96), 256, 0, s>>>(n->cat2, 224, 128, B, H2, W2, 96, n->p3);
    NCK(n, layer_fwd(n, BTA, n->p3, 96, 0, n->t3, nullptr, 128, 0, H3, W3));
    NCK(n, layer_fwd(n, BTB, n->t3, 128, 0, n->bt, nullptr, 128, 0, H3, W3));
    k_up2<<<blocks((long long)B * H2 * W2 * 128), 256, 0, s>>>(n->bt, B, H2, W2, 128, n->cat2, 224, 0);
    NCK(n, layer_fwd(n, D2A, n->cat2, 224, 0, n->u2, nullptr, 96, 0, H2, W2));
    NCK(n, layer_fwd(n, D2B, n->u2, 96, 0, n->d2, nullptr, 96, 0, H2, W2));
    k_up2<<<blocks((long long)B * H1 * W1 * 96), 256, 0, s>>>(n->d2, B, H1, W1, 96, n->cat1, 160, 0);
    NCK(n, layer_fwd(n, D1A, n->cat1, 160, 0, n->u1, nullptr, 64, 0, H1, W1));
    NCK(n, layer_fwd(n, D1B, n->u1, 64, 0, n->d1, nullptr, 64, 0, H1, W1));
    k_up2<<<blocks((long long)B * H * W * 64), 256, 0, s>>>(n->d1, B, H, W, 64, n->cat0, 96, 0);
    NCK(n, layer_fwd(n, D0A, n->cat0, 96, 0, n->u0, nullptr, 32, 0, H, W));
    NCK(n, layer_fwd(n, D0B, n->u0, 32, 0, n->d0, nullptr, 32, 0, H, W));
    NCK(n, layer_fwd(n, HEAD, n->d0, 32, 0, nullptr, n->y, 16, 0, H, W));
    NCK(n, cudaGetLastError());
    return LB_OK;
}

// gradients of sum(gy * y) for every parameter (overwritten), from the activations of the last
// forward; gy: FP32 [P0][16]
int net_backward(lb_net* n, const float* gy)
{
    const int H = n->H, W = n->W, B = n->B;
    const int H1 = H / 2, W1 = W / 2, H2 = H / 4, W2 = W / 4, H3 = H / 8, W3 = W / 8;
    cudaStream_t s = n->stream;
    bf16 *A = n->gs[0], *Bz = n->gs[1], *C = n->gs[2], *D = n->gs[3], *E = n->gs[4], *F = n->gs[5];
    const long long P0 = (long long)B * H * W;
    k_to_bf16<<<blocks(P0 * 16), 256, 0, s>>>(gy, P0 * 16, Bz);
    NCK(n, layer_bwd(n, HEAD, n->d0, 32, 0, nullptr, 0, 0, Bz, 16, 0, nullptr, A, H, W));            // A = g d0
    NCK(n, layer_bwd(n, D0B, n->u0, 32, 0, n->d0, 32, 0, A, 32, 0, Bz, A, H, W));                    // A = g u0
    NCK(n, layer_bwd(n, D0A, n->cat0, 96, 0, n->u0, 32, 0, A, 32, 0, Bz, C, H, W));                  // C = g cat0
    k_up2_bwd<<<blocks((long long)B * H1 * W1 * 64), 256, 0, s>>>(C, 96, 0, B, H, W, 64, A);         // A = g d1
    NCK(n, layer_bwd(n, D1B, n->u1, 64, 0, n->d1, 64, 0, A, 64, 0, Bz, A, H1, W1));                  // A = g u1
    NCK(n, layer_bwd(n, D1A, n->cat1, 160, 0, n->u1, 64, 0, A, 64, 0, Bz, D, H1, W1));               // D = g cat1
    k_up2_bwd<<<blocks((long long)B * H2 * W2 * 96), 256, 0, s>>>(D, 160, 0, B, H1, W1, 96, A);      // A = g d2
    NCK(n, layer_bwd(n, D2B, n->u2, 96, 0, n->d2, 96, 0, A, 96, 0, Bz, A, H2, W2));                  // A = g u2
    NCK(n, layer_bwd(n, D2A, n->cat2, 224, 0, n->u2, 96, 0, A, 96, 0, Bz, E, H2, W2));               // E = g cat2
    k_up2_bwd<<<blocks((long long)B * H3 * W3 * 128), 256, 0, s>>>(E, 224, 0, B, H2, W2, 128, A);    // A = g bt
    NCK(n, layer_bwd(n, BTB, n->t3, 128, 0, n->bt, 128, 0, A, 128, 0, Bz, A, H3, W3));               // A = g t3
    NCK(n, layer_bwd(n, BTA, n->p3, 96, 0, n->t3, 128, 0, A, 128, 0, Bz, F, H3, W3));                // F = g p3
    k_pool2_bwd_add<<<blocks((long long)B * H2 * W2 * 96), 256, 0, s>>>(F, E, 224, 128, B, H2, W2, 96, A);  // g e2
    NCK(n, layer_bwd(n, E2B, n->t2, 96, 0, n->cat2, 224, 128, A, 96, 0, Bz, A, H2, W2));             // A = g t2
    NCK(n, layer_bwd(n, E2A, n->p2, 64, 0, n->t2, 96, 0, A, 96, 0, Bz, F, H2, W2));                  // F = g p2
    k_pool2_bwd_add<<<blocks((long long)B * H1 * W1 * 64), 256, 0, s>>>(F, D, 160, 96, B, H1, W1, 64, A);   // g e1
    NCK(n, layer_bwd(n, E1B, n->t1, 64, 0, n->cat1, 160, 96, A, 64, 0, Bz, A, H1, W1));              // A = g t1
    NCK(n, layer_bwd(n, E1A, n->p1, 32, 0, n->t1, 64, 0, A, 64, 0, Bz, F, H1, W1));                  // F = g p1
    k_pool2_bwd_add<<<blocks((long long)B * H * W * 32), 256, 0, s>>>(F, C, 96, 64, B, H, W, 32, A);        // g e0
    NCK(n, layer_bwd(n, E0B, n->t0, 32, 0, n->cat0, 96, 64, A, 32, 0, Bz, A, H, W));                 // A = g t0
    NCK(n, layer_bwd(n, E0A, n->x_in, 16, 0, n->t0, 32, 0, A, 32, 0, Bz, nullptr, H, W));
    NCK(n, cudaGetLastError());
    return LB_OK;
}

}  // namespace

extern "C" {

int lb_net_create(int32_t batch, int32_t height, int32_t width, uint64_t seed, void* stream, lb_net** out)
{
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (batch < 1 || height < 8 || width < 8 || height % 8 || width % 8 || (long long)batch * height * width > (1LL << 28))
        return LB_EINVAL;
    lb_net* n = new lb_net();
    n->B = batch;
    n->H = height;
    n->W = width;
    n->stream = (cudaStream_t)stream;
    long long off = 0;
    for (int l = 0; l < N_LAYERS; ++l) {
        NetLayer& Ly = n->L[l];
        Ly.name = NET_LAYERS[l].name;
        Ly.ci = NET_LAYERS[l].ci;
        Ly.co = NET_LAYERS[l].co;
        Ly.act = NET_LAYERS[l].act;
        Ly.w_off = off;
        off += 9LL * Ly.ci * Ly.co;
        Ly.b_off = off;
        off += Ly.co;
    }
    n->n_params = off;
    auto cleanup = [&](int code) { lb_net_destroy(n); return code; };
    const long long P0 = (long long)batch * height * width, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
    long long max_part = 0;
    for (int l = 0; l < N_LAYERS; ++l) max_part = std::max<long long>(max_part, 9LL * n->L[l].co * n->L[l].ci);
    max_part = std::max<long long>(max_part, 128) * 64;
    n->part_n = max_part;
    if (nalloc(n, &n->p, off) || nalloc(n, &n->g, off) || nalloc(n, &n->m, off) || nalloc(n, &n->v, off) ||
        nalloc(n, &n->wb, off) || nalloc(n, &n->wt, off) || nalloc(n, &n->x_in, P0 * 16) ||
        nalloc(n, &n->t0, P0 * 32) || nalloc(n, &n->cat0, P0 * 96) || nalloc(n, &n->p1, P1 * 32) ||
        nalloc(n, &n->t1, P1 * 64) || nalloc(n, &n->cat1, P1 * 160) || nalloc(n, &n->p2, P2 * 64) ||
        nalloc(n, &n->t2, P2 * 96) || nalloc(n, &n->cat2, P2 * 224) || nalloc(n, &n->p3, P3 * 96) ||
        nalloc(n, &n->t3, P3 * 128) || nalloc(n, &n->bt, P3 * 128) || nalloc(n, &n->u2, P2 * 96) ||
        nalloc(n, &n->d2, P2 * 96) || nalloc(n, &n->u1, P1 * 64) || nalloc(n, &n->d1, P1 * 64) ||
        nalloc(n, &n->u0, P0 * 32) || nalloc(n, &n->d0, P0 * 32) || nalloc(n, &n->y, P0 * 16) ||
        nalloc(n, &n->gy, P0 * 16) || nalloc(n, &n->part, max_part) || nalloc(n, &n->lpart, 1024))
        return cleanup(LB_ENOMEM);
    for (int i = 0; i < 6; ++i)
        if (nalloc(n, &n->gs[i], P0 * 96)) return cleanup(LB_ENOMEM);
    // He initialisation from a seeded generator (host, FP64 Box-Muller), zero biases
    std::vector<float> h(off, 0.f);
    uint64_t st = seed * 0x9E3779B97F4A7C15ULL + 1;
    auto next = [&]() {   // splitmix64
        uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    for (int l = 0; l < N_LAYERS; ++l) {
        const NetLayer& Ly = n->L[l];
        const double sd = Ly.act ? std::sqrt(2.0 / (9.0 * Ly.ci)) : 0.1 * std::sqrt(1.0 / (9.0 * Ly.ci));
        for (long long i = 0; i < 9LL * Ly.ci * Ly.co; ++i) {
            const double u1 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            const double u2 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            h[Ly.w_off + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    const int rc = lb_net_set_params(n, h.data(), off);
    if (rc != LB_OK) return cleanup(rc);
    if (cudaMemset(n->m, 0, sizeof(float) * off) != cudaSuccess || cudaMemset(n->v, 0, sizeof(float) * off) != cudaSuccess ||
        cudaMemset(n->g, 0, sizeof(float) * off) != cudaSuccess)
        return cleanup(LB_ECUDA);
    *out = n;
    return LB_OK;
}

int64_t lb_net_num_params(const lb_net* n) { return n ? n->n_params : -1; }

int lb_net_shape(const lb_net* n, int32_t* batch, int32_t* height, int32_t* width)
{
    if (!n || !batch || !height || !width) return LB_EINVAL;
    *batch = n->B;
    *height = n->H;
    *width = n->W;
    return LB_OK;
}

int lb_net_set_params(lb_net* n, const float* host, int64_t count)
{
    if (!n || !host) return LB_EINVAL;
    if (count != n->n_params) return nfail(n, LB_EINVAL, "parameter count mismatch");
    NCK(n, cudaMemcpyAsync(n->p, host, sizeof(float) * count, cudaMemcpyHostToDevice, n->stream));
    k_to_bf16<<<blocks(count), 256, 0, n->stream>>>(n->p, count, n->wb);
    NCK(n, refresh_weights(n));
    NCK(n, cudaStreamSynchronize(n->stream));
    n->adam_t = 0;
    return LB_OK;
}

int lb_net_get_params(lb_net* n, float* host, int64_t count)
{
    if (!n || !host) return LB_EINVAL;
    if (count != n->n_params) return nfail(n, LB_EINVAL, "parameter count mismatch");
    NCK(n, cudaMemcpyAsync(host, n->p, sizeof(float) * count, cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    return LB_OK;
}

int lb_net_get_grads(lb_net* n, float* host, int64_t count)
{
    if (!n || !host) return LB_EINVAL;
    if (count != n->n_params) return nfail(n, LB_EINVAL, "parameter count mismatch");
    NCK(n, cudaMemcpyAsync(host, n->g, sizeof(float) * count, cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    return LB_OK;
}

int lb_net_forward(lb_net* n, const void* x, float* y)
{
    if (!n || !x) return LB_EINVAL;
    const long long P0 = (long long)n->B * n->H * n->W;
    NCK(n, cudaMemcpyAsync(n->x_in, x, sizeof(bf16) * P0 * 16, cudaMemcpyDeviceToDevice, n->stream));
    const int rc = net_forward(n);
    if (rc == LB_OK && y) NCK(n, cudaMemcpyAsync(y, n->y, sizeof(float) * P0 * 16, cudaMemcpyDeviceToDevice, n->stream));
    return rc;
}

const float* lb_net_output(const lb_net* n) { return n ? n->y : nullptr; }

int lb_net_backward(lb_net* n, const float* grad_out)
{
    if (!n || !grad_out) return LB_EINVAL;
    return net_backward(n, grad_out);
}

int lb_net_mse(lb_net* n, const float* target, const float* mask16, double* loss)
{
    if (!n || !target || !mask16) return LB_EINVAL;
    const long long P0 = (long long)n->B * n->H * n->W;
    float msum = 0.f;
    for (int c = 0; c < 16; ++c) msum += mask16[c];
    if (!(msum > 0.f)) return nfail(n, LB_EINVAL, "empty channel mask");
    float* mdev = reinterpret_cast<float*>(n->lpart + 512);   // 16 floats after the loss partials
    NCK(n, cudaMemcpyAsync(mdev, mask16, sizeof(float) * 16, cudaMemcpyHostToDevice, n->stream));
    const int nb = 256;
    k_mse<<<nb, 256, 0, n->stream>>>(n->y, target, mdev, P0, (float)(1.0 / ((double)P0 * msum)), n->gy, n->lpart);
    NCK(n, cudaGetLastError());
    if (loss) {
        std::vector<double> h(nb);
        NCK(n, cudaMemcpyAsync(h.data(), n->lpart, sizeof(double) * nb, cudaMemcpyDeviceToHost, n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
        double s = 0.0;
        for (int i = 0; i < nb; ++i) s += h[i];
        *loss = s / ((double)P0 * msum);
    }
    return LB_OK;
}

const float* lb_net_loss_grad(const lb_net* n) { return n ? n->gy : nullptr; }

int lb_net_adam(lb_net* n, float lr, float beta1, float beta2, float eps)
{
    if (!n || !(lr >= 0.f)) return LB_EINVAL;
    n->adam_t += 1;
    const float c1 = 1.f / (1.f - std::pow(beta1, (float)n->adam_t));
    const float c2 = 1.f / (1.f - std::pow(beta2, (float)n->adam_t));
    k_adam<<<blocks(n->n_params), 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, n->n_params, lr, beta1, beta2, eps, c1,
                                                       c2, n->wb);
    NCK(n, cudaGetLastError());
    NCK(n, refresh_weights(n));
    return LB_OK;
}

int lb_net_train_step(lb_net* n, const void* x, const float* target, const float* mask16, float lr, double* loss)
{
    int rc = lb_net_forward(n, x, nullptr);
    if (rc == LB_OK) rc = lb_net_mse(n, target, mask16, loss);
    if (rc == LB_OK) rc = net_backward(n, n->gy);
    if (rc == LB_OK) rc = lb_net_adam(n, lr, 0.9f, 0.999f, 1e-8f);
    return rc;
}

int lb_net_activation(lb_net* n, int32_t which, void* host, int64_t bytes)
{
    if (!n || !host) return LB_EINVAL;
    const long long P0 = (long long)n->B * n->H * n->W, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
    const struct {
        const void* p;
        long long n;
    } T[] = {{n->x_in, P0 * 16}, {n->t0, P0 * 32}, {n->cat0, P0 * 96}, {n->p1, P1 * 32}, {n->t1, P1 * 64},
             {n->cat1, P1 * 160}, {n->p2, P2 * 64}, {n->t2, P2 * 96}, {n->cat2, P2 * 224}, {n->p3, P3 * 96},
             {n->t3, P3 * 128}, {n->bt, P3 * 128}, {n->u2, P2 * 96}, {n->d2, P2 * 96}, {n->u1, P1 * 64},
             {n->d1, P1 * 64}, {n->u0, P0 * 32}, {n->d0, P0 * 32}};
    if (which < 0 || which >= (int)(sizeof T / sizeof T[0])) return nfail(n, LB_EINVAL, "no such activation");
    if (bytes != (int64_t)(T[which].n * sizeof(bf16))) return nfail(n, LB_EINVAL, "bytes mismatch");
    NCK(n, cudaMemcpyAsync(host, T[which].p, (size_t)bytes, cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    return LB_OK;
}

const char* lb_net_last_error(const lb_net* n) { return n ? n->err.c_str() : "null network"; }

void lb_net_destroy(lb_net* n)
{
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void* q : n->allocs) cudaFree(q);
    delete n;
}

// ---- single-layer entry points (the building blocks, for tests against the oracle) ----

int lb_conv_kernel(int32_t kernel)
{
    if (kernel != 0 && kernel != 1) return LB_EINVAL;
    g_conv_kernel = kernel;
    return LB_OK;
}

int lb_conv_status(void)
{
    if (!g_conv_err) return LB_OK;
    int e = 0;
    if (cudaMemcpy(&e, g_conv_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LB_ECUDA;
    if (e) {
        const int z = 0;
        cudaMemcpy(g_conv_err, &z, sizeof(int), cudaMemcpyHostToDevice);
        return LB_ETIMEOUT;
    }
    return LB_OK;
}

int lb_conv3x3(const void* x, int64_t ldx, int32_t xoff, const void* w, const float* bias, void* y, float* yf,
               int64_t ldy, int32_t yoff, int32_t B, int32_t H, int32_t W, int32_t Ci, int32_t Co, int32_t act,
               void* stream)
{
    if (!x || !w || (!y && !yf) || B < 1 || H < 1 || W < 1 || Ci < 16 || Co < 16 || Ci % 16 || Co % 8 || ldx % 8 ||
        xoff % 8 || ldx < xoff + Ci || ldy < yoff + Co || yoff % 2)
        return LB_EINVAL;
    return conv_fwd((cudaStream_t)stream, static_cast<const bf16*>(x), ldx, xoff, static_cast<const bf16*>(w), bias,
                    static_cast<bf16*>(y), yf, ldy, yoff, B, H, W, Ci, Co, act ? 1 : 0) == cudaSuccess
               ? LB_OK
               : LB_ECUDA;
}

int lb_conv3x3_dgrad(const void* gz, const void* w, void* gx, int32_t B, int32_t H, int32_t W, int32_t Ci, int32_t Co,
                     void* stream)
{
    if (!gz || !w || !gx || B < 1 || H < 1 || W < 1 || Ci < 16 || Co < 16 || Ci % 16 || Co % 16) return LB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    bf16* wt = nullptr;
    if (cudaMalloc(&wt, sizeof(bf16) * 9 * (size_t)Ci * Co) != cudaSuccess) return LB_ENOMEM;
    k_flip_transpose<<<blocks(9LL * Ci * Co), 256, 0, s>>>(static_cast<const bf16*>(w), Co, Ci, wt);
    cudaError_t e = conv_fwd(s, static_cast<const bf16*>(gz), Co, 0, wt, nullptr, static_cast<bf16*>(gx), nullptr, Ci, 0,
                             B, H, W, Co, Ci, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(wt);
    return e == cudaSuccess ? LB_OK : LB_ECUDA;
}

int lb_conv3x3_wgrad(const void* x, const void* gz, float* gw, float* gb, int32_t B, int32_t H, int32_t W, int32_t Ci,
                     int32_t Co, void* stream)
{
    if (!x || !gz || !gw || !gb || B < 1 || H < 1 || W < 1 || Ci < 16 || Co < 8 || Ci % 16 || Co % 8) return LB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int S = S_parts(B, H, W);
    float* part = nullptr;
    const long long np = (long long)S * std::max<long long>(9LL * Ci * Co, Co);
    if (cudaMalloc(&part, sizeof(float) * (size_t)np) != cudaSuccess) return LB_ENOMEM;
    cudaError_t e = conv_wgrad(s, static_cast<const bf16*>(x), Ci, 0, static_cast<const bf16*>(gz), B, H, W, Ci, Co,
                               part, gw, gb);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(part);
    return e == cudaSuccess ? LB_OK : LB_ECUDA;
}

}  // extern "C"
