// lb_nodes.cu -- the node kernel: one CTA per ring (App. A).
//
// Per step, after the fused lattice kernel of the same step has written u(t) (and, on readout
// steps, f^p(t)) onto the ring's work box:
//   * readout (t % every == 0): restoring force sum_a sum_r f^p(r) K(R_a - r) and the centre of
//     mass of R(t), FP64 sums in a fixed order; CTA 0 also reduces the per-CTA partial sums of
//     the lattice kernel (mass, momentum, total force) in a fixed order;
//   * overdamped advection dR/dt = v(R) by Heun on the frozen u(t): R* = R + v(R),
//     R' = R + (v(R) + v(R*))/2, v interpolated with the cosine kernel (FP32 weights);
//   * Lagrangian forces of R' (Eq. Const: springs, angle terms, constant pull split over the
//     nodes), gathered per node without atomics, and the work box of R' for the next step.
// Node positions are kept in FP64 (O(N_nodes) data); the lattice kernel sees them as int32 cell +
// FP32 fraction with FP32 forces.  The last CTA to finish advances the step counter.
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace vlb {

namespace {

constexpr int NTN = 256;
constexpr int MAXN = 1024;
constexpr int NW = NTN / 32;

// Node positions are kept in [0, n); one step moves a node by less than one cell, and offsets
// between nodes of a ring are below n/2, so single conditional corrections replace fmod.
__device__ __forceinline__ double wrap1(double x, double L)
{
    if (x < 0.0) x += L;
    else if (x >= L) x -= L;
    return x;
}

__device__ __forceinline__ double mimg1(double d, double L)
{
    if (d >= 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

__device__ __forceinline__ int wrapi1(int i, int n)
{
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    return i;
}

__device__ __forceinline__ float phi(float r)
{
    return fabsf(r) < 2.f ? 0.25f * (1.f + cospif(0.5f * r)) : 0.f;
}

// Interpolate a 2-component box field at the position (X, Y) in [0, n); returns false if a
// support cell lies outside the box.
__device__ __forceinline__ bool interp_box(const float* __restrict__ box, const RingDev& R, int bx0, int by0,
                                           int bw, int bh, int nx, int ny, double X, double Y,
                                           float& vx, float& vy)
{
    const int cx = (int)X, cy = (int)Y;              // X, Y >= 0
    const float fx = (float)(X - cx), fy = (float)(Y - cy);
    const long long cap = (long long)R.cap_w * R.cap_h;
    const int ox = wrapi1(cx - 1 - bx0, nx), oy = wrapi1(cy - 1 - by0, ny);
    vx = 0.f;
    vy = 0.f;
    if (ox + 3 >= bw || oy + 3 >= bh) return false;   // the box never wraps onto itself
    const float* p = box + R.box_off + (long long)oy * R.cap_w + ox;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float wy = phi(fy - (float)(j - 1));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float w = phi(fx - (float)(i - 1)) * wy;
            vx += w * p[j * R.cap_w + i];
            vy += w * p[j * R.cap_w + i + cap];
        }
    }
    return true;
}

// Fixed-order block sums of K doubles per thread; results valid in thread 0.
template <int K>
__device__ void block_sums(double (&v)[K], double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * NW + wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += red[k * NW + w];
            v[k] = s;
        }
    __syncthreads();
}

__global__ void __launch_bounds__(NTN) k_nodes(const NodeArgs a)
{
    extern __shared__ __align__(16) double smd[];
    double* rx = smd;               // positions relative to node 0
    double* ry = rx + MAXN;
    double* tex = ry + MAXN;        // spring tension vectors per edge (a, a+1)
    double* tey = tex + MAXN;
    double* dpx = tey + MAXN;       // d cos(gamma_b) / d p and / d q per node b
    double* dpy = dpx + MAXN;
    double* dqx = dpy + MAXN;
    double* dqy = dqx + MAXN;
    __shared__ double red[5 * NW];
    __shared__ int ired[4 * NW];
    __shared__ double sX0[2];

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const double Lx = nx, Ly = ny;
    const long long t = a.ctl->t;
    const bool readout = a.advance && (t % a.every) == 0;
    double* row = a.series + (long long)((t / a.every) % a.series_cap) * a.row_len;

    if (blockIdx.x < a.n_rings) {
        // the ring record is read once into registers (its box is written back at the end)
        const RingDev R = a.rings[blockIdx.x];
        const int n = R.n_nodes, off = R.node_off;
        const int bx0 = R.box_x0, by0 = R.box_y0, bw = R.box_w, bh = R.box_h;

        if (a.advance) {
            if (tid == 0) { sX0[0] = a.X[off].x; sX0[1] = a.X[off].y; }
            __syncthreads();
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            int bad = 0;
            for (int k = tid; k < n; k += NTN) {
                const double2 X = a.X[off + k];
                if (readout) {
                    float fx, fy;
                    if (!interp_box(a.fpbox, R, bx0, by0, bw, bh, nx, ny, X.x, X.y, fx, fy)) bad = 1;
                    acc[0] += (double)fx;
                    acc[1] += (double)fy;
                    acc[2] += mimg1(X.x - sX0[0], Lx);
                    acc[3] += mimg1(X.y - sX0[1], Ly);
                }
                float vx, vy, wx, wy;
                if (!interp_box(a.ubox, R, bx0, by0, bw, bh, nx, ny, X.x, X.y, vx, vy)) bad = 1;
                const double Xs = wrap1(X.x + (double)vx, Lx), Ys = wrap1(X.y + (double)vy, Ly);
                if (!interp_box(a.ubox, R, bx0, by0, bw, bh, nx, ny, Xs, Ys, wx, wy)) bad = 1;
                const double dX = 0.5 * ((double)vx + (double)wx), dY = 0.5 * ((double)vy + (double)wy);
                if (!(fabs(dX) < 1.0 && fabs(dY) < 1.0)) bad = 1;
                a.X[off + k] = make_double2(wrap1(X.x + dX, Lx), wrap1(X.y + dY, Ly));
            }
            if (bad) atomicExch(&a.ctl->err_body, 1);
            if (readout) {
                block_sums<4>(acc, red);
                if (tid == 0) {
                    double* rr = row + 6 + 4 * blockIdx.x;
                    rr[0] = acc[0];
                    rr[1] = acc[1];
                    rr[2] = wrap1(sX0[0] + acc[2] / n, Lx);
                    rr[3] = wrap1(sX0[1] + acc[3] / n, Ly);
                    if (!isfinite(acc[0]) || !isfinite(acc[1]) || !isfinite(acc[2]) || !isfinite(acc[3]))
                        atomicExch(&a.ctl->err_nonfinite, 1);
                }
            }
            __syncthreads();
        }

        // positions relative to node 0 (the ring spans less than half the lattice)
        const double2 X0 = a.X[off];
        for (int k = tid; k < n; k += NTN) {
            const double2 X = a.X[off + k];
            rx[k] = mimg1(X.x - X0.x, Lx);
            ry[k] = mimg1(X.y - X0.y, Ly);
        }
        __syncthreads();

        // spring tension vectors and angle gradients (Eq. Const)
        const double ks = R.k_spring, leq = R.l_eq, eps = R.eps_angle;
        for (int k = tid; k < n; k += NTN) {
            const int kp = (k + 1 == n) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            const double qx = rx[kp] - rx[k], qy = ry[kp] - ry[k];
            const double px = rx[km] - rx[k], py = ry[km] - ry[k];
            const double iq = rsqrt(qx * qx + qy * qy), ip = rsqrt(px * px + py * py);
            const double lq = (qx * qx + qy * qy) * iq;
            const double T = ks * (lq - leq) * iq;
            tex[k] = T * qx;
            tey[k] = T * qy;
            const double ipq = ip * iq;
            const double c = (px * qx + py * qy) * ipq;
            const double cp = c * ip * ip, cq = c * iq * iq;
            dpx[k] = qx * ipq - cp * px;
            dpy[k] = qy * ipq - cp * py;
            dqx[k] = px * ipq - cq * qx;
            dqy[k] = py * ipq - cq * qy;
        }
        __syncthreads();

        int mm[4] = {1 << 30, 1 << 30, 1 << 30, 1 << 30};   // min x, -max x, min y, -max y
        for (int k = tid; k < n; k += NTN) {
            const int kp = (k + 1 == n) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            // f_a = -dU/dR_a: springs (a, a+1) and (a-1, a); angle terms at a-1 (a is its next),
            // a, a+1 (a is its prev); the pull
            const double fx = tex[k] - tex[km] - eps * (dpx[kp] + dqx[km] - dpx[k] - dqx[k]) + R.pull_x;
            const double fy = tey[k] - tey[km] - eps * (dpy[kp] + dqy[km] - dpy[k] - dqy[k]) + R.pull_y;
            a.node_force[off + k] = make_float2((float)fx, (float)fy);
            const double2 X = a.X[off + k];
            int cx = (int)X.x, cy = (int)X.y;
            float frx = (float)(X.x - cx), fry = (float)(X.y - cy);
            if (frx >= 1.f) { frx = 0.f; cx += 1; }
            if (fry >= 1.f) { fry = 0.f; cy += 1; }
            a.node_cell[off + k] = make_int2(wrapi1(cx, nx), wrapi1(cy, ny));
            a.node_frac[off + k] = make_float2(frx, fry);
            // unwrapped cell relative to node 0
            const int ux = (int)floor(X0.x + rx[k]), uy = (int)floor(X0.y + ry[k]);
            mm[0] = min(mm[0], ux); mm[1] = min(mm[1], -ux);
            mm[2] = min(mm[2], uy); mm[3] = min(mm[3], -uy);
            if (!isfinite(fx) || !isfinite(fy)) atomicExch(&a.ctl->err_nonfinite, 1);
        }
        {
            const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                for (int o = 16; o > 0; o >>= 1) mm[q] = min(mm[q], __shfl_down_sync(0xffffffffu, mm[q], o));
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 4; ++q) ired[q * NW + wid] = mm[q];
            __syncthreads();
        }
        if (tid == 0) {
            for (int q = 0; q < 4; ++q)
                for (int w = 1; w < NW; ++w) mm[q] = min(mm[q], ired[q * NW + w]);
            const int mnx = mm[0], mxx = -mm[1], mny = mm[2], mxy = -mm[3];
            // cells min-2 .. max+3 cover the supports of R and of the Heun predictor R*
            int w = mxx - mnx + 6, h = mxy - mny + 6;
            if (w > R.cap_w || h > R.cap_h) {
                atomicExch(&a.ctl->err_body, 1);
                w = min(w, R.cap_w);
                h = min(h, R.cap_h);
            }
            RingDev& Rg = a.rings[blockIdx.x];
            Rg.box_x0 = wrapi1(wrapi1(mnx - 2, nx), nx);
            Rg.box_y0 = wrapi1(wrapi1(mny - 2, ny), ny);
            Rg.box_w = w;
            Rg.box_h = h;
        }
    }

    if (blockIdx.x == 0 && readout) {
        // fixed-order reduction of the lattice kernel's per-CTA sums
        double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = tid; k < a.n_partials; k += NTN)
#pragma unroll
            for (int c = 0; c < 5; ++c) v[c] += a.partials[(long long)k * 5 + c];
        block_sums<5>(v, red);
        if (tid == 0) {
            row[0] = (double)t;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                row[1 + c] = v[c];
                if (!isfinite(v[c])) atomicExch(&a.ctl->err_nonfinite, 1);
            }
        }
    }

    // the last CTA to arrive advances the step counter
    if (a.advance) {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&a.ctl->ticket, 1u);
            if (prev == gridDim.x - 1) {
                a.ctl->ticket = 0u;
                a.ctl->t = t + 1;
                __threadfence();
            }
        }
    }
}

}  // namespace

cudaError_t launch_nodes(const NodeArgs& a, cudaStream_t s)
{
    static bool attr = false;
    const size_t smem = 8 * MAXN * sizeof(double);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = a.n_rings > 0 ? a.n_rings : 1;
    k_nodes<<<grid, NTN, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace vlb
