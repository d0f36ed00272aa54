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

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ double wrapd(double x, int n)
{
    double L = (double)n;
    x = fmod(x, L);
    if (x < 0) x += L;
    if (x >= L) x -= L;
    return x;
}

__device__ __forceinline__ double minimg(double d, int n)
{
    double L = (double)n;
    d = fmod(d, L);
    if (d >= 0.5 * L) d -= L;
    if (d < -0.5 * L) d += L;
    return d;
}

__device__ __forceinline__ float phi(float r)
{
    return fabsf(r) < 2.f ? 0.25f * (1.f + cospif(0.5f * r)) : 0.f;
}

// Interpolate a 2-component box field at the (wrapped) position (X, Y); returns false if a
// support cell lies outside the box.
__device__ bool interp_box(const float* box, const RingDev& R, int bx0, int by0, int bw, int bh,
                           int nx, int ny, double X, double Y, float& vx, float& vy)
{
    const int cx = (int)floor(X), cy = (int)floor(Y);
    const float fx = (float)(X - cx), fy = (float)(Y - cy);
    const long long cap = (long long)R.cap_w * R.cap_h;
    vx = 0.f;
    vy = 0.f;
    bool ok = true;
    for (int j = -1; j <= 2; ++j) {
        const int by = wrapi(cy + j - by0, ny);
        const float wy = phi(fy - (float)j);
        for (int i = -1; i <= 2; ++i) {
            const int bx = wrapi(cx + i - bx0, nx);
            if (bx >= bw || by >= bh) {
                ok = false;
                continue;
            }
            const float w = phi(fx - (float)i) * wy;
            const long long o = R.box_off + (long long)by * R.cap_w + bx;
            vx += w * box[o];
            vy += w * box[o + cap];
        }
    }
    return ok;
}

// fixed-order block sum of one double per thread (result valid in thread 0)
__device__ double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NTN / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

__device__ int block_min_max(int v, int* red, bool is_max)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        int u = __shfl_down_sync(0xffffffffu, v, o);
        v = is_max ? max(v, u) : min(v, u);
    }
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = red[0];
        for (int w = 1; w < NTN / 32; ++w) s = is_max ? max(s, red[w]) : min(s, red[w]);
        red[NTN / 32] = s;
    }
    __syncthreads();
    int r = red[NTN / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(NTN) k_nodes(const NodeArgs a)
{
    extern __shared__ __align__(16) double smd[];
    double* rx = smd;               // unwrapped positions relative to node 0
    double* ry = rx + MAXN;
    double* tex = ry + MAXN;        // spring tension vectors per edge (a, a+1)
    double* tey = tex + MAXN;
    double* dpx = tey + MAXN;       // d cos(gamma_b) / d p and / d q per node b
    double* dpy = dpx + MAXN;
    double* dqx = dpy + MAXN;
    double* dqy = dqx + MAXN;
    __shared__ double red[NTN / 32 + 1];
    __shared__ int ired[NTN / 32 + 1];
    __shared__ double sX0[2];

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const long long t = a.ctl->t;
    const bool readout = a.advance && (t % a.every) == 0;
    double* row = a.series + (long long)((t / a.every) % a.series_cap) * a.row_len;

    if (blockIdx.x < a.n_rings) {
        RingDev& R = a.rings[blockIdx.x];
        const int n = R.n_nodes, off = R.node_off;
        const int bx0 = R.box_x0, by0 = R.box_y0, bw = R.box_w, bh = R.box_h;

        if (a.advance) {
            if (tid == 0) { sX0[0] = a.X[off].x; sX0[1] = a.X[off].y; }
            __syncthreads();
            double frx = 0.0, fry = 0.0, cmx = 0.0, cmy = 0.0;
            int bad = 0;
            for (int k = tid; k < n; k += NTN) {
                const double2 X = a.X[off + k];
                if (readout) {
                    float fx, fy;
                    if (!interp_box(a.fpbox, R, bx0, by0, bw, bh, nx, ny, X.x, X.y, fx, fy)) bad = 1;
                    frx += (double)fx;
                    fry += (double)fy;
                    cmx += minimg(X.x - sX0[0], nx);
                    cmy += minimg(X.y - sX0[1], ny);
                }
                float vx, vy, wx, wy;
                if (!interp_box(a.ubox, R, bx0, by0, bw, bh, nx, ny, X.x, X.y, vx, vy)) bad = 1;
                const double Xs = wrapd(X.x + (double)vx, nx), Ys = wrapd(X.y + (double)vy, ny);
                if (!interp_box(a.ubox, R, bx0, by0, bw, bh, nx, ny, Xs, Ys, wx, wy)) bad = 1;
                const double dX = 0.5 * ((double)vx + (double)wx), dY = 0.5 * ((double)vy + (double)wy);
                if (!(fabs(dX) < 1.0 && fabs(dY) < 1.0)) bad = 1;
                a.X[off + k] = make_double2(wrapd(X.x + dX, nx), wrapd(X.y + dY, ny));
            }
            if (bad) atomicExch(&a.ctl->err_body, 1);
            if (readout) {
                const double s0 = block_sum(frx, red);
                const double s1 = block_sum(fry, red);
                const double s2 = block_sum(cmx, red);
                const double s3 = block_sum(cmy, red);
                if (tid == 0) {
                    double* rr = row + 6 + 4 * blockIdx.x;
                    rr[0] = s0;
                    rr[1] = s1;
                    rr[2] = wrapd(sX0[0] + s2 / n, nx);
                    rr[3] = wrapd(sX0[1] + s3 / n, ny);
                    if (!isfinite(s0) || !isfinite(s1) || !isfinite(s2) || !isfinite(s3))
                        atomicExch(&a.ctl->err_nonfinite, 1);
                }
            }
            __syncthreads();
        }

        // positions relative to node 0 (the ring spans less than half the lattice)
        const double2 X0 = a.X[off];
        for (int k = tid; k < n; k += NTN) {
            const double2 X = a.X[off + k];
            rx[k] = minimg(X.x - X0.x, nx);
            ry[k] = minimg(X.y - X0.y, ny);
        }
        __syncthreads();

        // spring tension vectors and angle gradients (Eq. Const)
        const double ks = R.k_spring, leq = R.l_eq, eps = R.eps_angle;
        for (int k = tid; k < n; k += NTN) {
            const int kp = (k + 1 == n) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            const double dx = rx[kp] - rx[k], dy = ry[kp] - ry[k];
            const double l = sqrt(dx * dx + dy * dy);
            const double T = ks * (l - leq) / l;
            tex[k] = T * dx;
            tey[k] = T * dy;
            const double px = rx[km] - rx[k], py = ry[km] - ry[k];
            const double qx = dx, qy = dy;
            const double lp = sqrt(px * px + py * py), lq = l;
            const double c = (px * qx + py * qy) / (lp * lq);
            dpx[k] = qx / (lp * lq) - c * px / (lp * lp);
            dpy[k] = qy / (lp * lq) - c * py / (lp * lp);
            dqx[k] = px / (lp * lq) - c * qx / (lq * lq);
            dqy[k] = py / (lp * lq) - c * qy / (lq * lq);
        }
        __syncthreads();

        int mnx = 1 << 30, mxx = -(1 << 30), mny = 1 << 30, mxy = -(1 << 30);
        for (int k = tid; k < n; k += NTN) {
            const int kp = (k + 1 == n) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            // f_a = -dU/dR_a: springs (a, a+1) and (a-1, a); angle terms at a-1 (a is its next),
            // a, a+1 (a is its prev); the pull
            const double fx = tex[k] - tex[km] - eps * (dpx[kp] + dqx[km] - dpx[k] - dqx[k]) + R.pull_x;
            const double fy = tey[k] - tey[km] - eps * (dpy[kp] + dqy[km] - dpy[k] - dqy[k]) + R.pull_y;
            a.node_force[off + k] = make_float2((float)fx, (float)fy);
            const double2 X = a.X[off + k];
            int cx = (int)floor(X.x), cy = (int)floor(X.y);
            float frx = (float)(X.x - cx), fry = (float)(X.y - cy);
            if (frx >= 1.f) { frx = 0.f; cx += 1; }
            if (fry >= 1.f) { fry = 0.f; cy += 1; }
            a.node_cell[off + k] = make_int2(wrapi(cx, nx), wrapi(cy, ny));
            a.node_frac[off + k] = make_float2(frx, fry);
            // unwrapped cell relative to node 0's cell
            const int ux = (int)floor(X0.x + rx[k]), uy = (int)floor(X0.y + ry[k]);
            mnx = min(mnx, ux); mxx = max(mxx, ux);
            mny = min(mny, uy); mxy = max(mxy, uy);
            if (!isfinite(fx) || !isfinite(fy)) atomicExch(&a.ctl->err_nonfinite, 1);
        }
        mnx = block_min_max(mnx, ired, false);
        mxx = block_min_max(mxx, ired, true);
        mny = block_min_max(mny, ired, false);
        mxy = block_min_max(mxy, ired, true);
        if (tid == 0) {
            // cells min-2 .. max+3 cover the supports of R and of the Heun predictor R*
            int w = mxx - mnx + 6, h = mxy - mny + 6;
            if (w > R.cap_w || h > R.cap_h) {
                atomicExch(&a.ctl->err_body, 1);
                w = min(w, R.cap_w);
                h = min(h, R.cap_h);
            }
            R.box_x0 = wrapi(mnx - 2, nx);
            R.box_y0 = wrapi(mny - 2, ny);
            R.box_w = w;
            R.box_h = h;
        }
    }

    if (blockIdx.x == 0 && readout) {
        // fixed-order reduction of the lattice kernel's per-CTA sums
        double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k = tid; k < a.n_partials; k += NTN)
            for (int c = 0; c < 5; ++c) v[c] += a.partials[(long long)k * 5 + c];
        for (int c = 0; c < 5; ++c) {
            const double s = block_sum(v[c], red);
            if (tid == 0) {
                row[1 + c] = s;
                if (!isfinite(s)) atomicExch(&a.ctl->err_nonfinite, 1);
            }
        }
        if (tid == 0) row[0] = (double)t;
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
