// lb_node.cuh -- the node step (device code shared by the node kernel and the batched persistent
// kernel; App. A).
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
// Node positions are kept in FP64 (O(N_nodes) data) and advanced in FP64; the forces are
// evaluated in FP32 except the spring extension, whose l^2 - l_eq^2 is formed in FP64 (FP64 is
// a narrow unit on this GPU, so it is kept to a few operations per node).  The lattice kernel
// sees the nodes as int32 cell + FP32 fraction with FP32 forces.  One CTA owns NB nodes of one
// ring and recomputes the advance of HALO neighbours on each side, so no CTA waits for
// another; the last CTA of a ring writes the ring's box and readouts, the last CTA overall the
// lattice readouts and the step counter.
#pragma once
#include <cuda_runtime.h>

#include "lb_cell.cuh"
#include "lb_internal.h"

namespace vlb {
namespace node {

constexpr int HALO = 2;                       // neighbours whose advance a CTA recomputes

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

// The four cosine-kernel weights phi(f + 1), phi(f), phi(f - 1), phi(f - 2) of a node at
// fraction f in [0, 1) (App. A): with c = cos(pi f / 2), s = sin(pi f / 2) they are
// (1 - s)/4, (1 + c)/4, (1 + s)/4, (1 - c)/4 (quarter-period shifts of the cosine).
__device__ __forceinline__ void phi4(float f, float* w)
{
    float sn, cs;
    sincospif(0.5f * f, &sn, &cs);
    w[0] = 0.25f * (1.f - sn);
    w[1] = 0.25f * (1.f + cs);
    w[2] = 0.25f * (1.f + sn);
    w[3] = 0.25f * (1.f - cs);
}

// Interpolate a 2-component box field at the position (X, Y) in [0, n); returns false if a
// support cell lies outside the box.
__device__ __forceinline__ bool interp_box(const float* box, const RingDev& R, int bx0, int by0,
                                           int bw, int bh, int nx, int ny, double X, double Y,
                                           float& vx, float& vy)
{
    const int cx = (int)X, cy = (int)Y;              // X, Y >= 0
    const long long cap = (long long)R.cap_w * R.cap_h;
    const int ox = wrapi1(cx - 1 - bx0, nx), oy = wrapi1(cy - 1 - by0, ny);
    vx = 0.f;
    vy = 0.f;
    if (ox + 3 >= bw || oy + 3 >= bh) return false;   // the box never wraps onto itself
    float wx[4], wy[4];
    phi4((float)(X - cx), wx);
    phi4((float)(Y - cy), wy);
    const float* p = box + R.box_off + (long long)oy * R.cap_w + ox;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float w = wx[i] * wy[j];
            vx += w * __ldcg(p + j * R.cap_w + i);      // written by the lattice step
            vy += w * __ldcg(p + j * R.cap_w + i + cap);
        }
    }
    return true;
}

// The trap protocol at step t (doubles): k(t) and the trap's fraction g(t) of its way, from the
// sigmoids s(t; c) = 1 / (1 + exp(-8 (t - c) / w)).
__device__ __forceinline__ double trap_sigmoid(double t, double c, double w) { return 1.0 / (1.0 + exp(-8.0 * (t - c) / w)); }
__device__ __forceinline__ double trap_softplus(double z) { return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
__device__ __forceinline__ void trap_at(const RingDev& R, double t, double& k, double& g)
{
    const double w = R.trap_w, te = R.trap_t_eq, T = R.trap_pull;
    k = R.trap_k * trap_sigmoid(t, 0.5 * w, w) * (1.0 - trap_sigmoid(t, te + T + 0.5 * w, w));
    const double a = 8.0 / w;
    g = (trap_softplus(a * (t - te)) - trap_softplus(a * (t - te - T))) / (a * T);
}

__device__ __forceinline__ int half_wrap(int d, int n)   // d in (-n, n) -> [-n/2, n/2)
{
    if (d >= n - n / 2) d -= n;
    else if (d < -(n / 2)) d += n;
    return d;
}

// Fixed-order sums over the warps of a CTA (K values per thread); result valid in thread 0.
template <int K, class T>
__device__ void cta_reduce(T (&v)[K], T* red, bool is_min)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            const T u = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = is_min ? (u < v[k] ? u : v[k]) : v[k] + u;
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * 32 + wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T s = red[k * 32];
            for (int w = 1; w < nw; ++w) s = is_min ? (red[k * 32 + w] < s ? red[k * 32 + w] : s) : s + red[k * 32 + w];
            v[k] = s;
        }
    __syncthreads();
}

// Shared memory of one node block.  It is passed in rather than declared static: a kernel that
// runs node blocks after other work hands over space it no longer needs, so the node code takes
// nothing from the L1 share of that kernel's main work.
struct NodeSmem {
    double sx[NODE_THREADS], sy[NODE_THREADS];     // new positions relative to node j = 0
    double dred[4 * 32];
    float tex[NODE_THREADS], tey[NODE_THREADS];    // spring tension vector of edge (j, j+1)
    float dpx[NODE_THREADS], dpy[NODE_THREADS];    // d cos(gamma_j) / d p, / d q
    float dqx[NODE_THREADS], dqy[NODE_THREADS];
    int ired[4 * 32];
    int s_last;
    int flag[3];                                   // free for the caller
    unsigned mask;                                 // free for the caller
};

// Lattice readout of step t, run by the last CTA to arrive (all its threads): the sums of the
// per-CTA partials (double-float pairs, cell::store_partial) in a fixed order, merged in
// double-float on FP32 lanes, into columns 0-5 of the readout row; FP64 only for the five totals.
// dred: 4 * 32 doubles of shared scratch.
__device__ __forceinline__ void lattice_readout(const NodeArgs& a, long long t, double* dred)
{
    const int tid = threadIdx.x;
    double* row = a.series + (long long)((t / a.every) % a.series_cap) * a.row_len;
    cell::DF v[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    // the partials of other CTAs, read through L2 (after the caller's fence), several in flight
    const float2* P = reinterpret_cast<const float2*>(a.partials);
#pragma unroll 4
    for (int k = tid; k < a.n_partials; k += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float2 q = __ldcg(P + (long long)k * 5 + c);
            v[c] = cell::df_merge(v[c], cell::DF{q.x, q.y});
        }
    }
    const cell::DF s = cell::df_block_sum<5>(v, reinterpret_cast<float*>(dred));
    if (tid < 5) {
        const double val = (double)s.hi + (double)s.lo;
        row[1 + tid] = val;
        if (!isfinite(val)) atomicExch(&a.ctl->err_nonfinite, 1);
    }
    if (tid == 0) row[0] = (double)t;
}

// One CTA per block of NB nodes of one ring, with a halo of HALO nodes on each side whose
// advance is recomputed (identically) so that the forces of the owned nodes need no other CTA.
// One node block (cta: index into a.work) of the node step; called by k_nodes (one block per
// CTA), by the batched persistent kernel, and (whole_step = false: without the end of the step,
// which the caller then runs itself; t_in: the step index, else read from ctl->t) by the tail of
// the lattice kernel.
__device__ __forceinline__ void node_block(const NodeArgs& a, int cta, NodeSmem& S, bool whole_step = true,
                                           long long t_in = -1)
{
    double* sx = S.sx;
    double* sy = S.sy;
    float* tex = S.tex;
    float* tey = S.tey;
    float* dpx = S.dpx;
    float* dpy = S.dpy;
    float* dqx = S.dqx;
    float* dqy = S.dqy;
    double* dred = S.dred;
    int* ired = S.ired;
    int& s_last = S.s_last;

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const double Lx = nx, Ly = ny;
    const long long t = t_in >= 0 ? t_in : a.ctl->t;
    const bool readout = a.advance && (t % a.every) == 0;
    double* row = a.series + (long long)((t / a.every) % a.series_cap) * a.row_len;
    const int2 wk = a.work[cta];                           // (ring, first owned node)

    if (wk.x >= 0) {
        const RingDev R = a.rings[wk.x];
        const int n = R.n_nodes, off = R.node_off;
        const int k0 = wk.y, n_own = min(NB, n - k0);
        const int4 B0 = ring_box(R, t);
        const int bx0 = B0.x, by0 = B0.y, bw = B0.z, bh = B0.w;
        const int j = tid;                                   // local slot: node k0 - HALO + j
        const bool active = j < NODE_THREADS && j < n_own + 2 * HALO;   // larger CTAs: extra threads idle
        const bool own = j >= HALO && j < HALO + n_own;
        int k = k0 - HALO + j;
        k %= n;
        if (k < 0) k += n;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int bad = 0;
        double2 Xn = make_double2(0.0, 0.0);
        double2 X = make_double2(0.0, 0.0);
        if (active) X = a.X[off + k];              // written by the previous node kernel
        // u(t), f^p(t) and the lattice readout sums come from the lattice kernel just before
        cell::pdl_wait();
        cell::pdl_trigger();
        if (active) {
            Xn = X;
            if (a.advance) {
                if (readout && own) {
                    float fx, fy;
                    if (!interp_box(a.fpbox, R, bx0, by0, bw, bh, nx, ny, X.x, X.y, fx, fy)) bad = 1;
                    acc[0] = (double)fx;
                    acc[1] = (double)fy;
                    acc[2] = mimg1(X.x - (double)bx0, Lx);        // centre of mass relative to the box
                    acc[3] = mimg1(X.y - (double)by0, Ly);
                }
                float vx, vy, wx, wy;
                if (!interp_box(a.ubox, R, bx0, by0, bw, bh, nx, ny, X.x, X.y, vx, vy)) bad = 1;
                const double Xs = wrap1(X.x + (double)vx, Lx), Ys = wrap1(X.y + (double)vy, Ly);
                if (!interp_box(a.ubox, R, bx0, by0, bw, bh, nx, ny, Xs, Ys, wx, wy)) bad = 1;
                const double dX = 0.5 * ((double)vx + (double)wx), dY = 0.5 * ((double)vy + (double)wy);
                if (!(fabs(dX) < 1.0 && fabs(dY) < 1.0)) bad = 1;
                Xn = make_double2(wrap1(X.x + dX, Lx), wrap1(X.y + dY, Ly));
                if (a.walls_y && (Xn.y < 4.0 || Xn.y > Ly - 5.0)) bad = 1;   // supports stay off the walls
                if (a.walls_x && (Xn.x < 4.0 || Xn.x > Lx - 5.0)) bad = 1;
            }
        }
        if (bad && own) atomicExch(&a.ctl->err_body, 1);
        // positions relative to local slot 0 (the ring spans less than half the lattice)
        if (tid == 0) { dred[0] = Xn.x; dred[1] = Xn.y; }
        __syncthreads();
        const double X0x = dred[0], X0y = dred[1];
        __syncthreads();
        if (active) {
            sx[j] = mimg1(Xn.x - X0x, Lx);
            sy[j] = mimg1(Xn.y - X0y, Ly);
        }
        __syncthreads();
        const int last = n_own + 2 * HALO - 1;
        const float ks = (float)R.k_spring, leq = (float)R.l_eq, eps = (float)R.eps_angle;
        if (j >= 1 && j < last) {
            // Eq. Const.  Spring on the edge (j, j+1): the extension l - l_eq = (l^2 - l_eq^2) /
            // (l + l_eq) with l^2 - l_eq^2 formed in FP64 from the FP64 edge vector, so it keeps
            // its relative precision; the rest in FP32.
            const double qxd = sx[j + 1] - sx[j], qyd = sy[j + 1] - sy[j];
            const double ext2 = fma(qxd, qxd, fma(qyd, qyd, -R.l_eq * R.l_eq));
            const float qx = (float)qxd, qy = (float)qyd;
            const float px = (float)(sx[j - 1] - sx[j]), py = (float)(sy[j - 1] - sy[j]);
            const float lq = sqrtf(qx * qx + qy * qy), lp = sqrtf(px * px + py * py);
            const float T = ks * (float)ext2 / ((lq + leq) * lq);
            tex[j] = T * qx;
            tey[j] = T * qy;
            // angle term at j: gradients of cos(gamma_j) = p.q / (|p||q|)
            const float ip = 1.f / lp, iq = 1.f / lq;
            const float ipq = ip * iq;
            const float c = (px * qx + py * qy) * ipq;
            const float cp = c * ip * ip, cq = c * iq * iq;
            dpx[j] = qx * ipq - cp * px;
            dpy[j] = qy * ipq - cp * py;
            dqx[j] = px * ipq - cq * qx;
            dqy[j] = py * ipq - cq * qy;
        }
        __syncthreads();
        int mm[4] = {1 << 30, 1 << 30, 1 << 30, 1 << 30};   // min x, -max x, min y, -max y
        const bool trap = R.trap_k > 0.0;
        double cn[2] = {0.0, 0.0};                          // advanced positions, for the trap
        if (own && trap) {
            cn[0] = mimg1(Xn.x - (double)bx0, Lx);
            cn[1] = mimg1(Xn.y - (double)by0, Ly);
        }
        if (own) {
            // f_a = -dU/dR_a: springs (a, a+1) and (a-1, a); angle terms at a-1 (a is its next),
            // a, a+1 (a is its prev); the pull
            const float fx = tex[j] - tex[j - 1] - eps * (dpx[j + 1] + dqx[j - 1] - dpx[j] - dqx[j]) + (float)R.pull_x;
            const float fy = tey[j] - tey[j - 1] - eps * (dpy[j + 1] + dqy[j - 1] - dpy[j] - dqy[j]) + (float)R.pull_y;
            a.node_force[off + k] = make_float2(fx, fy);
            a.X_out[off + k] = Xn;
            int cx = (int)Xn.x, cy = (int)Xn.y;
            float frx = (float)(Xn.x - cx), fry = (float)(Xn.y - cy);
            if (frx >= 1.f) { frx = 0.f; cx += 1; }
            if (fry >= 1.f) { fry = 0.f; cy += 1; }
            a.node_cell[off + k] = make_int2(wrapi1(cx, nx), wrapi1(cy, ny));
            a.node_frac[off + k] = make_float2(frx, fry);
            // cell offsets from the previous box origin, for the new box
            const int ux = half_wrap(wrapi1(cx, nx) - bx0, nx), uy = half_wrap(wrapi1(cy, ny) - by0, ny);
            mm[0] = ux; mm[1] = -ux; mm[2] = uy; mm[3] = -uy;
            if (!isfinite(fx) || !isfinite(fy)) atomicExch(&a.ctl->err_nonfinite, 1);
        }
        cta_reduce<4, int>(mm, ired, true);
        if (readout) cta_reduce<4, double>(acc, dred, false);
        if (trap) cta_reduce<2, double>(cn, dred, false);
        double* np_ = a.node_partials + (long long)cta * NODE_PARTIALS;
        if (tid == 0) {
            for (int q = 0; q < 4; ++q) np_[q] = acc[q];
            for (int q = 0; q < 4; ++q) np_[4 + q] = (double)mm[q];
            np_[8] = cn[0];
            np_[9] = cn[1];
            __threadfence();
            const unsigned prev = atomicAdd(&a.ring_tickets[wk.x], 1u);
            s_last = (prev == (unsigned)(a.ring_ctas[wk.x] - 1));
        }
        __syncthreads();
        if (s_last && tid == 0) {
            // the ring's last CTA: box of the new positions and the ring's readouts
            __threadfence();
            const int c0 = a.ring_cta0[wk.x], nc = a.ring_ctas[wk.x];
            double sum[4] = {0.0, 0.0, 0.0, 0.0}, scn[2] = {0.0, 0.0};
            int m[4] = {1 << 30, 1 << 30, 1 << 30, 1 << 30};
            for (int c = 0; c < nc; ++c) {
                const volatile double* p = a.node_partials + (long long)(c0 + c) * NODE_PARTIALS;
                for (int q = 0; q < 4; ++q) {
                    sum[q] += p[q];
                    m[q] = min(m[q], (int)p[4 + q]);
                }
                scn[0] += p[8];
                scn[1] += p[9];
            }
            if (trap) {
                // Eq. Utrap at the step the nodes advance to: k (R_ext - R_com) / N on each node
                const double tn = (double)(t + a.advance);
                double kt, g;
                trap_at(R, tn, kt, g);
                const double ex = mimg1(R.trap_x0 + R.trap_dx * g - ((double)bx0 + scn[0] / n), Lx);
                const double ey = mimg1(R.trap_y0 + R.trap_dy * g - ((double)by0 + scn[1] / n), Ly);
                a.rings[wk.x].trap_f[(t + a.advance) & 1] = make_float2((float)(kt * ex / n), (float)(kt * ey / n));
            }
            int w = -m[1] - m[0] + 6, h = -m[3] - m[2] + 6;      // cells min-2 .. max+3
            if (w > R.cap_w || h > R.cap_h) {
                atomicExch(&a.ctl->err_body, 1);
                w = min(w, R.cap_w);
                h = min(h, R.cap_h);
            }
            // the box of the step the nodes advance to
            a.rings[wk.x].box[(t + a.advance) & 1] =
                make_int4(wrapi1(wrapi1(bx0 + m[0] - 2, nx), nx), wrapi1(wrapi1(by0 + m[2] - 2, ny), ny), w, h);
            if (readout) {
                double* rr = row + 6 + 4 * wk.x;
                rr[0] = sum[0];
                rr[1] = sum[1];
                rr[2] = wrap1((double)bx0 + sum[2] / n, Lx);
                rr[3] = wrap1((double)by0 + sum[3] / n, Ly);
                for (int q = 0; q < 4; ++q)
                    if (!isfinite(sum[q])) atomicExch(&a.ctl->err_nonfinite, 1);
            }
            a.ring_tickets[wk.x] = 0u;
        }
    }

    if (!whole_step) return;
    // the last CTA overall: lattice readout sums (fixed order) and the step counter
    if (wk.x < 0) {
        cell::pdl_wait();
        cell::pdl_trigger();
    }
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.ctl->ticket, 1u);
        s_last = (prev == (unsigned)a.n_ctas - 1u);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (readout) lattice_readout(a, t, dred);
        if (tid == 0) {
            a.ctl->ticket = 0u;
            if (a.advance) a.ctl->t = t + a.advance;      // advance: steps taken (1, or a jump)
            __threadfence();
        }
    }
}

}  // namespace node
}  // namespace vlb
