// lb_sweep.cu -- the fused time step as a column-strip sweep (the fast lattice kernel).
//
// The same step as lb_fused.cu (every field updated from the state at t, Fig. 2), organised for
// HBM streaming: a CTA owns a strip of 120 output columns (128 with the 4-cell halo) and a chunk
// of rows, and sweeps the chunk upwards two rows per iteration.  Rows of P, sigma and the
// populations stream from HBM into shared-memory ring buffers by asynchronous bulk copies
// (cp.async.bulk, completion on an mbarrier) issued one iteration ahead; the stages of the step
// run as a software pipeline on consecutive rows:
//   B  rows e+3, e+4   molecular field and Ericksen stress
//   C  rows e+2, e+3   forces (div sigma^p, div sigma^E, f_IB gathered from nearby ring nodes) and
//                      moments
//   D  rows e+1, e+2   velocity gradient, RHS, Heun predictor
//   E  rows e,   e+1   collision + push streaming, Heun corrector, ring-box writes, readout sums
// so each stage reads the rows its predecessor wrote in this or the previous iteration.  Only
// the x halo is recomputed (1.02x - 1.07x), and the per-cell arithmetic is lb_cell.cuh's, the
// same as the tile kernel's.  The first four iterations of a chunk prime the pipeline.
#include <cuda_runtime.h>

#include "lb_cell.cuh"
#include "lb_internal.h"

namespace vlb {

namespace {

using namespace cell;

constexpr int SW = 128;          // strip width including the halo (threads per row)
constexpr int TW = SW - 8;       // output columns per strip
constexpr int RB = 2;            // rows per stage per iteration
constexpr int NT = SW * RB;      // threads per CTA
constexpr int WARM = 4;          // iterations before the first output row

// ring buffers: rows x components x SW floats.  Each ring holds the rows its readers need in
// one iteration (k: rows relative to the chunk start), plus the rows being written or loaded:
//   P   reads 2k .. 2k+5, loads of the next iteration 2k+6, 2k+7            -> 8
//   sig reads 2k-1 .. 2k+4, next loads 2k+5, 2k+6                           -> 8
//   pop reads 2k .. 2k+3, next loads 2k+4, 2k+5                             -> 6
//   E   B writes 2k+3, 2k+4; C reads 2k+1 .. 2k+4                           -> 4
//   h   B writes 2k+3, 2k+4; D reads 2k+1, 2k+2                             -> 4
//   M   C writes 2k+2, 2k+3; D reads 2k .. 2k+3; E reads 2k-1 .. 2k+2       -> 6
//   y*  D writes 2k+1, 2k+2; E reads 2k-1 .. 2k+2                           -> 4
//   RHS D writes 2k+1, 2k+2; E reads 2k, 2k+1                               -> 4
constexpr int RP = 8, RS = 8, RQ = 6, RE = 4, RH = 4, RM = 6, RY = 4, RR = 4;
constexpr int OFF_P = 0;
constexpr int OFF_S = OFF_P + RP * 2 * SW;
constexpr int OFF_Q = OFF_S + RS * 3 * SW;
constexpr int OFF_E = OFF_Q + RQ * 9 * SW;
constexpr int OFF_H = OFF_E + RE * 4 * SW;
constexpr int OFF_M = OFF_H + RH * 2 * SW;
constexpr int OFF_Y = OFF_M + RM * 5 * SW;
constexpr int OFF_R = OFF_Y + RY * 5 * SW;
constexpr int OFF_L = OFF_R + RR * 5 * SW;
constexpr int OFF_N = (OFF_L + 3) & ~3;                       // node list [NT] float4 + [NT] float2
constexpr int OFF_NF = OFF_N + 4 * NT;
constexpr int OFF_SC = OFF_NF + 2 * NT;                        // scan scratch (int)
constexpr int OFF_RED = (OFF_SC + NT / 32 + 1 + 3) & ~3;       // readout [5][NT/32] (double)
constexpr int OFF_BAR = OFF_RED + 2 * 5 * (NT / 32);           // two mbarriers (8 B each)
constexpr int MAX_SH_RINGS = 32;                               // ring boxes kept in shared memory
constexpr int OFF_BOX = OFF_BAR + 4;                           // [MAX_SH_RINGS] int4 + cap, off
constexpr int SMEM_FLOATS = OFF_BOX + 8 * MAX_SH_RINGS;
constexpr size_t SMEM_BYTES = sizeof(float) * SMEM_FLOATS;
static_assert(OFF_BAR % 2 == 0 && OFF_N % 4 == 0 && OFF_RED % 2 == 0, "alignment");
static_assert(SMEM_BYTES <= 113 * 1024, "two CTAs per SM");
constexpr unsigned TX_BYTES = 14u * RB * SW * sizeof(float);   // bytes per iteration's loads

__device__ __forceinline__ int wrapn(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait on an mbarrier phase; returns false after the iteration limit
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const float* src, unsigned bytes, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// One strip row segment [x0 - 4, x0 + 124) of a plane row into shared memory (split at the
// periodic seam; nx is a multiple of 4 and >= SW, so each piece is 16-byte aligned).
__device__ __forceinline__ void load_row(float* dst, const float* plane, int gy, int xs, int nx, unsigned bar)
{
    const float* row = plane + (long long)gy * nx;
    if (xs < 0) {
        bulk_g2s(smem_addr(dst), row + nx + xs, (unsigned)(-xs) * 4u, bar);
        bulk_g2s(smem_addr(dst - xs), row, (unsigned)(SW + xs) * 4u, bar);
    } else if (xs + SW > nx) {
        const int a = nx - xs;
        bulk_g2s(smem_addr(dst), row + xs, (unsigned)a * 4u, bar);
        bulk_g2s(smem_addr(dst + a), row, (unsigned)(SW - a) * 4u, bar);
    } else {
        bulk_g2s(smem_addr(dst), row + xs, SW * 4u, bar);
    }
}

// Issue the loads of iteration k (rows relative to the chunk's first row e0): P rows 2k+4, 2k+5,
// sigma rows 2k+3, 2k+4, populations rows 2k+2, 2k+3.  Lanes 0..27 of warp 0 issue one row each.
__device__ __forceinline__ void issue_loads(float* sm, const float* src, long long NP, int nx, int ny, int e0,
                                            int xs, int k, unsigned bar, int lane)
{
    if (lane == 0) mbar_expect_tx(bar, TX_BYTES);
    __syncwarp();
    if (lane < 28) {
        const int r = lane & 1, q = lane >> 1;       // q: plane 0..13
        int rel, ring, slotbase;
        float* dst;
        if (q >= PL_PX) {                            // P
            rel = 2 * k + 4 + r;
            ring = RP;
            slotbase = OFF_P + (int)((unsigned)rel % (unsigned)ring) * 2 * SW + (q - PL_PX) * SW;
        } else if (q >= PL_SXX) {                    // sigma
            rel = 2 * k + 3 + r;
            ring = RS;
            slotbase = OFF_S + (int)((unsigned)rel % (unsigned)ring) * 3 * SW + (q - PL_SXX) * SW;
        } else {                                     // populations
            rel = 2 * k + 2 + r;
            ring = RQ;
            slotbase = OFF_Q + (int)((unsigned)rel % (unsigned)ring) * 9 * SW + q * SW;
        }
        dst = sm + slotbase;
        const int gy = wrapn(e0 + rel, ny);
        load_row(dst, src + q * NP, gy, xs, nx, bar);
    }
}

template <int R, int C>
__device__ __forceinline__ float* ring_row(float* base, int rel, int comp)
{
    return base + (((unsigned)rel % (unsigned)R) * C + comp) * SW;   // rel >= 0
}

// stencil of column c of row rel from a ring (rows rel - 1 .. rel + 1)
template <int R, int C>
__device__ __forceinline__ St ring_st(float* base, int rel, int comp, int c)
{
    const float* m = ring_row<R, C>(base, rel, comp);
    const float* n = ring_row<R, C>(base, rel + 1, comp);
    const float* s = ring_row<R, C>(base, rel - 1, comp);
    return St{m[c], m[c + 1], m[c - 1], n[c], s[c]};
}

__device__ __forceinline__ bool meets(int a, int aw, int b, int bw, int n)
{
    if (aw >= n || bw >= n) return true;
    int d1 = wrapn(a - b, n), d2 = wrapn(b - a, n);
    return d1 < bw || d2 < aw;
}

__global__ void __launch_bounds__(NT, 2) k_sweep(const FusedArgs a, const int chunk)
{
    extern __shared__ __align__(128) float sm[];
    float* sP = sm + OFF_P;
    float* sS = sm + OFF_S;
    float* sQ = sm + OFF_Q;
    float* sE = sm + OFF_E;
    float* sH = sm + OFF_H;
    float* sM = sm + OFF_M;
    float* sY = sm + OFF_Y;
    float* sR = sm + OFF_R;
    const float* sL = reinterpret_cast<const float*>(a.lut);   // C~ table (global, L1)
    float4* sNode = reinterpret_cast<float4*>(sm + OFF_N);
    float2* sNodeF = reinterpret_cast<float2*>(sm + OFF_NF);
    int* sScan = reinterpret_cast<int*>(sm + OFF_SC);
    double* sRed = reinterpret_cast<double*>(sm + OFF_RED);
    unsigned long long* sBar = reinterpret_cast<unsigned long long*>(sm + OFF_BAR);
    int4* sBox = reinterpret_cast<int4*>(sm + OFF_BOX);                 // x0, y0, w, h
    int4* sBoxB = sBox + MAX_SH_RINGS;                                  // cap_w, cap_h, off lo, off hi

    const int tid = threadIdx.x;
    const int c = tid % SW;               // column within the strip (0 .. 127)
    const int r = tid / SW;               // row slot (0, 1)
    const int lane = tid & 31, wid = tid >> 5;
    const int nx = a.nx, ny = a.ny;
    const long long NP = a.plane;
    const int x0 = blockIdx.x * TW;
    const int xs = x0 - 4;                // first staged column
    const int yc0 = blockIdx.y * chunk;
    const int yend = min(yc0 + chunk, ny);
    const int e0 = yc0 - 2 * WARM;        // row of E at iteration 0
    const int K = WARM + (yend - yc0 + 1) / 2;
    const Phys ph = a.ph;
    const float* __restrict__ src = static_cast<const float*>(a.src);   // FP32 state only
    float* __restrict__ dst = static_cast<float*>(a.dst);
    const int gx = wrapn(xs + c, nx);     // this thread's column
    const bool out_col = (c >= 4 && c < 4 + TW && x0 + c - 4 < nx);
    const long long t = a.ctl->t;
    const bool readout = (t % a.every) == 0;
    const unsigned bar0 = smem_addr(&sBar[0]), bar1 = smem_addr(&sBar[1]);

    const int n_sh_rings = min(a.n_rings, MAX_SH_RINGS);
    for (int i = tid; i < n_sh_rings; i += NT) {
        const RingDev& R = a.rings[i];
        sBox[i] = ring_box(R, t);
        sBoxB[i] = make_int4(R.cap_w, R.cap_h, (int)(R.box_off & 0xffffffffLL), (int)(R.box_off >> 32));
    }
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (wid == 0) issue_loads(sm, src, NP, nx, ny, e0, xs, 0, bar0, lane);

    const int c_cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int c_cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    DF acc[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    bool timed_out = false;

    for (int k = 0; k < K; ++k) {
        if (!mbar_wait((k & 1) ? bar1 : bar0, (unsigned)((k >> 1) & 1))) timed_out = true;

        // ---- B: molecular field and Ericksen stress (rows 2k+3, 2k+4; columns 1..126) ----
        {
            const int rel = 2 * k + 3 + r;
            if (c >= 1 && c < SW - 1) {
                const St px = ring_st<RP, 2>(sP, rel, 0, c);
                const St py = ring_st<RP, 2>(sP, rel, 1, c);
                float hx, hy, E[4];
                ericksen(ph, px, py, hx, hy, E);
                ring_row<RH, 2>(sH, rel, 0)[c] = hx;
                ring_row<RH, 2>(sH, rel, 1)[c] = hy;
#pragma unroll
                for (int q = 0; q < 4; ++q) ring_row<RE, 4>(sE, rel, q)[c] = ph.ericksen ? E[q] : 0.f;
            }
        }
        __syncthreads();
        if (wid == 0 && k + 1 < K) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_loads(sm, src, NP, nx, ny, e0, xs, k + 1, ((k + 1) & 1) ? bar1 : bar0, lane);
        }

        // ---- C: forces and moments (rows 2k+2, 2k+3; columns 2..125) ----
        {
            const int rel = 2 * k + 2 + r;
            float fibx = 0.f, fiby = 0.f;
            // immersed-boundary spreading from the nodes whose support meets these two rows
            const int gyc0 = wrapn(e0 + 2 * k + 2, ny);
            for (int ri = 0; ri < a.n_rings; ++ri) {
                const int4 bx = ri < MAX_SH_RINGS ? sBox[ri] : ring_box(a.rings[ri], t);
                if (!meets(gyc0, RB, bx.y, bx.w, ny) || !meets(xs + 2, SW - 4, bx.x, bx.z, nx))
                    continue;
                const RingDev& R = a.rings[ri];
                for (int base = 0; base < R.n_nodes; base += NT) {
                    const int kk = base + tid;
                    bool keep = false;
                    int cx = 0, cy = 0;
                    float2 fr = make_float2(0.f, 0.f), f = make_float2(0.f, 0.f);
                    if (kk < R.n_nodes) {
                        const int2 cc = a.node_cell[R.node_off + kk];
                        fr = a.node_frac[R.node_off + kk];
                        f = a.node_force[R.node_off + kk];
                        if (R.trap_k > 0.0) {     // the trap's force, the same on every node
                            const float2 tf = R.trap_f[t & 1];
                            f.x += tf.x;
                            f.y += tf.y;
                        }
                        // offsets of the node cell from the first C row and the first staged column
                        cy = wrapn(cc.y - gyc0, ny);
                        if (cy > RB) cy -= ny;
                        cx = wrapn(cc.x - xs, nx);
                        if (cx > SW) cx -= nx;
                        keep = cy >= -2 && cx >= -2;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    if (lane == 0) sScan[wid] = __popc(bal);
                    __syncthreads();
                    if (tid == 0) {
                        int s = 0;
                        for (int w = 0; w < NT / 32; ++w) {
                            const int v = sScan[w];
                            sScan[w] = s;
                            s += v;
                        }
                        sScan[NT / 32] = s;
                    }
                    __syncthreads();
                    if (keep) {
                        const int slot = sScan[wid] + __popc(bal & ((1u << lane) - 1u));
                        sNode[slot] = make_float4(__int_as_float(cx), __int_as_float(cy), fr.x, fr.y);
                        sNodeF[slot] = f;
                    }
                    __syncthreads();
                    const int cnt = sScan[NT / 32];
                    for (int j = 0; j < cnt; ++j) {
                        const float4 q = sNode[j];
                        const float dx = (float)(__float_as_int(q.x) - c) + q.z;
                        const float dy = (float)(__float_as_int(q.y) - r) + q.w;
                        if (fabsf(dx) < 2.f && fabsf(dy) < 2.f) {
                            const float w = phi(dx) * phi(dy);
                            const float2 fq = sNodeF[j];
                            fibx += fq.x * w;
                            fiby += fq.y * w;
                        }
                    }
                    __syncthreads();
                }
            }
            if (c >= 2 && c < SW - 2) {
                float Fx, Fy;
                div_sigma(ring_st<RS, 3>(sS, rel, 0, c), ring_st<RS, 3>(sS, rel, 1, c),
                          ring_st<RS, 3>(sS, rel, 2, c), Fx, Fy);
                if (ph.ericksen) {
                    float ex, ey;
                    div_ericksen(ring_st<RE, 4>(sE, rel, 0, c), ring_st<RE, 4>(sE, rel, 1, c),
                                 ring_st<RE, 4>(sE, rel, 2, c), ring_st<RE, 4>(sE, rel, 3, c), ex, ey);
                    Fx += ex;
                    Fy += ey;
                }
                Fx += fibx;
                Fy += fiby;
                float d[9];
#pragma unroll
                for (int n = 0; n < 9; ++n) d[n] = ring_row<RQ, 9>(sQ, rel, n)[c];
                float drho, ux, uy;
                moments(ph, d, Fx, Fy, drho, ux, uy);
                ring_row<RM, 5>(sM, rel, 0)[c] = drho;
                ring_row<RM, 5>(sM, rel, 1)[c] = ux;
                ring_row<RM, 5>(sM, rel, 2)[c] = uy;
                ring_row<RM, 5>(sM, rel, 3)[c] = Fx;
                ring_row<RM, 5>(sM, rel, 4)[c] = Fy;
            }
        }
        __syncthreads();

        // ---- D: predictor (rows 2k+1, 2k+2; columns 3..124) ----
        {
            const int rel = 2 * k + 1 + r;
            if (c >= 3 && c < SW - 3) {
                const float* u0 = ring_row<RM, 5>(sM, rel, 1);
                const float* v0 = ring_row<RM, 5>(sM, rel, 2);
                const float dxux = 0.5f * (u0[c + 1] - u0[c - 1]);
                const float dyux = 0.5f * (ring_row<RM, 5>(sM, rel + 1, 1)[c] - ring_row<RM, 5>(sM, rel - 1, 1)[c]);
                const float dxuy = 0.5f * (v0[c + 1] - v0[c - 1]);
                const float dyuy = 0.5f * (ring_row<RM, 5>(sM, rel + 1, 2)[c] - ring_row<RM, 5>(sM, rel - 1, 2)[c]);
                const float pxx = dxux, pyy = dyuy, pxy = 0.5f * (dxuy + dyux), om = 0.5f * (dxuy - dyux);
                const St s0 = ring_st<RS, 3>(sS, rel, 0, c);
                const St s1 = ring_st<RS, 3>(sS, rel, 1, c);
                const St s2 = ring_st<RS, 3>(sS, rel, 2, c);
                const St p0 = ring_st<RP, 2>(sP, rel, 0, c);
                const St p1 = ring_st<RP, 2>(sP, rel, 1, c);
                float rr[5];
                rhs_cell(ph, sL, u0[c], v0[c], pxx, pyy, pxy, om, s0, s1, s2, p0, p1,
                         ring_row<RH, 2>(sH, rel, 0)[c], ring_row<RH, 2>(sH, rel, 1)[c], rr);
                ring_row<RY, 5>(sY, rel, 0)[c] = s0.c + rr[0];
                ring_row<RY, 5>(sY, rel, 1)[c] = s1.c + rr[1];
                ring_row<RY, 5>(sY, rel, 2)[c] = s2.c + rr[2];
                ring_row<RY, 5>(sY, rel, 3)[c] = p0.c + rr[3];
                ring_row<RY, 5>(sY, rel, 4)[c] = p1.c + rr[4];
#pragma unroll
                for (int q = 0; q < 5; ++q) ring_row<RR, 5>(sR, rel, q)[c] = rr[q];
            }
        }
        __syncthreads();

        // ---- E: collision + push, corrector, ring boxes, readout (rows 2k, 2k+1) ----
        {
            const int rel = 2 * k + r;
            const int gy_abs = e0 + rel;
            if (k >= WARM && out_col && gy_abs < yend) {
                const int gy = gy_abs;            // inside [yc0, yend) and < ny
                const long long g = (long long)gy * nx + gx;
                const float drho = ring_row<RM, 5>(sM, rel, 0)[c];
                const float* u0 = ring_row<RM, 5>(sM, rel, 1);
                const float* v0 = ring_row<RM, 5>(sM, rel, 2);
                const float ux = u0[c], uy = v0[c];
                const float Fx = ring_row<RM, 5>(sM, rel, 3)[c], Fy = ring_row<RM, 5>(sM, rel, 4)[c];
                {
                    float dn[9], D[9];
#pragma unroll
                    for (int n = 0; n < 9; ++n) dn[n] = ring_row<RQ, 9>(sQ, rel, n)[c];
                    collide(ph, dn, drho, ux, uy, Fx, Fy, D);
                    const int gyp = (gy + 1 == ny) ? 0 : gy + 1, gym = (gy == 0) ? ny - 1 : gy - 1;
                    const int gxp = (gx + 1 == nx) ? 0 : gx + 1, gxm = (gx == 0) ? nx - 1 : gx - 1;
#pragma unroll
                    for (int n = 0; n < 9; ++n) {
                        const int yy = c_cy[n] > 0 ? gyp : (c_cy[n] < 0 ? gym : gy);
                        const int xx = c_cx[n] > 0 ? gxp : (c_cx[n] < 0 ? gxm : gx);
                        dst[n * NP + (long long)yy * nx + xx] = dn[n] + D[n];
                    }
                    if (readout) {
                        float dsum, jx, jy;
                        cell::cell_readout(dn, dsum, jx, jy);
                        cell::df_add(acc[0], dsum);
                        cell::df_add(acc[1], jx);
                        cell::df_add(acc[2], jy);
                        cell::df_add(acc[3], Fx);
                        cell::df_add(acc[4], Fy);
                    }
                }
                {
                    const float dxux = 0.5f * (u0[c + 1] - u0[c - 1]);
                    const float dyux = 0.5f * (ring_row<RM, 5>(sM, rel + 1, 1)[c] - ring_row<RM, 5>(sM, rel - 1, 1)[c]);
                    const float dxuy = 0.5f * (v0[c + 1] - v0[c - 1]);
                    const float dyuy = 0.5f * (ring_row<RM, 5>(sM, rel + 1, 2)[c] - ring_row<RM, 5>(sM, rel - 1, 2)[c]);
                    const float pxx = dxux, pyy = dyuy, pxy = 0.5f * (dxuy + dyux), om = 0.5f * (dxuy - dyux);
                    const St s0 = ring_st<RY, 5>(sY, rel, 0, c);
                    const St s1 = ring_st<RY, 5>(sY, rel, 1, c);
                    const St s2 = ring_st<RY, 5>(sY, rel, 2, c);
                    const St p0 = ring_st<RY, 5>(sY, rel, 3, c);
                    const St p1 = ring_st<RY, 5>(sY, rel, 4, c);
                    float hx, hy;
                    molecular(ph, p0, p1, hx, hy);
                    float rr[5];
                    rhs_cell(ph, sL, ux, uy, pxx, pyy, pxy, om, s0, s1, s2, p0, p1, hx, hy, rr);
                    const float y0s[5] = {ring_row<RS, 3>(sS, rel, 0)[c], ring_row<RS, 3>(sS, rel, 1)[c],
                                          ring_row<RS, 3>(sS, rel, 2)[c], ring_row<RP, 2>(sP, rel, 0)[c],
                                          ring_row<RP, 2>(sP, rel, 1)[c]};
#pragma unroll
                    for (int q = 0; q < 5; ++q)
                        dst[(PL_SXX + q) * NP + g] = y0s[q] + 0.5f * (ring_row<RR, 5>(sR, rel, q)[c] + rr[q]);
                }
                for (int ri = 0; ri < a.n_rings; ++ri) {
                    int4 B, C2;
                    if (ri < MAX_SH_RINGS) {
                        B = sBox[ri];
                        C2 = sBoxB[ri];
                    } else {
                        const RingDev& R = a.rings[ri];
                        B = ring_box(R, t);
                        C2 = make_int4(R.cap_w, R.cap_h, (int)(R.box_off & 0xffffffffLL), (int)(R.box_off >> 32));
                    }
                    int bx = gx - B.x; if (bx < 0) bx += nx;
                    int by = gy - B.y; if (by < 0) by += ny;
                    if (bx < B.z && by < B.w) {
                        const long long box_off = (long long)(unsigned)C2.z | ((long long)C2.w << 32);
                        const long long o = box_off + (long long)by * C2.x + bx;
                        const long long cap = (long long)C2.x * C2.y;
                        a.ubox[o] = ux;
                        a.ubox[o + cap] = uy;
                        if (readout) {
                            float fpx, fpy;
                            div_sigma(ring_st<RS, 3>(sS, rel, 0, c), ring_st<RS, 3>(sS, rel, 1, c),
                                      ring_st<RS, 3>(sS, rel, 2, c), fpx, fpy);
                            a.fpbox[o] = fpx;
                            a.fpbox[o + cap] = fpy;
                        }
                    }
                }
            }
        }
    }

    if (timed_out) {
        atomicExch(&a.ctl->err_timeout, 1);
        mbar_wait(bar0, 0);                                             // bounded: drain copies
        mbar_wait(bar1, 0);
    }
    if (readout) {
        __syncthreads();
        cell::store_partial(a.partials, (long long)blockIdx.y * gridDim.x + blockIdx.x, acc,
                            reinterpret_cast<float*>(sRed));
    }
}

}  // namespace

bool sweep_eligible(int nx, int ny) { return nx % 4 == 0 && nx >= 2 * SW && ny >= 16; }

// Rows per CTA chunk: enough CTAs for two per SM, chunks of 16 .. 64 rows (even).
int sweep_chunk(int nx, int ny, int n_sm)
{
    const int strips = (nx + TW - 1) / TW;
    int want = (2 * n_sm + strips - 1) / strips;
    int ch = (ny + want - 1) / want;
    ch = (ch + 1) & ~1;
    if (ch < 16) ch = 16;
    if (ch > 64) ch = 64;
    return ch;
}

int sweep_ctas(int nx, int ny, int chunk) { return ((nx + TW - 1) / TW) * ((ny + chunk - 1) / chunk); }

cudaError_t launch_sweep(const FusedArgs& a, int chunk, cudaStream_t s)
{
    static unsigned long long attr_done = 0;     // per device
    if (!done_on_device(attr_done)) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) {
            attr_done = 0;
            return e;
        }
    }
    dim3 grid((a.nx + TW - 1) / TW, (a.ny + chunk - 1) / chunk);
    k_sweep<<<grid, NT, SMEM_BYTES, s>>>(a, chunk);
    return cudaGetLastError();
}

}  // namespace vlb
