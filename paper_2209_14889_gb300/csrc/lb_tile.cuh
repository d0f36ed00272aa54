// lb_tile.cuh -- the fused lattice step of one tile (device code shared by the tile kernel and the
// batched persistent kernel): one whole time step of every lattice field.
//
// For an output tile of TX x TY cells a CTA stages, in shared memory, P with a 4-cell halo and
// sigma^p with a 3-cell halo, and then, from the state at t only (Fig. 2):
//   B  (halo 3)  molecular field h = (alpha + beta |P|^2) P - kappa lap P (Eq. Ffunctional) and
//                Ericksen stress sigma^E (Sec. II C 1, kappa on the gradient term);
//   IB (halo 2)  spreading f_IB(r) = sum_a f_a phi phi (App. A), gathered per cell over the
//                ring nodes near the tile in index order (no atomics, bitwise reproducible);
//   C  (halo 2)  F = f_IB + div sigma^p + div sigma^E; moments rho = rho0 + sum d_n,
//                u = (sum c_n d_n + F/2) / rho (Eq. rhoDef, Eq. vDef, Guo half force);
//   D  (halo 1)  velocity gradient (Psi, omega), RHS of Eq. StiffCons and Eq. BE, Heun
//                predictor y* = y + RHS(y);
//   E  (tile)    BGK collision with the Guo source, pushed to the neighbours (Eq. LB, BGK);
//                Heun corrector y' = y + (RHS(y) + RHS(y*))/2 with u frozen at t; u and f^p
//                on the ring work boxes for the node kernel; FP64 readout partial sums.
// Halo cells are recomputed redundantly, so one launch reads and writes each stored value
// once from HBM (the halo re-reads hit L2).  Populations are stored shifted, d_n = h_n - w_n rho0,
// so that FP32 keeps the small deviations that carry the flow.
#pragma once
#include <cuda_runtime.h>

#include "lb_cell.cuh"
#include "lb_internal.h"

namespace vlb {
namespace tile {

using namespace cell;

constexpr int NT = 256;
constexpr int TILE_X = 32, TILE_Y = 16;   // tile of the single-lattice kernel

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int al4(int x) { return (x + 3) & ~3; }   // 16-byte alignment in floats

// Geometry and shared-memory layout (in floats) of a TX x TY output tile.
template <int TX, int TY>
struct TileGeo {
    static constexpr int R4W = TX + 8, R4H = TY + 8, R4 = R4W * R4H;
    static constexpr int R3W = TX + 6, R3H = TY + 6, R3 = R3W * R3H;
    static constexpr int R2W = TX + 4, R2H = TY + 4, R2 = R2W * R2H;
    static constexpr int R1W = TX + 2, R1H = TY + 2, R1 = R1W * R1H;
    static constexpr int R0 = TX * TY;
    static constexpr int OFF_P = 0;                               // P        [2][R4]
    static constexpr int OFF_S = OFF_P + 2 * R4;                  // sigma    [3][R3]
    static constexpr int OFF_E = OFF_S + 3 * R3;                  // sigma^E  [4][R3]  | y* [5][R1]
    static constexpr int SZ_E = cmax(4 * R3, 5 * R1);
    static constexpr int OFF_H = OFF_E + SZ_E;                    // h        [2][R3]
    static constexpr int OFF_M = OFF_H + 2 * R3;                  // drho,ux,uy,Fx,Fy [5][R2]
    static constexpr int OFF_R = OFF_M + 5 * R2;                  // RHS(y)   [5][R0] | f_IB [2][R2]
    static constexpr int SZ_R = cmax(5 * R0, 2 * R2);
    static constexpr int OFF_N = al4(OFF_R + SZ_R);               // nodes    [NT] float4 (cell, frac)
    static constexpr int OFF_NF = OFF_N + 4 * NT;                 // node forces [NT] float2
    static constexpr int OFF_XI = OFF_NF + 2 * NT;                // wrapped x index [R4W] (int)
    static constexpr int OFF_YI = OFF_XI + R4W;                   // wrapped y index [R4H] (int)
    static constexpr int OFF_SC = OFF_YI + R4H;                   // scan scratch [NT/32 + 1] (int)
    static constexpr int OFF_RED = al4(OFF_SC + NT / 32 + 1);     // readout [5][NT/32] (double)
    static constexpr int SMEM_FLOATS = OFF_RED + 2 * 5 * (NT / 32);
    static constexpr size_t SMEM_BYTES = sizeof(float) * SMEM_FLOATS;
    static_assert(OFF_N % 4 == 0 && OFF_NF % 2 == 0 && OFF_RED % 2 == 0, "shared-memory alignment");
};

// One TX x TY tile (tile coordinates bx, by) of the step; sm: TileGeo<TX, TY>::SMEM_BYTES of
// shared memory.  Called by k_fused (one tile per CTA) and by the batched persistent kernel.
template <int MODE, int PREC, int TX, int TY, bool COH = false>
__device__ __forceinline__ void tile_step(const FusedArgs& a, int bx, int by, int tile_index, float* sm)
{
    using G = TileGeo<TX, TY>;
    constexpr int R4W = G::R4W, R4H = G::R4H, R4 = G::R4;
    constexpr int R3W = G::R3W, R3 = G::R3;
    constexpr int R2W = G::R2W, R2H = G::R2H, R2 = G::R2;
    constexpr int R1W = G::R1W, R1 = G::R1;
    constexpr int R0 = G::R0;
    constexpr int OFF_P = G::OFF_P, OFF_S = G::OFF_S, OFF_E = G::OFF_E, OFF_H = G::OFF_H;
    constexpr int OFF_M = G::OFF_M, OFF_R = G::OFF_R, OFF_N = G::OFF_N, OFF_NF = G::OFF_NF;
    constexpr int OFF_XI = G::OFF_XI, OFF_YI = G::OFF_YI, OFF_SC = G::OFF_SC, OFF_RED = G::OFF_RED;
    float* sP = sm + OFF_P;
    float* sS = sm + OFF_S;
    float* sE = sm + OFF_E;
    float* sY = sm + OFF_E;      // y* after sigma^E is dead
    float* sH = sm + OFF_H;
    float* sM = sm + OFF_M;
    float* sR = sm + OFF_R;
    float* sFib = sm + OFF_R;    // f_IB before RHS(y) is written
    const float* sL = reinterpret_cast<const float*>(a.lut);   // C~ table (global, L1)
    float4* sNode = reinterpret_cast<float4*>(sm + OFF_N);
    float2* sNodeF = reinterpret_cast<float2*>(sm + OFF_NF);
    int* sXi = reinterpret_cast<int*>(sm + OFF_XI);
    int* sYi = reinterpret_cast<int*>(sm + OFF_YI);
    int* sScan = reinterpret_cast<int*>(sm + OFF_SC);
    double* sRed = reinterpret_cast<double*>(sm + OFF_RED);

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const long long NP = a.plane;
    const int x0 = bx * TX, y0 = by * TY;
    const Phys ph = a.ph;
    const void* __restrict__ src = a.src;

    for (int i = tid; i < R4W; i += NT) sXi[i] = wrapn(x0 - 4 + i, nx);
    for (int i = tid; i < R4H; i += NT) sYi[i] = wrapn(y0 - 4 + i, ny);
    for (int i = tid; i < 2 * R2; i += NT) sFib[i] = 0.f;
    __syncthreads();

    // ---- A: stage P (halo 4) and sigma (halo 3) ---------------------------------------------
    for (int i = tid; i < R4; i += NT) {
        const int ly = i / R4W, lx = i - ly * R4W;
        const long long g = (long long)sYi[ly] * nx + sXi[lx];
        sP[i] = ld_fld<PREC, COH>(src, NP, PL_PX, g);
        sP[R4 + i] = ld_fld<PREC, COH>(src, NP, PL_PY, g);
    }
    for (int i = tid; i < R3; i += NT) {
        const int ly = i / R3W, lx = i - ly * R3W;
        const long long g = (long long)sYi[ly + 1] * nx + sXi[lx + 1];
        sS[i] = ld_fld<PREC, COH>(src, NP, PL_SXX, g);
        sS[R3 + i] = ld_fld<PREC, COH>(src, NP, PL_SYY, g);
        sS[2 * R3 + i] = ld_fld<PREC, COH>(src, NP, PL_SXY, g);
    }
    __syncthreads();

    // ---- B: molecular field and Ericksen stress on the halo-3 region ------------------------
    for (int i = tid; i < R3; i += NT) {
        const int ly = i / R3W, lx = i - ly * R3W;
        const St px = st_at(sP, R4W, lx + 1, ly + 1);         // dP stencils
        const St py = st_at(sP + R4, R4W, lx + 1, ly + 1);
        float hx, hy, E[4];
        ericksen(ph, px, py, hx, hy, E);
        sH[i] = hx;
        sH[R3 + i] = hy;
        if (ph.ericksen) {
            sE[i] = E[0];
            sE[R3 + i] = E[1];
            sE[2 * R3 + i] = E[2];
            sE[3 * R3 + i] = E[3];
        }
    }

    // The state at t was written two kernels back; the node forces, ring boxes, step counter and
    // readout buffers come from the node kernel just before this one.
    pdl_wait();
    pdl_trigger();

    // ---- IB: gather f_IB on the halo-2 region from the nodes of every ring near the tile ----
    // A node at cell c with fraction f sits at (c - o) + f relative to the region origin o; the
    // integer part is kept apart from the fraction so that kernel arguments stay exact in FP32.
    const bool small = (nx < R2W + 8) || (ny < R2H + 8);   // region may wrap onto itself
    for (int r = 0; r < a.n_rings; ++r) {
        const RingDev& R = a.rings[r];
        if (!meets(x0 - 2, R2W, R.box_x0, R.box_w, nx) || !meets(y0 - 2, R2H, R.box_y0, R.box_h, ny))
            continue;
        for (int base = 0; base < R.n_nodes; base += NT) {
            const int k = base + tid;
            bool keep = false;
            int cxr = 0, cyr = 0;
            float2 fr = make_float2(0.f, 0.f), f = make_float2(0.f, 0.f);
            if (k < R.n_nodes) {
                const int2 c = a.node_cell[R.node_off + k];
                fr = a.node_frac[R.node_off + k];
                f = a.node_force[R.node_off + k];
                // the image of the node nearest the region: support cells c-1 .. c+2 meet
                // [0, R2W) iff the offset lies in [-2, R2W]
                cxr = wrapn(c.x - (x0 - 2), nx);
                cyr = wrapn(c.y - (y0 - 2), ny);
                if (cxr > R2W) cxr -= nx;
                if (cyr > R2H) cyr -= ny;
                keep = small || (cxr >= -2 && cyr >= -2);
            }
            // order-preserving compaction of the kept nodes
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int lane = tid & 31, wid = tid >> 5;
            if (lane == 0) sScan[wid] = __popc(bal);
            __syncthreads();
            if (tid == 0) {
                int acc = 0;
                for (int w = 0; w < NT / 32; ++w) {
                    const int c = sScan[w];
                    sScan[w] = acc;
                    acc += c;
                }
                sScan[NT / 32] = acc;
            }
            __syncthreads();
            if (keep) {
                const int slot = sScan[wid] + __popc(bal & ((1u << lane) - 1u));
                sNode[slot] = make_float4(__int_as_float(cxr), __int_as_float(cyr), fr.x, fr.y);
                sNodeF[slot] = f;
            }
            __syncthreads();
            const int cnt = sScan[NT / 32];
            for (int i = tid; i < R2; i += NT) {
                const int ly = i / R2W, lx = i - ly * R2W;
                float fx = 0.f, fy = 0.f;
                for (int j = 0; j < cnt; ++j) {
                    const float4 q = sNode[j];
                    int ddx = __float_as_int(q.x) - lx, ddy = __float_as_int(q.y) - ly;
                    if (small) {
                        ddx = mimg(ddx, nx);
                        ddy = mimg(ddy, ny);
                    }
                    const float dx = (float)ddx + q.z, dy = (float)ddy + q.w;
                    if (fabsf(dx) < 2.f && fabsf(dy) < 2.f) {
                        const float w = phi(dx) * phi(dy);
                        const float2 fq = sNodeF[j];
                        fx += fq.x * w;
                        fy += fq.y * w;
                    }
                }
                sFib[i] += fx;
                sFib[R2 + i] += fy;
            }
            __syncthreads();
        }
    }
    __syncthreads();

    // ---- C: total force and moments on the halo-2 region ------------------------------------
    for (int i = tid; i < R2; i += NT) {
        const int ly = i / R2W, lx = i - ly * R2W;
        const int j3 = (ly + 1) * R3W + lx + 1;
        float Fx, Fy;
        div_sigma(st_at(sS, R3W, lx + 1, ly + 1), st_at(sS + R3, R3W, lx + 1, ly + 1),
                  st_at(sS + 2 * R3, R3W, lx + 1, ly + 1), Fx, Fy);
        if (ph.ericksen) {
            float ex, ey;
            div_ericksen(st_at(sE, R3W, lx + 1, ly + 1), st_at(sE + R3, R3W, lx + 1, ly + 1),
                         st_at(sE + 2 * R3, R3W, lx + 1, ly + 1), st_at(sE + 3 * R3, R3W, lx + 1, ly + 1),
                         ex, ey);
            Fx += ex;
            Fy += ey;
        }
        (void)j3;
        Fx += sFib[i];
        Fy += sFib[R2 + i];
        const long long g = (long long)sYi[ly + 2] * nx + sXi[lx + 2];
        float d[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) d[n] = ld_pop<PREC, COH>(src, NP, n, g);
        float drho, ux, uy;
        moments(ph, d, Fx, Fy, drho, ux, uy);
        sM[i] = drho;
        sM[R2 + i] = ux;
        sM[2 * R2 + i] = uy;
        sM[3 * R2 + i] = Fx;
        sM[4 * R2 + i] = Fy;
    }
    __syncthreads();

    if (MODE == MODE_MOMENTS) {
        for (int i = tid; i < R0; i += NT) {
            const int ly = i / TX, lx = i - ly * TX;
            const int gx = x0 + lx, gy = y0 + ly;
            if (gx >= nx || gy >= ny) continue;
            const int j = (ly + 2) * R2W + lx + 2;
            const long long g = (long long)gy * nx + gx;
            a.moments_out[g] = sM[j];
            a.moments_out[NP + g] = sM[R2 + j];
            a.moments_out[2 * NP + g] = sM[2 * R2 + j];
        }
        return;
    }

    // ---- D: predictor on the halo-1 region --------------------------------------------------
    for (int i = tid; i < R1; i += NT) {
        const int ly = i / R1W, lx = i - ly * R1W;
        const int j2 = (ly + 1) * R2W + lx + 1;
        float pxx, pyy, pxy, om;
        vgrad(sM + R2, sM + 2 * R2, R2W, j2, pxx, pyy, pxy, om);
        const St s0 = st_at(sS, R3W, lx + 2, ly + 2);
        const St s1 = st_at(sS + R3, R3W, lx + 2, ly + 2);
        const St s2 = st_at(sS + 2 * R3, R3W, lx + 2, ly + 2);
        const St p0 = st_at(sP, R4W, lx + 3, ly + 3);
        const St p1 = st_at(sP + R4, R4W, lx + 3, ly + 3);
        const int j3 = (ly + 2) * R3W + lx + 2;
        float r[5];
        rhs_cell(ph, sL, sM[R2 + j2], sM[2 * R2 + j2], pxx, pyy, pxy, om, s0, s1, s2, p0, p1,
                 sH[j3], sH[R3 + j3], r);
        // y* (the sigma^E buffer is dead: C has finished)
        sY[i] = s0.c + r[0];
        sY[R1 + i] = s1.c + r[1];
        sY[2 * R1 + i] = s2.c + r[2];
        sY[3 * R1 + i] = p0.c + r[3];
        sY[4 * R1 + i] = p1.c + r[4];
        if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY) {
            const int j0 = (ly - 1) * TX + (lx - 1);
#pragma unroll
            for (int c = 0; c < 5; ++c) sR[c * R0 + j0] = r[c];
        }
    }
    __syncthreads();

    // ---- E: collide + push-stream, corrector, box writes, readout sums ----------------------
    const long long t = a.ctl->t;
    const bool readout = (t % a.every) == 0;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    void* __restrict__ dst = a.dst;
    // D2Q9 (Sec. II A): c_n and w_n, n = 0..8
    const int c_cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int c_cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int i = tid; i < R0; i += NT) {
        const int ly = i / TX, lx = i - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const long long g = (long long)gy * nx + gx;
        const int j2 = (ly + 2) * R2W + lx + 2;
        const float drho = sM[j2], ux = sM[R2 + j2], uy = sM[2 * R2 + j2];
        const float Fx = sM[3 * R2 + j2], Fy = sM[4 * R2 + j2];

        // collision (Eq. LB, Eq. BGK, Guo source; exactly conservative FP32 increments),
        // pushed to x + c_n
        {
            float dn[9], D[9];
#pragma unroll
            for (int n = 0; n < 9; ++n) dn[n] = ld_pop<PREC, COH>(src, NP, n, g);
            collide(ph, dn, drho, ux, uy, Fx, Fy, D);
            long long gd[9];
            float out[9];
#pragma unroll
            for (int n = 0; n < 9; ++n) {
                gd[n] = (long long)sYi[ly + 4 + c_cy[n]] * nx + sXi[lx + 4 + c_cx[n]];
                out[n] = dn[n] + D[n];
            }
            st_pops<PREC>(dst, NP, gd, out, (unsigned long long)t, g);
            if (readout) {
                float dsum = 0.f;
                double jxs = 0.0, jys = 0.0;
#pragma unroll
                for (int n = 0; n < 9; ++n) {
                    dsum += dn[n];
                    jxs += (double)((float)c_cx[n] * dn[n]);
                    jys += (double)((float)c_cy[n] * dn[n]);
                }
                acc[0] += (double)dsum;
                acc[1] += jxs;
                acc[2] += jys;
                acc[3] += (double)Fx;
                acc[4] += (double)Fy;
            }
        }

        // corrector with the frozen u
        {
            float pxx, pyy, pxy, om;
            vgrad(sM + R2, sM + 2 * R2, R2W, j2, pxx, pyy, pxy, om);
            const St s0 = st_at(sY, R1W, lx + 1, ly + 1);
            const St s1 = st_at(sY + R1, R1W, lx + 1, ly + 1);
            const St s2 = st_at(sY + 2 * R1, R1W, lx + 1, ly + 1);
            const St p0 = st_at(sY + 3 * R1, R1W, lx + 1, ly + 1);
            const St p1 = st_at(sY + 4 * R1, R1W, lx + 1, ly + 1);
            float hx, hy;
            molecular(ph, p0, p1, hx, hy);
            float r[5];
            rhs_cell(ph, sL, ux, uy, pxx, pyy, pxy, om, s0, s1, s2, p0, p1, hx, hy, r);
            const int j3 = (ly + 3) * R3W + lx + 3;
            const int j4 = (ly + 4) * R4W + lx + 4;
            const float y0s[5] = {sS[j3], sS[R3 + j3], sS[2 * R3 + j3], sP[j4], sP[R4 + j4]};
            float ynew[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) ynew[c] = y0s[c] + 0.5f * (sR[c * R0 + i] + r[c]);
            st_flds<PREC>(dst, NP, g, ynew, (unsigned long long)t);
        }

        // u(t) (and f^p(t) on readout steps) on the work box of every ring containing the cell
        for (int rr = 0; rr < a.n_rings; ++rr) {
            const RingDev& R = a.rings[rr];
            int bx = gx - R.box_x0; if (bx < 0) bx += nx;
            int by = gy - R.box_y0; if (by < 0) by += ny;
            if (bx < R.box_w && by < R.box_h) {
                const long long o = R.box_off + (long long)by * R.cap_w + bx;
                const long long cap = (long long)R.cap_w * R.cap_h;
                a.ubox[o] = ux;
                a.ubox[o + cap] = uy;
                if (readout) {
                    const int j3 = (ly + 3) * R3W + lx + 3;
                    a.fpbox[o] = 0.5f * (sS[j3 + 1] - sS[j3 - 1]) + 0.5f * (sS[2 * R3 + j3 + R3W] - sS[2 * R3 + j3 - R3W]);
                    a.fpbox[o + cap] = 0.5f * (sS[2 * R3 + j3 + 1] - sS[2 * R3 + j3 - 1]) +
                                       0.5f * (sS[R3 + j3 + R3W] - sS[R3 + j3 - R3W]);
                }
            }
        }
    }

    if (readout) {
        // fixed-order block reduction of the FP64 readout sums
        const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            double v = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) sRed[c * (NT / 32) + wid] = v;
        }
        __syncthreads();
        if (tid < 5) {
            double v = 0.0;
            for (int w = 0; w < NT / 32; ++w) v += sRed[tid * (NT / 32) + w];
            a.partials[(long long)tile_index * 5 + tid] = v;
        }
    }
}

}  // namespace tile
}  // namespace vlb
