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
//                u = (sum c_n d_n + F/2) / rho (Eq. rhoDef, Eq. vDef, Guo half force); on the
//                owned cells the BGK collision with the Guo source, pushed to the neighbours
//                (Eq. LB, BGK), and the FP64 readout partial sums;
//   D  (halo 1)  velocity gradient (Psi, omega), RHS of Eq. StiffCons and Eq. BE, Heun
//                predictor y* = y + RHS(y);
//   E  (tile)    Heun corrector y' = y + (RHS(y) + RHS(y*))/2 with u frozen at t; u and f^p
//                on the ring work boxes for the node kernel.
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
    static constexpr int OFF_M = OFF_H + 2 * R3;                  // drho, ux, uy [3][R2]
    static constexpr int OFF_R = OFF_M + 3 * R2;                  // RHS(y)   [5][R0] | f_IB [2][R2]
    static constexpr int SZ_R = cmax(5 * R0, 2 * R2);
    static constexpr int OFF_N = al4(OFF_R + SZ_R);               // nodes    [NT] float4 (cell, frac)
    static constexpr int OFF_NF = OFF_N + 4 * NT;                 // node forces [NT] float2
    static constexpr int OFF_XI = OFF_NF + 2 * NT;                // wrapped x index [R4W] (int)
    static constexpr int OFF_YI = OFF_XI + R4W;                   // wrapped y index [R4H] (int)
    static constexpr int OFF_SC = OFF_YI + R4H;                   // scan scratch [NT/32 + 1] (int),
                                                                  // then the tile's ring masks [2]
    static constexpr int OFF_RED = al4(OFF_SC + NT / 32 + 3);     // readout [5][NT/32] (double)
    static constexpr int SMEM_FLOATS = OFF_RED + 2 * 5 * (NT / 32);
    static constexpr size_t SMEM_BYTES = sizeof(float) * SMEM_FLOATS;
    static_assert(OFF_N % 4 == 0 && OFF_NF % 2 == 0 && OFF_RED % 2 == 0, "shared-memory alignment");
};

// Shared-memory views of one tile (layout of TileGeo<TX, TY>).
template <int TX, int TY>
struct TileMem {
    using G = TileGeo<TX, TY>;
    float* sP;          // dP           [2][R4]
    float* sS;          // sigma        [3][R3]
    float* sE;          // sigma^E      [4][R3]
    float* sY;          // y*           [5][R1]  (over sigma^E once C is done)
    float* sH;          // h            [2][R3]
    float* sM;          // drho (moments mode only), ux, uy  [3][R2]
    float* sR;          // RHS(y)       [5][R0]
    float* sFib;        // f_IB         [2][R2]  (over RHS(y) until D)
    float4* sNode;
    float2* sNodeF;
    int* sXi;
    int* sYi;
    int* sScan;
    double* sRed;
    __device__ __forceinline__ explicit TileMem(float* sm)
        : sP(sm + G::OFF_P), sS(sm + G::OFF_S), sE(sm + G::OFF_E), sY(sm + G::OFF_E), sH(sm + G::OFF_H),
          sM(sm + G::OFF_M), sR(sm + G::OFF_R), sFib(sm + G::OFF_R),
          sNode(reinterpret_cast<float4*>(sm + G::OFF_N)), sNodeF(reinterpret_cast<float2*>(sm + G::OFF_NF)),
          sXi(reinterpret_cast<int*>(sm + G::OFF_XI)), sYi(reinterpret_cast<int*>(sm + G::OFF_YI)),
          sScan(reinterpret_cast<int*>(sm + G::OFF_SC)), sRed(reinterpret_cast<double*>(sm + G::OFF_RED))
    {
    }
};

// a pair of neighbouring values (flat indices g, g + 1, g even, plane size even) of one field
// plane of the state, as FP32
template <int PREC, bool COH>
__device__ __forceinline__ float2 ld_fld2(const void* src, long long NP, int plane, long long g)
{
    if (PREC == PREC_FP32)
        return ld_state<float2, COH>(reinterpret_cast<const float2*>(reinterpret_cast<const float*>(src) + plane * NP + g));
    const unsigned b = ld_state<unsigned, COH>(
        reinterpret_cast<const unsigned*>(reinterpret_cast<const unsigned short*>(src) + plane * NP + g));
    const unsigned short lo = (unsigned short)(b & 0xFFFFu), hi = (unsigned short)(b >> 16);
    if (plane >= PL_PX) return make_float2(__half2float(__ushort_as_half(lo)), __half2float(__ushort_as_half(hi)));
    return make_float2(__uint_as_float((unsigned)lo << 16), __uint_as_float((unsigned)hi << 16));
}

// Walls in y (App. C, half-way bounce-back): the walls sit at y = -1/2 and y = ny - 1/2, and a
// row beyond them is the mirror image of the row inside: zero-gradient fields (sigma, P) copy
// their image, the velocity (zero at the wall) and the Ericksen stress take it negated (the
// polar field exerts no traction on a free-anchoring wall, so f^E hands no momentum to it).
__device__ __forceinline__ int mirror_row(int y, int ny)
{
    for (int k = 0; k < 8 && (y < 0 || y >= ny); ++k) y = y < 0 ? -1 - y : 2 * ny - 1 - y;
    return y < 0 ? 0 : (y >= ny ? ny - 1 : y);   // rows this far out are never read
}

// Cells of a staged region (origin (xr, yr), W x H, nplanes planes of stride PS; value c of the
// region's cell q at f[c PS + q CS]) that lie beyond a wall take the value of their mirror image,
// times sgn for each wall crossed, where the image is in the region (images are inside the
// walls, so no cell is both read and written).  CS = 2, PS = 1: an interleaved pair plane.
__device__ __forceinline__ void mirror_ghosts(float* f, int PS, int nplanes, int W, int H, int xr, int yr,
                                              const FusedArgs& a, float sgn, int CS = 1)
{
    for (int q = threadIdx.x; q < W * H; q += NT) {
        const int ly = q / W, lx = q - ly * W;
        const int x = xr + lx, y = yr + ly;
        const bool ox = a.walls_x && (x < 0 || x >= a.nx), oy = a.walls_y && (y < 0 || y >= a.ny);
        if (!ox && !oy) continue;
        const int mx = (ox ? mirror_row(x, a.nx) : x) - xr, my = (oy ? mirror_row(y, a.ny) : y) - yr;
        if (mx < 0 || mx >= W || my < 0 || my >= H) continue;
        const float s = (ox ? sgn : 1.f) * (oy ? sgn : 1.f);
        for (int c = 0; c < nplanes; ++c) f[c * PS + (ly * W + lx) * CS] = s * f[c * PS + (my * W + mx) * CS];
    }
}

// ---- A: wrapped index tables, f_IB cleared, P staged with a 4-cell halo and sigma with 3 ----
// With nx even every staged row starts at an even column (x0 - 4, wrapped), so the rows are read
// as aligned pairs that never straddle the periodic seam; each thread issues all its loads
// before its shared-memory stores.  Odd nx takes single-value loads.
// PI: P staged as interleaved (dP_x, dP_y) pairs (the one-cell step), else as two planes.
template <int PREC, bool COH, int TX, int TY, bool SCALAR = false, bool PI = false>
__device__ __forceinline__ void stage(const FusedArgs& a, const TileMem<TX, TY>& m, int x0, int y0)
{
    using G = TileGeo<TX, TY>;
    constexpr int R4W = G::R4W, R4 = G::R4, R3W = G::R3W, R3 = G::R3;
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const long long NP = a.plane;
    const void* src = a.src;
    for (int i = tid; i < R4W; i += NT) m.sXi[i] = a.walls_x ? mirror_row(x0 - 4 + i, nx) : wrapn(x0 - 4 + i, nx);
    for (int i = tid; i < G::R4H; i += NT) m.sYi[i] = a.walls_y ? mirror_row(y0 - 4 + i, ny) : wrapn(y0 - 4 + i, ny);
    for (int i = tid; i < 2 * G::R2; i += NT) m.sFib[i] = 0.f;
    __syncthreads();
    // pairs need consecutive columns: not where mirrored columns (walls in x) enter the tile
    if ((nx & 1) == 0 && !(a.walls_x && (x0 - 4 < 0 || x0 + TX + 4 > nx))) {
        // P: pairs of the halo-4 rows; sigma: pairs of the rows y0-3 .. y0+TY+2 over the halo-4
        // columns, of which the outermost column on each side is dropped
        constexpr int HP = R4W / 2;                      // pairs per row
        constexpr int NPP = R4 / 2, NSP = HP * G::R3H;   // pairs of P, of sigma
        constexpr int KP = (NPP + NT - 1) / NT, KS = (NSP + NT - 1) / NT;
        float2 vp[KP][2], vs[KS][3];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int q = tid + k * NT;
            if (!SCALAR && q < NPP) {
                const int ly = q / HP, lx = 2 * (q - ly * HP);
                const long long g = (long long)m.sYi[ly] * nx + m.sXi[lx];
                vp[k][0] = ld_fld2<PREC, COH>(src, NP, PL_PX, g);
                vp[k][1] = ld_fld2<PREC, COH>(src, NP, PL_PY, g);
            }
        }
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int q = tid + k * NT;
            if (q < NSP) {
                const int ly = q / HP, lx = 2 * (q - ly * HP);
                const long long g = (long long)m.sYi[ly + 1] * nx + m.sXi[lx];
#pragma unroll
                for (int c = 0; c < 3; ++c) vs[k][c] = ld_fld2<PREC, COH>(src, NP, PL_SXX + c, g);
            }
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int q = tid + k * NT;
            if (!SCALAR && q < NPP) {
                if (PI) {
                    *reinterpret_cast<float4*>(m.sP + 4 * q) =
                        make_float4(vp[k][0].x, vp[k][1].x, vp[k][0].y, vp[k][1].y);
                } else {
                    st2<true>(m.sP + 2 * q, vp[k][0]);
                    st2<true>(m.sP + R4 + 2 * q, vp[k][1]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const int q = tid + k * NT;
            if (q < NSP) {
                const int ly = q / HP, lx = 2 * (q - ly * HP);   // halo-4 column of the pair
                const int i = ly * R3W + lx - 1;                 // halo-3 index of its first value
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (lx >= 1) m.sS[c * R3 + i] = vs[k][c].x;
                    if (lx + 1 <= R3W) m.sS[c * R3 + i + 1] = vs[k][c].y;
                }
            }
        }
    } else {
        for (int i = tid; i < (SCALAR ? 0 : R4); i += NT) {
            const int ly = i / R4W, lx = i - ly * R4W;
            const long long g = (long long)m.sYi[ly] * nx + m.sXi[lx];
            const float px = ld_fld<PREC, COH>(src, NP, PL_PX, g), py = ld_fld<PREC, COH>(src, NP, PL_PY, g);
            if (PI) {
                reinterpret_cast<float2*>(m.sP)[i] = make_float2(px, py);
            } else {
                m.sP[i] = px;
                m.sP[R4 + i] = py;
            }
        }
        for (int i = tid; i < R3; i += NT) {
            const int ly = i / R3W, lx = i - ly * R3W;
            const long long g = (long long)m.sYi[ly + 1] * nx + m.sXi[lx + 1];
            m.sS[i] = ld_fld<PREC, COH>(src, NP, PL_SXX, g);
            m.sS[R3 + i] = ld_fld<PREC, COH>(src, NP, PL_SYY, g);
            m.sS[2 * R3 + i] = ld_fld<PREC, COH>(src, NP, PL_SXY, g);
        }
    }
    __syncthreads();
}

// ---- IB: gather f_IB on the halo-2 region from the nodes of every ring near the tile ----
// A node at cell c with fraction f sits at (c - o) + f relative to the region origin o; the
// integer part is kept apart from the fraction so that kernel arguments stay exact in FP32.
// Each cell sums the nodes in ring and index order, so the result does not depend on the tile.
// the step index of a lattice launch: from the host with the node tail (which advances ctl->t
// while tiles still run), else from the device step counter
__device__ __forceinline__ long long step_index(const FusedArgs& a) { return a.node_tail ? a.t : a.ctl->t; }

template <int TX, int TY>
__device__ __forceinline__ void ib_gather(const FusedArgs& a, const TileMem<TX, TY>& m, int x0, int y0)
{
    using G = TileGeo<TX, TY>;
    constexpr int R2W = G::R2W, R2H = G::R2H, R2 = G::R2;
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const bool small = (nx < R2W + 8) || (ny < R2H + 8);   // region may wrap onto itself
    const long long t = step_index(a);
    const int nr = a.n_rings;
    // with up to 32 rings every warp tests one ring per lane: the rings whose box meets the
    // staged halo-2 region (meet) and the owned cells (own); beyond 32 rings each is tested below
    unsigned meet = 0xffffffffu, own = 0xffffffffu;
    if (nr <= 32) {
        const int lane = tid & 31;
        bool m2 = false, mo = false;
        if (lane < nr) {
            const int4 bx = ring_box(a.rings[lane], t);
            m2 = meets(x0 - 2, R2W, bx.x, bx.z, nx) && meets(y0 - 2, R2H, bx.y, bx.w, ny);
            mo = m2 && meets(x0, TX, bx.x, bx.z, nx) && meets(y0, TY, bx.y, bx.w, ny);
        }
        meet = __ballot_sync(0xffffffffu, m2);
        own = __ballot_sync(0xffffffffu, mo);
    }
    for (int r = 0; r < nr; ++r) {
        if (nr <= 32 && !((meet >> r) & 1u)) continue;
        const RingDev& R = a.rings[r];
        if (nr > 32) {
            const int4 bx = ring_box(R, t);
            if (!meets(x0 - 2, R2W, bx.x, bx.z, nx) || !meets(y0 - 2, R2H, bx.y, bx.w, ny)) continue;
        }
        for (int base = 0; base < R.n_nodes; base += NT) {
            const int k = base + tid;
            bool keep = false;
            int cxr = 0, cyr = 0;
            float2 fr = make_float2(0.f, 0.f), f = make_float2(0.f, 0.f);
            if (k < R.n_nodes) {
                const int2 c = a.node_cell[R.node_off + k];
                fr = a.node_frac[R.node_off + k];
                f = a.node_force[R.node_off + k];
                if (R.trap_k > 0.0) {             // the trap's force, the same on every node
                    const float2 tf = R.trap_f[t & 1];
                    f.x += tf.x;
                    f.y += tf.y;
                }
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
            if (lane == 0) m.sScan[wid] = __popc(bal);
            __syncthreads();
            if (tid == 0) {
                int acc = 0;
                for (int w = 0; w < NT / 32; ++w) {
                    const int c = m.sScan[w];
                    m.sScan[w] = acc;
                    acc += c;
                }
                m.sScan[NT / 32] = acc;
            }
            __syncthreads();
            if (keep) {
                const int slot = m.sScan[wid] + __popc(bal & ((1u << lane) - 1u));
                m.sNode[slot] = make_float4(__int_as_float(cxr), __int_as_float(cyr), fr.x, fr.y);
                m.sNodeF[slot] = f;
            }
            __syncthreads();
            const int cnt = m.sScan[NT / 32];
            for (int i = tid; i < R2; i += NT) {
                const int ly = i / R2W, lx = i - ly * R2W;
                float fx = 0.f, fy = 0.f;
                for (int j = 0; j < cnt; ++j) {
                    const float4 q = m.sNode[j];
                    int ddx = __float_as_int(q.x) - lx, ddy = __float_as_int(q.y) - ly;
                    if (small) {
                        ddx = mimg(ddx, nx);
                        ddy = mimg(ddy, ny);
                    }
                    const float dx = (float)ddx + q.z, dy = (float)ddy + q.w;
                    if (fabsf(dx) < 2.f && fabsf(dy) < 2.f) {
                        const float w = phi(dx) * phi(dy);
                        const float2 fq = m.sNodeF[j];
                        fx += fq.x * w;
                        fy += fq.y * w;
                    }
                }
                m.sFib[i] += fx;
                m.sFib[R2 + i] += fy;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        m.sScan[NT / 32 + 1] = (int)own;    // for the box writes of phase E
        m.sScan[NT / 32 + 2] = (int)meet;   // for the node tail
    }
    __syncthreads();
}

// u(t) (and f^p(t) = div sigma^p on readout steps) of the owned cell (gx, gy) on the work box of
// ring rr if it contains the cell; j3: the cell's index in the halo-3 sigma planes (width R3W).
template <int R3, int R3W>
__device__ __forceinline__ void box_write_ring(const FusedArgs& a, int rr, long long t, int gx, int gy, float ux,
                                               float uy, bool readout, const float* sS, int j3)
{
    const int nx = a.nx, ny = a.ny;
    {
        const RingDev& R = a.rings[rr];
        const int4 B = ring_box(R, t);
        int bx = gx - B.x; if (bx < 0) bx += nx;
        int by = gy - B.y; if (by < 0) by += ny;
        if (bx < B.z && by < B.w) {
            const long long o = R.box_off + (long long)by * R.cap_w + bx;
            const long long cap = (long long)R.cap_w * R.cap_h;
            a.ubox[o] = ux;
            a.ubox[o + cap] = uy;
            if (readout) {
                a.fpbox[o] = 0.5f * (sS[j3 + 1] - sS[j3 - 1]) + 0.5f * (sS[2 * R3 + j3 + R3W] - sS[2 * R3 + j3 - R3W]);
                a.fpbox[o + cap] = 0.5f * (sS[2 * R3 + j3 + 1] - sS[2 * R3 + j3 - 1]) +
                                   0.5f * (sS[R3 + j3 + R3W] - sS[R3 + j3 - R3W]);
            }
        }
    }
}

// u(t) (and f^p(t) on readout steps) of the owned cell (gx, gy) on the box of every ring that
// contains it; mask: the rings whose box meets the tile's owned cells (with up to 32 rings; all
// rings are tested when there are more).
template <int R3, int R3W>
__device__ __forceinline__ void box_write(const FusedArgs& a, unsigned mask, long long t, int gx, int gy, float ux,
                                          float uy, bool readout, const float* sS, int j3)
{
    if (a.n_rings > 32) {
        for (int rr = 0; rr < a.n_rings; ++rr) box_write_ring<R3, R3W>(a, rr, t, gx, gy, ux, uy, readout, sS, j3);
        return;
    }
    for (; mask; mask &= mask - 1)
        box_write_ring<R3, R3W>(a, __ffs(mask) - 1, t, gx, gy, ux, uy, readout, sS, j3);
}

// fixed-order reduction of the tile's double-float readout sums into its partial slot
__device__ __forceinline__ void readout_reduce(const FusedArgs& a, const DF* acc, double* sRed, int tile_index)
{
    store_partial(a.partials, tile_index, acc, reinterpret_cast<float*>(sRed));
}

// the moments of the owned cells to the moments_out planes (MODE_MOMENTS)
// IL: u staged as interleaved (u_x, u_y) pairs and drho after them (the one-cell step)
template <int TX, int TY, bool IL = false>
__device__ __forceinline__ void moments_out(const FusedArgs& a, const TileMem<TX, TY>& m, int x0, int y0)
{
    using G = TileGeo<TX, TY>;
    const long long NP = a.plane;
    for (int i = threadIdx.x; i < G::R0; i += NT) {
        const int ly = i / TX, lx = i - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= a.nx || gy >= a.ny) continue;
        const int j = (ly + 2) * G::R2W + lx + 2;
        const long long g = (long long)gy * a.nx + gx;
        if (IL) {
            const float2 u = reinterpret_cast<const float2*>(m.sM)[j];
            a.moments_out[g] = m.sM[2 * G::R2 + j];
            a.moments_out[NP + g] = u.x;
            a.moments_out[2 * NP + g] = u.y;
        } else {
            a.moments_out[g] = m.sM[j];
            a.moments_out[NP + g] = m.sM[G::R2 + j];
            a.moments_out[2 * NP + g] = m.sM[2 * G::R2 + j];
        }
        if (a.forces_out) {
            a.forces_out[g] = m.sFib[j];
            a.forces_out[NP + g] = m.sFib[G::R2 + j];
        }
    }
}

// Cell k of a region made of the TX x TY owned cells and a frame BD cells wide around them, in
// the order in which the tile step visits it: first the owned cells row by row (a warp covers
// one row of 32, so its stencil reads fall in distinct banks, and the owned cells, which carry
// most of the work, spread evenly over the threads), then the frame: BD rows on top, BD rows at
// the bottom, then the BD + BD side cells of each owned row.  (lx, ly): coordinates in the
// region, whose width is TX + 2 BD.
template <int TX, int TY, int BD>
__device__ __forceinline__ void region_cell(int k, int& lx, int& ly)
{
    constexpr int W = TX + 2 * BD, H = TY + 2 * BD;
    if (k < TX * TY) {
        ly = BD + k / TX;
        lx = BD + k % TX;
        return;
    }
    int h = k - TX * TY;
    if (h < 2 * BD * W) {
        const int r = h / W;
        lx = h - r * W;
        ly = r < BD ? r : H - 2 * BD + r;
        return;
    }
    h -= 2 * BD * W;
    const int r = h / (2 * BD), c = h - r * (2 * BD);
    ly = BD + r;
    lx = c < BD ? c : TX + c;
}

// D2Q9 (Sec. II A): c_n, n = 0..8
__device__ constexpr int C_CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int C_CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ constexpr int C_OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};   // c_opp(n) = -c_n

// Stencils of a shared-memory plane of interleaved pairs (a, b): one 8-byte load per stencil point.
__device__ __forceinline__ void st_pair(const float2* base, int W, int lx, int ly, St& a, St& b)
{
    const float2* p = base + ly * W + lx;
    const float2 c = p[0], e = p[1], w = p[-1], n = p[W], s = p[-W];
    a = St{c.x, e.x, w.x, n.x, s.x};
    b = St{c.y, e.y, w.y, n.y, s.y};
}

// One TX x TY tile (tile coordinates bx, by) of the step, one cell per thread and iteration;
// sm: TileGeo<TX, TY>::SMEM_BYTES of shared memory.  The two components of P, h, u, the
// predictor of sigma_xx, sigma_yy and of P, and of the right-hand sides live as interleaved
// pairs in the regions TileGeo gives their planes (same sizes), so that a stencil point is one
// 8-byte load that feeds the paired arithmetic of lb_cell.cuh directly.
template <int MODE, int PREC, int TX, int TY, bool COH = false, bool SCALAR = false>
__device__ __forceinline__ void tile_step(const FusedArgs& a, int bx, int by, int tile_index, float* sm)
{
    using G = TileGeo<TX, TY>;
    constexpr int R4W = G::R4W, R4 = G::R4;
    constexpr int R3W = G::R3W, R3 = G::R3;
    constexpr int R2W = G::R2W, R2 = G::R2;
    constexpr int R1W = G::R1W, R1 = G::R1;
    constexpr int R0 = G::R0;
    const TileMem<TX, TY> m(sm);
    static_assert(R4 % 2 == 0 && R3 % 2 == 0 && R2 % 2 == 0 && R1 % 2 == 0 && R0 % 2 == 0 &&
                  G::OFF_H % 2 == 0 && G::OFF_M % 2 == 0 && G::OFF_R % 2 == 0 && G::OFF_E % 2 == 0,
                  "pair planes need 8-byte alignment");
    const float2* sP2 = reinterpret_cast<const float2*>(m.sP);   // (dP_x, dP_y)        [R4]
    float2* sH2 = reinterpret_cast<float2*>(m.sH);               // (h_x, h_y)          [R3]
    float2* sU2 = reinterpret_cast<float2*>(m.sM);               // (u_x, u_y)          [R2]
    float* sRho = m.sM + 2 * R2;                                 // drho (moments mode) [R2]
    float2* sY01 = reinterpret_cast<float2*>(m.sY);              // y* of (s_xx, s_yy)  [R1]
    float2* sY34 = sY01 + R1;                                    // y* of (dP_x, dP_y)  [R1]
    float* sY2 = m.sY + 4 * R1;                                  // y* of s_xy          [R1]
    float2* sR01 = reinterpret_cast<float2*>(m.sR);              // RHS(y): (r0, r1)    [R0]
    float2* sR34 = sR01 + R0;                                    //         (r3, r4)    [R0]
    float* sR2 = m.sR + 4 * R0;                                  //          r2         [R0]
    const float* sL = reinterpret_cast<const float*>(a.lut);   // C~ table (global, L1)
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const long long NP = a.plane;
    const int x0 = bx * TX, y0 = by * TY;
    const Phys& ph = a.ph;
    const void* src = a.src;

    stage<PREC, COH, TX, TY, SCALAR, true>(a, m, x0, y0);
    // a tile whose staged cells reach beyond a wall (uniform over the CTA)
    const bool wall = (a.walls_y && (y0 - 4 < 0 || y0 + TY + 4 > ny)) || (a.walls_x && (x0 - 4 < 0 || x0 + TX + 4 > nx));

    // ---- B: molecular field and Ericksen stress on the halo-3 region (not in the scalar model)
    for (int k = tid; k < (SCALAR ? 0 : R3); k += NT) {
        int lx, ly;
        region_cell<TX, TY, 3>(k, lx, ly);
        const int i = ly * R3W + lx;
        St px, py;
        st_pair(sP2, R4W, lx + 1, ly + 1, px, py);               // dP stencils
        float hx, hy, E[4];
        ericksen(ph, px, py, hx, hy, E);
        sH2[i] = f2(hx, hy);
        if (ph.ericksen) {
#pragma unroll
            for (int c = 0; c < 4; ++c) m.sE[c * R3 + i] = E[c];
        }
    }

    if (wall && !SCALAR && ph.ericksen) {
        __syncthreads();
        mirror_ghosts(m.sE, R3, 4, R3W, G::R3H, x0 - 3, y0 - 3, a, -1.f);   // read in C, after the gather's barrier
    }

    // The state at t was written two kernels back; the node forces, ring boxes, step counter and
    // readout buffers come from the node kernel just before this one.
    pdl_wait();
    pdl_trigger();
    ib_gather(a, m, x0, y0);

    // ---- C: total force and moments on the halo-2 region; collision of the owned cells ------
    // Owned cells collide here, with their populations still in registers, and push to
    // x + c_n (Eq. LB, Eq. BGK, Guo source; exactly conservative FP32 increments).
    const long long t = step_index(a);
    const bool readout = (t % a.every) == 0;
    DF acc[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    void* dst = a.dst;
    for (int k = tid; k < R2; k += NT) {
        int lx, ly;
        region_cell<TX, TY, 2>(k, lx, ly);
        const int i = ly * R2W + lx;
        float2 F;
        div_sigma(st_at(m.sS, R3W, lx + 1, ly + 1), st_at(m.sS + R3, R3W, lx + 1, ly + 1),
                  st_at(m.sS + 2 * R3, R3W, lx + 1, ly + 1), F.x, F.y);
        if (ph.ericksen) {
            float2 E;
            div_ericksen(st_at(m.sE, R3W, lx + 1, ly + 1), st_at(m.sE + R3, R3W, lx + 1, ly + 1),
                         st_at(m.sE + 2 * R3, R3W, lx + 1, ly + 1), st_at(m.sE + 3 * R3, R3W, lx + 1, ly + 1),
                         E.x, E.y);
            F = F + E;
        }
        F = F + f2(m.sFib[i], m.sFib[R2 + i]);
        const float Fx = F.x, Fy = F.y;
        const long long g = (long long)m.sYi[ly + 2] * nx + m.sXi[lx + 2];
        float d[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) d[n] = ld_pop<PREC, COH>(src, NP, n, g);
        float drho, ux, uy;
        moments(ph, d, Fx, Fy, drho, ux, uy);
        sU2[i] = f2(ux, uy);
        if (MODE == MODE_MOMENTS) {
            sRho[i] = drho;
            m.sFib[i] = Fx;              // the total force replaces f_IB (read above, this cell only)
            m.sFib[R2 + i] = Fy;
        }
        const bool own = k < R0 && x0 + lx - 2 < nx && y0 + ly - 2 < ny;
        if (MODE == MODE_STEP && own) {
            float D[9];
            collide(ph, d, drho, ux, uy, Fx, Fy, D);
            long long gd[9];
            float out[9];
#pragma unroll
            for (int n = 0; n < 9; ++n) gd[n] = (long long)m.sYi[ly + 2 + C_CY[n]] * nx + m.sXi[lx + 2 + C_CX[n]];
            add_pops(d, D, out);
            const int gy = y0 + ly - 2, gxo = x0 + lx - 2;
            if (PREC == PREC_FP32 && wall &&
                ((a.walls_y && (gy == 0 || gy == ny - 1)) || (a.walls_x && (gxo == 0 || gxo == nx - 1)))) {
                // half-way bounce-back (FP32 state): a population that would leave through a
                // wall comes back into its own cell as the opposite population
                float* dd = reinterpret_cast<float*>(dst);
#pragma unroll
                for (int n = 0; n < 9; ++n) {
                    const int yd = gy + C_CY[n], xd = gxo + C_CX[n];
                    if ((a.walls_y && (yd < 0 || yd >= ny)) || (a.walls_x && (xd < 0 || xd >= nx)))
                        dd[C_OPP[n] * NP + g] = out[n];
                    else
                        dd[n * NP + gd[n]] = out[n];
                }
            } else {
                st_pops<PREC>(dst, NP, gd, out, (unsigned long long)t, g);
            }
            if (readout) {
                float dsum, jx, jy;
                cell_readout(d, dsum, jx, jy);
                df_add(acc[0], dsum);
                df_add(acc[1], jx);
                df_add(acc[2], jy);
                df_add(acc[3], Fx);
                df_add(acc[4], Fy);
            }
        }
    }
    __syncthreads();

    if (MODE == MODE_MOMENTS) {
        moments_out<TX, TY, true>(a, m, x0, y0);
        return;
    }
    if (wall) {
        // u beyond a wall: the negated image (zero velocity at the wall)
        mirror_ghosts(m.sM, 1, 2, R2W, G::R2H, x0 - 2, y0 - 2, a, -1.f, 2);
        __syncthreads();
    }

    // ---- D: predictor on the halo-1 region --------------------------------------------------
    for (int k = tid; k < R1; k += NT) {
        int lx, ly;
        region_cell<TX, TY, 1>(k, lx, ly);
        const int i = ly * R1W + lx;
        float pxx, pyy, pxy, om;
        St su, sv;
        st_pair(sU2, R2W, lx + 1, ly + 1, su, sv);
        vgrad(su, sv, pxx, pyy, pxy, om);
        const St s0 = st_at(m.sS, R3W, lx + 2, ly + 2);
        const St s1 = st_at(m.sS + R3, R3W, lx + 2, ly + 2);
        const St s2 = st_at(m.sS + 2 * R3, R3W, lx + 2, ly + 2);
        St p0{}, p1{};
        float2 h{0.f, 0.f};
        if (!SCALAR) {
            st_pair(sP2, R4W, lx + 3, ly + 3, p0, p1);
            h = sH2[(ly + 2) * R3W + lx + 2];
        }
        float r[5];
        rhs_cell<float, SCALAR>(ph, sL, su.c, sv.c, pxx, pyy, pxy, om, s0, s1, s2, p0, p1, h.x, h.y, r);
        // y* (the sigma^E buffer is dead: C has finished)
        {
            const float yc[5] = {s0.c, s1.c, s2.c, p0.c, p1.c};
            float ys[5];
            predict<SCALAR ? 3 : 5>(yc, r, ys);
            sY01[i] = f2(ys[0], ys[1]);
            sY2[i] = ys[2];
            if (!SCALAR) sY34[i] = f2(ys[3], ys[4]);
        }
        if (k < R0) {       // an owned cell: k = (ly - 1) TX + (lx - 1)
            sR01[k] = f2(r[0], r[1]);
            sR2[k] = r[2];
            if (!SCALAR) sR34[k] = f2(r[3], r[4]);
        }
    }
    __syncthreads();
    if (wall) {
        // the predictor beyond a wall: the image (zero gradient of sigma and P)
        mirror_ghosts(m.sY, 1, 2, R1W, G::R1H, x0 - 1, y0 - 1, a, 1.f, 2);
        mirror_ghosts(sY2, R1, 1, R1W, G::R1H, x0 - 1, y0 - 1, a, 1.f);
        if (!SCALAR) mirror_ghosts(m.sY + 2 * R1, 1, 2, R1W, G::R1H, x0 - 1, y0 - 1, a, 1.f, 2);
        __syncthreads();
    }

    // ---- E: corrector, field stores, box writes, readout sums -------------------------------
    const unsigned bmask = (unsigned)m.sScan[NT / 32 + 1];
    for (int i = tid; i < R0; i += NT) {
        const int ly = i / TX, lx = i - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const long long g = (long long)gy * nx + gx;
        St su, sv;
        st_pair(sU2, R2W, lx + 2, ly + 2, su, sv);
        const float ux = su.c, uy = sv.c;
        // corrector with the frozen u
        {
            float pxx, pyy, pxy, om;
            vgrad(su, sv, pxx, pyy, pxy, om);
            St s0, s1, p0{}, p1{};
            st_pair(sY01, R1W, lx + 1, ly + 1, s0, s1);
            const St s2 = st_at(sY2, R1W, lx + 1, ly + 1);
            if (!SCALAR) st_pair(sY34, R1W, lx + 1, ly + 1, p0, p1);
            float hx = 0.f, hy = 0.f;
            if (!SCALAR) molecular(ph, p0, p1, hx, hy);
            float r[5];
            rhs_cell<float, SCALAR>(ph, sL, ux, uy, pxx, pyy, pxy, om, s0, s1, s2, p0, p1, hx, hy, r);
            const int j3 = (ly + 3) * R3W + lx + 3;
            const int j4 = (ly + 4) * R4W + lx + 4;
            const float2 R01 = sR01[i];
            if (SCALAR) {
                // sigma only: the scalar model has no P field (its planes keep their values)
                float* d = reinterpret_cast<float*>(dst);
                const float Rs[3] = {R01.x, R01.y, sR2[i]};
                const float y0s[3] = {m.sS[j3], m.sS[R3 + j3], m.sS[2 * R3 + j3]};
                float ynew[3];
                heun<3>(Rs, r, y0s, ynew);
                d[PL_SXX * NP + g] = ynew[0];
                d[PL_SYY * NP + g] = ynew[1];
                d[PL_SXY * NP + g] = ynew[2];
            } else {
                const float2 P0 = sP2[j4], R34 = sR34[i];
                const float y0s[5] = {m.sS[j3], m.sS[R3 + j3], m.sS[2 * R3 + j3], P0.x, P0.y};
                const float Rs[5] = {R01.x, R01.y, sR2[i], R34.x, R34.y};
                float ynew[5];
                heun<5>(Rs, r, y0s, ynew);
                st_flds<PREC>(dst, NP, g, ynew, (unsigned long long)t);
            }
        }
        box_write<R3, R3W>(a, bmask, t, gx, gy, ux, uy, readout, m.sS, (ly + 3) * R3W + lx + 3);
    }
    if (readout) readout_reduce(a, acc, m.sRed, tile_index);
}

// ---------------------------------------------------------------------------------------------
// The same step with two neighbouring cells (lx, lx+1) per thread: the per-cell arithmetic runs
// on float2 (paired FP32 instructions), stencil pairs are read from shared memory as 8-byte
// words where aligned, and global loads and stores of a pair use 8-byte accesses where the
// pair is contiguous and aligned in the lattice.  Region widths are even, so pairs never
// straddle rows.  Every lane computes exactly what tile_step's arithmetic (with the same
// fused multiply-adds) computes for its cell.
// ---------------------------------------------------------------------------------------------

// populations n of the cell pair at flat indices g0, g1; vec: g1 = g0 + 1 with g0 and the plane
// size even (aligned 8-byte or 4-byte access)
template <int PREC, bool COH>
__device__ __forceinline__ float2 ld_pop2(const void* src, long long NP, int n, long long g0, long long g1,
                                          bool vec)
{
    if (vec) {
        if (PREC == PREC_FP32) {
            const float2* p = reinterpret_cast<const float2*>(reinterpret_cast<const float*>(src) + n * NP + g0);
            return ld_state<float2, COH>(p);
        } else {
            const unsigned* p = reinterpret_cast<const unsigned*>(reinterpret_cast<const unsigned short*>(src) + n * NP + g0);
            const unsigned b = ld_state<unsigned, COH>(p);
            return make_float2(__half2float(__ushort_as_half((unsigned short)(b & 0xFFFFu))) * pop_unscale(n),
                               __half2float(__ushort_as_half((unsigned short)(b >> 16))) * pop_unscale(n));
        }
    }
    return make_float2(ld_pop<PREC, COH>(src, NP, n, g0), ld_pop<PREC, COH>(src, NP, n, g1));
}

template <int MODE, int PREC, int TX, int TY, bool COH = false>
__device__ __forceinline__ void tile_step2(const FusedArgs& a, int bx, int by, int tile_index, float* sm)
{
    static_assert(TX % 2 == 0, "cell pairs along x");
    using G = TileGeo<TX, TY>;
    constexpr int R4W = G::R4W, R4 = G::R4;
    constexpr int R3W = G::R3W, R3 = G::R3;
    constexpr int R2W = G::R2W, R2 = G::R2;
    constexpr int R1W = G::R1W, R1 = G::R1;
    constexpr int R0 = G::R0;
    const TileMem<TX, TY> m(sm);
    const float* sL = reinterpret_cast<const float*>(a.lut);
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const long long NP = a.plane;
    // 8-byte pair accesses to the lattice need even flat indices: nx even makes every row start,
    // plane size and pair start (x0 + lx, lx even) even
    const bool nx_even = (nx & 1) == 0;
    const int x0 = bx * TX, y0 = by * TY;
    const Phys& ph = a.ph;
    const void* src = a.src;

    stage<PREC, COH>(a, m, x0, y0);

    // ---- B (pairs): molecular field and Ericksen stress on the halo-3 region --------------
    for (int q = tid; q < R3 / 2; q += NT) {
        const int ly = q / (R3W / 2), lx = 2 * (q - ly * (R3W / 2));
        const StT<float2> px = st2_at<false>(m.sP, R4W, lx + 1, ly + 1);
        const StT<float2> py = st2_at<false>(m.sP + R4, R4W, lx + 1, ly + 1);
        float2 hx, hy, E[4];
        ericksen(ph, px, py, hx, hy, E);
        const int i = ly * R3W + lx;
        st2<true>(m.sH + i, hx);
        st2<true>(m.sH + R3 + i, hy);
        if (ph.ericksen) {
#pragma unroll
            for (int c = 0; c < 4; ++c) st2<true>(m.sE + c * R3 + i, E[c]);
        }
    }

    pdl_wait();
    pdl_trigger();
    ib_gather(a, m, x0, y0);

    // ---- C (pairs): total force and moments on the halo-2 region; collision of the owned
    // pairs (the owned columns 2 .. TX+1 of the halo-2 frame start at an even column, so a pair
    // is owned or not as a whole) -------------------------------------------------------------
    const long long t = step_index(a);
    const bool readout = (t % a.every) == 0;
    DF acc[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    void* dst = a.dst;
    for (int q = tid; q < R2 / 2; q += NT) {
        const int ly = q / (R2W / 2), lx = 2 * (q - ly * (R2W / 2));
        const int i = ly * R2W + lx;
        float2 Fx, Fy;
        div_sigma(st2_at<false>(m.sS, R3W, lx + 1, ly + 1), st2_at<false>(m.sS + R3, R3W, lx + 1, ly + 1),
                  st2_at<false>(m.sS + 2 * R3, R3W, lx + 1, ly + 1), Fx, Fy);
        if (ph.ericksen) {
            float2 ex, ey;
            div_ericksen(st2_at<false>(m.sE, R3W, lx + 1, ly + 1), st2_at<false>(m.sE + R3, R3W, lx + 1, ly + 1),
                         st2_at<false>(m.sE + 2 * R3, R3W, lx + 1, ly + 1),
                         st2_at<false>(m.sE + 3 * R3, R3W, lx + 1, ly + 1), ex, ey);
            Fx = Fx + ex;
            Fy = Fy + ey;
        }
        Fx = Fx + ld2<true>(m.sFib + i);
        Fy = Fy + ld2<true>(m.sFib + R2 + i);
        const long long row = (long long)m.sYi[ly + 2] * nx;
        const int gx0 = m.sXi[lx + 2], gx1 = m.sXi[lx + 3];
        const long long g0 = row + gx0, g1 = row + gx1;
        const bool vec = nx_even && gx1 == gx0 + 1;
        float2 d[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) d[n] = ld_pop2<PREC, COH>(src, NP, n, g0, g1, vec);
        float2 drho, ux, uy;
        moments(ph, d, Fx, Fy, drho, ux, uy);
        st2<true>(m.sM + R2 + i, ux);
        st2<true>(m.sM + 2 * R2 + i, uy);
        if (MODE == MODE_MOMENTS) {
            st2<true>(m.sM + i, drho);
            st2<true>(m.sFib + i, Fx);
            st2<true>(m.sFib + R2 + i, Fy);
        }
        const int gx = x0 + lx - 2, gy = y0 + ly - 2;
        const bool own = lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2 && gx < nx && gy < ny;
        if (MODE == MODE_STEP && own) {
            const bool has1 = gx + 1 < nx;             // the second cell lies in the lattice
            float2 D[9];
            collide(ph, d, drho, ux, uy, Fx, Fy, D);
            float2 out[9];
#pragma unroll
            for (int n = 0; n < 9; ++n) out[n] = d[n] + D[n];
            if (PREC == PREC_FP32) {
                float* dd = reinterpret_cast<float*>(dst);
#pragma unroll
                for (int n = 0; n < 9; ++n) {
                    const long long rowd = (long long)m.sYi[ly + 2 + C_CY[n]] * nx;
                    const int xa = m.sXi[lx + 2 + C_CX[n]], xb = m.sXi[lx + 3 + C_CX[n]];
                    float* pa = dd + n * NP + rowd + xa;
                    if (C_CX[n] == 0 && vec) {
                        *reinterpret_cast<float2*>(pa) = out[n];     // the pair's own columns
                    } else {
                        *pa = out[n].x;
                        if (has1) dd[n * NP + rowd + xb] = out[n].y;
                    }
                }
            } else {
                long long gd[9];
                float o1[9];
#pragma unroll
                for (int n = 0; n < 9; ++n) {
                    gd[n] = (long long)m.sYi[ly + 2 + C_CY[n]] * nx + m.sXi[lx + 2 + C_CX[n]];
                    o1[n] = out[n].x;
                }
                st_pops<PREC>(dst, NP, gd, o1, (unsigned long long)t, g0);
                if (has1) {
#pragma unroll
                    for (int n = 0; n < 9; ++n) {
                        gd[n] = (long long)m.sYi[ly + 2 + C_CY[n]] * nx + m.sXi[lx + 3 + C_CX[n]];
                        o1[n] = out[n].y;
                    }
                    st_pops<PREC>(dst, NP, gd, o1, (unsigned long long)t, g1);
                }
            }
            if (readout) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (k == 1 && !has1) break;
                    float dk[9];
#pragma unroll
                    for (int n = 0; n < 9; ++n) dk[n] = lane(d[n], k);
                    float dsum, jx, jy;
                    cell_readout(dk, dsum, jx, jy);
                    df_add(acc[0], dsum);
                    df_add(acc[1], jx);
                    df_add(acc[2], jy);
                    df_add(acc[3], lane(Fx, k));
                    df_add(acc[4], lane(Fy, k));
                }
            }
        }
    }
    __syncthreads();

    if (MODE == MODE_MOMENTS) {
        moments_out(a, m, x0, y0);
        return;
    }

    // ---- D (pairs): predictor on the halo-1 region ----------------------------------------
    for (int q = tid; q < R1 / 2; q += NT) {
        const int ly = q / (R1W / 2), lx = 2 * (q - ly * (R1W / 2));
        const StT<float2> su = st2_at<false>(m.sM + R2, R2W, lx + 1, ly + 1);
        const StT<float2> sv = st2_at<false>(m.sM + 2 * R2, R2W, lx + 1, ly + 1);
        float2 pxx, pyy, pxy, om;
        vgrad(su, sv, pxx, pyy, pxy, om);
        const StT<float2> s0 = st2_at<true>(m.sS, R3W, lx + 2, ly + 2);
        const StT<float2> s1 = st2_at<true>(m.sS + R3, R3W, lx + 2, ly + 2);
        const StT<float2> s2 = st2_at<true>(m.sS + 2 * R3, R3W, lx + 2, ly + 2);
        const StT<float2> p0 = st2_at<false>(m.sP, R4W, lx + 3, ly + 3);
        const StT<float2> p1 = st2_at<false>(m.sP + R4, R4W, lx + 3, ly + 3);
        const int j3 = (ly + 2) * R3W + lx + 2;
        float2 r[5];
        rhs_cell(ph, sL, su.c, sv.c, pxx, pyy, pxy, om, s0, s1, s2, p0, p1, ld2<true>(m.sH + j3),
                 ld2<true>(m.sH + R3 + j3), r);
        const int i = ly * R1W + lx;
        st2<true>(m.sY + i, s0.c + r[0]);
        st2<true>(m.sY + R1 + i, s1.c + r[1]);
        st2<true>(m.sY + 2 * R1 + i, s2.c + r[2]);
        st2<true>(m.sY + 3 * R1 + i, p0.c + r[3]);
        st2<true>(m.sY + 4 * R1 + i, p1.c + r[4]);
        if (ly >= 1 && ly <= TY) {
            // interior cells of the pair (the halo-1 frame is offset by one column from the tile)
            const int j0 = (ly - 1) * TX + (lx - 1);
            if (lx >= 1) {
#pragma unroll
                for (int c = 0; c < 5; ++c) m.sR[c * R0 + j0] = r[c].x;
            }
            if (lx + 1 <= TX) {
#pragma unroll
                for (int c = 0; c < 5; ++c) m.sR[c * R0 + j0 + 1] = r[c].y;
            }
        }
    }
    __syncthreads();

    // ---- E (pairs): corrector, field stores, box writes, readout sums ---------------------
    const unsigned bmask = (unsigned)m.sScan[NT / 32 + 1];
    for (int q = tid; q < R0 / 2; q += NT) {
        const int ly = q / (TX / 2), lx = 2 * (q - ly * (TX / 2));
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const bool has1 = gx + 1 < nx;                 // the second cell lies in the lattice
        const long long g0 = (long long)gy * nx + gx;
        const long long g1 = has1 ? g0 + 1 : g0;
        const bool vec = has1 && nx_even;
        const int i = ly * TX + lx;
        const StT<float2> su = st2_at<true>(m.sM + R2, R2W, lx + 2, ly + 2);
        const StT<float2> sv = st2_at<true>(m.sM + 2 * R2, R2W, lx + 2, ly + 2);
        const float2 ux = su.c, uy = sv.c;
        // corrector with the frozen u
        {
            float2 pxx, pyy, pxy, om;
            vgrad(su, sv, pxx, pyy, pxy, om);
            const StT<float2> s0 = st2_at<false>(m.sY, R1W, lx + 1, ly + 1);
            const StT<float2> s1 = st2_at<false>(m.sY + R1, R1W, lx + 1, ly + 1);
            const StT<float2> s2 = st2_at<false>(m.sY + 2 * R1, R1W, lx + 1, ly + 1);
            const StT<float2> p0 = st2_at<false>(m.sY + 3 * R1, R1W, lx + 1, ly + 1);
            const StT<float2> p1 = st2_at<false>(m.sY + 4 * R1, R1W, lx + 1, ly + 1);
            float2 hx, hy;
            molecular(ph, p0, p1, hx, hy);
            float2 r[5];
            rhs_cell(ph, sL, ux, uy, pxx, pyy, pxy, om, s0, s1, s2, p0, p1, hx, hy, r);
            const int j3 = (ly + 3) * R3W + lx + 3;
            const int j4 = (ly + 4) * R4W + lx + 4;
            const float2 y0s[5] = {ld2<false>(m.sS + j3), ld2<false>(m.sS + R3 + j3), ld2<false>(m.sS + 2 * R3 + j3),
                                   ld2<true>(m.sP + j4), ld2<true>(m.sP + R4 + j4)};
            float2 ynew[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) ynew[c] = vfma(0.5f, ld2<true>(m.sR + c * R0 + i) + r[c], y0s[c]);
            if (PREC == PREC_FP32) {
                float* d = reinterpret_cast<float*>(dst);
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    float* p = d + (PL_SXX + c) * NP + g0;
                    if (vec) {
                        *reinterpret_cast<float2*>(p) = ynew[c];
                    } else {
                        p[0] = ynew[c].x;
                        if (has1) d[(PL_SXX + c) * NP + g1] = ynew[c].y;
                    }
                }
            } else {
                float o[5];
#pragma unroll
                for (int c = 0; c < 5; ++c) o[c] = ynew[c].x;
                st_flds<PREC>(dst, NP, g0, o, (unsigned long long)t);
                if (has1) {
#pragma unroll
                    for (int c = 0; c < 5; ++c) o[c] = ynew[c].y;
                    st_flds<PREC>(dst, NP, g1, o, (unsigned long long)t);
                }
            }
        }
        const int j3 = (ly + 3) * R3W + lx + 3;
        box_write<R3, R3W>(a, bmask, t, gx, gy, ux.x, uy.x, readout, m.sS, j3);
        if (has1) box_write<R3, R3W>(a, bmask, t, gx + 1, gy, ux.y, uy.y, readout, m.sS, j3 + 1);
    }
    if (readout) readout_reduce(a, acc, m.sRed, tile_index);
}

}  // namespace tile
}  // namespace vlb
