// lb_strip.cuh -- the fused time step as warp strips swept along y (device code of the warp-strip
// kernel, shared by its single-lattice launch in lb_strip.cu and the batched launches in lb_batch.cu).
//
// The step of lb_tile.cuh (every field updated from the state at t, Fig. 2), organised so that
// no stored value is staged through shared memory and no barrier stands between the stages:
// a warp owns a strip of 32 lattice columns (lane = column; the 24 inner columns are its output,
// 4 columns of halo on each side) and a chunk of H rows, and sweeps the chunk upwards one row
// per iteration.  The stages run as a software pipeline on consecutive rows; with e the row the
// corrector finishes in iteration i:
//   loads  P row e+4, sigma row e+3, populations row e+2 (FP32 or the 2-byte precision form)
//   B      row e+3   molecular field h and Ericksen stress sigma^E (Sec. II C 1)
//   C      row e+2   F = f_IB + div sigma^p + div sigma^E, moments (Guo half force); on the owned
//                    cells the BGK collision with the Guo source pushed to x + c_n (Eq. LB,
//                    Eq. BGK), the readout sums and the u / f^p values on the ring work boxes
//   D      row e+1   velocity gradient, RHS of Eq. StiffCons and Eq. BE, Heun predictor
//   E      row e     Heun corrector with u frozen at t; sigma and P stored
// Each stage's north and south neighbours are rows that earlier iterations left in registers
// (rolling windows), its east and west neighbours are the adjacent lanes (warp shuffles).  Each
// stage is valid on one lane fewer per side than the one before (B lanes 1..30, C 2..29, D
// 3..28, E 4..27), so only the x halo is recomputed (32 / 24), and the y halo only at the chunk
// ends ((H + 6) / H for B).  Every per-cell expression is lb_cell.cuh's, evaluated on the same
// operands as in the tile kernel, so the fields and node positions equal the tile kernel's bit
// for bit; the FP64 readout sums differ only in the order of their partial sums.
//
// Spreading (App. A): per sub-chunk of 16 C rows a warp scatters the nodes of the rings whose
// work box meets its strip into a shared-memory row buffer, node after node in ring and index
// order, each ring's contribution summed on its own before it is added (the tile kernel's
// gather order).  No float atomics, no cross-lane accumulation: each lane owns its column.
// The node step of the same time step runs in the node kernel launched after this one.
#pragma once
#include <cuda_runtime.h>

#include "lb_cell.cuh"
#include "lb_internal.h"

namespace vlb {

// each translation unit that includes this header gets its own copy of the device code
namespace {


using namespace cell;

constexpr unsigned FULL = 0xffffffffu;
constexpr int SWARPS = 4;                 // warps (strips) per CTA
constexpr int SNT = 32 * SWARPS;
constexpr int SOWN = 24;                  // owned columns per strip: lanes 4 .. 27
constexpr int SUB = 8;                    // C rows per spreading sub-chunk
constexpr int NST = 3;                    // row stages of the load pipeline (two in flight)
// shared memory per warp: the load stages, [NST][14 planes][32 words] (a word holds one FP32
// column, or two columns of the 2-byte form), then f_IB of a sub-chunk and one ring's part of
// it, [SUB][2][32] floats each
constexpr int STAGE_WORDS = N_PLANES * 32;
constexpr int FIB_FLOATS = SUB * 2 * 32;
constexpr int WARP_FLOATS = NST * STAGE_WORDS + 2 * FIB_FLOATS;
constexpr int OFF_RED = SWARPS * WARP_FLOATS;                    // readout [5][SWARPS] (double)
constexpr size_t STRIP_SMEM = sizeof(float) * (OFF_RED + 2 * 5 * SWARPS);
static_assert(OFF_RED % 2 == 0, "alignment of the readout scratch");

// D2Q9 (Sec. II A): c_n, n = 0..8
__device__ constexpr int S_CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int S_CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// the value of the east (+x) and west (-x) neighbour column: the adjacent lanes
__device__ __forceinline__ float sh_e(float v) { return __shfl_down_sync(FULL, v, 1); }
__device__ __forceinline__ float sh_w(float v) { return __shfl_up_sync(FULL, v, 1); }

// five-point stencil at a lane from the values of its row (c) and of the rows above (n) and below (s)
__device__ __forceinline__ St st5(float c, float n, float s) { return St{c, sh_e(c), sh_w(c), n, s}; }

// one stored value (plane, flat index g) as FP32, decoded as ld_pop / ld_fld decode it, with a
// 32-bit index (the state stays below 2^31 values per buffer)
template <int PREC>
__device__ __forceinline__ float ldp(const void* src, int NP, int plane, int g)
{
    const int o = plane * NP + g;
    if (PREC == PREC_FP32) return __ldg(reinterpret_cast<const float*>(src) + o);
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(src) + o);
    if (plane < PL_SXX) return __half2float(__ushort_as_half(b)) * pop_unscale(plane);
    if (plane >= PL_PX) return __half2float(__ushort_as_half(b));
    return __uint_as_float((unsigned)b << 16);
}

// asynchronous 4-byte copies global -> shared (completion tracked per thread in commit groups)
__device__ __forceinline__ void cp4(unsigned dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copy one row of `nplanes` planes from plane p0 (row y of the lattice, the strip's 32 columns
// from xs, wrapped) into the stage at word offset p0 * 32 of `st`.  FP32: lane l copies column
// xs + l.  2-byte form: lanes 0..15 copy the 4-byte word of columns xs + 2l, xs + 2l + 1 (xs and nx
// even, so a word never straddles the periodic seam).
template <int PREC>
__device__ __forceinline__ void stage_row(unsigned st, const void* src, int NP, int p0, int nplanes, int y, int nx,
                                          int xs, int gx)
{
    const int lane = threadIdx.x & 31;
    if (PREC == PREC_FP32) {
        const float* b = reinterpret_cast<const float*>(src) + (p0 * NP + y * nx + gx);
        for (int q = 0; q < nplanes; ++q) cp4(st + 4u * (unsigned)((p0 + q) * 32 + lane), b + q * NP);
    } else if (lane < 16) {
        int c0 = xs + 2 * lane;
        if (c0 < 0) c0 += nx;
        else if (c0 >= nx) c0 -= nx;
        const unsigned short* b = reinterpret_cast<const unsigned short*>(src) + (p0 * NP + y * nx + c0);
        for (int q = 0; q < nplanes; ++q) cp4(st + 4u * (unsigned)((p0 + q) * 32 + lane), b + q * NP);
    }
}

// one staged value of plane `plane` at this lane's column, decoded as ld_pop / ld_fld decode it
template <int PREC>
__device__ __forceinline__ float staged(const unsigned* st, int plane)
{
    const int lane = threadIdx.x & 31;
    if (PREC == PREC_FP32) return __uint_as_float(st[plane * 32 + lane]);
    const unsigned short b = reinterpret_cast<const unsigned short*>(st)[plane * 64 + lane];
    if (plane < PL_SXX) return __half2float(__ushort_as_half(b)) * pop_unscale(plane);
    if (plane >= PL_PX) return __half2float(__ushort_as_half(b));
    return __uint_as_float((unsigned)b << 16);
}

// f_IB on the C rows [yr0, yr0 + SUB) of this warp's strip (column gx per lane) into fib[SUB][2][32]:
// for every ring of `meet` whose box meets these rows, its nodes in index order, in chunks of 256
// as the tile kernel gathers them, each chunk's sum formed apart (tmp) and then added.
__device__ __noinline__ void strip_spread(const FusedArgs& a, unsigned meet, long long t, int yr0, int xs, int gx,
                                          float* fib, float* tmp)
{
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny;
    for (int k = 0; k < SUB; ++k) {
        fib[(2 * k) * 32 + lane] = 0.f;
        fib[(2 * k + 1) * 32 + lane] = 0.f;
    }
    const int nr = a.n_rings;
    for (int r = 0; r < nr; ++r) {
        if (nr <= 32 && !((meet >> r) & 1u)) continue;
        const RingDev& R = a.rings[r];
        const int4 bx = ring_box(R, t);
        if (!meets(yr0, SUB, bx.y, bx.w, ny) || !meets(xs, 32, bx.x, bx.z, nx)) continue;
        float2 tf = make_float2(0.f, 0.f);
        if (R.trap_k > 0.0) tf = R.trap_f[t & 1];
        for (int base = 0; base < R.n_nodes; base += 256) {
            for (int k = 0; k < SUB; ++k) {
                tmp[(2 * k) * 32 + lane] = 0.f;
                tmp[(2 * k + 1) * 32 + lane] = 0.f;
            }
            const int end = min(base + 256, R.n_nodes);
            for (int b32 = base; b32 < end; b32 += 32) {
                const int k = b32 + lane;
                bool keep = false;
                int cx = 0, cyr = 0;
                float2 fr = make_float2(0.f, 0.f), f = make_float2(0.f, 0.f);
                if (k < end) {
                    const int2 c = a.node_cell[R.node_off + k];
                    fr = a.node_frac[R.node_off + k];
                    f = a.node_force[R.node_off + k];
                    if (R.trap_k > 0.0) {
                        f.x += tf.x;
                        f.y += tf.y;
                    }
                    cx = c.x;
                    cyr = mimg(c.y - yr0, ny);                       // node row relative to yr0
                    const int cxr = mimg(c.x - xs, nx);
                    keep = cyr >= -2 && cyr <= SUB + 1 && cxr >= -2 && cxr <= 33;
                }
                unsigned bal = __ballot_sync(FULL, keep);
                while (bal) {
                    const int j = __ffs(bal) - 1;
                    bal &= bal - 1;
                    const int qcx = __shfl_sync(FULL, cx, j), qcy = __shfl_sync(FULL, cyr, j);
                    const float qfx = __shfl_sync(FULL, fr.x, j), qfy = __shfl_sync(FULL, fr.y, j);
                    const float qFx = __shfl_sync(FULL, f.x, j), qFy = __shfl_sync(FULL, f.y, j);
                    const float dx = (float)mimg(qcx - gx, nx) + qfx;   // node - cell, as in the gather
                    if (fabsf(dx) < 2.f) {
                        for (int kr = max(qcy - 1, 0); kr <= min(qcy + 2, SUB - 1); ++kr) {
                            const float dy = (float)(qcy - kr) + qfy;
                            if (fabsf(dy) < 2.f) {
                                const float w = phi(dx) * phi(dy);
                                tmp[(2 * kr) * 32 + lane] += qFx * w;
                                tmp[(2 * kr + 1) * 32 + lane] += qFy * w;
                            }
                        }
                    }
                }
            }
            for (int k = 0; k < SUB; ++k) {
                fib[(2 * k) * 32 + lane] += tmp[(2 * k) * 32 + lane];
                fib[(2 * k + 1) * 32 + lane] += tmp[(2 * k + 1) * 32 + lane];
            }
        }
    }
}

// One CTA of the step: warps wid = 0..3 take strips cx * SWARPS + wid of the rows chunk
// [cy * H, cy * H + H); t: the step index; part: the CTA's slot in the readout partials; smem:
// STRIP_SMEM bytes of shared memory.
template <int PREC, bool SCALAR>
__device__ __forceinline__ void strip_body(const FusedArgs& a, long long t, int H, int cx, int cy, long long part,
                                           float* smem)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nx = a.nx, ny = a.ny;
    const int NP = (int)a.plane;
    const int n_strips = (nx + SOWN - 1) / SOWN;
    const int strip = cx * SWARPS + wid;
    const int yc = cy * H;
    const int Hc = min(H, ny - yc);
    const bool readout = (t % a.every) == 0;
    const Phys& ph = a.ph;
    const float* lut = reinterpret_cast<const float*>(a.lut);
    const void* src = a.src;
    void* dst = a.dst;
    unsigned* stages = reinterpret_cast<unsigned*>(smem + wid * WARP_FLOATS);
    const unsigned stages_s = (unsigned)__cvta_generic_to_shared(stages);
    float* fib = smem + wid * WARP_FLOATS + NST * STAGE_WORDS;
    float* tmp = fib + FIB_FLOATS;
    DF acc[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};

    // the state at t was written two launches back; the ring records, node forces and boxes by
    // the node kernel just before this one
    pdl_wait();
    pdl_trigger();

    if (strip < n_strips) {
        const int xo = strip * SOWN;                  // first owned column
        const int xs = xo - 4;                        // column of lane 0
        const int gx = wrapn(xs + lane, nx);
        const bool own_lane = lane >= 4 && lane < 4 + SOWN && xo + lane - 4 < nx;
        const int gxp = gx + 1 == nx ? 0 : gx + 1, gxm = gx == 0 ? nx - 1 : gx - 1;

        // rings whose work box meets the strip's C region (spreading) and its owned cells (boxes)
        unsigned meet = 0u, bown = 0u;
        const int nr = a.n_rings;
        if (nr > 32) {
            meet = bown = FULL;
        } else if (nr > 0) {
            bool m2 = false, mo = false;
            if (lane < nr) {
                const int4 bx = ring_box(a.rings[lane], t);
                m2 = meets(xs + 2, 28, bx.x, bx.z, nx) && meets(yc - 2, Hc + 4, bx.y, bx.w, ny);
                mo = meets(xo, SOWN, bx.x, bx.z, nx) && meets(yc, Hc, bx.y, bx.w, ny);
            }
            meet = __ballot_sync(FULL, m2);
            bown = __ballot_sync(FULL, mo);
        }

        // rolling windows (index r: row e + r of the iteration, e the corrector's row)
        float P0[5], P1[5];              // dP (x, y), rows e .. e+4
        float S0[4], S1[4], S2[4];       // sigma (xx, yy, xy), rows e .. e+3
        float Exx2 = 0.f, Eyx2 = 0.f;    // sigma^E xx, yx at row e+2
        float Exy1 = 0.f, Exy2 = 0.f, Eyy1 = 0.f, Eyy2 = 0.f;   // xy, yy at rows e+1, e+2
        float H0[2], H1[2];              // h (x, y) at rows e+1, e+2
        float U0[4], U1[4];              // u (x, y) at rows e-1 .. e+2
        float Y[5][3];                   // y* (sxx, syy, sxy, Px, Py) at rows e-1 .. e+1
        float R[5];                      // RHS(y) at row e
#pragma unroll
        for (int r = 0; r < 5; ++r) P0[r] = P1[r] = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) S0[r] = S1[r] = S2[r] = U0[r] = U1[r] = 0.f;
        H0[0] = H0[1] = H1[0] = H1[1] = 0.f;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            R[c] = 0.f;
            Y[c][0] = Y[c][1] = Y[c][2] = 0.f;
        }
        // Load pipeline: iteration j reads P row yc + j (its e+4), sigma row yc + j - 1 (e+3) and,
        // from j = 0, the populations of row yc + j - 2 (e+2) from stage (j + 3) % NST; those rows
        // are copied two iterations ahead.  rP, rS, rC: the wrapped rows of the next copy.
        int rP = wrapn(yc - 2, ny), rS = wrapn(yc - 3, ny), rC = wrapn(yc - 4, ny);
        auto issue = [&](int j) {                     // the copies of iteration j, one commit group
            const unsigned st = stages_s + 4u * (unsigned)(((j + 3) % NST) * STAGE_WORDS);
            stage_row<PREC>(st, src, NP, PL_SXX, 3, rS, nx, xs, gx);
            if (!SCALAR) stage_row<PREC>(st, src, NP, PL_PX, 2, rP, nx, xs, gx);
            if (j >= 0) stage_row<PREC>(st, src, NP, 0, 9, rC, nx, xs, gx);
            cp_commit();
            if (++rP == ny) rP = 0;
            if (++rS == ny) rS = 0;
            if (++rC == ny) rC = 0;
        };
        issue(-2);
        issue(-1);
        // P rows yc - 4, yc - 3 ahead of the first iteration (they sit at e+2, e+3 when i = -2)
        if (!SCALAR) {
            const int g4 = wrapn(yc - 4, ny) * nx + gx, g3 = wrapn(yc - 3, ny) * nx + gx;
            P0[2] = ldp<PREC>(src, NP, PL_PX, g4);
            P1[2] = ldp<PREC>(src, NP, PL_PY, g4);
            P0[3] = ldp<PREC>(src, NP, PL_PX, g3);
            P1[3] = ldp<PREC>(src, NP, PL_PY, g3);
        }

        for (int i = -2; i <= Hc + 3; ++i) {
            const int e = yc + i - 4;
            // ---- this iteration's rows from the stage; the copies for iteration i + 2 --------
            cp_wait_prev();                           // the group of iteration i has landed
            __syncwarp();                             // ... for every lane (2-byte words are shared)
            const unsigned* st = stages + ((i + 3) % NST) * STAGE_WORDS;
            if (i + 2 <= Hc + 3) issue(i + 2);
            else cp_commit();                         // an empty group keeps the count
            S0[3] = staged<PREC>(st, PL_SXX);
            S1[3] = staged<PREC>(st, PL_SYY);
            S2[3] = staged<PREC>(st, PL_SXY);
            if (!SCALAR) {
                P0[4] = staged<PREC>(st, PL_PX);
                P1[4] = staged<PREC>(st, PL_PY);
            }
            float d[9];
            const int yC = e + 2;                     // the C row (may lie outside [0, ny))
            if (i >= 0) {
#pragma unroll
                for (int n = 0; n < 9; ++n) d[n] = staged<PREC>(st, n);
            }

            // ---- B: molecular field and Ericksen stress at row e+3 ------------------------
            float hx3 = 0.f, hy3 = 0.f, E3[4] = {0.f, 0.f, 0.f, 0.f};
            if (!SCALAR) {
                const St px = st5(P0[3], P0[4], P0[2]);
                const St py = st5(P1[3], P1[4], P1[2]);
                ericksen(ph, px, py, hx3, hy3, E3);      // E3 = (xx, xy, yx, yy)
            }

            // ---- C: forces, moments, collision of the owned cells at row e+2 ---------------
            if (i >= 0) {
                if ((i % SUB) == 0 && meet) strip_spread(a, meet, t, yC, xs, gx, fib, tmp);
                float Fx, Fy;
                {
                    const St sxx{S0[2], sh_e(S0[2]), sh_w(S0[2]), 0.f, 0.f};
                    const St syy{0.f, 0.f, 0.f, S1[3], S1[1]};
                    const St sxy{0.f, sh_e(S2[2]), sh_w(S2[2]), S2[3], S2[1]};
                    div_sigma(sxx, syy, sxy, Fx, Fy);
                    if (!SCALAR && ph.ericksen) {
                        const St exx{0.f, sh_e(Exx2), sh_w(Exx2), 0.f, 0.f};
                        const St exy{0.f, 0.f, 0.f, E3[1], Exy1};
                        const St eyx{0.f, sh_e(Eyx2), sh_w(Eyx2), 0.f, 0.f};
                        const St eyy{0.f, 0.f, 0.f, E3[3], Eyy1};
                        float ex, ey;
                        div_ericksen(exx, exy, eyx, eyy, ex, ey);
                        Fx += ex;
                        Fy += ey;
                    }
                    const int kr = i % SUB;
                    Fx += meet ? fib[(2 * kr) * 32 + lane] : 0.f;
                    Fy += meet ? fib[(2 * kr + 1) * 32 + lane] : 0.f;
                    float drho, ux, uy;
                    moments(ph, d, Fx, Fy, drho, ux, uy);
                    U0[3] = ux;
                    U1[3] = uy;
                    // owned cells of the chunk: collide, push, readout sums, ring work boxes
                    const int yo = yC - yc;                   // 0 .. Hc-1 for an owned row
                    if (own_lane && yo >= 0 && yo < Hc) {
                        float D[9], out[9];
                        int gd[9];
                        collide(ph, d, drho, ux, uy, Fx, Fy, D);
                        const int gy = yC;                    // inside [0, ny)
                        const int gC = gy * nx + gx;
                        const int gyp = gy + 1 == ny ? 0 : gy + 1, gym = gy == 0 ? ny - 1 : gy - 1;
#pragma unroll
                        for (int n = 0; n < 9; ++n) {
                            const int yy = S_CY[n] > 0 ? gyp : (S_CY[n] < 0 ? gym : gy);
                            const int xx = S_CX[n] > 0 ? gxp : (S_CX[n] < 0 ? gxm : gx);
                            gd[n] = yy * nx + xx;
                        }
                        add_pops(d, D, out);
                        long long gdl[9];
#pragma unroll
                        for (int n = 0; n < 9; ++n) gdl[n] = gd[n];
                        st_pops<PREC>(dst, NP, gdl, out, (unsigned long long)t, gC);
                        if (readout) {
                            float dsum, jx, jy;
                            cell_readout(d, dsum, jx, jy);
                            df_add(acc[0], dsum);
                            df_add(acc[1], jx);
                            df_add(acc[2], jy);
                            df_add(acc[3], Fx);
                            df_add(acc[4], Fy);
                        }
                        // u (and f^p on readout steps, as the tile kernel forms it) on the work
                        // box of every ring whose box holds this cell
                        auto box_put = [&](int r2) {
                            const RingDev& Rg = a.rings[r2];
                            const int4 B = ring_box(Rg, t);
                            int bx = gx - B.x; if (bx < 0) bx += nx;
                            int by = gy - B.y; if (by < 0) by += ny;
                            if (bx < B.z && by < B.w) {
                                const long long o = Rg.box_off + (long long)by * Rg.cap_w + bx;
                                const long long cap = (long long)Rg.cap_w * Rg.cap_h;
                                a.ubox[o] = ux;
                                a.ubox[o + cap] = uy;
                                if (readout) {
                                    a.fpbox[o] = 0.5f * (sxx.e - sxx.w) + 0.5f * (sxy.n - sxy.s);
                                    a.fpbox[o + cap] = 0.5f * (sxy.e - sxy.w) + 0.5f * (syy.n - syy.s);
                                }
                            }
                        };
                        if (nr > 32) {
                            for (int r2 = 0; r2 < nr; ++r2) box_put(r2);
                        } else {
                            for (unsigned m = bown; m; m &= m - 1) box_put(__ffs(m) - 1);
                        }
                    }
                }
            }

            // ---- D: predictor at row e+1 ------------------------------------------------------
            float Rn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            if (i >= 2) {
                float pxx, pyy, pxy, om;
                vgrad(st5(U0[2], U0[3], U0[1]), st5(U1[2], U1[3], U1[1]), pxx, pyy, pxy, om);
                const St s0 = st5(S0[1], S0[2], S0[0]);
                const St s1 = st5(S1[1], S1[2], S1[0]);
                const St s2 = st5(S2[1], S2[2], S2[0]);
                const St p0 = SCALAR ? St{} : st5(P0[1], P0[2], P0[0]);
                const St p1 = SCALAR ? St{} : st5(P1[1], P1[2], P1[0]);
                rhs_cell<float, SCALAR>(ph, lut, U0[2], U1[2], pxx, pyy, pxy, om, s0, s1, s2, p0, p1,
                                        SCALAR ? 0.f : H0[0], SCALAR ? 0.f : H1[0], Rn);
                const float yc[5] = {s0.c, s1.c, s2.c, p0.c, p1.c};
                float ys[5];
                predict<SCALAR ? 3 : 5>(yc, Rn, ys);
#pragma unroll
                for (int c = 0; c < (SCALAR ? 3 : 5); ++c) Y[c][2] = ys[c];
            }

            // ---- E: corrector at row e ----------------------------------------------------------
            if (i >= 4) {
                float pxx, pyy, pxy, om;
                vgrad(st5(U0[1], U0[2], U0[0]), st5(U1[1], U1[2], U1[0]), pxx, pyy, pxy, om);
                const St y0 = st5(Y[0][1], Y[0][2], Y[0][0]);
                const St y1 = st5(Y[1][1], Y[1][2], Y[1][0]);
                const St y2 = st5(Y[2][1], Y[2][2], Y[2][0]);
                const St y3 = SCALAR ? St{} : st5(Y[3][1], Y[3][2], Y[3][0]);
                const St y4 = SCALAR ? St{} : st5(Y[4][1], Y[4][2], Y[4][0]);
                float hx = 0.f, hy = 0.f;
                if (!SCALAR) molecular(ph, y3, y4, hx, hy);
                float r[5];
                rhs_cell<float, SCALAR>(ph, lut, U0[1], U1[1], pxx, pyy, pxy, om, y0, y1, y2, y3, y4, hx, hy, r);
                if (own_lane) {
                    const int g = e * nx + gx;            // e inside [yc, yc + Hc)
                    if (SCALAR) {
                        float* dd = reinterpret_cast<float*>(dst);
                        const float y0s[3] = {S0[0], S1[0], S2[0]};
                        float ynew[3];
                        heun<3>(R, r, y0s, ynew);
                        dd[PL_SXX * NP + g] = ynew[0];
                        dd[PL_SYY * NP + g] = ynew[1];
                        dd[PL_SXY * NP + g] = ynew[2];
                    } else {
                        const float y0s[5] = {S0[0], S1[0], S2[0], P0[0], P1[0]};
                        float ynew[5];
                        heun<5>(R, r, y0s, ynew);
                        st_flds<PREC>(dst, NP, g, ynew, (unsigned long long)t);
                    }
                }
            }

            // ---- advance the windows by one row ------------------------------------------------
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                P0[r] = P0[r + 1];
                P1[r] = P1[r + 1];
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                S0[r] = S0[r + 1];
                S1[r] = S1[r + 1];
                S2[r] = S2[r + 1];
                U0[r] = U0[r + 1];
                U1[r] = U1[r + 1];
            }
            Exx2 = E3[0];
            Eyx2 = E3[2];
            Exy1 = Exy2;
            Exy2 = E3[1];
            Eyy1 = Eyy2;
            Eyy2 = E3[3];
            H0[0] = H0[1];
            H1[0] = H1[1];
            H0[1] = hx3;
            H1[1] = hy3;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                Y[c][0] = Y[c][1];
                Y[c][1] = Y[c][2];
                R[c] = Rn[c];
            }
        }
        cp_wait_all();                                // no copy outlives the warp's work
    }

    if (readout) {
        // fixed-order reduction of the CTA's double-float readout sums into its partial slot
        store_partial(a.partials, part, acc, smem + OFF_RED);
    }
}

}  // namespace
}  // namespace vlb
