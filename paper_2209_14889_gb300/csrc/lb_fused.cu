// lb_fused.cu -- the fused lattice kernel: one whole time step of every lattice field.
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
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace vlb {

namespace {

constexpr int TX = 32;
constexpr int TY = 16;
constexpr int NT = 256;

constexpr int R4W = TX + 8, R4H = TY + 8, R4 = R4W * R4H;
constexpr int R3W = TX + 6, R3H = TY + 6, R3 = R3W * R3H;
constexpr int R2W = TX + 4, R2H = TY + 4, R2 = R2W * R2H;
constexpr int R1W = TX + 2, R1H = TY + 2, R1 = R1W * R1H;
constexpr int R0 = TX * TY;

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int al4(int x) { return (x + 3) & ~3; }   // 16-byte alignment in floats

// shared-memory layout (in floats)
constexpr int OFF_P = 0;                                  // P        [2][R4]
constexpr int OFF_S = OFF_P + 2 * R4;                     // sigma    [3][R3]
constexpr int OFF_E = OFF_S + 3 * R3;                     // sigma^E  [4][R3]  | y* [5][R1]
constexpr int SZ_E = cmax(4 * R3, 5 * R1);
constexpr int OFF_H = OFF_E + SZ_E;                       // h        [2][R3]
constexpr int OFF_M = OFF_H + 2 * R3;                     // drho,ux,uy,Fx,Fy [5][R2]
constexpr int OFF_R = OFF_M + 5 * R2;                     // RHS(y)   [5][R0] | f_IB [2][R2]
constexpr int SZ_R = cmax(5 * R0, 2 * R2);
constexpr int OFF_L = OFF_R + SZ_R;                       // LUT      [2][LUT_N+1]
constexpr int OFF_N = al4(OFF_L + 2 * (LUT_N + 1));       // nodes    [NT] float4 (cell, frac)
constexpr int OFF_NF = OFF_N + 4 * NT;                    // node forces [NT] float2
constexpr int OFF_XI = OFF_NF + 2 * NT;                   // wrapped x index [R4W] (int)
constexpr int OFF_YI = OFF_XI + R4W;                      // wrapped y index [R4H] (int)
constexpr int OFF_SC = OFF_YI + R4H;                      // scan scratch [NT/32 + 1] (int)
constexpr int OFF_RED = al4(OFF_SC + NT / 32 + 1);        // readout [5][NT/32] (double)
constexpr int SMEM_FLOATS = OFF_RED + 2 * 5 * (NT / 32);
constexpr size_t SMEM_BYTES = sizeof(float) * SMEM_FLOATS;
static_assert(OFF_N % 4 == 0 && OFF_NF % 2 == 0 && OFF_RED % 2 == 0, "shared-memory alignment");
static_assert(SMEM_BYTES <= 75 * 1024, "three CTAs per SM");

__device__ __forceinline__ int wrapn(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// minimum image of an integer offset on a periodic axis of length n, in [-n/2, n/2)
__device__ __forceinline__ int mimg(int d, int n)
{
    d %= n;
    if (d < -(n / 2)) d += n;
    else if (d >= n - n / 2) d -= n;
    return d;
}

// cosine IB kernel phi(r) = (1 + cos(pi r / 2)) / 4 for |r| < 2 (App. A)
__device__ __forceinline__ float phi(float r)
{
    return fabsf(r) < 2.f ? 0.25f * (1.f + cospif(0.5f * r)) : 0.f;
}

__device__ __forceinline__ void lut_eval(const float* L, const Phys& ph, float q, float& a2, float& a4)
{
    float qq = fminf(q, ph.q_cap);
    float t = qq * ph.lut_scale;
    int i = min(max((int)t, 1), LUT_N - 2);
    float f = t - (float)i;
    float fm1 = f - 1.f, fm2 = f - 2.f, fp1 = f + 1.f;
    float w0 = -f * fm1 * fm2 * (1.f / 6.f);
    float w1 = fp1 * fm1 * fm2 * 0.5f;
    float w2 = -fp1 * f * fm2 * 0.5f;
    float w3 = fp1 * f * fm1 * (1.f / 6.f);
    const float* v = L + 2 * (i - 1);
    a2 = w0 * v[0] + w1 * v[2] + w2 * v[4] + w3 * v[6];
    a4 = w0 * v[1] + w1 * v[3] + w2 * v[5] + w3 * v[7];
    if (q > ph.q_cap) {
        float s = ph.q_cap / q;
        a2 *= s;
        a4 *= s * s;
    }
}

// Stencil values of one component: centre, east (+x), west, north (+y), south.
struct St {
    float c, e, w, n, s;
};

__device__ __forceinline__ St st_at(const float* base, int W, int lx, int ly)
{
    const float* p = base + ly * W + lx;
    return St{p[0], p[1], p[-1], p[W], p[-W]};
}

// Molecular field h = (alpha + beta |P|^2) P - kappa lap P (Eq. Ffunctional) from the stencil
// of dP = P - P_ref: alpha + beta |P|^2 = A0 + beta (2 P_ref.dP + |dP|^2) has no cancellation.
__device__ __forceinline__ void molecular(const Phys& ph, const St& dx, const St& dy, float& hx,
                                          float& hy)
{
    const float A = ph.A0 + ph.beta * (2.f * (ph.prx * dx.c + ph.pry * dy.c) + (dx.c * dx.c + dy.c * dy.c));
    hx = A * (ph.prx + dx.c) - ph.kappa * (dx.e + dx.w + dx.n + dx.s - 4.f * dx.c);
    hy = A * (ph.pry + dy.c) - ph.kappa * (dy.e + dy.w + dy.n + dy.s - 4.f * dy.c);
}

// Right-hand sides of Eq. StiffCons (with the Jaumann derivative) and Eq. BE at one cell, for
// the frozen u, Psi = (pxx, pyy, pxy), omega = Omega_xy; s = sigma (xx, yy, xy), p = dP (x, y).
__device__ __forceinline__ void rhs_cell(const Phys& ph, const float* lut, float ux, float uy,
                                         float pxx, float pyy, float pxy, float om,
                                         const St& s0, const St& s1, const St& s2,
                                         const St& p0, const St& p1, float hx, float hy,
                                         float* r)
{
    // stiffness C~(P) (App. B) from the table of a2, a4 and polynomials in P = P_ref + dP
    const float Px = ph.prx + p0.c, Py = ph.pry + p1.c;
    const float q = Px * Px + Py * Py;
    float a2, a4;
    lut_eval(lut, ph, q, a2, a4);
    const float c2q = Px * Px - Py * Py, s2q = 2.f * Px * Py;
    const float r2c2 = a2 * c2q, r2s2 = a2 * s2q;
    const float r4c4 = a4 * (c2q * c2q - s2q * s2q), r4s4 = a4 * (2.f * c2q * s2q);
    const float C11 = ph.kS8 + 0.5f * ph.dK * r2c2 + 0.125f * ph.kX * r4c4;
    const float C12 = ph.kC12 - 0.125f * ph.kX * r4c4;
    const float C13 = 0.25f * ph.kX * r4s4 + 0.5f * ph.dK * r2s2;
    const float C22 = C11 - ph.dK * r2c2;
    const float C23 = 0.5f * ph.dK * r2s2 - 0.25f * ph.kX * r4s4;
    const float C33 = ph.kC33 - 0.25f * ph.kX * r4c4;

    // C psi - C s / eta_p = C (psi - s / eta_p)
    const float v0 = pxx - ph.inv_eta * s0.c;
    const float v1 = pyy - ph.inv_eta * s1.c;
    const float v2 = pxy - ph.inv_eta * s2.c;
    const float Cv0 = C11 * v0 + C12 * v1 + C13 * v2;
    const float Cv1 = C12 * v0 + C22 * v1 + C23 * v2;
    const float Cv2 = 0.5f * C13 * v0 + 0.5f * C23 * v1 + C33 * v2;

    // Jaumann rotation (Omega s - s Omega) = (2 w sxy, -2 w sxy, w (syy - sxx))
    const float J0 = 2.f * om * s2.c;
    const float J2 = om * (s1.c - s0.c);

    const float D = ph.Dp;
    r[0] = -(ux * 0.5f * (s0.e - s0.w) + uy * 0.5f * (s0.n - s0.s)) - J0 + Cv0 +
           D * (s0.e + s0.w + s0.n + s0.s - 4.f * s0.c);
    r[1] = -(ux * 0.5f * (s1.e - s1.w) + uy * 0.5f * (s1.n - s1.s)) + J0 + Cv1 +
           D * (s1.e + s1.w + s1.n + s1.s - 4.f * s1.c);
    r[2] = -(ux * 0.5f * (s2.e - s2.w) + uy * 0.5f * (s2.n - s2.s)) - J2 + Cv2 +
           D * (s2.e + s2.w + s2.n + s2.s - 4.f * s2.c);
    // Eq. BE: -(u.grad)P - Omega P + xi Psi P - Gamma h
    r[3] = -(ux * 0.5f * (p0.e - p0.w) + uy * 0.5f * (p0.n - p0.s)) - om * Py +
           ph.xi * (pxx * Px + pxy * Py) - ph.Gamma * hx;
    r[4] = -(ux * 0.5f * (p1.e - p1.w) + uy * 0.5f * (p1.n - p1.s)) + om * Px +
           ph.xi * (pxy * Px + pyy * Py) - ph.Gamma * hy;
}

// Velocity gradient at the cell (lx, ly) of a region of width W (u planes at ux, uy).
__device__ __forceinline__ void vgrad(const float* ux, const float* uy, int W, int i, float& pxx,
                                      float& pyy, float& pxy, float& om)
{
    const float dxux = 0.5f * (ux[i + 1] - ux[i - 1]);
    const float dyux = 0.5f * (ux[i + W] - ux[i - W]);
    const float dxuy = 0.5f * (uy[i + 1] - uy[i - 1]);
    const float dyuy = 0.5f * (uy[i + W] - uy[i - W]);
    pxx = dxux;
    pyy = dyuy;
    pxy = 0.5f * (dxuy + dyux);
    om = 0.5f * (dxuy - dyux);
}

// Does the periodic interval [b, b + bw) meet [a, a + aw) on an axis of length n?
__device__ __forceinline__ bool meets(int a, int aw, int b, int bw, int n)
{
    if (aw >= n || bw >= n) return true;
    int d1 = wrapn(a - b, n), d2 = wrapn(b - a, n);
    return d1 < bw || d2 < aw;
}

template <int MODE>
__global__ void __launch_bounds__(NT, 3) k_fused(const FusedArgs a)
{
    extern __shared__ __align__(16) float sm[];
    float* sP = sm + OFF_P;
    float* sS = sm + OFF_S;
    float* sE = sm + OFF_E;
    float* sY = sm + OFF_E;      // y* after sigma^E is dead
    float* sH = sm + OFF_H;
    float* sM = sm + OFF_M;
    float* sR = sm + OFF_R;
    float* sFib = sm + OFF_R;    // f_IB before RHS(y) is written
    float* sL = sm + OFF_L;
    float4* sNode = reinterpret_cast<float4*>(sm + OFF_N);
    float2* sNodeF = reinterpret_cast<float2*>(sm + OFF_NF);
    int* sXi = reinterpret_cast<int*>(sm + OFF_XI);
    int* sYi = reinterpret_cast<int*>(sm + OFF_YI);
    int* sScan = reinterpret_cast<int*>(sm + OFF_SC);
    double* sRed = reinterpret_cast<double*>(sm + OFF_RED);

    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const long long NP = a.plane;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const Phys ph = a.ph;
    const float* __restrict__ src = a.src;

    for (int i = tid; i < R4W; i += NT) sXi[i] = wrapn(x0 - 4 + i, nx);
    for (int i = tid; i < R4H; i += NT) sYi[i] = wrapn(y0 - 4 + i, ny);
    for (int i = tid; i < 2 * (LUT_N + 1); i += NT) sL[i] = reinterpret_cast<const float*>(a.lut)[i];
    for (int i = tid; i < 2 * R2; i += NT) sFib[i] = 0.f;
    __syncthreads();

    // ---- A: stage P (halo 4) and sigma (halo 3) ---------------------------------------------
    for (int i = tid; i < R4; i += NT) {
        const int ly = i / R4W, lx = i - ly * R4W;
        const long long g = (long long)sYi[ly] * nx + sXi[lx];
        sP[i] = __ldg(src + PL_PX * NP + g);
        sP[R4 + i] = __ldg(src + PL_PY * NP + g);
    }
    for (int i = tid; i < R3; i += NT) {
        const int ly = i / R3W, lx = i - ly * R3W;
        const long long g = (long long)sYi[ly + 1] * nx + sXi[lx + 1];
        sS[i] = __ldg(src + PL_SXX * NP + g);
        sS[R3 + i] = __ldg(src + PL_SYY * NP + g);
        sS[2 * R3 + i] = __ldg(src + PL_SXY * NP + g);
    }
    __syncthreads();

    // ---- B: molecular field and Ericksen stress on the halo-3 region ------------------------
    for (int i = tid; i < R3; i += NT) {
        const int ly = i / R3W, lx = i - ly * R3W;
        const St px = st_at(sP, R4W, lx + 1, ly + 1);         // dP stencils
        const St py = st_at(sP + R4, R4W, lx + 1, ly + 1);
        float hx, hy;
        molecular(ph, px, py, hx, hy);
        sH[i] = hx;
        sH[R3 + i] = hy;
        if (ph.ericksen) {
            const float Px = ph.prx + px.c, Py = ph.pry + py.c;
            const float gxPx = 0.5f * (px.e - px.w), gyPx = 0.5f * (px.n - px.s);
            const float gxPy = 0.5f * (py.e - py.w), gyPy = 0.5f * (py.n - py.s);
            const float anti = Px * hy - hx * Py;
            const float sym = Px * hy + hx * Py;
            const float cross = ph.kappa * (gxPx * gyPx + gxPy * gyPy);
            sE[i] = ph.xi * Px * hx - ph.kappa * (gxPx * gxPx + gxPy * gxPy);            // xx
            sE[R3 + i] = -0.5f * anti + 0.5f * ph.xi * sym - cross;                       // xy
            sE[2 * R3 + i] = 0.5f * anti + 0.5f * ph.xi * sym - cross;                    // yx
            sE[3 * R3 + i] = ph.xi * Py * hy - ph.kappa * (gyPx * gyPx + gyPy * gyPy);    // yy
        }
    }

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
        float Fx = 0.5f * (sS[j3 + 1] - sS[j3 - 1]) + 0.5f * (sS[2 * R3 + j3 + R3W] - sS[2 * R3 + j3 - R3W]);
        float Fy = 0.5f * (sS[2 * R3 + j3 + 1] - sS[2 * R3 + j3 - 1]) + 0.5f * (sS[R3 + j3 + R3W] - sS[R3 + j3 - R3W]);
        if (ph.ericksen) {
            Fx += 0.5f * (sE[j3 + 1] - sE[j3 - 1]) + 0.5f * (sE[R3 + j3 + R3W] - sE[R3 + j3 - R3W]);
            Fy += 0.5f * (sE[2 * R3 + j3 + 1] - sE[2 * R3 + j3 - 1]) +
                  0.5f * (sE[3 * R3 + j3 + R3W] - sE[3 * R3 + j3 - R3W]);
        }
        Fx += sFib[i];
        Fy += sFib[R2 + i];
        const long long g = (long long)sYi[ly + 2] * nx + sXi[lx + 2];
        float d[9];
#pragma unroll
        for (int n = 0; n < 9; ++n) d[n] = __ldg(src + n * NP + g);
        const float drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        const float jy = (d[2] - d[4]) + (d[5] - d[8]) + (d[6] - d[7]);
        const float inv = 1.f / (ph.rho0 + drho);
        sM[i] = drho;
        sM[R2 + i] = (jx + 0.5f * Fx) * inv;
        sM[2 * R2 + i] = (jy + 0.5f * Fy) * inv;
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
    float* __restrict__ dst = a.dst;
    // D2Q9 (Sec. II A): c_n and w_n, n = 0..8
    const int c_cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int c_cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const float w9[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                         1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
    for (int i = tid; i < R0; i += NT) {
        const int ly = i / TX, lx = i - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const long long g = (long long)gy * nx + gx;
        const int j2 = (ly + 2) * R2W + lx + 2;
        const float drho = sM[j2], ux = sM[R2 + j2], uy = sM[2 * R2 + j2];
        const float Fx = sM[3 * R2 + j2], Fy = sM[4 * R2 + j2];

        // collision: d*_n = d_n + omega (d^eq_n - d_n) + guo * S_n, pushed to x + c_n.
        // The change D_n = d*_n - d_n of one cell carries no mass and the momentum F in exact
        // arithmetic; in FP32 the rounding of u (coherent over a uniform flow) would leak
        // momentum into every cell alike, so the FP32 changes are corrected to exactly
        // sum D_n = 0 and sum c_n D_n = F (pair and rest-population corrections).
        {
            const float rho = ph.rho0 + drho;
            const float uu = 1.5f * (ux * ux + uy * uy);
            const float uF = ux * Fx + uy * Fy;
            float dn[9], D[9];
#pragma unroll
            for (int n = 0; n < 9; ++n) {
                dn[n] = __ldg(src + n * NP + g);
                const float cu = (float)c_cx[n] * ux + (float)c_cy[n] * uy;
                const float cF = (float)c_cx[n] * Fx + (float)c_cy[n] * Fy;
                const float deq = w9[n] * (drho + rho * (3.f * cu + 4.5f * cu * cu - uu));
                const float S = w9[n] * (3.f * (cF - uF) + 9.f * cu * cF);
                D[n] = ph.omega * (deq - dn[n]) + ph.guo * S;
            }
            const float ex = ((D[1] - D[3]) + (D[5] - D[6]) + (D[8] - D[7])) - Fx;
            const float ey = ((D[2] - D[4]) + (D[5] - D[8]) + (D[6] - D[7])) - Fy;
            D[1] -= 0.5f * ex;
            D[3] += 0.5f * ex;
            D[2] -= 0.5f * ey;
            D[4] += 0.5f * ey;
            D[0] -= ((D[1] + D[2]) + (D[3] + D[4])) + ((D[5] + D[6]) + (D[7] + D[8])) + D[0];
#pragma unroll
            for (int n = 0; n < 9; ++n) {
                const long long gd = (long long)sYi[ly + 4 + c_cy[n]] * nx + sXi[lx + 4 + c_cx[n]];
                dst[n * NP + gd] = dn[n] + D[n];
            }
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
#pragma unroll
            for (int c = 0; c < 5; ++c)
                dst[(PL_SXX + c) * NP + g] = y0s[c] + 0.5f * (sR[c * R0 + i] + r[c]);
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
            a.partials[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * 5 + tid] = v;
        }
    }
}

}  // namespace

int fused_ctas(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

cudaError_t launch_fused(const FusedArgs& a, int mode, cudaStream_t s, int* grid_ctas)
{
    static bool attr_done[2] = {false, false};
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
    if (grid_ctas) *grid_ctas = grid.x * grid.y;
    if (mode == MODE_STEP) {
        if (!attr_done[0]) {
            cudaError_t e = cudaFuncSetAttribute(k_fused<MODE_STEP>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
            if (e != cudaSuccess) return e;
            attr_done[0] = true;
        }
        k_fused<MODE_STEP><<<grid, NT, SMEM_BYTES, s>>>(a);
    } else {
        if (!attr_done[1]) {
            cudaError_t e = cudaFuncSetAttribute(k_fused<MODE_MOMENTS>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
            if (e != cudaSuccess) return e;
            attr_done[1] = true;
        }
        k_fused<MODE_MOMENTS><<<grid, NT, SMEM_BYTES, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace vlb
