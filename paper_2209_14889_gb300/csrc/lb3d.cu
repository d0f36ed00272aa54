// lb3d.cu -- the three-dimensional form of the step (include/lb3d.h): D3Q19 lattice Boltzmann
// with the Guo force, the polymer stress of Eq. StiffCons with the stiffness averaged over the
// unit sphere, and the Beris-Edwards field P, as four HBM-streaming stencil kernels per step.
//
// Kernels of one step (one thread per cell, CTAs of 32 x 4 x 2 cells, x fastest so that a warp
// reads 128 contiguous bytes of a plane; neighbour values come through L1/L2):
//   k3_molecular  sigma^E (Sec. II C 1) of the state, from h = (alpha + beta |P|^2) P - kappa lap P
//                 (launched with the Ericksen force only)
//   k3_collide    F = div sigma^p + div sigma^E + f_ext, moments with the Guo half force, BGK
//                 collision with the Guo source pushed to the neighbours (Eq. LB, Eq. BGK); u;
//                 on readout steps the FP64 sums (mass, momentum, force) in a fixed order
//   k3_predict    RHS(y) of Eq. StiffCons and Eq. BE at y = (sigma^p, P) (h from the P stencils it
//                 loads), u(t) frozen; y* = y + RHS
//   k3_correct    RHS(y*) (h* from P*), y' = y + (RHS(y) + RHS(y*)) / 2 into the next state
// The stiffness C(P) = int g(n) K(n) dOmega is applied in its transversely isotropic form about
// P^: with the orientation moments m2 = <mu^2>, m4 = <mu^4> of the Fisher density (their
// combinations below tabulated against |P| in FP64 and stored as FP32),
// M2 = <nn> = A d + B pp and M4 = <nnnn> = e1 pppp + e2 Sym(pp d) + e3 Sym(d d), and
// K(n) = a1 nnnn + a2 (nn d + d nn) + a3 d d + a4 Sym'(nn d) + a5 (d d + d d), the contraction
// C:X of a symmetric X is
//   c_pp pp + c_d d + c_s (p (Xp) + (Xp) p) + c_X X
// with c_pp = a1 e1 pXp + (a1 e2 + a2 B) trX, c_d = (a1 e2 + a2 B) pXp + (a1 e3 + 2 a2 A + a3) trX,
// c_s = 2 (a1 e2 + a4 B), c_X = 2 (a1 e3 + 2 a4 A + a5).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lb3d.h"

namespace v3 {

constexpr int NQ = 19;
constexpr int NPL = 28;                 // 19 populations, 6 sigma, 3 P
constexpr int PL_S = 19, PL_P = 25;
constexpr int LUT_N = 8192;             // table intervals in |P| up to P_cap (linear interpolation:
                                        // coefficient error below 1e-7 of their scale)
constexpr int BX = 32, BY = 4, BZ = 2, NT = BX * BY * BZ;

// D3Q19 (the order of include/lb3d.h)
__device__ constexpr int CX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int CY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int CZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

__device__ __forceinline__ float wq(int n) { return n == 0 ? 1.f / 3.f : (n < 7 ? 1.f / 18.f : 1.f / 36.f); }

struct Args3 {
    const float* src;            // state at t (NPL planes)
    float* dst;                  // state at t + 1
    float* sE;                   // Ericksen stress [9] (i * 3 + j)
    float* u;                    // u(t) [3]
    float* ys;                   // predictor y* [9]
    float* r0;                   // RHS(y) [9]
    float* mom;                  // moments pass: drho, ux, uy, uz [4]
    const float4* lut;           // coefficients of C:X against |P| (two float4 per entry)
    long long NP;
    int nx, ny, nz;
    float tau_inv, guo, rho0;
    float inv_eta, Dp, alpha, beta, xi, Gamma, kappa, P_cap, lut_scale;
    float fx, fy, fz;
    float prx, pry, prz, A0;     // P_ref and alpha + beta |P_ref|^2 (formed in FP64)
    int ericksen;
    int readout;                 // k3_collide: sum the readouts of this step
    long long t;
    double* partials;            // [CTAs][7]
    double* gpartials;           // [groups of NT CTAs][7]
    double* row;                 // readout row of this step (8 values)
    int* err_nonfinite;
};

struct Cell {
    int x, y, z, c;
    int xp, xm, yp, ym, zp, zm;  // flat indices of the six face neighbours
};

__device__ __forceinline__ bool cell_of(const Args3& a, Cell& q)
{
    q.x = blockIdx.x * BX + threadIdx.x;
    q.y = blockIdx.y * BY + threadIdx.y;
    q.z = blockIdx.z * BZ + threadIdx.z;
    if (q.x >= a.nx || q.y >= a.ny || q.z >= a.nz) return false;
    const int nx = a.nx, nxy = a.nx * a.ny;
    q.c = q.z * nxy + q.y * nx + q.x;
    // neighbour offsets compose: the +x neighbour of the +y neighbour is c + (xp - c) + (yp - c)
    q.xp = q.c + (q.x + 1 == nx ? 1 - nx : 1);
    q.xm = q.c + (q.x == 0 ? nx - 1 : -1);
    q.yp = q.c + (q.y + 1 == a.ny ? nx - nxy : nx);
    q.ym = q.c + (q.y == 0 ? nxy - nx : -nx);
    q.zp = q.c + (q.z + 1 == a.nz ? nxy - nxy * a.nz : nxy);
    q.zm = q.c + (q.z == 0 ? nxy * a.nz - nxy : -nxy);
    return true;
}

// value of plane f at the cell and its six neighbours: v[0] centre, then +x -x +y -y +z -z
__device__ __forceinline__ void stencil(const float* f, const Cell& q, float* v)
{
    v[0] = __ldg(f + q.c);
    v[1] = __ldg(f + q.xp); v[2] = __ldg(f + q.xm);
    v[3] = __ldg(f + q.yp); v[4] = __ldg(f + q.ym);
    v[5] = __ldg(f + q.zp); v[6] = __ldg(f + q.zm);
}

__device__ __forceinline__ float lap7(const float* v) { return v[1] + v[2] + v[3] + v[4] + v[5] + v[6] - 6.f * v[0]; }
__device__ __forceinline__ float dif(const float* v, int a) { return 0.5f * (v[1 + 2 * a] - v[2 + 2 * a]); }

// alpha + beta |P|^2 at P = P_ref + dP without the cancellation near the equilibrium modulus
__device__ __forceinline__ float bulk(const Args3& a, float dx, float dy, float dz)
{
    const float pd = a.prx * dx + a.pry * dy + a.prz * dz;
    const float dd = dx * dx + dy * dy + dz * dz;
    return a.A0 + a.beta * (2.f * pd + dd);
}

// symmetric-tensor component (xx, yy, zz, yz, xz, xy) of (i, j)
__device__ __forceinline__ int sym6(int i, int j)
{
    return i == j ? i : (i + j == 3 ? 3 : (i + j == 2 ? 4 : 5));
}

// ---- stiffness: the transversely isotropic contraction C(P):X --------------------------------
struct Stiff {
    float n[3];
    float cpp_n, g;              // c_pp = cpp_n pXp + g trX
    float cd_t;                  // c_d  = g pXp + cd_t trX
    float cs, cX;
};

// The table holds, per |P|, the five scalar coefficients of C:X (formed on the host in FP64 from
// the orientation moments and K^x, so the cancellations in e1, e2, e3 never happen in FP32):
// (cpp_n, g, cd_t, cs) and (cX, -, -, -).
__device__ __forceinline__ Stiff stiffness(const Args3& a, float px, float py, float pz)
{
    Stiff S;
    const float P2 = px * px + py * py + pz * pz;
    const float Pm = sqrtf(P2);
    if (Pm > 0.f) {
        const float r = 1.f / Pm;
        S.n[0] = px * r; S.n[1] = py * r; S.n[2] = pz * r;
    } else {
        S.n[0] = 1.f; S.n[1] = 0.f; S.n[2] = 0.f;
    }
    const float q = fminf(Pm, a.P_cap) * a.lut_scale;
    int i = (int)q;
    if (i > LUT_N - 1) i = LUT_N - 1;
    const float f = q - (float)i;
    const float4 u0 = __ldg(a.lut + 2 * i), u1 = __ldg(a.lut + 2 * i + 2);
    const float v0 = __ldg(&a.lut[2 * i + 1].x), v1 = __ldg(&a.lut[2 * i + 3].x);
    S.cpp_n = u0.x + f * (u1.x - u0.x);
    S.g = u0.y + f * (u1.y - u0.y);
    S.cd_t = u0.z + f * (u1.z - u0.z);
    S.cs = u0.w + f * (u1.w - u0.w);
    S.cX = v0 + f * (v1 - v0);
    return S;
}

// out = C:X for the symmetric X (6 components)
__device__ __forceinline__ void apply_c(const Stiff& S, const float* X, float* out)
{
    const float* n = S.n;
    const float Xn0 = X[0] * n[0] + X[5] * n[1] + X[4] * n[2];
    const float Xn1 = X[5] * n[0] + X[1] * n[1] + X[3] * n[2];
    const float Xn2 = X[4] * n[0] + X[3] * n[1] + X[2] * n[2];
    const float nXn = n[0] * Xn0 + n[1] * Xn1 + n[2] * Xn2;
    const float tr = X[0] + X[1] + X[2];
    const float cpp = S.cpp_n * nXn + S.g * tr;
    const float cd = S.g * nXn + S.cd_t * tr;
    const float Xn[3] = {Xn0, Xn1, Xn2};
    const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int i = I[c], j = J[c];
        out[c] = cpp * n[i] * n[j] + (i == j ? cd : 0.f) + S.cs * (n[i] * Xn[j] + Xn[i] * n[j]) + S.cX * X[c];
    }
}

// ---- right-hand sides of Eq. StiffCons (Jaumann derivative) and Eq. BE -----------------------
// y = (sigma (6), dP = P - P_ref (3)) at the cell, reduced from each component's stencil as it is
// loaded: the value, the advection u.grad (central differences) and the 7-point Laplacian
struct Y9 {
    float c[9], adv[9], lap[9];
};

__device__ __forceinline__ void load_y9(const float* base, long long NP, const Cell& q, const float* uc, Y9& y)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float v[7];
        stencil(base + k * NP, q, v);
        y.c[k] = v[0];
        y.adv[k] = uc[0] * dif(v, 0) + uc[1] * dif(v, 1) + uc[2] * dif(v, 2);
        y.lap[k] = lap7(v);
    }
}

// uc: u at the cell; G[i][j] = d_i u_j; h: molecular field at the cell
__device__ __forceinline__ void rhs9(const Args3& a, const Y9& y, const float (*G)[3], const float* h, float* r)
{
    float Psi[3][3], Om[3][3], s[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Psi[i][j] = 0.5f * (G[i][j] + G[j][i]);
            Om[i][j] = 0.5f * (G[i][j] - G[j][i]);
            s[i][j] = y.c[sym6(i, j)];
        }
    const float P[3] = {a.prx + y.c[6], a.pry + y.c[7], a.prz + y.c[8]};
    const Stiff S = stiffness(a, P[0], P[1], P[2]);
    // C Psi - C sigma / eta_p = C (Psi - sigma / eta_p): one contraction (C is linear in X)
    const float psi6[6] = {Psi[0][0], Psi[1][1], Psi[2][2], Psi[1][2], Psi[0][2], Psi[0][1]};
    float X6[6], CX6[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) X6[c] = psi6[c] - a.inv_eta * y.c[c];
    apply_c(S, X6, CX6);
    const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int i = I[c], j = J[c];
        float Jc = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) Jc += Om[i][k] * s[k][j] - s[i][k] * Om[k][j];
        r[c] = -y.adv[c] - Jc + CX6[c] + a.Dp * y.lap[c];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float rot = 0.f, str = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            rot += Om[i][k] * P[k];
            str += Psi[i][k] * P[k];
        }
        r[6 + i] = -y.adv[6 + i] - rot + a.xi * str - a.Gamma * h[i];
    }
}

// u at the cell and its gradient G[i][j] = d_i u_j (central differences)
__device__ __forceinline__ void flow(const Args3& a, const Cell& q, float* uc, float (*G)[3])
{
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float v[7];
        stencil(a.u + j * a.NP, q, v);
        uc[j] = v[0];
#pragma unroll
        for (int i = 0; i < 3; ++i) G[i][j] = dif(v, i);
    }
}

// ---- kernels ---------------------------------------------------------------------------------

__global__ void __launch_bounds__(NT) k3_molecular(const Args3 a, const float* dP)
{
    Cell q;
    if (!cell_of(a, q)) return;
    float v[3][7];                  // stencils of dP = P - P_ref
#pragma unroll
    for (int i = 0; i < 3; ++i) stencil(dP + i * a.NP, q, v[i]);
    const float A = bulk(a, v[0][0], v[1][0], v[2][0]);
    const float P[3] = {a.prx + v[0][0], a.pry + v[1][0], a.prz + v[2][0]};
    float h[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) h[i] = A * P[i] - a.kappa * lap7(v[i]);
    float gP[3][3];                 // gP[i][k] = d_i P_k
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) gP[i][k] = dif(v[k], i);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float Pi = P[i], Pj = P[j];
            const float gg = gP[i][0] * gP[j][0] + gP[i][1] * gP[j][1] + gP[i][2] * gP[j][2];
            a.sE[(i * 3 + j) * a.NP + q.c] = -0.5f * (Pi * h[j] - h[i] * Pj) + 0.5f * a.xi * (Pi * h[j] + h[i] * Pj)
                                             - a.kappa * gg;
        }
}

// Fixed-order sums of the readout values v[7] of a CTA into out[7]: FP32 within each warp (a
// warp's cells are 32 consecutive FP32 values), FP64 across the warps, one thread per value (FP64
// is a narrow unit on this GPU: seven short chains, not one long one).
__device__ __forceinline__ void cta_sum7(const float* v, double* out, float* sm)
{
    const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[wid * 7 + k] = x;
    }
    __syncthreads();
    if (tid < 7) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += (double)sm[w * 7 + tid];
        out[tid] = s;
    }
}

// fixed-order FP64 block sum of v[7] (thread 0 returns the totals)
__device__ __forceinline__ void block_sum7(double* v, double* sm)
{
    const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[wid * 7 + k] = x;
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < 7; ++k) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += sm[w * 7 + k];
            v[k] = s;
        }
    }
}

// mode 0: the step's collision and streaming; mode 1: moments of the current state only
__global__ void __launch_bounds__(NT, 4) k3_collide(const Args3 a, int mode)
{
    __shared__ float sRedF[(NT / 32) * 7];
    Cell q;
    const bool in = cell_of(a, q);
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (in) {
        // F_i = d_j sigma^p_ij + d_j sigma^E_ij + f_ext,i
        float F[3] = {a.fx, a.fy, a.fz};
        const int nb[3][2] = {{q.xp, q.xm}, {q.yp, q.ym}, {q.zp, q.zm}};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float* sp = a.src + (long long)(PL_S + sym6(i, j)) * a.NP;
                F[i] += 0.5f * (__ldg(sp + nb[j][0]) - __ldg(sp + nb[j][1]));
                if (a.ericksen) {
                    const float* se = a.sE + (long long)(i * 3 + j) * a.NP;
                    F[i] += 0.5f * (__ldg(se + nb[j][0]) - __ldg(se + nb[j][1]));
                }
            }
        float d[NQ];
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int n = 0; n < NQ; ++n) {
            d[n] = __ldg(a.src + (long long)n * a.NP + q.c);
            drho += d[n];
            jx += (float)CX[n] * d[n];
            jy += (float)CY[n] * d[n];
            jz += (float)CZ[n] * d[n];
        }
        const float rho = a.rho0 + drho;
        const float ir = 1.f / rho;
        const float ux = (jx + 0.5f * F[0]) * ir, uy = (jy + 0.5f * F[1]) * ir, uz = (jz + 0.5f * F[2]) * ir;
        if (mode == 1) {
            a.mom[q.c] = drho;
            a.mom[a.NP + q.c] = ux;
            a.mom[2 * a.NP + q.c] = uy;
            a.mom[3 * a.NP + q.c] = uz;
            return;
        }
        a.u[q.c] = ux;
        a.u[a.NP + q.c] = uy;
        a.u[2 * a.NP + q.c] = uz;
        // BGK with the Guo source: d* = d - (d - d_eq)/tau + (1 - 1/(2 tau)) w [3 (c - u) + 9 (c.u) c].F,
        // d_eq = w (drho + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)); pushed to x + c_n (periodic: the
        // neighbour offsets of the cell, combined per direction)
        const float rq = 1.5f * rho * (ux * ux + uy * uy + uz * uz);
        const float uF3 = 3.f * (ux * F[0] + uy * F[1] + uz * F[2]);
        const int ox[2] = {q.xp - q.c, q.xm - q.c}, oy[2] = {q.yp - q.c, q.ym - q.c}, oz[2] = {q.zp - q.c, q.zm - q.c};
        const float keep = 1.f - a.tau_inv;
        auto push = [&](int n, float out) {
            int dstc = q.c;
            if (CX[n]) dstc += ox[CX[n] > 0 ? 0 : 1];
            if (CY[n]) dstc += oy[CY[n] > 0 ? 0 : 1];
            if (CZ[n]) dstc += oz[CZ[n] > 0 ? 0 : 1];
            a.dst[(long long)n * a.NP + dstc] = out;
        };
        // rest population, then each direction n with its opposite n + 1 (the order of
        // include/lb3d.h pairs them) from the even and odd parts in c of d_eq and of the source
        const float base = drho - rq;
        push(0, keep * d[0] + a.tau_inv * (wq(0) * base) + (a.guo * wq(0)) * (-uF3));
#pragma unroll
        for (int n = 1; n < NQ; n += 2) {
            float cu = 0.f, cF = 0.f;
            if (CX[n]) { cu += CX[n] > 0 ? ux : -ux; cF += CX[n] > 0 ? F[0] : -F[0]; }
            if (CY[n]) { cu += CY[n] > 0 ? uy : -uy; cF += CY[n] > 0 ? F[1] : -F[1]; }
            if (CZ[n]) { cu += CZ[n] > 0 ? uz : -uz; cF += CZ[n] > 0 ? F[2] : -F[2]; }
            const float w = wq(n), gw = a.guo * w;
            const float ev = a.tau_inv * (w * (base + 4.5f * rho * cu * cu));     // even part of d_eq / tau
            const float od = a.tau_inv * (w * (3.f * rho * cu));                   // odd part
            const float Sev = gw * (9.f * cu * cF - uF3), Sod = gw * (3.f * cF);
            push(n, keep * d[n] + (ev + od) + (Sev + Sod));
            push(n + 1, keep * d[n + 1] + (ev - od) + (Sev - Sod));
        }
        if (a.readout) {
            acc[0] = drho;
            acc[1] = jx; acc[2] = jy; acc[3] = jz;
            acc[4] = F[0]; acc[5] = F[1]; acc[6] = F[2];
        }
    }
    if (mode == 1 || !a.readout) return;
    // readout: the CTA's sums; the groups of NT CTAs are added by the next kernel and the groups by
    // the one after (kernel boundaries order the writes: no fence or atomic in this kernel)
    const unsigned cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    cta_sum7(acc, a.partials + (long long)cta * 7, sRedF);
}

// Readout, second level (in k3_predict): CTA g < groups adds the sums of CTAs g NT .. g NT + NT - 1
// of k3_collide in a fixed tree.
__device__ __forceinline__ void readout_groups(const Args3& a, double* sm)
{
    const unsigned n_ctas = gridDim.x * gridDim.y * gridDim.z;
    const unsigned cta = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned n_grp = (n_ctas + NT - 1) / NT;
    if (!a.readout || cta >= n_grp) return;
    const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
    const unsigned g0 = cta * NT;
    double s[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (g0 + tid < n_ctas) {
#pragma unroll
        for (int k = 0; k < 7; ++k) s[k] = a.partials[(long long)(g0 + tid) * 7 + k];
    }
    block_sum7(s, sm);
    if (tid == 0)
        for (int k = 0; k < 7; ++k) a.gpartials[(long long)cta * 7 + k] = s[k];
}

// Readout, last level (in k3_correct, CTA 0): the group sums, each thread a fixed contiguous range,
// then the fixed tree; the row (t, mass, momentum, force) of the step.
__device__ __forceinline__ void readout_total(const Args3& a, double* sm)
{
    if (!a.readout || blockIdx.x + blockIdx.y + blockIdx.z != 0) return;
    const unsigned n_ctas = gridDim.x * gridDim.y * gridDim.z;
    const unsigned n_grp = (n_ctas + NT - 1) / NT;
    const int tid = threadIdx.x + BX * (threadIdx.y + BY * threadIdx.z);
    const unsigned per = (n_grp + NT - 1) / NT;
    const unsigned b0 = min(n_grp, tid * per), b1 = min(n_grp, b0 + per);
    double s[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (unsigned b = b0; b < b1; ++b) {
#pragma unroll
        for (int k = 0; k < 7; ++k) s[k] += a.gpartials[(long long)b * 7 + k];
    }
    block_sum7(s, sm);
    if (tid == 0) {
        a.row[0] = (double)a.t;
        for (int k = 0; k < 7; ++k) {
            a.row[1 + k] = s[k];
            if (!isfinite(s[k])) atomicExch(a.err_nonfinite, 1);
        }
    }
}

__global__ void __launch_bounds__(NT) k3_predict(const Args3 a)
{
    __shared__ double sRed[(NT / 32) * 7];
    readout_groups(a, sRed);
    Cell q;
    if (!cell_of(a, q)) return;
    float uc[3], G[3][3];
    flow(a, q, uc, G);
    Y9 y;
    load_y9(a.src + (long long)PL_S * a.NP, a.NP, q, uc, y);
    // h(P): Eq. Ffunctional from the folded dP stencils
    const float A = bulk(a, y.c[6], y.c[7], y.c[8]);
    const float Pr[3] = {a.prx, a.pry, a.prz};
    float h[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) h[i] = A * (Pr[i] + y.c[6 + i]) - a.kappa * y.lap[6 + i];
    float r[9];
    rhs9(a, y, G, h, r);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        a.r0[k * a.NP + q.c] = r[k];
        a.ys[k * a.NP + q.c] = y.c[k] + r[k];
    }
}

__global__ void __launch_bounds__(NT) k3_correct(const Args3 a)
{
    __shared__ double sRed[(NT / 32) * 7];
    readout_total(a, sRed);
    Cell q;
    if (!cell_of(a, q)) return;
    float uc[3], G[3][3];
    flow(a, q, uc, G);
    Y9 y;
    load_y9(a.ys, a.NP, q, uc, y);
    // h(P*): Eq. Ffunctional at the predictor
    const float A = bulk(a, y.c[6], y.c[7], y.c[8]);
    const float Pr[3] = {a.prx, a.pry, a.prz};
    float h[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) h[i] = A * (Pr[i] + y.c[6 + i]) - a.kappa * y.lap[6 + i];
    float r[9];
    rhs9(a, y, G, h, r);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float y0 = __ldg(a.src + (long long)(PL_S + k) * a.NP + q.c);
        const float r0 = __ldg(a.r0 + k * a.NP + q.c);
        a.dst[(long long)(PL_S + k) * a.NP + q.c] = y0 + 0.5f * (r0 + r[k]);
    }
}

// out = plane + c (the readout of P = P_ref + dP)
__global__ void k3_add(const float* plane, float c, float* out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = plane[i] + c;
}

// ---- host: the orientation-moment table (FP64) ------------------------------------------------

double langevin(double k)
{
    if (k < 0.05) {
        const double k2 = k * k;
        return k * (1.0 / 3.0 - k2 * (1.0 / 45.0 - k2 * (2.0 / 945.0 - k2 / 4725.0)));
    }
    return 1.0 / std::tanh(k) - 1.0 / k;
}

// concentration of the Fisher density with mean projection P (bisection on the increasing L)
double concentration(double P)
{
    if (P <= 0.0) return 0.0;
    double lo = 0.0, hi = 1.0;
    while (langevin(hi) < P) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (langevin(mid) < P) lo = mid;
        else hi = mid;
        if (hi - lo <= 1e-15 * hi) break;
    }
    return 0.5 * (lo + hi);
}

// <mu^2>, <mu^4> of exp(k mu) on [-1, 1]: the power series of both integrals below k = 4, the
// integration-by-parts recursion m_n = [1 or coth k] - (n / k) m_{n-1} above
void fisher_moments(double k, double& m2, double& m4)
{
    if (k < 4.0) {
        double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        double t = 1.0;                  // k^j / j!
        for (int j = 0; j < 80; ++j) {
            for (int n = 0; n <= 4; n += 2)
                if ((n + j) % 2 == 0) s[n] += t * 2.0 / (n + j + 1);
            t *= k / (j + 1);
        }
        m2 = s[2] / s[0];
        m4 = s[4] / s[0];
        return;
    }
    const double c = 1.0 / std::tanh(k);
    const double m1 = c - 1.0 / k;
    m2 = 1.0 - 2.0 / k * m1;
    const double m3 = c - 3.0 / k * m2;
    m4 = 1.0 - 4.0 / k * m3;
}

void moment_table(double P_cap, std::vector<float>& out)
{
    out.resize(2 * (LUT_N + 1));
    for (int i = 0; i <= LUT_N; ++i) {
        const double P = P_cap * i / LUT_N;
        double m2, m4;
        fisher_moments(concentration(P), m2, m4);
        out[2 * i] = (float)m2;
        out[2 * i + 1] = (float)m4;
    }
}

// The coefficients of C:X per table entry (8 floats: cpp_n, g, cd_t, cs, cX, 0, 0, 0), in FP64:
// K(n) in the transversely isotropic basis about n (K2323 = (K2222 - K2233) / 2), the moment
// tensors M2 = A d + B pp, M4 = e1 pppp + e2 Sym(pp d) + e3 Sym(d d) of the Fisher density.
void coefficient_table(const lb3d_params& p, std::vector<float>& out)
{
    const double a5 = 0.5 * (p.K2222 - p.K2233), a3 = p.K2233, a4 = p.K1212 - a5, a2 = p.K1122 - a3;
    const double a1 = p.K1111 - 2.0 * a2 - a3 - 4.0 * a4 - 2.0 * a5;
    out.assign(8 * (LUT_N + 1), 0.f);
    for (int i = 0; i <= LUT_N; ++i) {
        double m2, m4;
        fisher_moments(concentration(p.P_cap * i / LUT_N), m2, m4);
        const double A = 0.5 * (1.0 - m2), B = 0.5 * (3.0 * m2 - 1.0);
        const double e3 = (A - B + m4) / 8.0, e2 = A - 5.0 * e3, e1 = B - 7.0 * e2;
        float* o = out.data() + 8 * i;
        o[0] = (float)(a1 * e1);
        o[1] = (float)(a1 * e2 + a2 * B);
        o[2] = (float)(a1 * e3 + 2.0 * a2 * A + a3);
        o[3] = (float)(2.0 * (a1 * e2 + a4 * B));
        o[4] = (float)(2.0 * (a1 * e3 + 2.0 * a4 * A + a5));
    }
}

}  // namespace v3

// ---- host: the handle --------------------------------------------------------------------------

struct lb3d_handle {
    lb3d_params p;
    cudaStream_t stream = nullptr;
    long long NP = 0;
    float* state[2] = {nullptr, nullptr};
    int cur = 0;
    float* sE = nullptr;
    float* u = nullptr;
    float* ys = nullptr;
    float* r0 = nullptr;
    float* mom = nullptr;
    float4* lut = nullptr;
    double* partials = nullptr;
    double* gpartials = nullptr;
    double* series = nullptr;
    int* err = nullptr;
    long long t = 0;
    long long rows = 0;           // readout rows written since lb3d_init_fields
    bool ready = false;
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::string msg;
};

namespace {

int fail(lb3d_handle* h, int code, const char* fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->msg = buf;
    }
    return code;
}

#define CK3(h, call)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(h, e_ == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, "%s: %s", #call,     \
                        cudaGetErrorString(e_));                                                       \
    } while (0)

template <class T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

dim3 grid_of(const lb3d_handle* h)
{
    return dim3((unsigned)((h->p.nx + v3::BX - 1) / v3::BX), (unsigned)((h->p.ny + v3::BY - 1) / v3::BY),
                (unsigned)((h->p.nz + v3::BZ - 1) / v3::BZ));
}

v3::Args3 args_of(lb3d_handle* h)
{
    const lb3d_params& p = h->p;
    v3::Args3 a = {};
    a.src = h->state[h->cur];
    a.dst = h->state[h->cur ^ 1];
    a.sE = h->sE; a.u = h->u; a.ys = h->ys; a.r0 = h->r0; a.mom = h->mom;
    a.lut = h->lut;
    a.NP = h->NP;
    a.nx = p.nx; a.ny = p.ny; a.nz = p.nz;
    a.tau_inv = (float)(1.0 / p.tau);
    a.guo = (float)(1.0 - 0.5 / p.tau);
    a.rho0 = (float)p.rho0;
    a.inv_eta = (float)(1.0 / p.eta_p);
    a.Dp = (float)p.Dp;
    a.alpha = (float)p.alpha; a.beta = (float)p.beta; a.xi = (float)p.xi;
    a.Gamma = (float)p.Gamma; a.kappa = (float)p.kappa;
    a.P_cap = (float)p.P_cap;
    a.lut_scale = (float)(v3::LUT_N / p.P_cap);
    a.fx = (float)p.fext[0]; a.fy = (float)p.fext[1]; a.fz = (float)p.fext[2];
    a.prx = (float)p.P_ref[0]; a.pry = (float)p.P_ref[1]; a.prz = (float)p.P_ref[2];
    a.A0 = (float)(p.alpha + p.beta * (p.P_ref[0] * p.P_ref[0] + p.P_ref[1] * p.P_ref[1] + p.P_ref[2] * p.P_ref[2]));
    a.ericksen = p.ericksen;
    a.partials = h->partials;
    a.gpartials = h->gpartials;
    a.err_nonfinite = h->err;
    a.t = h->t;
    return a;
}

int launch_check(lb3d_handle* h, const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, LB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return LB_OK;
}

// h and sigma^E of the current state, then the moments pass or the step's collision
int launch_front(lb3d_handle* h, v3::Args3& a, int mode)
{
    const dim3 g = grid_of(h), b(v3::BX, v3::BY, v3::BZ);
    if (h->p.ericksen) {
        v3::k3_molecular<<<g, b, 0, h->stream>>>(a, a.src + (long long)v3::PL_P * h->NP);
        int rc = launch_check(h, "k3_molecular");
        if (rc) return rc;
    }
    v3::k3_collide<<<g, b, 0, h->stream>>>(a, mode);
    return launch_check(h, "k3_collide");
}

}  // namespace

extern "C" {

int lb3d_create(const lb3d_params* p, lb3d_handle** out)
{
    if (!p || !out) return LB_EINVAL;
    *out = nullptr;
    if (p->nx < 3 || p->ny < 3 || p->nz < 3 || (long long)p->nx * p->ny * p->nz >= (1LL << 31) ||
        p->readout_every < 1 || p->max_samples < 1 || !(p->tau > 0.5) || !(p->eta_p > 0.0) ||
        !(p->P_cap > 0.0 && p->P_cap < 1.0) || !(p->rho0 > 0.0) || p->Dp < 0.0 || p->Gamma < 0.0 ||
        p->kappa < 0.0)
        return LB_EINVAL;
    // Heun on the 7-point Laplacian (eigenvalues down to -12) and on the relaxation of P: the
    // explicit bounds 12 D_p <= 2, 12 Gamma kappa <= 2, 2 Gamma |alpha| <= 2
    if (12.0 * p->Dp > 2.0 || 12.0 * p->Gamma * p->kappa > 2.0 || p->Gamma * std::fabs(p->alpha) > 1.0)
        return LB_EUNSTABLE;
    lb3d_handle* h = new lb3d_handle();
    h->p = *p;
    h->NP = (long long)p->nx * p->ny * p->nz;
    auto bail = [&](int code) {
        lb3d_destroy(h);
        return code;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    const size_t pb = sizeof(float) * (size_t)h->NP;
    const dim3 g = grid_of(h);
    const size_t n_ctas = (size_t)g.x * g.y * g.z;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&h->state[b], v3::NPL * pb);
    if (e == cudaSuccess && p->ericksen) e = cudaMalloc(&h->sE, 9 * pb);
    if (e == cudaSuccess) e = cudaMalloc(&h->u, 3 * pb);
    if (e == cudaSuccess) e = cudaMalloc(&h->ys, 9 * pb);
    if (e == cudaSuccess) e = cudaMalloc(&h->r0, 9 * pb);
    if (e == cudaSuccess) e = cudaMalloc(&h->mom, 4 * pb);
    if (e == cudaSuccess) e = cudaMalloc(&h->lut, sizeof(float4) * 2 * (v3::LUT_N + 1));
    const size_t n_grp = (n_ctas + v3::NT - 1) / v3::NT;
    if (e == cudaSuccess) e = cudaMalloc(&h->partials, sizeof(double) * 7 * n_ctas);
    if (e == cudaSuccess) e = cudaMalloc(&h->gpartials, sizeof(double) * 7 * n_grp);
    if (e == cudaSuccess) e = cudaMalloc(&h->series, sizeof(double) * 8 * (size_t)p->max_samples);
    if (e == cudaSuccess) e = cudaMalloc(&h->err, sizeof(int));
    if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA);
    std::vector<float> lut;
    v3::coefficient_table(*p, lut);
    e = cudaMemcpy(h->lut, lut.data(), sizeof(float) * lut.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
    if (e != cudaSuccess) return bail(LB_ECUDA);
    *out = h;
    return LB_OK;
}

void lb3d_destroy(lb3d_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    dfree(h->state[0]); dfree(h->state[1]);
    dfree(h->sE); dfree(h->u); dfree(h->ys); dfree(h->r0); dfree(h->mom);
    dfree(h->lut); dfree(h->partials); dfree(h->gpartials); dfree(h->series); dfree(h->err);
    for (auto e : h->ev) cudaEventDestroy(e);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char* lb3d_last_error(const lb3d_handle* h) { return h ? h->msg.c_str() : "null handle"; }

int lb3d_init_fields(lb3d_handle* h, const double* P_init)
{
    if (!h) return LB_EINVAL;
    const size_t N = (size_t)h->NP, pb = sizeof(float) * N;
    CK3(h, cudaStreamSynchronize(h->stream));
    // fluid at rest at rho0: every shifted population is 0; sigma^p = 0
    CK3(h, cudaMemset(h->state[0], 0, (size_t)v3::PL_P * pb));
    if (P_init) {
        std::vector<float> P(3 * N);
        for (int c = 0; c < 3; ++c)
            for (size_t i = 0; i < N; ++i) P[c * N + i] = (float)(P_init[c * N + i] - h->p.P_ref[c]);
        CK3(h, cudaMemcpy(h->state[0] + (size_t)v3::PL_P * N, P.data(), 3 * pb, cudaMemcpyHostToDevice));
    } else {
        // P = 0: dP = -P_ref
        std::vector<float> P(3 * N);
        for (int c = 0; c < 3; ++c)
            for (size_t i = 0; i < N; ++i) P[c * N + i] = (float)(-h->p.P_ref[c]);
        CK3(h, cudaMemcpy(h->state[0] + (size_t)v3::PL_P * N, P.data(), 3 * pb, cudaMemcpyHostToDevice));
    }
    CK3(h, cudaMemset(h->state[1], 0, v3::NPL * pb));
    CK3(h, cudaMemset(h->err, 0, sizeof(int)));
    h->cur = 0;
    h->t = 0;
    h->rows = 0;
    h->ready = true;
    return LB_OK;
}

int lb3d_step(lb3d_handle* h, int64_t n)
{
    if (!h) return LB_EINVAL;
    if (n < 0) return fail(h, LB_EINVAL, "n < 0");
    if (!h->ready) return fail(h, LB_ESTATE, "lb3d_init_fields not called");
    const dim3 g = grid_of(h), b(v3::BX, v3::BY, v3::BZ);
    for (int64_t k = 0; k < n; ++k) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->timing) {
            for (int i = 0; i < 2; ++i) {
                if (h->ev_used == h->ev.size()) {
                    cudaEvent_t e;
                    CK3(h, cudaEventCreate(&e));
                    h->ev.push_back(e);
                }
                (i ? e1 : e0) = h->ev[h->ev_used++];
            }
            CK3(h, cudaEventRecord(e0, h->stream));
        }
        v3::Args3 a = args_of(h);
        a.readout = (h->t % h->p.readout_every) == 0;
        if (a.readout) {
            a.row = h->series + (size_t)(h->rows % h->p.max_samples) * 8;
            h->rows += 1;
        }
        int rc = launch_front(h, a, 0);
        if (rc) return rc;
        v3::k3_predict<<<g, b, 0, h->stream>>>(a);
        rc = launch_check(h, "k3_predict");
        if (rc) return rc;
        v3::k3_correct<<<g, b, 0, h->stream>>>(a);
        rc = launch_check(h, "k3_correct");
        if (rc) return rc;
        if (h->timing) CK3(h, cudaEventRecord(e1, h->stream));
        h->cur ^= 1;
        h->t += 1;
    }
    return LB_OK;
}

int lb3d_sync(lb3d_handle* h)
{
    if (!h) return LB_EINVAL;
    CK3(h, cudaStreamSynchronize(h->stream));
    int err = 0;
    CK3(h, cudaMemcpy(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CK3(h, cudaMemset(h->err, 0, sizeof(int)));
        return fail(h, LB_ENONFINITE, "a readout sum became NaN/Inf");
    }
    return LB_OK;
}

int64_t lb3d_time(const lb3d_handle* h) { return h ? h->t : -1; }

int lb3d_readout(lb3d_handle* h, int32_t field, float* dst, size_t count, int32_t dst_is_device)
{
    if (!h || !dst) return fail(h, LB_EINVAL, "null argument");
    if (field < 0 || field >= LB3D_N_FIELDS) return fail(h, LB_EINVAL, "unknown field %d", field);
    if (count < (size_t)h->NP) return fail(h, LB_EINVAL, "need %lld values", h->NP);
    if (!h->ready) return fail(h, LB_ESTATE, "lb3d_init_fields not called");
    const float* srcp;
    if (field <= 3) {
        v3::Args3 a = args_of(h);
        a.readout = 0;
        int rc = launch_front(h, a, 1);
        if (rc) return rc;
        srcp = h->mom + (size_t)field * h->NP;
    } else if (field < LB3D_FIELD_P) {
        srcp = h->state[h->cur] + (size_t)(v3::PL_S + field - LB3D_FIELD_SIGMA) * h->NP;
    } else if (field < LB3D_FIELD_POP0) {
        const int c = field - LB3D_FIELD_P;
        v3::k3_add<<<1024, 256, 0, h->stream>>>(h->state[h->cur] + (size_t)(v3::PL_P + c) * h->NP,
                                                (float)h->p.P_ref[c], h->mom, h->NP);
        int rc = launch_check(h, "k3_add");
        if (rc) return rc;
        srcp = h->mom;
    } else {
        srcp = h->state[h->cur] + (size_t)(field - LB3D_FIELD_POP0) * h->NP;
    }
    CK3(h, cudaMemcpyAsync(dst, srcp, sizeof(float) * (size_t)h->NP,
                           dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CK3(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb3d_series(lb3d_handle* h, double* dst, int32_t max_rows, int32_t* rows_written)
{
    if (!h || !dst || max_rows < 0) return fail(h, LB_EINVAL, "bad argument");
    CK3(h, cudaStreamSynchronize(h->stream));
    const long long cap = h->p.max_samples;
    const long long n = std::min<long long>(h->rows, cap);
    const long long first = h->rows - n;
    std::vector<double> all((size_t)cap * 8);
    CK3(h, cudaMemcpy(all.data(), h->series, sizeof(double) * all.size(), cudaMemcpyDeviceToHost));
    const long long k = std::min<long long>(n, max_rows);
    for (long long i = 0; i < k; ++i) {
        const long long slot = (first + i) % cap;
        memcpy(dst + 8 * i, all.data() + 8 * slot, sizeof(double) * 8);
    }
    if (rows_written) *rows_written = (int32_t)k;
    return LB_OK;
}

int lb3d_timing(lb3d_handle* h, int32_t enable)
{
    if (!h) return LB_EINVAL;
    CK3(h, cudaStreamSynchronize(h->stream));
    h->timing = enable != 0;
    h->ev_used = 0;
    return LB_OK;
}

int lb3d_kernel_time(lb3d_handle* h, double* ms, int64_t* steps)
{
    if (!h) return LB_EINVAL;
    CK3(h, cudaStreamSynchronize(h->stream));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        float m = 0.f;
        CK3(h, cudaEventElapsedTime(&m, h->ev[i], h->ev[i + 1]));
        tot += m;
    }
    if (ms) *ms = tot;
    if (steps) *steps = (int64_t)(h->ev_used / 2);
    return LB_OK;
}

int32_t lb3d_launches_per_step(const lb3d_handle* h) { return h ? (h->p.ericksen ? 4 : 3) : 0; }

int32_t lb3d_moment_table(double P_cap, float* dst, int32_t max_entries)
{
    if (!(P_cap > 0.0 && P_cap < 1.0)) return LB_EINVAL;
    if (!dst) return v3::LUT_N + 1;
    if (max_entries < v3::LUT_N + 1) return LB_EINVAL;
    std::vector<float> t;
    v3::moment_table(P_cap, t);
    memcpy(dst, t.data(), sizeof(float) * t.size());
    return v3::LUT_N + 1;
}

double lb3d_bytes_per_cell(const lb3d_handle* h) { return h ? 2.0 * v3::NPL * sizeof(float) : 0.0; }

}  // extern "C"
