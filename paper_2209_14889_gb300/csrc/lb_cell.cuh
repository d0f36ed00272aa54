// lb_cell.cuh -- per-cell arithmetic of the fused time step, shared by the lattice kernels so
// that every kernel variant evaluates the same expressions (see lb_fused.cu for the step).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace vlb {
namespace cell {

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

__device__ __forceinline__ void lut_eval(const float* __restrict__ L, const Phys& ph, float q, float& a2,
                                         float& a4)
{
    const float t = fminf(q, ph.q_cap) * ph.lut_scale;
    const int i = min((int)t, LUT_N - 1);                 // t >= 0; NaN converts to 0
    const float f = t - (float)i;
    const float2 v0 = __ldg(reinterpret_cast<const float2*>(L) + i);
    const float2 v1 = __ldg(reinterpret_cast<const float2*>(L) + i + 1);
    a2 = fmaf(f, v1.x - v0.x, v0.x);
    a4 = fmaf(f, v1.y - v0.y, v0.y);
    if (q > ph.q_cap) {
        const float s = ph.q_cap * __frcp_rn(q);
        a2 *= s;
        a4 *= s * s;
    }
}

// Programmatic dependent launch (the lattice and node kernels of consecutive steps overlap):
// pdl_wait blocks until the preceding kernel in the stream has completed and its writes are
// visible; pdl_trigger lets the following kernel start its prologue.  Each kernel triggers only
// after its own wait, so a kernel's prologue may read anything written two kernels back.
// Both are no-ops for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

// Ericksen stress (Sec. II C 1, kappa on the gradient term) and molecular field at one cell
// from the stencils of dP = P - P_ref; E = (xx, xy, yx, yy).
__device__ __forceinline__ void ericksen(const Phys& ph, const St& px, const St& py, float& hx,
                                         float& hy, float* E)
{
    molecular(ph, px, py, hx, hy);
    const float Px = ph.prx + px.c, Py = ph.pry + py.c;
    const float gxPx = 0.5f * (px.e - px.w), gyPx = 0.5f * (px.n - px.s);
    const float gxPy = 0.5f * (py.e - py.w), gyPy = 0.5f * (py.n - py.s);
    const float anti = Px * hy - hx * Py;
    const float sym = Px * hy + hx * Py;
    const float cross = ph.kappa * (gxPx * gyPx + gxPy * gyPy);
    E[0] = ph.xi * Px * hx - ph.kappa * (gxPx * gxPx + gxPy * gxPy);
    E[1] = -0.5f * anti + 0.5f * ph.xi * sym - cross;
    E[2] = 0.5f * anti + 0.5f * ph.xi * sym - cross;
    E[3] = ph.xi * Py * hy - ph.kappa * (gyPx * gyPx + gyPy * gyPy);
}

// div sigma^p from the stencils of (sxx, syy, sxy).
__device__ __forceinline__ void div_sigma(const St& sxx, const St& syy, const St& sxy, float& fx, float& fy)
{
    fx = 0.5f * (sxx.e - sxx.w) + 0.5f * (sxy.n - sxy.s);
    fy = 0.5f * (sxy.e - sxy.w) + 0.5f * (syy.n - syy.s);
}

// div sigma^E from the stencils of (xx, xy, yx, yy): only e, w of xx, yx and n, s of xy, yy are read.
__device__ __forceinline__ void div_ericksen(const St& exx, const St& exy, const St& eyx, const St& eyy,
                                             float& fx, float& fy)
{
    fx = 0.5f * (exx.e - exx.w) + 0.5f * (exy.n - exy.s);
    fy = 0.5f * (eyx.e - eyx.w) + 0.5f * (eyy.n - eyy.s);
}

// Moments (Eq. rhoDef, Eq. vDef, Guo half force) of the shifted populations d_n.
__device__ __forceinline__ void moments(const Phys& ph, const float* d, float Fx, float Fy, float& drho,
                                        float& ux, float& uy)
{
    drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const float jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const float jy = (d[2] - d[4]) + (d[5] - d[8]) + (d[6] - d[7]);
    const float inv = __frcp_rn(ph.rho0 + drho);
    ux = (jx + 0.5f * Fx) * inv;
    uy = (jy + 0.5f * Fy) * inv;
}

// BGK collision with the Guo source (Eq. LB, Eq. BGK): the changes D_n = d*_n - d_n of one cell,
// D_n = omega (d^eq_n - d_n) + (1 - 1/2tau) S_n with
//   d^eq_n = w_n (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)),
//   S_n    = w_n (3 (c - u).F + 9 (c.u)(c.F)),
// evaluated per pair of opposite velocities from their even and odd parts in c.
// They carry no mass and the momentum F in exact arithmetic; in FP32 the rounding of u (coherent
// over a uniform flow) would leak momentum into every cell alike, so the FP32 changes are
// corrected to exactly sum D_n = 0 and sum c_n D_n = F (pair and rest-population corrections).
// Order: n = 0 rest; 1..4 = +x, +y, -x, -y; 5..8 = (+,+), (-,+), (-,-), (+,-).
__device__ __forceinline__ void collide(const Phys& ph, const float* d, float drho, float ux, float uy,
                                        float Fx, float Fy, float* D)
{
    const float w0 = 4.f / 9.f, w1 = 1.f / 9.f, w5 = 1.f / 36.f;
    const float rho = ph.rho0 + drho;
    const float uu = 1.5f * (ux * ux + uy * uy);
    const float uF3 = 3.f * (ux * Fx + uy * Fy);
    const float om = ph.omega, g = ph.guo;
    const float base = drho - rho * uu;                 // even part common to all directions
    const float rho3 = 3.f * rho;
    D[0] = om * (w0 * base - d[0]) - g * w0 * uF3;
    // one pair (n, opposite m) with velocity c: cu = c.u, cF = c.F
    auto pair = [&](int n, int m, float w, float cu, float cF) {
        const float ev = w * fmaf(4.5f * rho * cu, cu, base);      // even part of d^eq
        const float od = w * rho3 * cu;                              // odd part of d^eq
        const float Sev = w * fmaf(9.f * cu, cF, -uF3);             // even part of S
        const float Sod = 3.f * w * cF;                              // odd part of S
        D[n] = om * ((ev + od) - d[n]) + g * (Sev + Sod);
        D[m] = om * ((ev - od) - d[m]) + g * (Sev - Sod);
    };
    pair(1, 3, w1, ux, Fx);
    pair(2, 4, w1, uy, Fy);
    pair(5, 7, w5, ux + uy, Fx + Fy);
    pair(6, 8, w5, uy - ux, Fy - Fx);
    const float ex = ((D[1] - D[3]) + (D[5] - D[6]) + (D[8] - D[7])) - Fx;
    const float ey = ((D[2] - D[4]) + (D[5] - D[8]) + (D[6] - D[7])) - Fy;
    D[1] -= 0.5f * ex;
    D[3] += 0.5f * ex;
    D[2] -= 0.5f * ey;
    D[4] += 0.5f * ey;
    D[0] -= ((D[1] + D[2]) + (D[3] + D[4])) + ((D[5] + D[6]) + (D[7] + D[8])) + D[0];
}

// ---------------------------------------------------------------------------------------------
// Storage forms of the lattice state.  PREC_FP32: FP32 planes.  PREC_LP (the precision form):
// populations as FP16 of s_n = d_n 2^POP_SHIFT / w_n (scaled deviations from w_n rho0, so the
// diagonal directions stay out of the FP16 subnormals), sigma^p as BF16 and dP = P - P_ref as
// FP16.  dP needs the 3 extra mantissa bits: the rounding noise of P_y (of order the director
// noise) enters alpha + beta |P|^2 and hence the Ericksen force; with BF16 it alone raised the
// restoring-force error to 1.3 %, with FP16 it is 0.14 % (oracle emulation, 128^2, 300 steps).
// Arithmetic is FP32 in both forms; LP stores round stochastically (hardware cvt.rs with
// counter-hashed random bits keyed by step, cell and value), which keeps the small per-step
// increments of sigma and P from being rounded away and the rounding errors unbiased.
// ---------------------------------------------------------------------------------------------
enum { PREC_FP32 = 0, PREC_LP = 1 };
constexpr int POP_SHIFT = 12;

__device__ __forceinline__ float pop_scale(int n)     // 2^POP_SHIFT / w_n
{
    return n == 0 ? 4096.f * 9.f / 4.f : (n < 5 ? 4096.f * 9.f : 4096.f * 36.f);
}
__device__ __forceinline__ float pop_unscale(int n)   // w_n / 2^POP_SHIFT
{
    return n == 0 ? (4.f / 9.f) / 4096.f : (n < 5 ? (1.f / 9.f) / 4096.f : (1.f / 36.f) / 4096.f);
}

// COH: the state was written earlier in the same launch (persistent kernel) -- load through L2
// (ld.global.cg) instead of the non-coherent read-only path
template <class T, bool COH>
__device__ __forceinline__ T ld_state(const T* p)
{
    if (COH) return __ldcg(p);
    return __ldg(p);
}

template <int PREC, bool COH = false>
__device__ __forceinline__ float ld_pop(const void* src, long long NP, int n, long long g)
{
    if (PREC == PREC_FP32) return ld_state<float, COH>(reinterpret_cast<const float*>(src) + n * NP + g);
    const unsigned short b = ld_state<unsigned short, COH>(reinterpret_cast<const unsigned short*>(src) + n * NP + g);
    return __half2float(__ushort_as_half(b)) * pop_unscale(n);
}

template <int PREC, bool COH = false>
__device__ __forceinline__ float ld_fld(const void* src, long long NP, int plane, long long g)
{
    if (PREC == PREC_FP32) return ld_state<float, COH>(reinterpret_cast<const float*>(src) + plane * NP + g);
    const unsigned short b = ld_state<unsigned short, COH>(reinterpret_cast<const unsigned short*>(src) + plane * NP + g);
    if (plane >= PL_PX) return __half2float(__ushort_as_half(b));      // dP: FP16
    return __uint_as_float((unsigned)b << 16);                         // sigma: BF16
}

// counter-based 32-bit hash (a bijective integer mixer) for the stochastic-rounding bits
__device__ __forceinline__ unsigned sr_bits(unsigned long long t, long long g, unsigned k)
{
    unsigned x = (unsigned)g * 0x9E3779B1u ^ ((unsigned)t * 0x85EBCA77u + k * 0xC2B2AE3Du);
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

// two FP32 values to FP16 / BF16 with stochastic rounding: a -> upper, b -> lower half
__device__ __forceinline__ unsigned cvt_sr_f16x2(float a, float b, unsigned rbits)
{
    unsigned d;
    asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    return d;
}
__device__ __forceinline__ unsigned cvt_sr_bf16x2(float a, float b, unsigned rbits)
{
    unsigned d;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    return d;
}

// Store the 9 post-collision populations v[n] of one cell at the flat indices gd[n].
template <int PREC>
__device__ __forceinline__ void st_pops(void* dst, long long NP, const long long* gd, const float* v,
                                        unsigned long long t, long long g)
{
    if (PREC == PREC_FP32) {
        float* d = reinterpret_cast<float*>(dst);
#pragma unroll
        for (int n = 0; n < 9; ++n) d[n * NP + gd[n]] = v[n];
    } else {
        unsigned short* d = reinterpret_cast<unsigned short*>(dst);
#pragma unroll
        for (int n = 0; n < 9; n += 2) {
            const float a = v[n] * pop_scale(n);
            const float b = (n + 1 < 9) ? v[n + 1] * pop_scale(n + 1) : 0.f;
            const unsigned p = cvt_sr_f16x2(a, b, sr_bits(t, g, (unsigned)n));
            d[n * NP + gd[n]] = (unsigned short)(p >> 16);
            if (n + 1 < 9) d[(n + 1) * NP + gd[n + 1]] = (unsigned short)(p & 0xFFFFu);
        }
    }
}

// Store sigma (xx, yy, xy) and dP (x, y) of one cell.
template <int PREC>
__device__ __forceinline__ void st_flds(void* dst, long long NP, long long g, const float* v,
                                        unsigned long long t)
{
    if (PREC == PREC_FP32) {
        float* d = reinterpret_cast<float*>(dst);
#pragma unroll
        for (int c = 0; c < 5; ++c) d[(PL_SXX + c) * NP + g] = v[c];
    } else {
        unsigned short* d = reinterpret_cast<unsigned short*>(dst);
        const unsigned s01 = cvt_sr_bf16x2(v[0], v[1], sr_bits(t, g, 16u));
        const unsigned s2 = cvt_sr_bf16x2(v[2], 0.f, sr_bits(t, g, 17u));
        const unsigned pp = cvt_sr_f16x2(v[3], v[4], sr_bits(t, g, 18u));
        d[PL_SXX * NP + g] = (unsigned short)(s01 >> 16);
        d[PL_SYY * NP + g] = (unsigned short)(s01 & 0xFFFFu);
        d[PL_SXY * NP + g] = (unsigned short)(s2 >> 16);
        d[PL_PX * NP + g] = (unsigned short)(pp >> 16);
        d[PL_PY * NP + g] = (unsigned short)(pp & 0xFFFFu);
    }
}

}  // namespace cell
}  // namespace vlb
