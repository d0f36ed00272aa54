// lb_cell.cuh -- per-cell arithmetic of the fused time step, shared by the lattice kernels so
// that every kernel variant evaluates the same expressions (see lb_fused.cu for the step).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_internal.h"
#include "lb_vec.cuh"

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
__device__ __forceinline__ void lut_eval(const float* __restrict__ L, const Phys& ph, float2 q, float2& a2,
                                         float2& a4)
{
    lut_eval(L, ph, q.x, a2.x, a4.x);
    lut_eval(L, ph, q.y, a2.y, a4.y);
}

// Programmatic dependent launch (the lattice and node kernels of consecutive steps overlap):
// pdl_wait blocks until the preceding kernel in the stream has completed and its writes are
// visible; pdl_trigger lets the following kernel start its prologue.  Each kernel triggers only
// after its own wait, so a kernel's prologue may read anything written two kernels back.
// Both are no-ops for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

using namespace vec;

// One cell per thread (T = float): the per-cell functions below then pair the x and y parts of
// a vector, two components of a tensor or two lattice directions onto the paired FP32
// instructions, each lane evaluating the scalar expression (same operations, same order, same
// fused multiply-adds), so the results are those of the scalar form: on GB300 every normal FP32
// result agreed bit for bit with the scalar build, and only values in the subnormal range (below
// 1e-37, in the nearly quiescent corners of a closed box) differed.  Per time step this cuts the
// FP32 instruction count, and the kernels, which are issue-bound, by 5-7 %.
template <class T>
constexpr bool ONE_CELL = std::is_same<T, float>::value;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// A paired product rounded on its own.  The compiler fuses a paired product with the paired sum
// or difference that consumes it when every use of the product is such a sum (even under
// -fmad=false and with the .rn intrinsics; measured on GB300), which rounds the two as one and
// makes the result depend on the surrounding code.  Written as a paired fused multiply-add with
// a +0 addend, the product rounds exactly as a plain product (up to the sign of a zero result)
// and is not fused.  Products that are only multiplied further, used as a factor or addend of a
// fused multiply-add, or scaled by a power of two (exact) need no such care.
__device__ __forceinline__ float2 mul_r(float2 a, float2 b) { return __ffma2_rn(a, b, make_float2(0.f, 0.f)); }
__device__ __forceinline__ float2 mul_r(float a, float2 b)
{
    return __ffma2_rn(make_float2(a, a), b, make_float2(0.f, 0.f));
}

// Stencil values of one component: centre, east (+x), west, north (+y), south; T = float for
// one cell, float2 for two neighbouring cells (x, x+1).
template <class T>
struct StT {
    T c, e, w, n, s;
};
using St = StT<float>;

__device__ __forceinline__ St st_at(const float* base, int W, int lx, int ly)
{
    const float* p = base + ly * W + lx;
    return St{p[0], p[1], p[-1], p[W], p[-W]};
}

// Stencils of the cell pair (lx, lx+1) of a shared-memory plane of even width W.  EVEN: the
// flat index of (lx, ly) is even (8-byte aligned pairs at the centre row and at +-W);
// otherwise the pairs at -1 and +1 are the aligned ones and hold w and e exactly.
template <bool EVEN>
__device__ __forceinline__ StT<float2> st2_at(const float* base, int W, int lx, int ly)
{
    const float* p = base + ly * W + lx;
    StT<float2> r;
    if (EVEN) {
        const float2 c = *reinterpret_cast<const float2*>(p);
        const float2 rr = *reinterpret_cast<const float2*>(p + 2);
        const float2 ll = *reinterpret_cast<const float2*>(p - 2);
        r.c = c;
        r.e = make_float2(c.y, rr.x);
        r.w = make_float2(ll.y, c.x);
        r.n = *reinterpret_cast<const float2*>(p + W);
        r.s = *reinterpret_cast<const float2*>(p - W);
    } else {
        const float2 ww = *reinterpret_cast<const float2*>(p - 1);
        const float2 ee = *reinterpret_cast<const float2*>(p + 1);
        r.c = make_float2(ww.y, ee.x);
        r.e = ee;
        r.w = ww;
        r.n = make_float2(p[W], p[W + 1]);
        r.s = make_float2(p[-W], p[-W + 1]);
    }
    return r;
}

// a pair of neighbouring values of a plane; EVEN as for st2_at
template <bool EVEN>
__device__ __forceinline__ float2 ld2(const float* p)
{
    if (EVEN) return *reinterpret_cast<const float2*>(p);
    return make_float2(p[0], p[1]);
}
template <bool EVEN>
__device__ __forceinline__ void st2(float* p, float2 v)
{
    if (EVEN) {
        *reinterpret_cast<float2*>(p) = v;
    } else {
        p[0] = v.x;
        p[1] = v.y;
    }
}

// Molecular field h = (alpha + beta |P|^2) P - kappa lap P (Eq. Ffunctional) from the stencil
// of dP = P - P_ref: alpha + beta |P|^2 = A0 + beta (2 P_ref.dP + |dP|^2) has no cancellation.
template <class T>
__device__ __forceinline__ void molecular(const Phys& ph, const StT<T>& dx, const StT<T>& dy, T& hx, T& hy)
{
    if constexpr (ONE_CELL<T>) {
        // the two components of P as one pair (lanes x, y): the Laplacians and h on paired FP32
        const float two_pd = fmaf(ph.prx, dx.c, ph.pry * dy.c);
        const float dd = fmaf(dx.c, dx.c, dy.c * dy.c);
        const float A = fmaf(ph.beta, fmaf(2.f, two_pd, dd), ph.A0);
        const float2 c = f2(dx.c, dy.c);
        const float2 L = vfma(-4.f, c, (f2(dx.e, dy.e) + f2(dx.w, dy.w)) + (f2(dx.n, dy.n) + f2(dx.s, dy.s)));
        const float2 H = vfma(A, c + f2(ph.prx, ph.pry), (-ph.kappa) * L);
        hx = H.x;
        hy = H.y;
        return;
    }
    const T two_pd = vfma(ph.prx, dx.c, ph.pry * dy.c);
    const T dd = vfma(dx.c, dx.c, dy.c * dy.c);
    const T A = vfma(ph.beta, vfma(2.f, two_pd, dd), bc<T>(ph.A0));
    const T lx = vfma(-4.f, dx.c, (dx.e + dx.w) + (dx.n + dx.s));
    const T ly = vfma(-4.f, dy.c, (dy.e + dy.w) + (dy.n + dy.s));
    hx = vfma(A, dx.c + ph.prx, -ph.kappa * lx);
    hy = vfma(A, dy.c + ph.pry, -ph.kappa * ly);
}

// Right-hand sides of Eq. StiffCons (with the Jaumann derivative) and Eq. BE at one cell, for
// the frozen u, Psi = (pxx, pyy, pxy), omega = Omega_xy; s = sigma (xx, yy, xy), p = dP (x, y).
// SCALAR: the scalar model of Eq. MaxDiff (Sec. II B): a constant modulus C = ph.kS8 in place of
// C~(P), and no P field (p0, p1, hx, hy unused; r[3], r[4] not written).  It rounds exactly as
// the tensorial form does for the isotropic K^x (K2222 = K1111, K1122 = 0, K1212 = K1111 / 2),
// whose C~ is C times the identity for every P.
template <class T, bool SCALAR = false>
__device__ __forceinline__ void rhs_cell(const Phys& ph, const float* lut, T ux, T uy, T pxx, T pyy, T pxy,
                                         T om, const StT<T>& s0, const StT<T>& s1, const StT<T>& s2,
                                         const StT<T>& p0, const StT<T>& p1, T hx, T hy, T* r)
{
    if constexpr (ONE_CELL<T>) {
        // pairs: (sigma_xx, sigma_yy) stencils, (P_x, P_y) stencils, (u_x, u_y), (Psi_xx, Psi_yy),
        // the first two rows of C~ v, the right-hand sides (r0, r1) and (r3, r4)
        const float2 V01 = vfma(-ph.inv_eta, f2(s0.c, s1.c), f2(pxx, pyy));   // (v0, v1)
        const float v2 = fmaf(-ph.inv_eta, s2.c, pxy);
        // Jaumann rotation: (-J0, J0) with J0 = 2 w sxy (the negation is exact), J2 = w (syy - sxx)
        const float2 nJ = f2(-2.f, 2.f) * (om * s2.c);
        const float J2 = om * (s1.c - s0.c);
        const float2 uh = 0.5f * f2(ux, uy);
        const float D = ph.Dp;
        const float2 E01 = f2(s0.e, s1.e), W01 = f2(s0.w, s1.w), N01 = f2(s0.n, s1.n), S01 = f2(s0.s, s1.s);
        const float2 nadv01 = vfma(uh.x, W01 - E01, uh.y * (S01 - N01));
        const float2 lap01 = vfma(-4.f, f2(s0.c, s1.c), (E01 + W01) + (N01 + S01));
        const float nadv2 = fmaf(uh.x, s2.w - s2.e, uh.y * (s2.s - s2.n));
        const float lap2 = fmaf(-4.f, s2.c, (s2.e + s2.w) + (s2.n + s2.s));
        if (SCALAR) {
            const float2 r01 = vfma(D, lap01, (mul_r(ph.kS8, V01) + nJ) + nadv01);
            r[0] = r01.x;
            r[1] = r01.y;
            r[2] = fmaf(D, lap2, ((ph.kS8 * v2) - J2) + nadv2);
            return;
        }
        const float2 P = f2(p0.c, p1.c) + f2(ph.prx, ph.pry);
        const float2 PP = mul_r(P, P);
        float a2, a4;
        lut_eval(lut, ph, PP.x + PP.y, a2, a4);
        const float c2q = PP.x - PP.y, s2q = 2.f * (P.x * P.y);
        const float2 R2 = a2 * f2(c2q, s2q);                                              // (r2c2, r2s2)
        const float2 R4 = a4 * f2((c2q - s2q) * (c2q + s2q), 2.f * (c2q * s2q));          // (r4c4, r4s4)
        const float hds = (0.5f * ph.dK) * R2.y;
        const float2 X = mul_r(f2(0.125f * ph.kX, 0.25f * ph.kX), R4);                     // (xc, xs)
        const float C11 = fmaf(0.5f * ph.dK, R2.x, ph.kS8) + X.x;
        const float C12 = ph.kC12 - X.x;
        const float C13 = X.y + hds;
        const float C22 = fmaf(-ph.dK, R2.x, C11);
        const float C23 = hds - X.y;
        const float C33 = fmaf(-2.f, X.x, ph.kC33);
        const float2 C3 = f2(C13, C23);
        const float2 Cv01 = vfma(f2(C11, C12), V01.x, vfma(f2(C12, C22), V01.y, C3 * v2));
        const float2 hC3 = 0.5f * C3;
        const float Cv2 = fmaf(hC3.x, V01.x, fmaf(hC3.y, V01.y, C33 * v2));
        const float2 r01 = vfma(D, lap01, (Cv01 + nJ) + nadv01);
        r[0] = r01.x;
        r[1] = r01.y;
        r[2] = fmaf(D, lap2, (Cv2 - J2) + nadv2);
        // Eq. BE
        const float xp0 = fmaf(pxx, P.x, pxy * P.y), xp1 = fmaf(pxy, P.x, pyy * P.y);
        const float2 Ep = f2(p0.e, p1.e), Wp = f2(p0.w, p1.w), Np = f2(p0.n, p1.n), Sp = f2(p0.s, p1.s);
        const float2 nadvp = vfma(uh.x, Wp - Ep, uh.y * (Sp - Np));
        const float2 r34 = vfma(-ph.Gamma, f2(hx, hy),
                                vfma(ph.xi, f2(xp0, xp1), f2(nadvp.x - om * P.y, fmaf(om, P.x, nadvp.y))));
        r[3] = r34.x;
        r[4] = r34.y;
        return;
    }
    // C psi - C s / eta_p = C (psi - s / eta_p)
    const T v0 = vfma(-ph.inv_eta, s0.c, pxx);
    const T v1 = vfma(-ph.inv_eta, s1.c, pyy);
    const T v2 = vfma(-ph.inv_eta, s2.c, pxy);
    T Cv0, Cv1, Cv2;
    // Jaumann rotation (Omega s - s Omega) = (2 w sxy, -2 w sxy, w (syy - sxx))
    const T J0 = 2.f * (om * s2.c);
    const T J2 = om * (s1.c - s0.c);
    // advection -(u.grad) y with central differences (uh = u / 2 times the plain differences)
    const T uxh = 0.5f * ux, uyh = 0.5f * uy;
    const float D = ph.Dp;
    auto nadv = [&](const StT<T>& f) { return vfma(uxh, f.w - f.e, uyh * (f.s - f.n)); };
    auto lap = [&](const StT<T>& f) { return vfma(-4.f, f.c, (f.e + f.w) + (f.n + f.s)); };
    if (SCALAR) {
        Cv0 = ph.kS8 * v0;
        Cv1 = ph.kS8 * v1;
        Cv2 = ph.kS8 * v2;
        r[0] = vfma(D, lap(s0), (Cv0 - J0) + nadv(s0));
        r[1] = vfma(D, lap(s1), (Cv1 + J0) + nadv(s1));
        r[2] = vfma(D, lap(s2), (Cv2 - J2) + nadv(s2));
        return;
    }
    // stiffness C~(P) (App. B) from the table of a2, a4 and polynomials in P = P_ref + dP
    const T Px = p0.c + ph.prx, Py = p1.c + ph.pry;
    const T PxPx = Px * Px, PyPy = Py * Py;
    const T q = PxPx + PyPy;
    T a2, a4;
    lut_eval(lut, ph, q, a2, a4);
    const T c2q = PxPx - PyPy, s2q = 2.f * (Px * Py);
    const T r2c2 = a2 * c2q, r2s2 = a2 * s2q;
    const T r4c4 = a4 * ((c2q - s2q) * (c2q + s2q)), r4s4 = a4 * (2.f * (c2q * s2q));
    const T hds = (0.5f * ph.dK) * r2s2;
    const T xc = (0.125f * ph.kX) * r4c4, xs = (0.25f * ph.kX) * r4s4;
    const T C11 = vfma(0.5f * ph.dK, r2c2, bc<T>(ph.kS8)) + xc;
    const T C12 = ph.kC12 - xc;
    const T C13 = xs + hds;
    const T C22 = vfma(-ph.dK, r2c2, C11);
    const T C23 = hds - xs;
    const T C33 = vfma(-2.f, xc, bc<T>(ph.kC33));
    Cv0 = vfma(C11, v0, vfma(C12, v1, C13 * v2));
    Cv1 = vfma(C12, v0, vfma(C22, v1, C23 * v2));
    Cv2 = vfma(0.5f * C13, v0, vfma(0.5f * C23, v1, C33 * v2));
    r[0] = vfma(D, lap(s0), (Cv0 - J0) + nadv(s0));
    r[1] = vfma(D, lap(s1), (Cv1 + J0) + nadv(s1));
    r[2] = vfma(D, lap(s2), (Cv2 - J2) + nadv(s2));
    // Eq. BE: -(u.grad)P - Omega P + xi Psi P - Gamma h
    const T xp0 = vfma(pxx, Px, pxy * Py), xp1 = vfma(pxy, Px, pyy * Py);
    r[3] = vfma(-ph.Gamma, hx, vfma(ph.xi, xp0, nadv(p0) - om * Py));
    r[4] = vfma(-ph.Gamma, hy, vfma(ph.xi, xp1, vfma(om, Px, nadv(p1))));
}

// Velocity gradient from the stencils of u: Psi = (pxx, pyy, pxy), omega = Omega_xy.
template <class T>
__device__ __forceinline__ void vgrad(const StT<T>& ux, const StT<T>& uy, T& pxx, T& pyy, T& pxy, T& om)
{
    if constexpr (ONE_CELL<T>) {
        const float2 A = 0.5f * (f2(ux.e, uy.e) - f2(ux.w, uy.w));   // (d_x u_x, d_x u_y)
        const float2 B = 0.5f * (f2(ux.n, uy.n) - f2(ux.s, uy.s));   // (d_y u_x, d_y u_y)
        pxx = A.x;
        pyy = B.y;
        pxy = 0.5f * (A.y + B.x);
        om = 0.5f * (A.y - B.x);
        return;
    }
    const T dxux = 0.5f * (ux.e - ux.w);
    const T dyux = 0.5f * (ux.n - ux.s);
    const T dxuy = 0.5f * (uy.e - uy.w);
    const T dyuy = 0.5f * (uy.n - uy.s);
    pxx = dxux;
    pyy = dyuy;
    pxy = 0.5f * (dxuy + dyux);
    om = 0.5f * (dxuy - dyux);
}

// the same from two planes of width W at the flat index i (one cell)
__device__ __forceinline__ void vgrad(const float* ux, const float* uy, int W, int i, float& pxx,
                                      float& pyy, float& pxy, float& om)
{
    const St sx{ux[i], ux[i + 1], ux[i - 1], ux[i + W], ux[i - W]};
    const St sy{uy[i], uy[i + 1], uy[i - 1], uy[i + W], uy[i - W]};
    vgrad(sx, sy, pxx, pyy, pxy, om);
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
template <class T>
__device__ __forceinline__ void ericksen(const Phys& ph, const StT<T>& px, const StT<T>& py, T& hx, T& hy, T* E)
{
    if constexpr (ONE_CELL<T>) {
        // (P_x, P_y) pairs at every stencil point: the Laplacians and h as in molecular, the
        // gradients as (d P_x, d P_y) pairs along x and along y
        const float two_pd = fmaf(ph.prx, px.c, ph.pry * py.c);
        const float dd = fmaf(px.c, px.c, py.c * py.c);
        const float A = fmaf(ph.beta, fmaf(2.f, two_pd, dd), ph.A0);
        const float2 c = f2(px.c, py.c), Ee = f2(px.e, py.e), Ww = f2(px.w, py.w), Nn = f2(px.n, py.n),
                     Ss = f2(px.s, py.s);
        const float2 L = vfma(-4.f, c, (Ee + Ww) + (Nn + Ss));
        const float2 P = c + f2(ph.prx, ph.pry);
        const float2 H = vfma(A, P, (-ph.kappa) * L);
        hx = H.x;
        hy = H.y;
        const float2 GX = 0.5f * (Ee - Ww);               // (d_x P_x, d_x P_y)
        const float2 GY = 0.5f * (Nn - Ss);               // (d_y P_x, d_y P_y)
        const float Pxhy = P.x * H.y, hxPy = H.x * P.y;
        const float anti = Pxhy - hxPy;
        const float sym = Pxhy + hxPy;
        const float cross = ph.kappa * fmaf(GX.x, GY.x, GX.y * GY.y);
        const float xs = (0.5f * ph.xi) * sym;
        const float2 g2 = f2(fmaf(GX.x, GX.x, GX.y * GX.y), fmaf(GY.x, GY.x, GY.y * GY.y));
        const float2 E03 = vfma(ph.xi, P * H, (-ph.kappa) * g2);
        E[0] = E03.x;
        E[1] = fmaf(-0.5f, anti, xs) - cross;
        E[2] = fmaf(0.5f, anti, xs) - cross;
        E[3] = E03.y;
        return;
    }
    molecular(ph, px, py, hx, hy);
    const T Px = px.c + ph.prx, Py = py.c + ph.pry;
    const T gxPx = 0.5f * (px.e - px.w), gyPx = 0.5f * (px.n - px.s);
    const T gxPy = 0.5f * (py.e - py.w), gyPy = 0.5f * (py.n - py.s);
    const T Pxhy = Px * hy, hxPy = hx * Py;
    const T anti = Pxhy - hxPy;
    const T sym = Pxhy + hxPy;
    const T cross = ph.kappa * vfma(gxPx, gyPx, gxPy * gyPy);
    const T xs = (0.5f * ph.xi) * sym;
    E[0] = vfma(ph.xi, Px * hx, -ph.kappa * vfma(gxPx, gxPx, gxPy * gxPy));
    E[1] = vfma(-0.5f, anti, xs) - cross;
    E[2] = vfma(0.5f, anti, xs) - cross;
    E[3] = vfma(ph.xi, Py * hy, -ph.kappa * vfma(gyPx, gyPx, gyPy * gyPy));
}

// div sigma^p from the stencils of (sxx, syy, sxy).
template <class T>
__device__ __forceinline__ void div_sigma(const StT<T>& sxx, const StT<T>& syy, const StT<T>& sxy, T& fx, T& fy)
{
    if constexpr (ONE_CELL<T>) {
        const float2 F = 0.5f * ((f2(sxx.e, sxy.e) - f2(sxx.w, sxy.w)) + (f2(sxy.n, syy.n) - f2(sxy.s, syy.s)));
        fx = F.x;
        fy = F.y;
        return;
    }
    fx = 0.5f * ((sxx.e - sxx.w) + (sxy.n - sxy.s));
    fy = 0.5f * ((sxy.e - sxy.w) + (syy.n - syy.s));
}

// div sigma^E from the stencils of (xx, xy, yx, yy): only e, w of xx, yx and n, s of xy, yy are read.
template <class T>
__device__ __forceinline__ void div_ericksen(const StT<T>& exx, const StT<T>& exy, const StT<T>& eyx,
                                             const StT<T>& eyy, T& fx, T& fy)
{
    if constexpr (ONE_CELL<T>) {
        const float2 F = 0.5f * ((f2(exx.e, eyx.e) - f2(exx.w, eyx.w)) + (f2(exy.n, eyy.n) - f2(exy.s, eyy.s)));
        fx = F.x;
        fy = F.y;
        return;
    }
    fx = 0.5f * ((exx.e - exx.w) + (exy.n - exy.s));
    fy = 0.5f * ((eyx.e - eyx.w) + (eyy.n - eyy.s));
}

// Moments (Eq. rhoDef, Eq. vDef, Guo half force) of the shifted populations d_n.
template <class T>
__device__ __forceinline__ void moments(const Phys& ph, const T* d, T Fx, T Fy, T& drho, T& ux, T& uy)
{
    if constexpr (ONE_CELL<T>) {
        // (j_x, j_y) and u as pairs; populations pair as (1, 2), (3, 4), (5, 6), (7, 8)
        drho = (((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7]))) + d[8];
        const float2 J = ((f2(d[1], d[2]) - f2(d[3], d[4])) + f2(d[5] - d[6], d[5] - d[8])) +
                         f2(d[8] - d[7], d[6] - d[7]);
        const float inv = __frcp_rn(drho + ph.rho0);
        const float2 U = mul_r(inv, vfma(0.5f, f2(Fx, Fy), J));
        ux = U.x;
        uy = U.y;
        return;
    }
    drho = (((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7]))) + d[8];
    const T jx = ((d[1] - d[3]) + (d[5] - d[6])) + (d[8] - d[7]);
    const T jy = ((d[2] - d[4]) + (d[5] - d[8])) + (d[6] - d[7]);
    const T inv = vrcp(drho + ph.rho0);
    ux = vfma(0.5f, Fx, jx) * inv;
    uy = vfma(0.5f, Fy, jy) * inv;
}

// Post-collision populations out_n = d_n + D_n, the (1, 2), (3, 4), (5, 6), (7, 8) sums paired.
__device__ __forceinline__ void add_pops(const float* d, const float* D, float* out)
{
    out[0] = d[0] + D[0];
#pragma unroll
    for (int n = 1; n < 9; n += 2) {
        const float2 o = f2(d[n], d[n + 1]) + f2(D[n], D[n + 1]);
        out[n] = o.x;
        out[n + 1] = o.y;
    }
}

// Heun corrector of the five fields y' = y + (R + r) / 2 (components 0, 1 and 3, 4 paired);
// NC = 3 for the scalar model (sigma only).
template <int NC>
__device__ __forceinline__ void heun(const float* R, const float* r, const float* y, float* out)
{
    const float2 a = vfma(0.5f, f2(R[0], R[1]) + f2(r[0], r[1]), f2(y[0], y[1]));
    out[0] = a.x;
    out[1] = a.y;
    out[2] = fmaf(0.5f, R[2] + r[2], y[2]);
    if (NC == 5) {
        const float2 b = vfma(0.5f, f2(R[3], R[4]) + f2(r[3], r[4]), f2(y[3], y[4]));
        out[3] = b.x;
        out[4] = b.y;
    }
}

// Heun predictor y* = y + r of the five fields (NC as for heun)
template <int NC>
__device__ __forceinline__ void predict(const float* y, const float* r, float* out)
{
    const float2 a = f2(y[0], y[1]) + f2(r[0], r[1]);
    out[0] = a.x;
    out[1] = a.y;
    out[2] = y[2] + r[2];
    if (NC == 5) {
        const float2 b = f2(y[3], y[4]) + f2(r[3], r[4]);
        out[3] = b.x;
        out[4] = b.y;
    }
}

// Readout sums in double-float: a sum is kept as hi + lo, two FP32 numbers (about 48 significant
// bits), accumulated with the error-free two-sum (Knuth): s = a + b, e = (a - (s - b')) + (b - b')
// with b' = s - a is exactly a + b - s.  These sources are built without FMA contraction, so every
// operation rounds as written.  FP64 is a narrow unit on this GPU (the per-cell FP64 accumulation
// and FP64 warp shuffles of the readout made a readout step 40 % slower than a plain one at
// 1024^2); here the cells and the warp trees run on FP32 lanes and only a CTA's five totals are
// formed in FP64.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void df_add(DF& x, float v)
{
    const float s = x.hi + v;
    const float bp = s - x.hi;
    const float e = (x.hi - (s - bp)) + (v - bp);
    x.hi = s;
    x.lo += e;
}

__device__ __forceinline__ DF df_merge(DF x, DF y)
{
    const float s = x.hi + y.hi;
    const float bp = s - x.hi;
    const float e = (x.hi - (s - bp)) + (y.hi - bp);
    const float l = (x.lo + y.lo) + e;
    const float h = s + l;
    return DF{h, l - (h - s)};
}

// Fixed-order sum over the CTA (1-D, whole warps, at most 16 of them) of K double-float values
// per thread: a shuffle tree within each warp, then the warps in order by thread k < K, which
// returns the total of value k (other threads return zero).  red: 2 K (warps) floats of shared
// memory, reusable when the call returns.
template <int K>
__device__ __forceinline__ DF df_block_sum(const DF* v, float* red)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        DF x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const DF y{__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)};
            x = df_merge(x, y);
        }
        if (lane == 0) {
            red[2 * (k * nw + wid)] = x.hi;
            red[2 * (k * nw + wid) + 1] = x.lo;
        }
    }
    __syncthreads();
    DF s{0.f, 0.f};
    if (tid < K) {
        s = DF{red[2 * (tid * nw)], red[2 * (tid * nw) + 1]};
        for (int w = 1; w < nw; ++w) s = df_merge(s, DF{red[2 * (tid * nw + w)], red[2 * (tid * nw + w) + 1]});
    }
    __syncthreads();
    return s;
}

// A CTA's readout partial: value k as the double-float pair (hi, lo) at float2 index 5 slot + k of
// the partials buffer (5 values per CTA); the lattice readout merges them in double-float and
// forms FP64 only for the five totals.
__device__ __forceinline__ void store_partial(double* partials, long long slot, const DF* acc, float* red)
{
    const DF s = df_block_sum<5>(acc, red);
    if (threadIdx.x < 5)
        reinterpret_cast<float2*>(partials)[slot * 5 + threadIdx.x] = make_float2(s.hi, s.lo);
}

// Readout values of one cell from its shifted populations: the mass excess and the bare momentum
// as FP32 sums in a fixed order (the momentum as moments forms it); every lattice kernel
// accumulates these and the cell's force in double-float (above).
__device__ __forceinline__ void cell_readout(const float* d, float& dsum, float& jx, float& jy)
{
    dsum = 0.f;
#pragma unroll
    for (int n = 0; n < 9; ++n) dsum += d[n];
    jx = ((d[1] - d[3]) + (d[5] - d[6])) + (d[8] - d[7]);
    jy = ((d[2] - d[4]) + (d[5] - d[8])) + (d[6] - d[7]);
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
template <class T>
__device__ __forceinline__ void collide(const Phys& ph, const T* d, T drho, T ux, T uy, T Fx, T Fy, T* D)
{
    const float w0 = 4.f / 9.f, w1 = 1.f / 9.f, w5 = 1.f / 36.f;
    const float om = ph.omega, g = ph.guo;
    if constexpr (ONE_CELL<T>) {
        // the opposite pairs (1, 3) and (2, 4) share w1 and run as the lanes of one paired
        // evaluation, likewise (5, 7) and (6, 8) with w5: D_12 = (D1, D2), D_34 = (D3, D4), ...
        const float nrho = (-ph.rho0) - drho;
        const float uu = 1.5f * fmaf(ux, ux, uy * uy);
        const float nuF3 = -3.f * fmaf(ux, Fx, uy * Fy);
        const float base = fmaf(nrho, uu, drho);
        const float rho3 = -3.f * nrho, rho45 = -4.5f * nrho;
        D[0] = fmaf(om, w0 * base - d[0], (g * w0) * nuF3);
        auto quad = [&](float w, float2 cu, float2 cF, float2 dn, float2 dm, float2& Dn, float2& Dm) {
            const float2 ev = mul_r(w, vfma(rho45 * cu, cu, base));
            const float2 od = mul_r(w, rho3 * cu);
            const float2 Sev = mul_r(w, vfma(9.f * cu, cF, nuF3));
            const float2 Sod = mul_r(3.f * w, cF);
            Dn = vfma(om, (ev + od) - dn, g * (Sev + Sod));
            Dm = vfma(om, (ev - od) - dm, g * (Sev - Sod));
        };
        float2 D12, D34, D56, D78;
        quad(w1, f2(ux, uy), f2(Fx, Fy), f2(d[1], d[2]), f2(d[3], d[4]), D12, D34);
        quad(w5, f2(ux + uy, uy - ux), f2(Fx + Fy, Fy - Fx), f2(d[5], d[6]), f2(d[7], d[8]), D56, D78);
        const float2 e = (((D12 - D34) + f2(D56.x - D56.y, D56.x - D78.y)) + f2(D78.y - D78.x, D56.y - D78.x)) -
                         f2(Fx, Fy);                      // (ex, ey)
        D12 = vfma(-0.5f, e, D12);
        D34 = vfma(0.5f, e, D34);
        D[1] = D12.x; D[2] = D12.y; D[3] = D34.x; D[4] = D34.y;
        D[5] = D56.x; D[6] = D56.y; D[7] = D78.x; D[8] = D78.y;
        D[0] = D[0] - ((((D[1] + D[2]) + (D[3] + D[4])) + ((D[5] + D[6]) + (D[7] + D[8]))) + D[0]);
        return;
    }
    const T nrho = (-ph.rho0) - drho;                   // -rho
    const T uu = 1.5f * vfma(ux, ux, uy * uy);
    const T nuF3 = -3.f * vfma(ux, Fx, uy * Fy);        // -3 u.F
    const T base = vfma(nrho, uu, drho);                // even part common to all directions
    const T rho3 = -3.f * nrho, rho45 = -4.5f * nrho;
    D[0] = vfma(om, w0 * base - d[0], (g * w0) * nuF3);
    // one pair (n, opposite m) with velocity c: cu = c.u, cF = c.F
    auto pair = [&](int n, int m, float w, T cu, T cF) {
        const T ev = w * vfma(rho45 * cu, cu, base);              // even part of d^eq
        const T od = w * (rho3 * cu);                              // odd part of d^eq
        const T Sev = w * vfma(9.f * cu, cF, nuF3);               // even part of S
        const T Sod = (3.f * w) * cF;                              // odd part of S
        D[n] = vfma(om, (ev + od) - d[n], g * (Sev + Sod));
        D[m] = vfma(om, (ev - od) - d[m], g * (Sev - Sod));
    };
    pair(1, 3, w1, ux, Fx);
    pair(2, 4, w1, uy, Fy);
    pair(5, 7, w5, ux + uy, Fx + Fy);
    pair(6, 8, w5, uy - ux, Fy - Fx);
    const T ex = (((D[1] - D[3]) + (D[5] - D[6])) + (D[8] - D[7])) - Fx;
    const T ey = (((D[2] - D[4]) + (D[5] - D[8])) + (D[6] - D[7])) - Fy;
    D[1] = vfma(-0.5f, ex, D[1]);
    D[3] = vfma(0.5f, ex, D[3]);
    D[2] = vfma(-0.5f, ey, D[2]);
    D[4] = vfma(0.5f, ey, D[4]);
    D[0] = D[0] - ((((D[1] + D[2]) + (D[3] + D[4])) + ((D[5] + D[6]) + (D[7] + D[8]))) + D[0]);
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
