/*
 * vlb3d_oracle.c -- plain FP64 CPU oracle of the three-dimensional step (TEST INFRASTRUCTURE
 * ONLY; see vlb3d_oracle.h).
 *
 * The two-dimensional method of Sec. II written for three dimensions, in the paper's order
 * (Fig. 2); slow on purpose: every stage is a full-lattice loop in natural (z, y, x) order.
 * Readings of points the paper leaves open are marked "Reading:" where they are used.
 */
#include "vlb3d_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

/* D3Q19 (Sec. II A with d = 3): rest, the six faces, the twelve edges. */
static const int CV[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double wq(int n) { return n == 0 ? 1.0 / 3.0 : (n < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

void o3_lattice(int32_t* c, double* w)
{
    for (int n = 0; n < 19; ++n) {
        for (int a = 0; a < 3; ++a) c[3 * n + a] = CV[n][a];
        w[n] = wq(n);
    }
}

/* Symmetric-tensor storage: component index of (i, j) in (xx, yy, zz, yz, xz, xy). */
static int sym(int i, int j)
{
    if (i == j) return i;
    int s = i + j;          /* (1,2) -> 3, (0,2) -> 2, (0,1) -> 1 */
    return s == 3 ? 3 : (s == 2 ? 4 : 5);
}

/* ------------------------------------------------------------------------------------ */
/* Periodic indexing and central differences                                            */
/* ------------------------------------------------------------------------------------ */

static int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

static double at(const o3_params* p, const double* f, int x, int y, int z)
{
    x = wrapi(x, p->nx); y = wrapi(y, p->ny); z = wrapi(z, p->nz);
    return f[((size_t)z * p->ny + y) * p->nx + x];
}

/* Central first difference along axis a (0: x, 1: y, 2: z) and the 7-point Laplacian (second
 * order, the three-dimensional form of the 2D stencils). */
static double D(const o3_params* p, const double* f, int a, int x, int y, int z)
{
    int dx = a == 0, dy = a == 1, dz = a == 2;
    return 0.5 * (at(p, f, x + dx, y + dy, z + dz) - at(p, f, x - dx, y - dy, z - dz));
}

static double Lap(const o3_params* p, const double* f, int x, int y, int z)
{
    return at(p, f, x + 1, y, z) + at(p, f, x - 1, y, z) + at(p, f, x, y + 1, z)
         + at(p, f, x, y - 1, z) + at(p, f, x, y, z + 1) + at(p, f, x, y, z - 1)
         - 6.0 * at(p, f, x, y, z);
}

/* ------------------------------------------------------------------------------------ */
/* Orientation distribution on the sphere and the stiffness tensor (Sec. II C, Sec. IV)  */
/* ------------------------------------------------------------------------------------ */

double o3_langevin(double k)
{
    /* Reading: the maximum-entropy density on the unit sphere with a given mean direction is
     * the Fisher density g(n) = k exp(k n.P^) / (4 pi sinh k) (the three-dimensional von Mises
     * density); its mean projection is coth k - 1/k.  Series below k = 0.05. */
    if (k < 0.05) {
        double k2 = k * k;
        return k * (1.0 / 3.0 - k2 * (1.0 / 45.0 - k2 * (2.0 / 945.0 - k2 / 4725.0)));
    }
    return 1.0 / tanh(k) - 1.0 / k;
}

double o3_k_of_P(double P)
{
    /* Newton on L(k) = P with a bisection bracket; L'(k) = 1/k^2 - 1/sinh^2 k. */
    if (P <= 0.0) return 0.0;
    double lo = 0.0, hi = 1.0;
    while (o3_langevin(hi) < P) { lo = hi; hi *= 2.0; }
    double k = 3.0 * P / (1.0 - P * P);                      /* small-k estimate */
    if (k <= lo || k >= hi) k = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double g = o3_langevin(k) - P;
        if (g > 0) hi = k; else lo = k;
        double d;
        if (k < 0.05) d = 1.0 / 3.0 - k * k / 15.0;
        else { double sh = sinh(k); d = 1.0 / (k * k) - 1.0 / (sh * sh); }
        double kn = k - g / d;
        if (!(kn > lo && kn < hi)) kn = 0.5 * (lo + hi);
        if (fabs(kn - k) <= 1e-15 * (1.0 + k)) { k = kn; break; }
        k = kn;
    }
    return k;
}

void o3_gauss_legendre(int32_t n, double* x, double* w)
{
    /* Roots of the Legendre polynomial P_n by Newton from the asymptotic estimate, weights
     * 2 / ((1 - x^2) P_n'(x)^2). */
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double r = cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = r;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * r * p1 - (j - 1.0) * p0) / j;
                p0 = p1; p1 = p2;
            }
            if (n == 1) p0 = 1.0;
            dp = n * (r * p1 - p0) / (r * r - 1.0);
            double dr = p1 / dp;
            r -= dr;
            if (fabs(dr) < 1e-16) break;
        }
        /* the final derivative at the converged root */
        double p0 = 1.0, p1 = r;
        for (int j = 2; j <= n; ++j) {
            double p2 = ((2.0 * j - 1.0) * r * p1 - (j - 1.0) * p0) / j;
            p0 = p1; p1 = p2;
        }
        dp = n * (r * p1 - p0) / (r * r - 1.0);
        x[i] = -r; x[n - 1 - i] = r;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
}

void o3_orientation_moments(double k, int32_t n_quad, double* m)
{
    /* <mu^j> = int mu^j exp(k mu) dOmega / int exp(k mu) dOmega with mu = n.P^; the azimuth
     * gives 2 pi to both.  Reading (Sec. IV leaves the method open): Gauss-Legendre in mu on
     * [-1, 1] for k < 1; for larger k in s = k (1 - mu) on the panels [0, 1], [1, 2], [2, 4],
     * ... up to 2k, where exp(-s) is smooth on every panel. */
    double* x = (double*)malloc(sizeof(double) * (size_t)n_quad);
    double* w = (double*)malloc(sizeof(double) * (size_t)n_quad);
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    o3_gauss_legendre(n_quad, x, w);
    if (k < 1.0) {
        for (int q = 0; q < n_quad; ++q) {
            double mu = x[q], e = w[q] * exp(k * (mu - 1.0)), pw = 1.0;
            for (int j = 0; j < 5; ++j) { s[j] += e * pw; pw *= mu; }
        }
    } else {
        double a = 0.0, b = 1.0, top = 2.0 * k;
        while (a < top) {
            if (b > top) b = top;
            for (int q = 0; q < n_quad; ++q) {
                double sv = a + 0.5 * (b - a) * (x[q] + 1.0);
                double e = 0.5 * (b - a) * w[q] * exp(-sv) / k;
                double mu = 1.0 - sv / k, pw = 1.0;
                for (int j = 0; j < 5; ++j) { s[j] += e * pw; pw *= mu; }
            }
            a = b;
            b = 2.0 * a;
        }
    }
    for (int j = 0; j < 5; ++j) m[j] = s[j] / s[0];
    free(x); free(w);
}

static double kd(int i, int j) { return i == j ? 1.0 : 0.0; }

void o3_stiffness(const o3_params* p, const double* P, double* C)
{
    /* Eq. CTens over the unit sphere: C = int g(n) K(n) dOmega with g the Fisher density about
     * P^ (concentration k from |P| capped at P_cap) and K(n) the rotation of K^x (Eq. rotate).
     * Reading (three dimensions): K^x is transversely isotropic about x, so besides the four
     * constants of Eq. Kmatrix (with K1133 = K1122, K3333 = K2222, K1313 = K1212) it has K2233,
     * and K2323 = (K2222 - K2233)/2.  Such a tensor about an axis n is
     *   K = a1 nnnn + a2 (nn d + d nn) + a3 d d + a4 (n_i n_k d_jl + n_i n_l d_jk + n_j n_k d_il
     *       + n_j n_l d_ik) + a5 (d_ik d_jl + d_il d_jk),
     * so by linearity C follows from the moment tensors M2 = <nn> and M4 = <nnnn> of g, which
     * are transversely isotropic about P^ and fixed by <mu^2>, <mu^4> (numerical quadrature). */
    double a5 = 0.5 * (p->K2222 - p->K2233);
    double a3 = p->K2233;
    double a4 = p->K1212 - a5;
    double a2 = p->K1122 - a3;
    double a1 = p->K1111 - 2.0 * a2 - a3 - 4.0 * a4 - 2.0 * a5;
    double Pm = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    double pc = Pm < p->P_cap ? Pm : p->P_cap;
    double n[3] = {1.0, 0.0, 0.0};
    if (Pm > 0.0) { n[0] = P[0] / Pm; n[1] = P[1] / Pm; n[2] = P[2] / Pm; }
    double m[5];
    o3_orientation_moments(pc > 0.0 ? o3_k_of_P(pc) : 0.0, p->n_quad, m);
    /* M2 = A d + B pp (trace 1, p.M2.p = <mu^2>); M4 = e1 pppp + e2 Sym(pp d) + e3 Sym(d d)
     * with the contractions M4_iikk... : e1 + 6 e2 + 3 e3 = <mu^4>, e1 + 7 e2 = B, e2 + 5 e3 = A */
    double A = 0.5 * (1.0 - m[2]), B = 0.5 * (3.0 * m[2] - 1.0);
    double e3 = (A - B + m[4]) / 8.0, e2 = A - 5.0 * e3, e1 = B - 7.0 * e2;
    double M2[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M2[i][j] = A * kd(i, j) + B * n[i] * n[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double M4 = e1 * n[i] * n[j] * n[k] * n[l]
                              + e2 * (n[i] * n[j] * kd(k, l) + n[i] * n[k] * kd(j, l) + n[i] * n[l] * kd(j, k)
                                      + n[j] * n[k] * kd(i, l) + n[j] * n[l] * kd(i, k) + n[k] * n[l] * kd(i, j))
                              + e3 * (kd(i, j) * kd(k, l) + kd(i, k) * kd(j, l) + kd(i, l) * kd(j, k));
                    C[((i * 3 + j) * 3 + k) * 3 + l] =
                        a1 * M4
                        + a2 * (M2[i][j] * kd(k, l) + kd(i, j) * M2[k][l])
                        + a3 * kd(i, j) * kd(k, l)
                        + a4 * (M2[i][k] * kd(j, l) + M2[i][l] * kd(j, k) + M2[j][k] * kd(i, l) + M2[j][l] * kd(i, k))
                        + a5 * (kd(i, k) * kd(j, l) + kd(i, l) * kd(j, k));
                }
}

/* ------------------------------------------------------------------------------------ */
/* Forces, moments, right-hand sides                                                      */
/* ------------------------------------------------------------------------------------ */

static void molecular_field(const o3_params* p, const double* P, int x, int y, int z, double* h)
{
    /* h_i = (alpha + beta |P|^2) P_i - kappa lap P_i (Eq. Ffunctional, three components) */
    size_t N = (size_t)p->nx * p->ny * p->nz;
    double Pc[3], P2 = 0.0;
    for (int i = 0; i < 3; ++i) { Pc[i] = at(p, P + i * N, x, y, z); P2 += Pc[i] * Pc[i]; }
    for (int i = 0; i < 3; ++i) h[i] = (p->alpha + p->beta * P2) * Pc[i] - p->kappa * Lap(p, P + i * N, x, y, z);
}

void o3_forces(const o3_params* p, const double* sigma, const double* P, const double* fext,
               double* F, double* h, double* fp)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    size_t N = (size_t)nx * ny * nz;
    double* sE = (double*)malloc(9 * N * sizeof(double));
    /* molecular field and Ericksen stress of every cell (Sec. II C 1):
     * sigma^E_ij = -1/2 (P_i h_j - h_i P_j) + xi/2 (P_i h_j + h_i P_j) - kappa d_i P_k d_j P_k
     * (kappa on the gradient term as in the two-dimensional oracle's reading) */
    #pragma omp parallel for collapse(2)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = ((size_t)z * ny + y) * nx + x;
                double hc[3], Pc[3], G[3][3];
                molecular_field(p, P, x, y, z, hc);
                for (int i = 0; i < 3; ++i) {
                    h[i * N + c] = hc[i];
                    Pc[i] = P[i * N + c];
                    for (int a = 0; a < 3; ++a) G[a][i] = D(p, P + i * N, a, x, y, z);   /* d_a P_i */
                }
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double gg = 0.0;
                        for (int k = 0; k < 3; ++k) gg += G[i][k] * G[j][k];
                        sE[(i * 3 + j) * N + c] = -0.5 * (Pc[i] * hc[j] - hc[i] * Pc[j])
                                                + 0.5 * p->xi * (Pc[i] * hc[j] + hc[i] * Pc[j]) - p->kappa * gg;
                    }
            }
    /* f^p_i = d_j sigma^p_ij, f^E_i = d_j sigma^E_ij; F = f^p + f^E + external */
    #pragma omp parallel for collapse(2)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = ((size_t)z * ny + y) * nx + x;
                for (int i = 0; i < 3; ++i) {
                    double fpi = 0.0, fei = 0.0;
                    for (int j = 0; j < 3; ++j) {
                        fpi += D(p, sigma + sym(i, j) * N, j, x, y, z);
                        if (p->ericksen) fei += D(p, sE + (i * 3 + j) * N, j, x, y, z);
                    }
                    F[i * N + c] = fpi + fei + (fext ? fext[i] : 0.0);
                    if (fp) fp[i * N + c] = fpi;
                }
            }
    free(sE);
}

void o3_moments(const o3_params* p, const double* h, const double* F, double* rho, double* u)
{
    /* Eq. rhoDef, Eq. vDef with the Guo half-force correction */
    size_t N = (size_t)p->nx * p->ny * p->nz;
    #pragma omp parallel for
    for (size_t c = 0; c < N; ++c) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int n = 0; n < 19; ++n) {
            double hn = h[n * N + c];
            r += hn;
            for (int a = 0; a < 3; ++a) j[a] += CV[n][a] * hn;
        }
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u[a * N + c] = (j[a] + 0.5 * F[a * N + c]) / r;
    }
}

void o3_rhs(const o3_params* p, const double* sigma, const double* P, const double* u,
            double* dsigma, double* dP)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    size_t N = (size_t)nx * ny * nz;
    #pragma omp parallel for collapse(2)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = ((size_t)z * ny + y) * nx + x;
                double uc[3], G[3][3], Psi[3][3], Om[3][3], s[3][3], Pc[3], C[81];
                for (int a = 0; a < 3; ++a) { uc[a] = u[a * N + c]; Pc[a] = P[a * N + c]; }
                /* velocity gradient G_ij = d_i u_j of the frozen u; Psi its symmetric part,
                 * Omega_ij = (G_ij - G_ji)/2 */
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) G[i][j] = D(p, u + j * N, i, x, y, z);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        Psi[i][j] = 0.5 * (G[i][j] + G[j][i]);
                        Om[i][j] = 0.5 * (G[i][j] - G[j][i]);
                        s[i][j] = sigma[sym(i, j) * N + c];
                    }
                o3_stiffness(p, Pc, C);
                /* Eq. StiffCons with the Jaumann derivative:
                 * d_t s = -(u.grad) s - (Omega s - s Omega) + C:Psi - C:s / eta_p + D_p lap s */
                for (int i = 0; i < 3; ++i)
                    for (int j = i; j < 3; ++j) {
                        int comp = sym(i, j);
                        const double* sc = sigma + comp * N;
                        double adv = 0.0, J = 0.0, Cpsi = 0.0, Cs = 0.0;
                        for (int a = 0; a < 3; ++a) adv += uc[a] * D(p, sc, a, x, y, z);
                        for (int k = 0; k < 3; ++k) J += Om[i][k] * s[k][j] - s[i][k] * Om[k][j];
                        for (int k = 0; k < 3; ++k)
                            for (int l = 0; l < 3; ++l) {
                                double Cijkl = C[((i * 3 + j) * 3 + k) * 3 + l];
                                Cpsi += Cijkl * Psi[k][l];
                                Cs += Cijkl * s[k][l];
                            }
                        dsigma[comp * N + c] = -adv - J + Cpsi - Cs / p->eta_p + p->Dp * Lap(p, sc, x, y, z);
                    }
                /* Eq. BE: d_t P_i = -(u.grad) P_i - Omega_ik P_k + xi Psi_ik P_k - Gamma h_i */
                double hc[3];
                molecular_field(p, P, x, y, z, hc);
                for (int i = 0; i < 3; ++i) {
                    double adv = 0.0, rot = 0.0, str = 0.0;
                    for (int a = 0; a < 3; ++a) adv += uc[a] * D(p, P + i * N, a, x, y, z);
                    for (int k = 0; k < 3; ++k) { rot += Om[i][k] * Pc[k]; str += Psi[i][k] * Pc[k]; }
                    dP[i * N + c] = -adv - rot + p->xi * str - p->Gamma * hc[i];
                }
            }
}

/* ------------------------------------------------------------------------------------ */
/* One time step                                                                          */
/* ------------------------------------------------------------------------------------ */

int o3_step(const o3_params* p, double* h, double* sigma, double* P, const double* fext, o3_diag* diag)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    size_t N = (size_t)nx * ny * nz;
    double* F = (double*)malloc(3 * N * sizeof(double));
    double* hm = (double*)malloc(3 * N * sizeof(double));
    double* rho = (double*)malloc(N * sizeof(double));
    double* u = (double*)malloc(3 * N * sizeof(double));
    double* hs = (double*)malloc(19 * N * sizeof(double));
    double* ds0 = (double*)malloc(6 * N * sizeof(double));
    double* dP0 = (double*)malloc(3 * N * sizeof(double));
    double* ds1 = (double*)malloc(6 * N * sizeof(double));
    double* dP1 = (double*)malloc(3 * N * sizeof(double));
    double* s1 = (double*)malloc(6 * N * sizeof(double));
    double* P1 = (double*)malloc(3 * N * sizeof(double));
    if (!F || !hm || !rho || !u || !hs || !ds0 || !dP0 || !ds1 || !dP1 || !s1 || !P1) return -1;

    /* 1-4. forces of the state at t: f^p, molecular field, f^E, F (Fig. 2) */
    o3_forces(p, sigma, P, fext, F, hm, NULL);
    /* 5. moments rho, u */
    o3_moments(p, h, F, rho, u);
    if (diag) {
        double m = 0.0, j[3] = {0.0, 0.0, 0.0}, f[3] = {0.0, 0.0, 0.0};
        for (size_t c = 0; c < N; ++c) {
            m += rho[c] - p->rho0;
            for (int n = 0; n < 19; ++n)
                for (int a = 0; a < 3; ++a) j[a] += CV[n][a] * h[n * N + c];
            for (int a = 0; a < 3; ++a) f[a] += F[a * N + c];
        }
        diag->mass_excess = m;
        for (int a = 0; a < 3; ++a) { diag->mom[a] = j[a]; diag->force[a] = f[a]; }
    }
    /* 6. BGK collision with Guo forcing:
     * h* = h - (h - h^eq)/tau + (1 - 1/(2 tau)) w_n [3 (c_n - u) + 9 (c_n.u) c_n] . F */
    double tau = p->tau;
    #pragma omp parallel for
    for (size_t c = 0; c < N; ++c) {
        double uc[3] = {u[c], u[N + c], u[2 * N + c]}, Fc[3] = {F[c], F[N + c], F[2 * N + c]};
        double uu = uc[0] * uc[0] + uc[1] * uc[1] + uc[2] * uc[2];
        for (int n = 0; n < 19; ++n) {
            double cu = CV[n][0] * uc[0] + CV[n][1] * uc[1] + CV[n][2] * uc[2];
            double heq = wq(n) * rho[c] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            double S = 0.0;
            for (int a = 0; a < 3; ++a) S += (3.0 * (CV[n][a] - uc[a]) + 9.0 * cu * CV[n][a]) * Fc[a];
            S *= (1.0 - 0.5 / tau) * wq(n);
            hs[n * N + c] = h[n * N + c] - (h[n * N + c] - heq) / tau + S;
        }
    }
    /* 7. streaming h_n(r + c_n, t + 1) = h*_n(r) (periodic) */
    #pragma omp parallel for collapse(2)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t c = ((size_t)z * ny + y) * nx + x;
                for (int n = 0; n < 19; ++n) {
                    int xd = wrapi(x + CV[n][0], nx), yd = wrapi(y + CV[n][1], ny), zd = wrapi(z + CV[n][2], nz);
                    h[n * N + ((size_t)zd * ny + yd) * nx + xd] = hs[n * N + c];
                }
            }
    /* 8-9. Heun predictor-corrector on (sigma, P) jointly, u(t) frozen */
    o3_rhs(p, sigma, P, u, ds0, dP0);
    #pragma omp parallel for
    for (size_t i = 0; i < 6 * N; ++i) s1[i] = sigma[i] + ds0[i];
    #pragma omp parallel for
    for (size_t i = 0; i < 3 * N; ++i) P1[i] = P[i] + dP0[i];
    o3_rhs(p, s1, P1, u, ds1, dP1);
    #pragma omp parallel for
    for (size_t i = 0; i < 6 * N; ++i) sigma[i] += 0.5 * (ds0[i] + ds1[i]);
    #pragma omp parallel for
    for (size_t i = 0; i < 3 * N; ++i) P[i] += 0.5 * (dP0[i] + dP1[i]);

    free(F); free(hm); free(rho); free(u); free(hs); free(ds0); free(dP0); free(ds1); free(dP1);
    free(s1); free(P1);
    return 0;
}
